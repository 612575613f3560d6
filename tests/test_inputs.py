"""The seeded input generators shared by the CUDA path and the oracle
(paper_2003_01490_gb300/workloads.py), CPU only: SplitMix64 against the
published reference output, the moments of its uniform and normal draws,
non-overlapping sphere placement, and reproducibility from the seed."""
import itertools
import math

import numpy as np

from paper_2003_01490_gb300 import workloads
from paper_2003_01490_gb300.workloads import SplitMix64


def test_splitmix64_matches_the_published_reference_output():
    # first outputs of the reference SplitMix64 (Steele, Lea and Flood's
    # generator as published with Vigna's reference code) for seed 1234567
    rng = SplitMix64(1234567)
    assert [rng.next_u64() for _ in range(5)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423,
        4593380528125082431, 16408922859458223821]


def test_uniform_and_normal_draws_have_the_right_moments():
    rng = SplitMix64(20030149)
    u = np.array([rng.uniform() for _ in range(100_000)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.005 and abs(u.var() - 1 / 12) < 0.002
    z = np.array([rng.normal(2.0) for _ in range(100_000)])
    assert abs(z.mean()) < 0.03 and abs(z.std() - 2.0) < 0.03
    assert abs(np.mean(np.abs(z) < 2.0) - math.erf(1 / math.sqrt(2))) < 0.01


def test_random_sequential_addition_places_non_overlapping_spheres():
    shape, n, D = (40, 36, 48), 60, 9.0
    pts = workloads.random_sequential_addition(shape, n, D, SplitMix64(5))
    pts = np.asarray(pts)
    assert pts.shape == (n, 3)
    L = np.array(shape, dtype=float)
    assert (pts >= 0).all() and (pts < L).all()
    for i, j in itertools.combinations(range(n), 2):
        d = pts[i] - pts[j]
        d -= L * np.round(d / L)
        assert d @ d >= D * D


def test_workloads_are_reproducible_from_their_seed():
    a = workloads.suspension(shape=(48, 48, 64), n=24, D=12.0, seed=7, storage='f32', steps=0)
    b = workloads.suspension(shape=(48, 48, 64), n=24, D=12.0, seed=7, storage='f32', steps=0)
    c = workloads.suspension(shape=(48, 48, 64), n=24, D=12.0, seed=8, storage='f32', steps=0)
    assert np.array_equal(a['pos'], b['pos']) and np.array_equal(a['vel'], b['vel'])
    assert not np.array_equal(a['pos'], c['pos'])
    # the full suspension's solid fraction: 10,000 spheres of D = 12 in 256 x 256 x 512
    assert abs(10_000 * math.pi * 12 ** 3 / 6 / (256 * 256 * 512) - 0.2696) < 1e-4
