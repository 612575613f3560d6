"""Seeded synthetic inputs shaped like the paper's runs (no method arithmetic here).

Used by ``bench.py`` and by the tests to feed the CUDA path and the oracle the
same inputs. Random numbers come from SplitMix64 (Steele, Lea & Flood 2014,
the generator of Java's SplittableRandom) implemented from its published
definition; normal deviates use the Box-Muller transform.

Workloads:
  * :func:`sphere_wall` -- one sphere settling towards a no-slip wall
    (32 x 32 x 64 cells, D = 8, density ratio 8, tau = 0.6, 2000 steps),
    shaped like the sphere-wall collision tests of Sec. 4.4.
  * :func:`suspension` -- dense periodic sedimenting suspension
    (256 x 256 x 512 cells, 10,000 spheres of D = 12 by random sequential
    addition, density ratio 2.5, tau = 0.55).
"""
import math

import numpy as np

MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 pseudo-random generator (64-bit state, golden-ratio increment)."""

    def __init__(self, seed):
        self.state = seed & MASK64

    def next_u64(self):
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self):
        """Double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def normal(self, sigma=1.0):
        """One N(0, sigma^2) deviate by Box-Muller (the cosine branch)."""
        u1 = 1.0 - self.uniform()
        u2 = self.uniform()
        return sigma * math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)


def random_sequential_addition(shape, n, diameter, rng, max_attempts=10_000_000):
    """Non-overlapping sphere centres in a periodic box: a uniform candidate is
    accepted iff its minimum-image distance to every accepted centre is >= D."""
    L = np.array(shape, dtype=np.float64)
    cell = diameter
    nb = np.maximum(1, np.floor(L / cell).astype(int))
    bs = L / nb
    grid = {}
    out = []
    attempts = 0
    while len(out) < n:
        attempts += 1
        if attempts > max_attempts:
            raise RuntimeError('random sequential addition did not reach %d spheres' % n)
        p = np.array([rng.uniform() * L[0], rng.uniform() * L[1], rng.uniform() * L[2]])
        b = np.minimum((p / bs).astype(int), nb - 1)
        ok = True
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    key = tuple((b + (dx, dy, dz)) % nb)
                    for q in grid.get(key, ()):
                        d = p - q
                        d -= L * np.round(d / L)
                        if d @ d < diameter * diameter:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if not ok:
                break
        if ok:
            out.append(p)
            grid.setdefault(tuple(b), []).append(p)
    return np.array(out)


def sphere_wall():
    """One sphere released at rest above a no-slip wall (shape of Sec. 4.4).

    Gravity gives a terminal Stokes number of about 10 by the Schiller-Naumann
    balance u_s = 9 St nu / ((rho_p/rho_f) D), g = 18 nu u_s (1 + 0.15 Re^0.687)
    / ((rho_p/rho_f - 1) D^2).
    """
    tau, D, ratio, St = 0.6, 8.0, 8.0, 10.0
    nu = (tau - 0.5) / 3.0
    u_s = 9.0 * St * nu / (ratio * D)
    Re = u_s * D / nu
    g = 18.0 * nu * u_s * (1.0 + 0.15 * Re ** 0.687) / ((ratio - 1.0) * D * D)
    return dict(
        name='sphere-wall 32x32x64, D=8, f64',
        shape=(32, 32, 64), periodic=(1, 1, 0), tau=tau, storage='f64', steps=2000,
        pos=np.array([[16.0, 16.0, 48.0]]), vel=np.zeros((1, 3)), omega=np.zeros((1, 3)),
        radius=np.array([D / 2]), density=np.array([ratio]),
        dem=dict(e_dry=0.97, Tc=0.0, nu_p=0.23, mu_p=0.15, n_sub=10, gravity=(0.0, 0.0, -g)),
        body_force=(0.0, 0.0, 0.0))


def suspension(shape=(256, 256, 512), n=10000, D=12.0, seed=20030149, storage='f32', steps=5000):
    """Dense periodic suspension: RSA placement, velocities N(0, (1e-3)^2) per
    component, density ratio 2.5, tau = 0.55, gravity for an isolated Stokes
    settling speed of 0.005, fluid counter force for zero net momentum input."""
    rng = SplitMix64(seed)
    pos = random_sequential_addition(shape, n, D, rng)
    vel = np.array([[rng.normal(1e-3) for _ in range(3)] for _ in range(n)])
    tau, ratio = 0.55, 2.5
    nu = (tau - 0.5) / 3.0
    g = 0.005 * 18.0 * nu / ((ratio - 1.0) * D * D)
    return dict(
        name='suspension %dx%dx%d, %d spheres D=%g, %s' % (shape + (n, D, storage)),
        shape=tuple(shape), periodic=(1, 1, 1), tau=tau, storage=storage, steps=steps,
        pos=pos, vel=vel, omega=np.zeros((n, 3)), radius=np.full(n, D / 2),
        density=np.full(n, ratio),
        dem=dict(e_dry=0.97, Tc=0.0, nu_p=0.23, mu_p=0.15, n_sub=10, gravity=(0.0, 0.0, -g),
                 fluid_counterforce=1),
        body_force=(0.0, 0.0, 0.0))


def reduced_suspension(storage='f32', seed=20030149):
    """64 x 64 x 128 cells at the same solid fraction (150 spheres of D = 12)."""
    return suspension(shape=(64, 64, 128), n=150, D=12.0, seed=seed, storage=storage, steps=1000)



def batched(n=64, seed=20030149, storage='f32', steps_divisor=20):
    """Many small independent boxes of the sphere-wall family (shape of
    Sec. 4.4, scaled down): instance k draws from SplitMix64(seed + k) a side
    s in {32, 40, ..., 96} (box s x s x 2s, no-slip walls at the z faces), a
    sphere of D = clamp(round(s / 4), 8, 24) at (s/2, s/2, 1.5 s), a density
    ratio log-uniform in [1.5, 10], tau log-uniform in [0.52, 0.8] and a step
    count uniform in {2000, ..., 10000} (divided by steps_divisor). Gravity
    follows the Schiller-Naumann balance of sphere_wall() for a settling speed
    of 0.02."""
    out = []
    for k in range(n):
        rng = SplitMix64(seed + k)
        s = 32 + 8 * int(rng.uniform() * 9)
        s = min(s, 96)
        D = float(min(24, max(8, int(round(s / 4.0)))))
        ratio = math.exp(math.log(1.5) + rng.uniform() * (math.log(10.0) - math.log(1.5)))
        tau = math.exp(math.log(0.52) + rng.uniform() * (math.log(0.8) - math.log(0.52)))
        steps = 2000 + int(rng.uniform() * 8001)
        steps = max(1, steps // steps_divisor)
        nu = (tau - 0.5) / 3.0
        u_s = 0.02
        Re = u_s * D / nu
        g = 18.0 * nu * u_s * (1.0 + 0.15 * Re ** 0.687) / ((ratio - 1.0) * D * D)
        out.append(dict(
            name='instance %d: %dx%dx%d, D=%g, ratio %.2f, tau %.3f, %s' % (k, s, s, 2 * s, D, ratio, tau, storage),
            shape=(s, s, 2 * s), periodic=(1, 1, 0), tau=tau, storage=storage, steps=steps,
            pos=np.array([[s / 2.0, s / 2.0, 1.5 * s]]), vel=np.zeros((1, 3)), omega=np.zeros((1, 3)),
            radius=np.array([D / 2]), density=np.array([ratio]),
            dem=dict(e_dry=0.97, Tc=0.0, nu_p=0.23, mu_p=0.15, n_sub=10, gravity=(0.0, 0.0, -g)),
            body_force=(0.0, 0.0, 0.0)))
    return out


def served(n=48, seed=20030149, storage='f16', steps_divisor=50, max_side=128, gap=0.004):
    """A seeded stream of independent jobs for the served mode: Poisson
    arrivals with mean gap `gap` seconds; half are sphere-wall jobs (one
    sphere, no-slip walls at the z faces), half periodic suspensions (random
    sequential addition). Every job is a cube s^3 with s in {32, 48, ...,
    max_side}; sphere diameters are uniform in [8, 16] (one per job);
    suspensions hold up to 2000 spheres, capped at 27 % solids; step counts
    are log-uniform in [1000, 20000], divided by steps_divisor."""
    rng = SplitMix64(seed)
    jobs = []
    t = 0.0
    sides = list(range(32, max_side + 1, 16))
    for k in range(n):
        t += -gap * math.log(1.0 - rng.uniform())
        s = sides[min(len(sides) - 1, int(rng.uniform() * len(sides)))]
        D = 8.0 + 8.0 * rng.uniform()
        steps = int(round(math.exp(math.log(1000.0) + rng.uniform() * (math.log(20000.0) - math.log(1000.0)))))
        steps = max(1, steps // steps_divisor)
        tau = 0.6
        nu = (tau - 0.5) / 3.0
        if rng.uniform() < 0.5:
            ratio = 4.0
            u_s = 0.02
            Re = u_s * D / nu
            g = 18.0 * nu * u_s * (1.0 + 0.15 * Re ** 0.687) / ((ratio - 1.0) * D * D)
            job = dict(name='job %d: sphere-wall %d^3, D=%.1f' % (k, s, D), shape=(s, s, s), periodic=(1, 1, 0),
                       pos=np.array([[s / 2.0, s / 2.0, 0.75 * s]]), vel=np.zeros((1, 3)), omega=np.zeros((1, 3)),
                       radius=np.array([D / 2]), density=np.array([ratio]),
                       dem=dict(e_dry=0.97, Tc=0.0, nu_p=0.23, mu_p=0.15, n_sub=10, gravity=(0.0, 0.0, -g)))
        else:
            cap = int(0.27 * s ** 3 / (math.pi * D ** 3 / 6.0))
            m = min(int(rng.uniform() * 2001), cap)
            pos = random_sequential_addition((s, s, s), m, D, rng) if m else np.zeros((0, 3))
            ratio = 2.5
            g = 0.005 * 18.0 * nu / ((ratio - 1.0) * D * D)
            job = dict(name='job %d: suspension %d^3, %d spheres D=%.1f' % (k, s, m, D), shape=(s, s, s),
                       periodic=(1, 1, 1), pos=pos, vel=np.zeros((m, 3)), omega=np.zeros((m, 3)),
                       radius=np.full(m, D / 2), density=np.full(m, ratio),
                       dem=dict(e_dry=0.97, Tc=0.0, nu_p=0.23, mu_p=0.15, n_sub=10, gravity=(0.0, 0.0, -g),
                                fluid_counterforce=1))
        job.update(tau=tau, storage=storage, steps=steps, arrival=t, body_force=(0.0, 0.0, 0.0))
        jobs.append(job)
    return jobs
