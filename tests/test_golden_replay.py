"""The stored oracle trajectory (tests/golden/suspension_32x32x64_trajectory.txt,
which the long-run GPU precision test compares against) is the output of the
oracle as it stands: its first checkpoint is recomputed here (CPU only)."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, 'golden'))

import make_precision_trajectory as gen  # noqa: E402
from oracle.sim import Domain, Params, Simulation  # noqa: E402


def test_first_checkpoint_of_the_stored_trajectory_is_reproduced():
    w = gen.case()
    dem = w['dem']
    p = Params(tau=w['tau'], body_force=w['body_force'], e_dry=dem['e_dry'], Tc=dem['Tc'],
               nu_p=dem['nu_p'], mu_p=dem['mu_p'], n_sub=dem['n_sub'], gravity=dem['gravity'],
               fluid_counterforce=bool(dem.get('fluid_counterforce', 0)))
    sim = Simulation(Domain(*w['shape'], periodic=tuple(bool(v) for v in w['periodic'])), p)
    sim.add_spheres(w['pos'], w['vel'], w['omega'], w['radius'], w['density'])
    sim.step(gen.CHECKPOINTS[0])
    lines = open(gen.OUT).read().splitlines()
    i = lines.index('step %d' % gen.CHECKPOINTS[0])
    n = len(w['radius'])
    ref = np.array([[float(v) for v in lines[i + 1 + k].split()] for k in range(n)])
    stats = np.array([float(v) for v in lines[i + 1 + n].split()[1:]])
    assert np.abs(sim.X - ref[:, :3]).max() <= 1e-12 * np.abs(ref[:, :3]).max()
    assert np.abs(sim.U - ref[:, 3:]).max() <= 1e-12 * np.abs(ref[:, 3:]).max()
    assert np.allclose(gen.field_stats(sim), stats, rtol=1e-10, atol=0)


def test_sphere_wall_golden_is_the_oracle_as_it_stands():
    # the first steps of tests/golden/sphere_wall_2000.npz, recomputed: the
    # stored trajectory is what the oracle computes (bit for bit on this host)
    import numpy as np
    sys.path.insert(0, os.path.join(HERE, 'golden'))
    import make_long_runs
    from cases import build_oracle
    gold = np.load(os.path.join(HERE, 'golden', 'sphere_wall_2000.npz'))['states']
    sim = build_oracle(make_long_runs.sphere_wall_case())
    for k in range(5):
        sim.step()
        got = np.concatenate([sim.X[0], sim.U[0], sim.Om[0], sim.Ffp[0], sim.Tfp[0]])
        assert np.allclose(got, gold[k], rtol=1e-13, atol=1e-16), k


def test_storage_rounding_of_the_floor_runs_matches_torch_conversions():
    # the storage floor rounds f - w as the GPU stores it: float32 round to
    # nearest even, float16 and bfloat16 from the float32 value
    import numpy as np
    import torch
    sys.path.insert(0, os.path.join(HERE, 'golden'))
    import make_long_runs
    rng = np.random.default_rng(3)
    v = np.concatenate([rng.normal(0, 1e-3, 5000), rng.normal(0, 1e-6, 5000), [0.0, -0.0, 1e-40, 65504.0]])
    t = torch.tensor(v.astype(np.float32))
    assert np.array_equal(make_long_runs.round_storage(v, 'f32'), t.double().numpy())
    assert np.array_equal(make_long_runs.round_storage(v, 'f16'), t.to(torch.float16).double().numpy())
    assert np.array_equal(make_long_runs.round_storage(v, 'bf16'), t.to(torch.bfloat16).double().numpy())
