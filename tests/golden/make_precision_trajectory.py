"""Writes suspension_32x32x64_trajectory.txt: the float64 oracle's particle
positions and velocities, and fluid-field statistics, along 1000 steps of a
32 x 32 x 64 periodic suspension (19 spheres of D = 12, 26 % solids, the
parameters of the 256 x 256 x 512 suspension). Uses only the oracle and the
seeded input generator. Run from the repository root:

    python tests/golden/make_precision_trajectory.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, 'tests'))

from oracle.sim import Domain, Params, Simulation  # noqa: E402
from paper_2003_01490_gb300 import workloads       # noqa: E402

CHECKPOINTS = (100, 250, 500, 1000)
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), 'suspension_32x32x64_trajectory.txt')


def case():
    return workloads.suspension(shape=(32, 32, 64), n=19, D=12.0, seed=20030149, storage='f64', steps=1000)


def field_stats(sim):
    rho, u = sim.fields()
    fluid = sim.owner < 0
    uf = u[:, fluid]
    return [float(uf[0].mean()), float(uf[1].mean()), float(uf[2].mean()),
            float(np.sqrt((uf ** 2).sum(0).mean())), float(np.sqrt(((rho[fluid] - 1.0) ** 2).mean()))]


def main():
    w = case()
    dem = w['dem']
    p = Params(tau=w['tau'], body_force=w['body_force'], e_dry=dem['e_dry'], Tc=dem['Tc'], nu_p=dem['nu_p'],
               mu_p=dem['mu_p'], n_sub=dem['n_sub'], gravity=dem['gravity'],
               fluid_counterforce=bool(dem.get('fluid_counterforce', 0)))
    sim = Simulation(Domain(*w['shape'], periodic=tuple(bool(v) for v in w['periodic'])), p)
    sim.add_spheres(w['pos'], w['vel'], w['omega'], w['radius'], w['density'])
    lines = ['# float64 oracle, 32x32x64 periodic suspension, 19 spheres D=12 (seed 20030149),',
             '# tau 0.55, density ratio 2.5, gravity for a Stokes speed of 0.005, fluid counter force.',
             '# per checkpoint: "step N", 19 rows "x y z ux uy uz", then',
             '# "fields mean_ux mean_uy mean_uz rms_u rms_rho-1" over the fluid cells']
    done = 0
    for cp in CHECKPOINTS:
        sim.step(cp - done)
        done = cp
        lines.append('step %d' % cp)
        for x, u in zip(sim.X, sim.U):
            lines.append(' '.join('%.17e' % v for v in list(x) + list(u)))
        lines.append('fields ' + ' '.join('%.17e' % v for v in field_stats(sim)))
        print('step', cp, flush=True)
    with open(OUT, 'w') as fh:
        fh.write('\n'.join(lines) + '\n')


if __name__ == '__main__':
    main()
