"""Build the oracle and the CUDA context from one case description.

A case is a dict with keys shape, periodic, tau, storage, body_force, and
optional wall_vel_lo / wall_vel_hi ([axis][component]), relax (overrides of
magic, lambda_b_shell, lambda_b_bulk, shell_width), dem (overrides of the DEM
parameters) and spheres (pos, vel, omega, radius, density arrays).
"""
import numpy as np

from oracle import Domain, Params, Simulation

DEM_DEFAULTS = dict(e_dry=0.97, Tc=0.0, nu_p=0.23, mu_p=0.15, n_sub=10, lub_cut_n=2.0 / 3.0,
                    lub_cut_tt=0.5, lub_cut_tr=0.5, lub_min_a=0.001, lub_min_b=0.00007,
                    gravity=(0.0, 0.0, 0.0), lubrication=1, tangential_lubrication=1,
                    force_averaging=1, fluid_counterforce=0, fixed_particles=0, missing_links=1)
RELAX_DEFAULTS = dict(magic=3.0 / 16.0, lambda_b_shell=100.0, lambda_b_bulk=1.0, shell_width=2.0)


def _merged(case):
    dem = dict(DEM_DEFAULTS)
    dem.update(case.get('dem', {}))
    relax = dict(RELAX_DEFAULTS)
    relax.update(case.get('relax', {}))
    return relax, dem


def build_oracle(case):
    relax, dem = _merged(case)
    dom = Domain(*case['shape'], periodic=tuple(bool(p) for p in case['periodic']),
                 wall_vel_lo=case.get('wall_vel_lo'), wall_vel_hi=case.get('wall_vel_hi'))
    p = Params(tau=case['tau'], magic=relax['magic'], lambda_b_shell=relax['lambda_b_shell'],
               lambda_b_bulk=relax['lambda_b_bulk'], shell_width=relax['shell_width'],
               body_force=case.get('body_force', (0, 0, 0)), e_dry=dem['e_dry'], Tc=dem['Tc'],
               nu_p=dem['nu_p'], mu_p=dem['mu_p'], n_sub=dem['n_sub'],
               lub_cut_n=dem['lub_cut_n'], lub_cut_tt=dem['lub_cut_tt'],
               lub_cut_tr=dem['lub_cut_tr'], lub_min_a=dem['lub_min_a'],
               lub_min_b=dem['lub_min_b'], gravity=dem['gravity'],
               lubrication=bool(dem['lubrication']),
               tangential_lubrication=bool(dem['tangential_lubrication']),
               force_averaging=bool(dem['force_averaging']),
               fluid_counterforce=bool(dem['fluid_counterforce']),
               fixed_particles=int(dem['fixed_particles']) == 1,
               prescribed_motion=int(dem['fixed_particles']) == 2,
               missing_links=bool(dem['missing_links']))
    sim = Simulation(dom, p)
    if 'init_pdfs' in case:
        sim.set_pdfs(case['init_pdfs'])
    sp = case.get('spheres')
    if sp is not None and len(sp['radius']):
        sim.add_spheres(sp['pos'], sp['vel'], sp['omega'], sp['radius'], sp['density'])
    return sim


def build_gpu(case, max_particles=None):
    from paper_2003_01490_gb300 import lbmdem as L
    relax, dem = _merged(case)
    r, d = L.lbm_default_params()
    r.tau = case['tau']
    for k, v in relax.items():
        setattr(r, k, v)
    for k, v in dem.items():
        if k == 'gravity':
            for a in range(3):
                d.gravity[a] = float(v[a])
        else:
            setattr(d, k, v)
    g = L.make_grid(case['shape'], case['periodic'], case.get('wall_vel_lo'),
                    case.get('wall_vel_hi'))
    sp = case.get('spheres')
    n = 0 if sp is None else len(sp['radius'])
    ctx = L.lbm_create(g, r, case.get('body_force', (0, 0, 0)), d, case['storage'],
                       max_particles if max_particles is not None else max(n, 1))
    if 'init_pdfs' in case:
        L.lbm_set_pdfs(ctx, case['init_pdfs'])
    if n:
        L.lbm_add_spheres(ctx, sp['pos'], sp['vel'], sp['omega'], sp['radius'], sp['density'])
    return ctx


def spheres(pos, radius, density=None, vel=None, omega=None):
    pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    n = len(pos)
    return dict(pos=pos, radius=np.asarray(radius, dtype=np.float64).reshape(n),
                density=np.full(n, 2.0) if density is None else np.asarray(density, float).reshape(n),
                vel=np.zeros((n, 3)) if vel is None else np.asarray(vel, float).reshape(n, 3),
                omega=np.zeros((n, 3)) if omega is None else np.asarray(omega, float).reshape(n, 3))


def rel_l2(a, b, mask=None):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    if mask is not None:
        a = a[..., mask]
        b = b[..., mask]
    den = np.sqrt((b * b).sum())
    return np.sqrt(((a - b) ** 2).sum()) / (den if den > 0 else 1.0)
