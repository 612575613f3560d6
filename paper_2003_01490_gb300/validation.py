"""Full-size validation runs on the GPU, against the values the paper prints.

These cases are too large for the float64 oracle; they check the CUDA path
against the paper's own simulation results instead.

* :func:`shear_drag_lift` -- Sec. 2.5: a fixed sphere (D = 20) at height
  L D above the resting bottom wall of a [48 x 16 x 8] D box, periodic in x
  and y, with the top wall moving at u_w = 0.1. The flow starts from the
  linear shear profile and runs until the drag and lift coefficients
  C_D = F_x / (pi/8 rho G^2 L^2 D^4) and C_L (F_z alike), G = u_w / H, settle.
  The paper prints them for L = 0.505, 1 and Re_s = G D^2 / nu = 1, 25
  (TRT+aB column of its drag/lift tables), next to the correlation of its
  reference.
* :func:`stokes_array` -- Sec. 2.4: the normalised drag C of a periodic array
  of fixed spheres in Stokes flow for the relaxation times of the paper's
  sweep and the collision models SRT, TRT, TRT+B and TRT+aB, against the
  quasi-analytical C_ref = 2.842 (the paper plots the errors).
* :func:`sphere_wall_rebound` -- Sec. 4.4: a sphere (St = 27) driven towards
  the bottom wall of a closed box with the prescribed approach velocity, then
  released (DEM with gravity) when the gap is below one diameter; reports the
  rebound height H_r = max gap / D after the first contact, which the paper
  tabulates against n_sub (mean 0.3274 at n_sub = 10).
* :func:`artificial_acceleration` -- Sec. 2.3.3: a sphere whose settling
  velocity is prescribed every step, u_p(t) = -u_s (1 - exp(-c_acc t / t_St)),
  with a density probe moving along at x_p + (D, 0, 0) (trilinear
  interpolation, every step); the paper shows the probe's spectrum for TRT,
  TRT+B (10, 100) and TRT+aB as a figure and states that the fluctuations
  stay below 0.01 % of the mean density, so the run reports the relative
  fluctuation and the spectrum's power per frequency band for each model.

Command line: ``python -m paper_2003_01490_gb300.validation shear --re 1``
prints one JSON line per case.
"""
import argparse
import json
import math
import time

import numpy as np

from . import lbmdem as L

# lattice directions and weights in the order of App. A (cx, cy, cz)
_C = np.array([[0, 0, 0], [0, 1, 0], [0, -1, 0], [-1, 0, 0], [1, 0, 0], [0, 0, 1], [0, 0, -1],
               [-1, 1, 0], [1, 1, 0], [-1, -1, 0], [1, -1, 0], [0, 1, 1], [0, -1, 1], [-1, 0, 1],
               [1, 0, 1], [0, 1, -1], [0, -1, -1], [-1, 0, -1], [1, 0, -1]], dtype=np.float64)
_W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)

# the paper's drag/lift tables (Sec. 2.5): (Re_s, L) -> (C_D, C_L) of its
# TRT+aB simulation and of the reference correlation
PAPER_SHEAR = {
    (1, 0.505): dict(sim=(44.00, 3.43), ref=(44.88, 3.54)),
    (1, 1.0): dict(sim=(34.44, 2.30), ref=(35.77, 2.32)),
    (25, 0.505): dict(sim=(3.70, 0.92), ref=(3.53, 0.88)),
    (25, 1.0): dict(sim=(2.78, 0.41), ref=(2.81, 0.45)),
}


def equilibrium_planes(ux_of_z):
    """Equilibrium PDFs (rho = 1, u = (u_x(z), 0, 0)) per z plane: (19, nz)."""
    ux = np.asarray(ux_of_z, dtype=np.float64)
    cu = _C[:, 0][:, None] * ux[None, :]
    return _W[:, None] * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * (ux * ux)[None, :])


def shear_drag_lift(L_dist, re, D=20.0, storage='f32', box=(48, 16, 8), u_w=0.1, block=1000,
                    window=5, rtol=1e-3, max_steps=200000, re_def='particle', log=None):
    """Drag and lift coefficients of the fixed sphere near the bottom wall.

    re_def 'shear': re = G D^2 / nu; 'particle': re = G L D^2 / nu, the
    Reynolds number of the undisturbed velocity G L D at the sphere centre
    (the two agree at L = 1). Runs blocks of `block` steps until C_D and C_L
    each changed by less than `rtol` (relative) over the last `window`
    blocks, or max_steps."""
    nx, ny, nz = int(box[0] * D), int(box[1] * D), int(box[2] * D)
    H = float(nz)
    G = u_w / H
    nu = G * D * D * (L_dist if re_def == 'particle' else 1.0) / re
    tau = 3.0 * nu + 0.5
    r, d = L.lbm_default_params()
    r.tau = tau
    d.fixed_particles = L.MOTION_FIXED
    wall_hi = [[0.0] * 3 for _ in range(3)]
    wall_hi[2] = [u_w, 0.0, 0.0]
    grid = L.make_grid((nx, ny, nz), (1, 1, 0), wall_vel_hi=wall_hi)
    ctx = L.lbm_create(grid, r, (0.0, 0.0, 0.0), d, storage, max_particles=1)
    # linear shear profile at the cell centres (halfway walls at z = 0 and H)
    z = np.arange(nz) + 0.5
    feq = equilibrium_planes(u_w * z / H)
    f = np.empty((19, nz, ny, nx))
    for q in range(19):
        f[q] = feq[q][:, None, None]
    L.lbm_set_pdfs(ctx, f.reshape(19, -1))
    del f
    pos = np.array([[box[0] / 2.0 * D, box[1] / 2.0 * D, L_dist * D]])
    L.lbm_add_spheres(ctx, pos, np.zeros((1, 3)), np.zeros((1, 3)), np.array([D / 2.0]), np.array([1.0]))
    norm = math.pi / 8.0 * G * G * L_dist * L_dist * D ** 4
    hist = []
    steps = 0
    t0 = time.time()
    while steps < max_steps:
        L.lbm_step(ctx, block)
        steps += block
        F = L.lbm_get_particle_state(ctx)['force_hyd'][0]
        hist.append((F[0] / norm, F[2] / norm))
        if log:
            log('step %d: C_D %.4f C_L %.4f' % (steps, hist[-1][0], hist[-1][1]))
        if len(hist) > window:
            a, b = np.array(hist[-window - 1]), np.array(hist[-1])
            if np.all(np.abs(b - a) <= rtol * np.abs(b)):
                break
    wall = time.time() - t0
    cells = nx * ny * nz
    del ctx
    cd, cl = hist[-1]
    paper = PAPER_SHEAR.get((int(re), float(L_dist)))
    out = dict(case='shear drag/lift', Re=re, re_def=re_def, Re_s=round(G * D * D / nu, 4), L=L_dist, D=D,
               shape=[nx, ny, nz], tau=tau, storage=storage,
               steps=steps, converged=steps < max_steps, C_D=round(cd, 4), C_L=round(cl, 4),
               mlups=round(cells * steps / wall / 1e6, 1))
    if paper:
        out['paper_sim'] = dict(C_D=paper['sim'][0], C_L=paper['sim'][1])
        out['paper_ref'] = dict(C_D=paper['ref'][0], C_L=paper['ref'][1])
        out['rel_dev_from_paper_sim'] = dict(C_D=round(cd / paper['sim'][0] - 1, 4),
                                             C_L=round(cl / paper['sim'][1] - 1, 4))
    return out


# Lambda_b of the settling test of Sec. 2.3.3: (shell, bulk)
ACCEL_MODELS = {'TRT': (1.0, 1.0), 'TRT+B(10)': (10.0, 10.0), 'TRT+B(100)': (100.0, 100.0),
                'TRT+aB': (100.0, 1.0)}


def artificial_acceleration(model='TRT+aB', D=20.0, box=(4, 4, 8), u_s=0.02, re=164.0, ratio=8.34,
                            c_acc=10.0, storage='f32', t_ref_units=24.0, max_steps=None):
    """Sphere with the prescribed settling velocity of Sec. 2.3.3 and a
    density probe moving with it at x_p + (D, 0, 0), sampled every step.
    Reports the probe's relative density fluctuation over the second half of
    the run and the share of its power spectrum in three frequency bands."""
    nx, ny, nz = int(box[0] * D), int(box[1] * D), int(box[2] * D)
    nu = u_s * D / re
    r, d = L.lbm_default_params()
    r.tau = 3.0 * nu + 0.5
    r.lambda_b_shell, r.lambda_b_bulk = ACCEL_MODELS[model]
    d.fixed_particles = L.MOTION_PRESCRIBED
    grid = L.make_grid((nx, ny, nz), (0, 0, 1))
    ctx = L.lbm_create(grid, r, (0.0, 0.0, 0.0), d, storage, max_particles=1)
    L.lbm_add_spheres(ctx, [[nx / 2.0, ny / 2.0, nz / 2.0]], np.zeros((1, 3)), np.zeros((1, 3)),
                      np.array([D / 2.0]), np.array([ratio]))
    t_st = ratio * D * D / (18.0 * nu)
    steps = int(t_ref_units * D / u_s) if max_steps is None else max_steps
    rho = np.empty(steps)
    x = np.array([nx / 2.0, ny / 2.0, nz / 2.0])
    t0 = time.time()
    for t in range(1, steps + 1):
        u = -u_s * (1.0 - math.exp(-c_acc * t / t_st))
        L.lbm_set_particle_velocity(ctx, np.array([[0.0, 0.0, u]]))
        L.lbm_step(ctx, 1)
        x[2] = (x[2] + u) % nz
        rho[t - 1] = L.lbm_sample_density(ctx, x + np.array([D, 0.0, 0.0]))[0]
    wall = time.time() - t0
    del ctx
    late = rho[steps // 2:]
    dev = late - late.mean()
    power = np.abs(np.fft.rfft(dev)) ** 2
    freq = np.fft.rfftfreq(len(dev))
    total = power[1:].sum()
    bands = {'low (< 1e-3 / step)': (0.0, 1e-3), 'mid (1e-3 - 1e-2)': (1e-3, 1e-2), 'high (> 1e-2)': (1e-2, 1.0)}
    share = {k: float(power[(freq > lo) & (freq <= hi)].sum() / total) for k, (lo, hi) in bands.items()}
    # fluctuation about the slow pressure signal of the moving sphere: the
    # deviation from a 1000-step running mean
    k = 1000
    slow = np.convolve(rho, np.ones(k) / k, mode='same')
    fast = (rho - slow)[steps // 2:steps - k // 2]
    return dict(case='artificial acceleration', model=model, D=D, shape=[nx, ny, nz], tau=r.tau, storage=storage,
                steps=steps, probe_rho_mean=float(late.mean()), probe_rel_fluctuation=float(dev.std() / late.mean()),
                probe_rel_fluctuation_fast=float(fast.std() / late.mean()),
                probe_rel_max=float(np.abs(dev).max() / late.mean()), spectrum_share=share,
                band_power={k: float(v * total) for k, v in share.items()}, wall_s=round(wall, 1))


# collision models of Sec. 2.4 as relaxation parameters: magic Lambda (None: (tau - 1/2)^2, which
# makes s- = s+, i.e. SRT), Lambda_b in the shell and in the bulk
STOKES_MODELS = {'SRT': (None, 1.0, 1.0), 'TRT': (3.0 / 16.0, 1.0, 1.0), 'TRT+B': (3.0 / 16.0, 100.0, 100.0),
                 'TRT+aB': (3.0 / 16.0, 100.0, 1.0)}
C_REF_STOKES = 2.842


def stokes_array(tau, model='TRT+aB', D=20.0, a=1e-8, storage='f64', block=500, rtol=1e-6, max_steps=400000):
    """Normalised drag C = (F_x + pi/6 D^3 a) / (3 pi mu D u_bar) of a fixed sphere in a periodic
    [2 x 2 x 2] D box driven by the body force a (Sec. 2.4), run until C changes by less than
    rtol over one block; the reference is C_ref = 2.842."""
    n = int(2 * D)
    magic, lb_shell, lb_bulk = STOKES_MODELS[model]
    r, d = L.lbm_default_params()
    r.tau = tau
    r.magic = (tau - 0.5) ** 2 if magic is None else magic
    r.lambda_b_shell, r.lambda_b_bulk = lb_shell, lb_bulk
    d.fixed_particles = L.MOTION_FIXED
    ctx = L.lbm_create(L.make_grid((n, n, n), (1, 1, 1)), r, (a, 0.0, 0.0), d, storage, max_particles=1)
    L.lbm_add_spheres(ctx, [[n / 2.0] * 3], np.zeros((1, 3)), np.zeros((1, 3)), np.array([D / 2.0]),
                      np.array([1.0]))
    nu = (tau - 0.5) / 3.0
    prev, steps, C = None, 0, float('nan')
    while steps < max_steps:
        L.lbm_step(ctx, block)
        steps += block
        F = L.lbm_get_particle_state(ctx)['force_hyd'][0, 0]
        _, u, _ = L.lbm_get_fields(ctx)
        u_bar = u[0].sum() / n ** 3
        C = (F + math.pi / 6.0 * D ** 3 * a) / (3.0 * math.pi * nu * D * u_bar)
        if prev is not None and abs(C - prev) <= rtol * abs(C):
            break
        prev = C
    del ctx
    return dict(case='stokes array', model=model, tau=tau, D=D, storage=storage, steps=steps,
                converged=steps < max_steps, C=round(C, 5), rel_err=round(C / C_REF_STOKES - 1, 5))


# Sec. 4.4, St = 27 (the experiments' fluid and sphere): Re, rho_f, mu_f, D_p, rho_p, box / D_p
SPHERE_WALL_ST27 = dict(Re=30.0, rho_f=965.0, mu_f=0.1, D_p=0.006, rho_p=7800.0, box=(12, 12, 48), e_dry=0.97)
# the paper's rebound heights for n_sub = 10 (ten runs, start perturbed by up to a cell): min, max, mean
PAPER_REBOUND_NSUB10 = (0.3269, 0.3276, 0.3274)


def sphere_wall_rebound(n_sub=10, D=20.0, dz=0.0, u_s=0.02, c_acc=10.0, storage='f32', setup=SPHERE_WALL_ST27,
                        max_steps=200000, log=None):
    """Rebound height H_r = max gap / D after the first contact of a sphere
    hitting the bottom wall of a closed box (Sec. 4.4): its settling velocity
    is prescribed by the artificial acceleration until the gap is below one
    diameter, then it moves freely under gravity and buoyancy (DEM). Lattice
    units from D cells per diameter and u_s; gravity from 9.81 m/s^2 with the
    time step that matches the fluid's viscosity."""
    nx, ny, nz = (int(b * D) for b in setup['box'])
    nu = u_s * D / setup['Re']
    dx = setup['D_p'] / D
    dt = nu * dx * dx / (setup['mu_f'] / setup['rho_f'])
    g = 9.81 * dt * dt / dx
    ratio = setup['rho_p'] / setup['rho_f']
    r, d = L.lbm_default_params()
    r.tau = 3.0 * nu + 0.5
    d.fixed_particles = L.MOTION_PRESCRIBED
    d.n_sub = int(n_sub)
    d.e_dry = setup['e_dry']
    d.gravity[2] = -g
    grid = L.make_grid((nx, ny, nz), (0, 0, 0))
    ctx = L.lbm_create(grid, r, (0.0, 0.0, 0.0), d, storage, max_particles=1)
    R = D / 2.0
    z0 = nz - 1.5 * D + dz
    L.lbm_add_spheres(ctx, [[nx / 2.0, ny / 2.0, z0]], np.zeros((1, 3)), np.zeros((1, 3)), np.array([R]),
                      np.array([ratio]))
    t_st = ratio * D * D / (18.0 * nu)
    t0 = time.time()
    step, z = 0, z0
    while z - R >= D and step < max_steps:   # prescribed approach until the gap is below D
        step += 1
        L.lbm_set_particle_velocity(ctx, np.array([[0.0, 0.0, -u_s * (1.0 - math.exp(-c_acc * step / t_st))]]))
        L.lbm_step(ctx, 1)
        z = L.lbm_get_particle_state(ctx)['pos'][0, 2]
    release = step
    L.lbm_set_motion(ctx, L.MOTION_DEM)
    contact, h_max, falling = None, -1.0, 0
    while step < max_steps:
        L.lbm_step(ctx, 1)
        step += 1
        gap = (L.lbm_get_particle_state(ctx)['pos'][0, 2] - R) / D
        if contact is None:
            if gap <= 0.0:
                contact = step
            continue
        if gap > h_max:
            h_max, falling = gap, 0
        elif h_max > 0.0:
            falling += 1
            if falling > 200:   # well past the apex of the rebound
                break
        if log and step % 1000 == 0:
            log('step %d: gap/D %.4f, H_r so far %.4f' % (step, gap, h_max))
    wall = time.time() - t0
    del ctx
    mn, mx, mean = PAPER_REBOUND_NSUB10
    return dict(case='sphere-wall rebound', St=round(ratio * setup['Re'] / 9.0, 1), n_sub=n_sub, D=D, dz=dz,
                shape=[nx, ny, nz], tau=r.tau, g=g, storage=storage, release_step=release, contact_step=contact,
                steps=step, H_r=round(h_max, 4),
                paper_n_sub10=dict(min=mn, max=mx, mean=mean), wall_s=round(wall, 1))


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split('\n')[0])
    sub = ap.add_subparsers(dest='case', required=True)
    a = sub.add_parser('shear')
    a.add_argument('--re', type=float, nargs='+', default=[1.0])
    a.add_argument('--L', type=float, nargs='+', default=[0.505, 1.0])
    a.add_argument('--D', type=float, default=20.0)
    a.add_argument('--storage', default='f32')
    a.add_argument('--max-steps', type=int, default=200000)
    a.add_argument('--block', type=int, default=1000)
    a.add_argument('--re-def', choices=('particle', 'shear'), default='particle')
    a.add_argument('--verbose', action='store_true')
    c = sub.add_parser('rebound')
    c.add_argument('--n-sub', type=int, nargs='+', default=[10])
    c.add_argument('--dz', type=float, nargs='+', default=[0.0])
    c.add_argument('--D', type=float, default=20.0)
    c.add_argument('--storage', default='f32')
    c.add_argument('--verbose', action='store_true')
    d = sub.add_parser('stokes')
    d.add_argument('--tau', type=float, nargs='+', default=[0.55, 0.6, 0.7, 0.8, 0.9, 1.0, 1.5])
    d.add_argument('--model', nargs='+', default=list(STOKES_MODELS))
    d.add_argument('--storage', default='f64')
    b = sub.add_parser('acceleration')
    b.add_argument('--model', nargs='+', default=list(ACCEL_MODELS))
    b.add_argument('--D', type=float, default=20.0)
    b.add_argument('--storage', default='f32')
    b.add_argument('--max-steps', type=int, default=None)
    args = ap.parse_args(argv)
    if args.case == 'shear':
        for re in args.re:
            for Ld in args.L:
                res = shear_drag_lift(Ld, re, D=args.D, storage=args.storage, max_steps=args.max_steps,
                                      block=args.block, re_def=args.re_def, log=print if args.verbose else None)
                print(json.dumps(res), flush=True)
    elif args.case == 'stokes':
        for m in args.model:
            for tau in args.tau:
                print(json.dumps(stokes_array(tau, m, storage=args.storage)), flush=True)
    elif args.case == 'rebound':
        for n in args.n_sub:
            for dz in args.dz:
                print(json.dumps(sphere_wall_rebound(n_sub=n, D=args.D, dz=dz, storage=args.storage,
                                                     log=print if args.verbose else None)), flush=True)
    else:
        for m in args.model:
            print(json.dumps(artificial_acceleration(m, D=args.D, storage=args.storage, max_steps=args.max_steps)),
                  flush=True)


if __name__ == '__main__':
    main()
