"""Complete four-way coupled time step of the oracle (Sec. 4.2, Algorithm 1).

Test infrastructure only (see ``oracle/__init__.py``).

One call of :meth:`Simulation.step` advances t -> t+1:
  1. boundary conditions + pull streaming + per-link momentum exchange
     (Eqs. (2), (14)-(17)), plus the missing-link correction (Sec. 2.2);
  2. averaging of F^fp, T^fp over the current and the previous step
     (Sec. 4.2);
  3. TRT+aB collision (Eq. (5) with S of Eq. (12); Lambda_b inside the shell
     of Sec. 2.3.2, Lambda_b,bulk elsewhere);
  4. n_sub DEM subcycles with dt_p = 1/n_sub (Algorithm 1, inner loop):
     Velocity-Verlet position update (Eq. (37)), lubrication (Eqs. (25)-(33)),
     contact (Eqs. (39)-(50)), external force V (rho_p - rho_f) g
     (Sec. 4.1.1), Velocity-Verlet velocity update (Eq. (38));
  5. mapping update and refill (Sec. 2.2, Eq. (18)).
Readings where the paper is silent:
  * first step: F^fp(t-1) := F^fp(0); the force F(t) that the first
    Velocity-Verlet position update needs is the lubrication + contact +
    external force at the initial state (no history update).
  * particle mass from the analytic volume, m = rho_p pi D^3 / 6.
  * fluid_counterforce: in periodic sedimentation the fluid gets the uniform
    body force -sum_i V_i (rho_p,i - rho_f) g / N_fluid (N_fluid = fluid
    cell count of the current mapping) so that no net momentum is injected.
  * positions are wrapped into [0, L) on periodic axes after each
    position update.
  * prescribed motion (Sec. 2.3.3 sets a sphere's velocity every step): the
    velocity set before a step is the boundary velocity of that step, the
    position advances by it over the step, the refill uses it; switching to
    the DEM later evaluates the first Velocity-Verlet force at the current
    state with the current averaged fluid force.
"""
import math

import numpy as np

from .d3q19 import (Q, RHO0, relaxation_rates, s_minus_from_magic, s_b_from_lambda_b,
                    viscosity)
from .lbm import collide, equilibrium, density, velocity_from_post_collision
from .coupling import stream_and_couple, missing_links, refill
from .particles import (map_cells, cell_centres, rel_vec, lubrication_on_i, lubrication_min_gap,
                        contact_coefficients, collision_time, contact_force)


class Domain:
    """Box of nx x ny x nz cells (Sec. 4.2); cell (i, j, k) has its centre at
    (i+1/2, j+1/2, k+1/2).

    An axis is either periodic or bounded by two no-slip walls on its faces.
    wall_vel[side][axis] is the velocity of the wall at the low (side 0) or
    high (side 1) face of that axis.
    """

    def __init__(self, nx, ny, nz, periodic=(True, True, True), wall_vel_lo=None, wall_vel_hi=None):
        self.shape = (int(nx), int(ny), int(nz))
        self.periodic = tuple(bool(p) for p in periodic)
        lo = np.zeros((3, 3)) if wall_vel_lo is None else np.asarray(wall_vel_lo, dtype=np.float64)
        hi = np.zeros((3, 3)) if wall_vel_hi is None else np.asarray(wall_vel_hi, dtype=np.float64)
        self.wall_vel = (lo, hi)


class Params:
    """Method parameters with the paper's defaults.

    tau = 1/s_nu; magic Lambda = 3/16 (Eq. (11)); Lambda_b = 100 in the shell
    and 1 elsewhere with shell width 2 (Sec. 2.3.2); lubrication cut-offs
    2/3, 1/2, 1/2 (Eq. (34)); minimum gap (0.001 + 0.00007 R) R (Eq. (56));
    T_c <= 0 selects Eq. (55); n_sub = 10 (Sec. 4.4).
    """

    def __init__(self, tau, magic=3.0 / 16.0, lambda_b_shell=100.0, lambda_b_bulk=1.0,
                 shell_width=2.0, body_force=(0.0, 0.0, 0.0), e_dry=0.97, Tc=0.0, nu_p=0.23,
                 mu_p=0.15, n_sub=10, lub_cut_n=2.0 / 3.0, lub_cut_tt=0.5, lub_cut_tr=0.5,
                 lub_min_a=0.001, lub_min_b=0.00007, gravity=(0.0, 0.0, 0.0), lubrication=True,
                 tangential_lubrication=True, force_averaging=True, fluid_counterforce=False,
                 fixed_particles=False, missing_links=True, prescribed_motion=False):
        self.tau = tau
        self.magic = magic
        self.lambda_b_shell = lambda_b_shell
        self.lambda_b_bulk = lambda_b_bulk
        self.shell_width = shell_width
        self.body_force = np.asarray(body_force, dtype=np.float64)
        self.e_dry, self.Tc, self.nu_p, self.mu_p, self.n_sub = e_dry, Tc, nu_p, mu_p, n_sub
        self.lub_cut_n, self.lub_cut_tt, self.lub_cut_tr = lub_cut_n, lub_cut_tt, lub_cut_tr
        self.lub_min_a, self.lub_min_b = lub_min_a, lub_min_b
        self.gravity = np.asarray(gravity, dtype=np.float64)
        self.lubrication = lubrication
        self.tangential_lubrication = tangential_lubrication
        self.force_averaging = force_averaging
        self.fluid_counterforce = fluid_counterforce
        self.fixed_particles = fixed_particles
        self.missing_links = missing_links
        # prescribed motion (Sec. 2.3.3 prescribes a sphere's velocity per
        # step): positions advance by the velocities the caller sets, no DEM
        self.prescribed_motion = prescribed_motion

    def rates(self):
        """Relaxation rates (bulk cells, shell cells) as two S diagonals (Eq. (12))."""
        s_nu = 1.0 / self.tau
        s_m = s_minus_from_magic(s_nu, self.magic)
        s_bulk = relaxation_rates('trtb', s_nu, s_m, s_b_from_lambda_b(s_nu, self.lambda_b_bulk))
        s_shell = relaxation_rates('trtb', s_nu, s_m, s_b_from_lambda_b(s_nu, self.lambda_b_shell))
        return s_bulk, s_shell


class Simulation:
    """Plain float64 restatement of Algorithm 1 on a small box."""

    def __init__(self, dom, params):
        self.dom = dom
        self.p = params
        nx, ny, nz = dom.shape
        self.ft = equilibrium(np.ones((nz, ny, nx)), np.zeros((3, nz, ny, nx)))
        self.owner = np.full((nz, ny, nx), -1, dtype=np.int64)
        self.shell = np.zeros((nz, ny, nx), dtype=bool)
        self.X = np.zeros((0, 3))
        self.U = np.zeros((0, 3))
        self.Om = np.zeros((0, 3))
        self.R = np.zeros(0)
        self.rho_p = np.zeros(0)
        self.hist = {}
        self.F_prev = None
        self.T_prev = None
        self.Ffp_old = None
        self.Tfp_old = None
        self.Ffp = np.zeros((0, 3))
        self.Tfp = np.zeros((0, 3))
        self.Fbar = np.zeros((0, 3))
        self.Tbar = np.zeros((0, 3))
        self.accel = self.p.body_force.copy()
        self.t = 0
        self.refilled = []

    # ------------------------------------------------------------------ setup
    def add_spheres(self, X, U, Om, R, rho_p):
        """Add spheres (centre, velocity, angular velocity, radius, density
        ratio rho_p / rho_f) and map them onto the cells (Sec. 2.2)."""
        self.X = np.vstack([self.X, np.asarray(X, dtype=np.float64).reshape(-1, 3)])
        self.U = np.vstack([self.U, np.asarray(U, dtype=np.float64).reshape(-1, 3)])
        self.Om = np.vstack([self.Om, np.asarray(Om, dtype=np.float64).reshape(-1, 3)])
        self.R = np.concatenate([self.R, np.asarray(R, dtype=np.float64).reshape(-1)])
        self.rho_p = np.concatenate([self.rho_p, np.asarray(rho_p, dtype=np.float64).reshape(-1)])
        self.remap()

    def remap(self):
        """Solid cells, owners and the TRT+aB shell from the current positions
        (Sec. 2.2, Sec. 2.3.2)."""
        self.owner, self.shell = map_cells(cell_centres(self.dom), self.X, self.R, self.dom,
                                           self.p.shell_width)

    def set_pdfs(self, ft):
        """Replace the post-collision PDFs f~ of Eq. (1), shape (19, nz, ny, nx)."""
        self.ft = np.array(ft, dtype=np.float64)

    @property
    def volume(self):
        """Analytic sphere volume pi D^3 / 6 (a reading: the paper gives no
        other volume for the particle mass)."""
        return math.pi * (2.0 * self.R) ** 3 / 6.0

    @property
    def mass(self):
        """m = rho_p V (Sec. 4.1)."""
        return self.rho_p * self.volume

    @property
    def inertia(self):
        """Moment of inertia of a solid sphere, 2/5 m R^2 (Sec. 4.1)."""
        return 0.4 * self.mass * self.R * self.R

    # ---------------------------------------------------------------- DEM
    def external_force(self):
        """Gravity and buoyancy V (rho_p - rho_f) g with rho_f = rho0 (Sec. 4.1.1)."""
        return (self.volume * (self.rho_p - RHO0))[:, None] * self.p.gravity[None, :]

    def dem_forces(self, Fbar, Tbar, dt_p, update_history):
        """Total force and torque on every particle at the current state
        (Algorithm 1, inner loop): lubrication (Eqs. (25)-(34), (56)), contact
        (Eqs. (39)-(52)), the averaged fluid force and torque (Sec. 4.2) and
        V (rho_p - rho_f) g (Sec. 4.1.1)."""
        p, dom = self.p, self.dom
        X, U, Om, R, m = self.X, self.U, self.Om, self.R, self.mass
        N = len(R)
        F = Fbar + self.external_force()
        T = Tbar.copy()
        mu = RHO0 * viscosity(1.0 / p.tau)
        cut_max = max(p.lub_cut_n, p.lub_cut_tt, p.lub_cut_tr)
        seen = set()
        for i, j in self._close_pairs(cut_max):
            d = rel_vec(X[i], X[j], dom)
            dist = math.sqrt(d @ d)
            delta = dist - (R[i] + R[j])
            key = (i, j)
            if delta >= cut_max and delta >= 0.0:
                continue
            n = d / dist
            u_ij = U[i] - U[j]
            if p.lubrication:
                dmin = lubrication_min_gap(0.5 * (R[i] + R[j]), p.lub_min_a, p.lub_min_b)
                Fi, Ti = lubrication_on_i(R[i], R[j], delta, n, u_ij, Om[i], Om[j], mu,
                                          p.lub_cut_n, p.lub_cut_tt, p.lub_cut_tr, dmin,
                                          p.tangential_lubrication)
                Fj, Tj = lubrication_on_i(R[j], R[i], delta, -n, -u_ij, Om[j], Om[i], mu,
                                          p.lub_cut_n, p.lub_cut_tt, p.lub_cut_tr, dmin,
                                          p.tangential_lubrication)
                F[i] += Fi
                T[i] += Ti
                F[j] += Fj
                T[j] += Tj
            if delta < 0.0:
                ri = -0.5 * d
                rj = 0.5 * d
                u_cp = (U[i] + np.cross(Om[i], ri)) - (U[j] + np.cross(Om[j], rj))
                m_eff = m[i] * m[j] / (m[i] + m[j])
                Tc = collision_time(R[i] + R[j], p.Tc)
                kn, dn, kt, dt_ = contact_coefficients(m_eff, p.e_dry, Tc, p.nu_p)
                old = self.hist.get(key, np.zeros(3))
                Fn, Ft, new = contact_force(n, delta, u_cp, u_ij, kn, dn, kt, dt_, p.mu_p, old,
                                            dt_p)
                F[i] += Fn + Ft
                F[j] -= Fn + Ft
                T[i] += np.cross(ri, Ft)
                T[j] += np.cross(rj, -Ft)
                if update_history:
                    self.hist[key] = new
                seen.add(key)
        for a in range(3):
            if dom.periodic[a]:
                continue
            for side in (0, 1):
                n_w = np.zeros(3)
                n_w[a] = 1.0 if side == 0 else -1.0
                x_w = 0.0 if side == 0 else float(dom.shape[a])
                u_w = dom.wall_vel[side][a]
                for i in range(N):
                    delta = (X[i, a] - x_w) * n_w[a] - R[i]
                    key = (i, 'wall', a, side)
                    u_ij = U[i] - u_w
                    if p.lubrication:
                        dmin = lubrication_min_gap(R[i], p.lub_min_a, p.lub_min_b)
                        Fi, Ti = lubrication_on_i(R[i], None, delta, n_w, u_ij, Om[i], np.zeros(3),
                                                  mu, p.lub_cut_n, p.lub_cut_tt, p.lub_cut_tr,
                                                  dmin, p.tangential_lubrication)
                        F[i] += Fi
                        T[i] += Ti
                    if delta < 0.0:
                        ri = -(R[i] + 0.5 * delta) * n_w
                        u_cp = (U[i] + np.cross(Om[i], ri)) - u_w
                        Tc = collision_time(2.0 * R[i], p.Tc)
                        kn, dn, kt, dt_ = contact_coefficients(m[i], p.e_dry, Tc, p.nu_p)
                        old = self.hist.get(key, np.zeros(3))
                        Fn, Ft, new = contact_force(n_w, delta, u_cp, u_ij, kn, dn, kt, dt_,
                                                    p.mu_p, old, dt_p)
                        F[i] += Fn + Ft
                        T[i] += np.cross(ri, Ft)
                        if update_history:
                            self.hist[key] = new
                        seen.add(key)
        if update_history:
            self.hist = {k: v for k, v in self.hist.items() if k in seen}
        return F, T

    def _close_pairs(self, cut_max):
        """Pairs i < j whose surface gap may be below cut_max (a superset: the
        exact test is repeated per pair), found with one vectorised distance
        matrix so that far pairs, which add nothing, are not visited."""
        X, R, dom = self.X, self.R, self.dom
        N = len(R)
        if N < 2:
            return []
        d = X[:, None, :] - X[None, :, :]
        for a in range(3):
            if dom.periodic[a]:
                L = float(dom.shape[a])
                d[..., a] = np.where(d[..., a] > 0.5 * L, d[..., a] - L, d[..., a])
                d[..., a] = np.where(d[..., a] < -0.5 * L, d[..., a] + L, d[..., a])
        gap = np.sqrt((d * d).sum(-1)) - (R[:, None] + R[None, :])
        ii, jj = np.nonzero(np.triu(gap < cut_max + 1e-6, k=1))
        return list(zip(ii.tolist(), jj.tolist()))

    def wrap_positions(self):
        """Positions back into [0, L) on periodic axes after an update (reading
        of the periodic boxes of Sec. 4.2)."""
        for a in range(3):
            if self.dom.periodic[a]:
                L = float(self.dom.shape[a])
                x = self.X[:, a]
                x = np.where(x >= L, x - L, x)
                x = np.where(x < 0.0, x + L, x)
                self.X[:, a] = x

    def dem_subcycles(self, Fbar, Tbar):
        """Inner loop of Algorithm 1 with Velocity Verlet, Eqs. (37)-(38)."""
        n_sub = self.p.n_sub
        dt = 1.0 / n_sub
        m = self.mass[:, None]
        I = self.inertia[:, None]
        for _ in range(n_sub):
            self.X = self.X + dt * self.U + (dt * dt / (2.0 * m)) * self.F_prev
            self.wrap_positions()
            Fn, Tn = self.dem_forces(Fbar, Tbar, dt, update_history=True)
            self.U = self.U + (dt / (2.0 * m)) * (self.F_prev + Fn)
            self.Om = self.Om + (dt / (2.0 * I)) * (self.T_prev + Tn)
            self.F_prev, self.T_prev = Fn, Tn

    # --------------------------------------------------------------- step
    def fluid_accel(self):
        """Fluid body force of the step: the given a, minus the particles'
        V (rho_p - rho_f) g spread over the fluid cells when the counterforce
        reading is on (periodic sedimentation)."""
        a = self.p.body_force.copy()
        if self.p.fluid_counterforce and len(self.R):
            n_fluid = int((self.owner < 0).sum())
            a = a - self.external_force().sum(axis=0) / (RHO0 * n_fluid)
        return a

    def set_motion(self, dem=False, fixed=False, prescribed=False):
        """Switch how particles move from the next step on. Switching to the
        DEM after the first step evaluates the force of the first Velocity-
        Verlet position update at the current state, with the current
        averaged fluid force (at t = 0 that force is zero)."""
        if dem and (self.p.fixed_particles or self.p.prescribed_motion) and self.t > 0:
            self.F_prev = None
        self.p.fixed_particles, self.p.prescribed_motion = fixed, prescribed

    def step(self, n=1):
        """n time steps of Algorithm 1 (Sec. 4.2)."""
        for _ in range(n):
            self._step()

    def _step(self):
        """One time step of Algorithm 1 in the order of the module doc."""
        p, dom = self.p, self.dom
        N = len(self.R)
        if self.F_prev is None and N and not p.fixed_particles and not p.prescribed_motion:
            Fb = self.Fbar if self.t > 0 else np.zeros((N, 3))
            Tb = self.Tbar if self.t > 0 else np.zeros((N, 3))
            self.F_prev, self.T_prev = self.dem_forces(Fb, Tb, 0.0, update_history=False)
        self.accel = self.fluid_accel()
        # Algorithm 1, lines 1-2: boundary conditions, interaction force
        f, Ffp, Tfp = stream_and_couple(self.ft, dom, self.owner, self.X, self.U, self.Om, self.R)
        if p.missing_links and N:
            Fm, Tm = missing_links(dom, self.owner, self.X, self.R)
            Ffp = Ffp + Fm
            Tfp = Tfp + Tm
        if self.Ffp_old is None:
            self.Ffp_old, self.Tfp_old = Ffp, Tfp
        if p.force_averaging:
            Fbar, Tbar = 0.5 * (Ffp + self.Ffp_old), 0.5 * (Tfp + self.Tfp_old)
        else:
            Fbar, Tbar = Ffp, Tfp
        self.Ffp_old, self.Tfp_old = Ffp, Tfp
        self.Ffp, self.Tfp, self.Fbar, self.Tbar = Ffp, Tfp, Fbar, Tbar
        # Algorithm 1, line 3: collision of the streamed PDFs in fluid cells
        fluid = self.owner < 0
        s_bulk, s_shell = p.rates()
        ft = self.ft.copy()
        ft[:, fluid] = collide(f[:, fluid], self.accel, s_bulk, s_shell, self.shell[fluid])
        self.ft = ft
        # Algorithm 1, lines 4-10: DEM subcycles; prescribed motion instead
        # moves each particle by its velocity over the step (Eq. (37), no force)
        if N and p.prescribed_motion:
            self.X = self.X + self.U
            self.wrap_positions()
        elif N and not p.fixed_particles:
            self.dem_subcycles(Fbar, Tbar)
        # Algorithm 1, line 11: mapping update and refill
        self.refilled = []
        if N:
            owner_old = self.owner
            self.remap()
            self.refilled = refill(self.ft, dom, owner_old, self.owner, self.X, self.U, self.Om,
                                   1.0 / p.tau, self.accel)
        self.t += 1

    # ------------------------------------------------------------- output
    def fields(self):
        """(rho, u) per cell (Eq. (2)) from the stored post-collision PDFs; zero in solid cells."""
        fluid = self.owner < 0
        rho = np.where(fluid, density(self.ft), 0.0)
        u = np.where(fluid[None], velocity_from_post_collision(self.ft, self.accel), 0.0)
        return rho, u
