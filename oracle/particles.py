"""Particle geometry, mapping, lubrication and contact laws of the oracle.

Test infrastructure only (see ``oracle/__init__.py``).

Paper passages followed:
  * Sec. 2.2: explicit mapping (a cell is solid iff its centre lies inside a
    particle); delta_q of Eq. (14) is the normalised distance from the cell
    centre to the surface along the link.
  * Sec. 2.3.2: TRT+aB shell of thickness delta_aB around each particle.
  * Sec. 3.1, Eqs. (25)-(33): lubrication correction, with cut-offs Eq. (34)
    and minimum gap Eq. (56).
  * Sec. 4.1.2, Eqs. (39)-(52): linear spring-dashpot contact with Coulomb
    limited tangential spring.
  * App. B, Eqs. (B.1)-(B.8): particle and pair definitions.
Readings where the paper is silent or ambiguous:
  * Eq. (B.1) is printed as u + (x - x_p) x omega, which is the rigid-body
    velocity with the wrong sign; the oracle uses u + omega x (x - x_p).
  * cell centres are at index + 1/2; the inside test is
    ((dx*dx + dy*dy) + dz*dz) <= R*R in float64 (ties count as inside),
    with minimum-image dx on periodic axes; on overlap the lowest particle
    index owns the cell; the shell holds fluid cells with
    R^2 < d^2 <= (R + delta_aB)^2.
  * the lubrication step function uses the actual gap, lambda = 1 iff
    0 < delta_ij,n < delta_cut; the capped gap of Eq. (28) is used inside the
    formulas; the torque sum of Eq. (26) is read as acting on particle i.
  * for two spheres the minimum gap of Eq. (56) uses the mean radius.
  * contact point: midpoint of the centres (App. B) for two spheres,
    x_i - (R_i + delta/2) n_w for a wall.
"""
import math

import numpy as np

CS = 1.0 / math.sqrt(3.0)


# --------------------------------------------------------------------------
# geometry
# --------------------------------------------------------------------------

def min_image(d, length, periodic):
    """Minimum-image wrap of a coordinate difference along one axis (periodic
    boxes of Sec. 4.2; the nearest image is the one the mapping and the pair
    laws see).

    Works elementwise on arrays. Uses one conditional shift by the box length
    (exact in float64 for |d| < 1.5 L).
    """
    if not periodic:
        return d
    half = 0.5 * length
    d = np.where(d > half, d - length, d)
    d = np.where(d < -half, d + length, d)
    return d


def rel_vec(x, xp, dom):
    """x - xp with minimum image on periodic axes (Sec. 2.2 mapping and the
    pair laws of Secs. 3.1, 4.1). x, xp: (..., 3), broadcast."""
    x = np.asarray(x, dtype=np.float64)
    xp = np.asarray(xp, dtype=np.float64)
    out = np.empty(np.broadcast(x, xp).shape, dtype=np.float64)
    for a in range(3):
        out[..., a] = min_image(x[..., a] - xp[..., a], dom.shape[a], dom.periodic[a])
    return out


def dist2(x, xp, dom):
    """Squared distance in the fixed summation order ((dx dx + dy dy) + dz dz),
    the inside test of the mapping (Sec. 2.2, reading of the cell centre)."""
    r = rel_vec(x, xp, dom)
    return (r[..., 0] * r[..., 0] + r[..., 1] * r[..., 1]) + r[..., 2] * r[..., 2]


def cell_centres(dom):
    """Centres of all cells (Sec. 2.2 maps a cell by its centre), shape
    (nz, ny, nx, 3), centre of cell i is i + 1/2."""
    nx, ny, nz = dom.shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing='ij')
    return np.stack([x + 0.5, y + 0.5, z + 0.5], axis=-1).astype(np.float64)


def map_cells(centres, X, R, dom, shell_width):
    """Explicit mapping of Sec. 2.2 plus the TRT+aB shell of Sec. 2.3.2.

    centres: (..., 3) cell centres (any subset of cells). Returns
    (owner int64 (-1 = fluid), shell bool). Brute force over all particles.
    """
    owner = np.full(centres.shape[:-1], -1, dtype=np.int64)
    shell = np.zeros(centres.shape[:-1], dtype=bool)
    for i in range(len(R)):
        d2 = dist2(centres, X[i], dom)
        r2 = R[i] * R[i]
        rs = R[i] + shell_width
        rs2 = rs * rs
        inside = d2 <= r2
        owner = np.where(inside & (owner < 0), i, owner)
        shell |= (d2 > r2) & (d2 <= rs2)
    shell &= owner < 0
    return owner, shell


def link_fraction(x, c, xp, radius, dom):
    """delta_q of Eq. (14): smallest t in [0, 1] with |x + t c - x_p| = R.

    x: (..., 3) cell centres outside the sphere, c: (3,) lattice direction.
    """
    r = rel_vec(x, xp, dom)
    cf = np.asarray(c, dtype=np.float64)
    a = float(cf @ cf)
    b = 2.0 * (r @ cf)
    cc = (r * r).sum(axis=-1) - np.asarray(radius) * np.asarray(radius)
    disc = b * b - 4.0 * a * cc
    t = (-b - np.sqrt(np.maximum(disc, 0.0))) / (2.0 * a)
    t = np.where(disc < 0.0, 0.5, t)
    return np.clip(t, 0.0, 1.0)


def rigid_velocity(u, omega, r):
    """Velocity of a rigid body at offset r from its centre, u + omega x r.

    This is Eq. (B.1) with the sign order of the cross product corrected.
    """
    return u + np.cross(omega, r)


# --------------------------------------------------------------------------
# lubrication correction, Sec. 3.1
# --------------------------------------------------------------------------

def lubrication_min_gap(radius, a=0.001, b=0.00007):
    """Eq. (56): delta_min = (0.001 + 0.00007 R) R."""
    return (a + b * radius) * radius


def lubrication_on_i(Ri, Rj, delta_n, n, u_ij, om_i, om_j, mu, cut_n, cut_tt, cut_tr,
                     delta_min, tangential=True):
    """Lubrication force and torque on particle i due to j, Eqs. (27)-(33).

    Rj = None means a plane wall (the kappa -> infinity limits stated at the
    end of Sec. 3.1). n points from j (or the wall) to i. u_ij = u_i - u_j.
    Returns (F, T) as float64 3-vectors.
    """
    F = np.zeros(3)
    T = np.zeros(3)
    dl = max(delta_n, delta_min)                                       # Eq. (28)
    u_n = (u_ij @ n) * n
    u_t = u_ij - u_n
    if Rj is None:
        c_n, c_ftt, c_ttt, c_ftr, c_ttr = 1.0, 8.0 / 15.0, 1.0 / 10.0, 2.0 / 15.0, 2.0 / 5.0
        om_sum = om_i                                  # wall: omega_j = 0
        om_ftr = om_i
        om_ttr = om_i
    else:
        k = Rj / Ri
        c_n = k * k / ((1.0 + k) ** 2)
        c_ftt = 4.0 * k * (2.0 + k + 2.0 * k * k) / (15.0 * (1.0 + k) ** 3)
        c_ttt = k * (4.0 + k) / (10.0 * (1.0 + k) ** 2)
        c_ftr = 2.0 * k * k / (15.0 * (1.0 + k) ** 2)
        c_ttr = 2.0 * k / (5.0 * (1.0 + k))
        om_sum = om_i + om_j
        om_ftr = om_sum + (4.0 / k) * om_i + 4.0 * k * om_j
        om_ttr = om_i + (k / 4.0) * om_j
    # Eq. (29) step function on the actual gap.
    if 0.0 < delta_n < cut_n:
        F += -6.0 * math.pi * mu * Ri * Ri * c_n * (1.0 / dl - 1.0 / cut_n) * u_n     # Eq. (27)
    if tangential and 0.0 < delta_n < cut_tt:
        lg = math.log(dl / cut_tt)
        F += 6.0 * math.pi * mu * Ri * c_ftt * lg * u_t                                  # Eq. (30)
        T += 8.0 * math.pi * mu * Ri * Ri * c_ttt * lg * np.cross(u_ij, n)               # Eq. (31)
    if tangential and 0.0 < delta_n < cut_tr:
        lg = math.log(dl / cut_tr)
        F += -6.0 * math.pi * mu * Ri * Ri * c_ftr * lg * np.cross(om_ftr, n)            # Eq. (32)
        T += 8.0 * math.pi * mu * Ri ** 3 * c_ttr * lg * (om_ttr - (om_ttr @ n) * n)     # Eq. (33)
    return F, T


# --------------------------------------------------------------------------
# contact model, Sec. 4.1.2
# --------------------------------------------------------------------------

def contact_coefficients(m_eff, e_dry, Tc, nu_p):
    """Eq. (43) for k_n, d_n and Eqs. (51)-(52) for k_t, d_t."""
    le = math.log(e_dry)
    k_n = m_eff * (math.pi ** 2 + le * le) / (Tc * Tc)
    d_n = -2.0 * m_eff * le / Tc
    kappa = 2.0 * (1.0 - nu_p) / (2.0 - nu_p)
    return k_n, d_n, kappa * k_n, math.sqrt(kappa) * d_n


def collision_time(diameter, Tc):
    """Eq. (55) T_c = 2.31 D / c_s when no explicit T_c > 0 is given."""
    return Tc if Tc > 0.0 else 2.31 * diameter / CS


def contact_force(n, delta_n, u_cp, u_ij, k_n, d_n, k_t, d_t, mu_p, delta_t, dt_p):
    """Normal and Coulomb-limited tangential contact force on i, Eqs. (41)-(50).

    u_cp: relative surface velocity at the contact point (Eq. (B.7)),
    u_ij: relative centre velocity (Eq. (B.4)). delta_t: stored tangential
    spring (zero for a new contact). Returns (F_n, F_t, new delta_t).
    """
    u_n = (u_ij @ n) * n                                   # Eqs. (B.5), (B.8)
    u_t = u_cp - u_n                                       # Eq. (B.8)
    F_n = -k_n * delta_n * n - d_n * u_n                   # Eq. (41)
    proj = delta_t - (delta_t @ n) * n                     # Eq. (49)
    lp = math.sqrt(proj @ proj)
    rot = (math.sqrt(delta_t @ delta_t) / lp) * proj if lp > 0.0 else np.zeros(3)
    F_sd = -k_t * rot - d_t * u_t                          # Eq. (45)
    f_c = mu_p * math.sqrt(F_n @ F_n)
    l_sd = math.sqrt(F_sd @ F_sd)
    if l_sd < f_c:                                         # Eq. (50), sticking
        return F_n, F_sd, rot + dt_p * u_t
    t = F_sd / l_sd if l_sd > 0.0 else np.zeros(3)         # Eq. (48)
    F_t = f_c * t                                          # Eq. (47)
    return F_n, F_t, -(f_c * t + d_t * u_t) / k_t          # Eq. (50), slipping
