"""Fluid part of the oracle: equilibrium, moments, MRT collision with forcing.

Test infrastructure only (see ``oracle/__init__.py``).

Paper passages followed:
  * Sec. 2.1, Eqs. (1)-(3): collide-then-stream, moments rho = sum f and
    u = (1/rho0) sum f c (incompressible form with rho0 = 1).
  * Sec. 2.1.1, Eq. (5): collision in moment space C = M^-1 S (m^eq - M f).
  * App. A, Eq. (A.2): equilibrium moments.
Readings where the paper is silent:
  * body force: Guo forcing in moment space, m += (I - S/2) M F with
    F_q = w_q [3 (c_q - u).a + 9 (c_q.u)(c_q.a)], and the velocity that
    enters m^eq is u = (j + a/2)/rho0.
  * initial PDFs: the incompressible equilibrium
    f_q = w_q [rho + rho0 (3 c.u + 4.5 (c.u)^2 - 1.5 u.u)], whose moments
    under M are exactly Eq. (A.2).

Arrays are laid out as f[q, z, y, x]; every routine is plain float64 numpy.
"""
import numpy as np

from .d3q19 import C, W, M, M_INV, Q, RHO0, equilibrium_moments


def equilibrium(rho, u):
    """Incompressible second-order equilibrium (Sec. 2.1; its moments under M
    are Eq. (A.2); reading, see module doc).

    rho: (...); u: (3, ...). Returns f_eq with shape (19, ...).
    """
    cu = np.tensordot(C.astype(np.float64), u, axes=([1], [0]))       # (19, ...)
    uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2]
    shape = (Q,) + (1,) * np.ndim(rho)
    w = W.reshape(shape)
    return w * (rho + RHO0 * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu))


def density(f):
    """Eq. (3): rho = sum_q f_q."""
    return f.sum(axis=0)


def momentum(f):
    """Eq. (3) without the 1/rho0 factor: j = sum_q f_q c_q, shape (3, ...)."""
    return np.tensordot(C.T.astype(np.float64), f, axes=([1], [0]))


def guo_source(u, accel):
    """Forcing populations F_q = w_q [3 (c_q - u).a + 9 (c_q.u)(c_q.a)].

    u: (3, ...); accel: (3,). Reading of the forcing scheme, which the paper
    leaves open (the body force a of Sec. 2.4 and of the suspension).
    """
    a = np.asarray(accel, dtype=np.float64)
    cf = C.astype(np.float64)
    ca = cf @ a                                                          # (19,)
    cu = np.tensordot(cf, u, axes=([1], [0]))                            # (19, ...)
    ua = u[0] * a[0] + u[1] * a[1] + u[2] * a[2]
    shape = (Q,) + (1,) * (np.ndim(u) - 1)
    return W.reshape(shape) * (3.0 * (ca.reshape(shape) - ua) + 9.0 * cu * ca.reshape(shape))


def collide(f, accel, s_diag, s_diag_alt=None, alt_mask=None):
    """Moment-space collision of Eq. (5) with the forcing reading above.

    f: pre-collision PDFs (19, ...). accel: body force per unit volume (3,).
    s_diag: the 19 relaxation rates (diagonal of S). Where ``alt_mask`` is
    True the rates ``s_diag_alt`` are used instead (TRT+aB shell cells,
    Sec. 2.3.2). Returns the post-collision PDFs f~ (Eq. (1)).
    """
    shp = f.shape[1:]
    fl = f.reshape(Q, -1)
    m = M @ fl                                                            # (19, N)
    rho = m[0]
    j = m[1:4]
    a = np.asarray(accel, dtype=np.float64).reshape(3, 1)
    u = (j + 0.5 * a) / RHO0
    meq = equilibrium_moments(rho, u)
    mF = M @ guo_source(u, accel)
    S = np.repeat(np.asarray(s_diag, dtype=np.float64).reshape(Q, 1), fl.shape[1], axis=1)
    if alt_mask is not None:
        S2 = np.asarray(s_diag_alt, dtype=np.float64).reshape(Q, 1)
        mask = np.asarray(alt_mask).reshape(-1)
        S[:, mask] = np.repeat(S2, int(mask.sum()), axis=1)
    m_post = m + S * (meq - m) + (1.0 - 0.5 * S) * mF
    return (M_INV @ m_post).reshape((Q,) + shp)


def velocity_from_post_collision(ft, accel):
    """Physical velocity of a cell whose PDFs are post-collision values
    (moments of Eq. (2) with the forcing reading of the module doc).

    The collision adds the body force a to j, while the velocity used in the
    collision was (j_pre + a/2)/rho0; hence u = (sum f~ c - a/2)/rho0.
    """
    a = np.asarray(accel, dtype=np.float64).reshape((3,) + (1,) * (ft.ndim - 1))
    return (momentum(ft) - 0.5 * a) / RHO0
