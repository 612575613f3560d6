"""D3Q19 lattice, moment basis and relaxation matrices of the paper.

Test infrastructure only (see ``oracle/__init__.py``).

Sources in the paper (Rettinger & Ruede, arXiv 2003.01490):
  * Sec. 2.1   -- D3Q19 velocity set, lattice units (dx = dt = rho0 = 1,
                 c_s^2 = 1/3), moments Eq. (3).
  * Sec. 2.1.1 -- MRT collision Eq. (5), rate matrix Eq. (6), viscosity
                 relations Eqs. (7)-(8).
  * Sec. 2.1.2 -- SRT matrix Eq. (9), TRT matrix Eq. (10), magic parameter
                 Eq. (11).
  * Sec. 2.1.3 -- TRT+B matrix Eq. (12), Lambda_b relation Eq. (13).
  * App. A     -- moment matrix M, Eq. (A.1), and equilibrium moments,
                 Eq. (A.2).

Everything here is float64 and written for readability, not speed.
"""
import numpy as np

Q = 19
CS2 = 1.0 / 3.0          # lattice speed of sound squared, Sec. 2.1
RHO0 = 1.0               # reference density, Sec. 2.1

# Moment matrix M exactly as printed in App. A, Eq. (A.1).
M = np.array([
    [1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1],
    [0, 0, 0, -1, 1, 0, 0, -1, 1, -1, 1, 0, 0, -1, 1, 0, 0, -1, 1],
    [0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, -1, 0, 0, 1, -1, 0, 0],
    [0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, 1, 1, -1, -1, -1, -1],
    [-1, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1],
    [1, -2, -2, -2, -2, -2, -2, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1],
    [0, 0, 0, 2, -2, 0, 0, -1, 1, -1, 1, 0, 0, -1, 1, 0, 0, -1, 1],
    [0, -2, 2, 0, 0, 0, 0, 1, 1, -1, -1, 1, -1, 0, 0, 1, -1, 0, 0],
    [0, 0, 0, 0, 0, -2, 2, 0, 0, 0, 0, 1, 1, 1, 1, -1, -1, -1, -1],
    [0, -1, -1, 2, 2, -1, -1, 1, 1, 1, 1, -2, -2, 1, 1, -2, -2, 1, 1],
    [0, 1, 1, 0, 0, -1, -1, 1, 1, 1, 1, 0, 0, -1, -1, 0, 0, -1, -1],
    [0, 0, 0, 0, 0, 0, 0, -1, 1, 1, -1, 0, 0, 0, 0, 0, 0, 0, 0],
    [0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, -1, 0, 0, -1, 1, 0, 0],
    [0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, -1, 1, 0, 0, 1, -1],
    [0, 1, 1, -2, -2, 1, 1, 1, 1, 1, 1, -2, -2, 1, 1, -2, -2, 1, 1],
    [0, -1, -1, 0, 0, 1, 1, 1, 1, 1, 1, 0, 0, -1, -1, 0, 0, -1, -1],
    [0, 0, 0, 0, 0, 0, 0, -1, 1, -1, 1, 0, 0, 1, -1, 0, 0, 1, -1],
    [0, 0, 0, 0, 0, 0, 0, -1, -1, 1, 1, 1, -1, 0, 0, 1, -1, 0, 0],
    [0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, -1, -1, 1, 1, 1, 1, -1, -1],
], dtype=np.float64)

# App. A states that rows 2-4 of M fix the ordering of the lattice velocities:
# c_q = (M[1, q], M[2, q], M[3, q]).
C = M[1:4].T.astype(np.int64).copy()            # (19, 3)

# Lattice weights of D3Q19 (Qian et al., cited in Sec. 2.1): rest 1/3,
# axis directions 1/18, face diagonals 1/36.
_norm2 = (C * C).sum(axis=1)
W = np.where(_norm2 == 0, 1.0 / 3.0, np.where(_norm2 == 1, 1.0 / 18.0, 1.0 / 36.0))

# Opposite direction index qbar with c_qbar = -c_q (Sec. 2.2).
OPP = np.array([int(np.nonzero((C == -C[q]).all(axis=1))[0][0]) for q in range(Q)])

M_INV = np.linalg.inv(M)


def equilibrium_moments(rho, u):
    """Equilibrium moments m^eq of App. A, Eq. (A.2).

    rho: array (...); u: array (3, ...). Returns (19, ...).
    """
    ux, uy, uz = u[0], u[1], u[2]
    z = np.zeros_like(rho)
    return np.stack([
        rho, ux, uy, uz,
        ux * ux + uy * uy + uz * uz,
        z, z, z, z,
        2.0 * ux * ux - uy * uy - uz * uz,
        uy * uy - uz * uz,
        ux * uy, uy * uz, ux * uz,
        z, z, z, z, z,
    ])


def relaxation_rates(variant, s_nu, s_minus=None, s_b=None, s_general=None):
    """Diagonal of the relaxation matrix S for the collision variants.

    variant:
      'mrt'  -- Eq. (6) with s_general = (s1, s2, s3, s4, s5, s6)
      'srt'  -- Eq. (9): every non-conserved moment relaxes with s_nu
      'trt'  -- Eq. (10): even moments s_nu, odd moments s_minus
      'trtb' -- Eq. (12): as TRT but moments 4 and 5 relax with s_b
    """
    if variant == 'mrt':
        s1, s2, s3, s4, s5, s6 = s_general
        d = [0, 0, 0, 0, s1, s2, s3, s3, s3, s4, s4, s4, s4, s4, s5, s5, s6, s6, s6]
    elif variant == 'srt':
        d = [0, 0, 0, 0] + [s_nu] * 15
    elif variant == 'trt':
        d = [0, 0, 0, 0, s_nu, s_nu, s_minus, s_minus, s_minus,
             s_nu, s_nu, s_nu, s_nu, s_nu, s_nu, s_nu, s_minus, s_minus, s_minus]
    elif variant == 'trtb':
        d = [0, 0, 0, 0, s_b, s_b, s_minus, s_minus, s_minus,
             s_nu, s_nu, s_nu, s_nu, s_nu, s_nu, s_nu, s_minus, s_minus, s_minus]
    else:
        raise ValueError(variant)
    return np.array(d, dtype=np.float64)


def s_nu_from_tau(tau):
    """s_nu = 1/tau; the kinematic viscosity follows Eq. (7)."""
    return 1.0 / tau


def viscosity(s_nu):
    """Eq. (7): nu = (1/s_nu - 1/2) / 3."""
    return (1.0 / s_nu - 0.5) / 3.0


def bulk_viscosity(s_b):
    """Eq. (8): nu_b = (2/9) (1/s_b - 1/2)."""
    return (2.0 / 9.0) * (1.0 / s_b - 0.5)


def s_minus_from_magic(s_nu, magic):
    """Solve Eq. (11), Lambda = (1/s_nu - 1/2)(1/s_minus - 1/2), for s_minus."""
    return 1.0 / (0.5 + magic / (1.0 / s_nu - 0.5))


def s_b_from_lambda_b(s_nu, lambda_b):
    """Solve Eq. (13), Lambda_b = (1/s_b - 1/2)/(1/s_nu - 1/2), for s_b."""
    return 1.0 / (0.5 + lambda_b * (1.0 / s_nu - 0.5))
