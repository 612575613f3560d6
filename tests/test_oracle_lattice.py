"""Pins of the oracle's lattice, moment basis and collision (CPU only).

Each test checks the oracle against something other than itself: textbook
identities of the D3Q19 velocity set, the printed equilibrium moments of
App. A, and an independent population-form TRT / BGK collision written here.
"""
import itertools

import numpy as np
import pytest

from oracle import d3q19
from oracle.d3q19 import C, W, M, OPP, Q
from oracle.lbm import collide, equilibrium, guo_source

rng = np.random.default_rng(20030149)


def textbook_feq(rho, u):
    """D3Q19 incompressible equilibrium written out per direction (Qian et al.)."""
    out = np.zeros((19,) + np.shape(rho))
    for q in range(19):
        cu = C[q, 0] * u[0] + C[q, 1] * u[1] + C[q, 2] * u[2]
        uu = u[0] ** 2 + u[1] ** 2 + u[2] ** 2
        out[q] = W[q] * (rho + 3 * cu + 4.5 * cu * cu - 1.5 * uu)
    return out


def test_velocity_set_is_d3q19():
    vecs = {tuple(c) for c in C}
    assert len(vecs) == 19
    expected = {v for v in itertools.product((-1, 0, 1), repeat=3) if sum(abs(x) for x in v) <= 2}
    assert vecs == expected
    assert tuple(C[0]) == (0, 0, 0)
    # ordering pinned by the printed rows 2-4 of M (App. A): q1 = (0,1,0), q3 = (-1,0,0)
    assert tuple(C[1]) == (0, 1, 0) and tuple(C[3]) == (-1, 0, 0) and tuple(C[5]) == (0, 0, 1)
    for q in range(Q):
        assert (C[OPP[q]] == -C[q]).all()


def test_lattice_isotropy():
    # sum w = 1, sum w c = 0, sum w c_a c_b = delta/3, fourth moment = (dd+dd+dd)/9
    assert abs(W.sum() - 1) < 1e-15
    assert np.abs(W @ C).max() < 1e-15
    second = np.einsum('q,qa,qb->ab', W, C, C)
    assert np.allclose(second, np.eye(3) / 3, atol=1e-15)
    fourth = np.einsum('q,qa,qb,qc,qd->abcd', W, C, C, C, C)
    I = np.eye(3)
    ref = (np.einsum('ab,cd->abcd', I, I) + np.einsum('ac,bd->abcd', I, I)
           + np.einsum('ad,bc->abcd', I, I)) / 9
    assert np.allclose(fourth, ref, atol=1e-15)
    third = np.einsum('q,qa,qb,qc->abc', W, C, C, C)
    assert np.abs(third).max() < 1e-15


def test_moment_rows_are_the_stated_polynomials():
    c2 = (C * C).sum(axis=1)
    assert (M[0] == 1).all()
    assert (M[4] == c2 - 1).all()
    assert (M[9] == 2 * C[:, 0] ** 2 - C[:, 1] ** 2 - C[:, 2] ** 2).all()
    assert (M[10] == C[:, 1] ** 2 - C[:, 2] ** 2).all()
    assert (M[11] == C[:, 0] * C[:, 1]).all()
    assert (M[12] == C[:, 1] * C[:, 2]).all()
    assert (M[13] == C[:, 0] * C[:, 2]).all()


def test_rows_of_M_are_weight_orthogonal():
    G = M @ np.diag(W) @ M.T
    off = G - np.diag(np.diag(G))
    assert np.abs(off).max() < 1e-15
    assert np.allclose(d3q19.M_INV @ M, np.eye(19), atol=1e-13)


def test_M_of_equilibrium_gives_printed_moments():
    rho = 1 + 0.05 * rng.standard_normal(50)
    u = 0.05 * rng.standard_normal((3, 50))
    feq = textbook_feq(rho, u)
    m = M @ feq
    meq = d3q19.equilibrium_moments(rho, u)
    assert np.abs(m - meq).max() < 1e-15
    assert np.abs(equilibrium(rho, u) - feq).max() < 1e-15


def test_relaxation_parameter_relations():
    s_nu = 1 / 0.6
    assert abs(d3q19.viscosity(s_nu) - 1 / 30) < 1e-15
    s_m = d3q19.s_minus_from_magic(s_nu, 3 / 16)
    assert abs((1 / s_nu - 0.5) * (1 / s_m - 0.5) - 3 / 16) < 1e-15
    assert abs(1 / s_m - 2.375) < 1e-12
    s_b = d3q19.s_b_from_lambda_b(s_nu, 100)
    assert abs((1 / s_b - 0.5) / (1 / s_nu - 0.5) - 100) < 1e-12
    assert abs(d3q19.s_b_from_lambda_b(s_nu, 1.0) - s_nu) < 1e-15
    assert abs(d3q19.bulk_viscosity(s_nu) - 2 / 9 * 0.1) < 1e-15


def test_guo_source_moments():
    u = 0.03 * rng.standard_normal((3, 7))
    a = np.array([1e-3, -2e-3, 5e-4])
    F = guo_source(u, a)
    assert np.abs(F.sum(axis=0)).max() < 1e-17
    first = np.einsum('qa,qn->an', C, F)
    assert np.abs(first - a[:, None]).max() < 1e-17
    second = np.einsum('qa,qb,qn->abn', C, C, F)
    ref = np.einsum('an,b->abn', u, a) + np.einsum('a,bn->abn', a, u)
    assert np.abs(second - ref).max() < 1e-17


def random_pdfs(n):
    rho = 1 + 0.02 * rng.standard_normal(n)
    u = 0.04 * rng.standard_normal((3, n))
    return textbook_feq(rho, u) * (1 + 0.05 * rng.standard_normal((19, n)))


def test_collision_conserves_mass_and_momentum():
    f = random_pdfs(40)
    s_nu = 1 / 0.55
    S = d3q19.relaxation_rates('trtb', s_nu, d3q19.s_minus_from_magic(s_nu, 3 / 16),
                               d3q19.s_b_from_lambda_b(s_nu, 100))
    a = np.array([2e-4, 0, -1e-4])
    ft = collide(f, np.zeros(3), S)
    assert np.abs(ft.sum(0) - f.sum(0)).max() < 1e-15
    assert np.abs(C.T @ ft - C.T @ f).max() < 1e-15
    ft = collide(f, a, S)
    assert np.abs(ft.sum(0) - f.sum(0)).max() < 1e-15
    assert np.abs(C.T @ ft - C.T @ f - a[:, None]).max() < 1e-15


def population_trt(f, s_plus, s_minus, a):
    """Independent two-relaxation-time collision in population form with Guo forcing."""
    rho = f.sum(0)
    j = np.einsum('qa,qn->an', C, f)
    u = j + 0.5 * a[:, None]
    feq = textbook_feq(rho, u)
    out = np.empty_like(f)
    for q in range(19):
        qb = OPP[q]
        fp, fm = 0.5 * (f[q] + f[qb]), 0.5 * (f[q] - f[qb])
        ep, em = 0.5 * (feq[q] + feq[qb]), 0.5 * (feq[q] - feq[qb])
        cu_q = C[q] @ u
        Fq = W[q] * (3 * (C[q] @ a - (u * a[:, None]).sum(0)) + 9 * cu_q * (C[q] @ a))
        cu_b = C[qb] @ u
        Fb = W[qb] * (3 * (C[qb] @ a - (u * a[:, None]).sum(0)) + 9 * cu_b * (C[qb] @ a))
        Fp, Fm = 0.5 * (Fq + Fb), 0.5 * (Fq - Fb)
        out[q] = f[q] - s_plus * (fp - ep) - s_minus * (fm - em) \
            + (1 - s_plus / 2) * Fp + (1 - s_minus / 2) * Fm
    return out


@pytest.mark.parametrize("tau", [0.52, 0.6, 1.0, 1.7])
def test_mrt_with_trt_rates_equals_population_trt(tau):
    f = random_pdfs(30)
    s_nu = 1 / tau
    s_m = d3q19.s_minus_from_magic(s_nu, 3 / 16)
    a = np.array([1e-3, 2e-4, -3e-4])
    S = d3q19.relaxation_rates('trt', s_nu, s_m)
    assert np.abs(collide(f, a, S) - population_trt(f, s_nu, s_m, a)).max() < 1e-15
    # TRT+B with Lambda_b = 1 is the TRT model (Sec. 2.1.3)
    S_b1 = d3q19.relaxation_rates('trtb', s_nu, s_m, d3q19.s_b_from_lambda_b(s_nu, 1.0))
    assert np.abs(S_b1 - S).max() < 1e-15


def test_mrt_with_srt_rates_equals_bgk():
    f = random_pdfs(30)
    s = 1 / 0.7
    a = np.array([0, 5e-4, 1e-4])
    S = d3q19.relaxation_rates('srt', s)
    assert np.abs(collide(f, a, S) - population_trt(f, s, s, a)).max() < 1e-15


def test_bulk_moments_relax_with_s_b_in_shell_cells():
    f = random_pdfs(10)
    s_nu = 1 / 0.6
    s_m = d3q19.s_minus_from_magic(s_nu, 3 / 16)
    s_b = d3q19.s_b_from_lambda_b(s_nu, 100)
    S = d3q19.relaxation_rates('trtb', s_nu, s_m, s_nu)
    S_shell = d3q19.relaxation_rates('trtb', s_nu, s_m, s_b)
    mask = np.array([True, False] * 5)
    ft = collide(f, np.zeros(3), S, S_shell, mask)
    m, mt = M @ f, M @ ft
    meq = d3q19.equilibrium_moments(m[0], m[1:4])
    for k in (4, 5):
        rate = (mt[k] - m[k]) / (meq[k] - m[k])
        assert np.allclose(rate[mask], s_b, rtol=1e-9)
        assert np.allclose(rate[~mask], s_nu, rtol=1e-9)
    for k in (9, 10, 11):
        rate = (mt[k] - m[k]) / (meq[k] - m[k])
        assert np.allclose(rate, s_nu, rtol=1e-9)
    for k in (6, 16):
        rate = (mt[k] - m[k]) / (meq[k] - m[k])
        assert np.allclose(rate, s_m, rtol=1e-9)
