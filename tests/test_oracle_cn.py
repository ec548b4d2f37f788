"""Pins of the oracle's Crank-Nicolson step (Sec. 2.3, the paper's comparison
method; reading: (I - tau/2 A_n) u^{n+1} = (I + tau/2 A_n) u^n + tau f_n)
against closed forms and properties the scheme fixes.  CPU only."""
import math

import numpy as np
import pytest
import scipy.fft

import oracle
from oracle import cn
from paper_2402_02273_gb300 import phantom


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def _neumann_eigs(N, h):
    k = np.arange(N)
    return -(4.0 / h ** 2) * np.sin(np.pi * k / (2 * N)) ** 2


@pytest.mark.parametrize("shape", [(6, 10, 14), (16, 16, 16)])
def test_constant_D_pure_diffusion_matches_cosine_modes(shape):
    """Constant D, rho = 0: the conservative operator is diagonal in DCT-II modes,
    and one step multiplies mode k by (1 + tau lam_k / 2) / (1 - tau lam_k / 2)."""
    Dc, h, tau = 0.13, 1.0, 7.3
    D = np.full(shape, Dc)
    _, u0 = phantom.case(shape, seed=0)
    P = oracle.Problem(D, h=h, rho=0.0, op="conservative", scheme="expeuler")
    got, _ = cn.cn_step(P, u0, tau)
    nz, ny, nx = shape
    lam = (_neumann_eigs(nz, h)[:, None, None] + _neumann_eigs(ny, h)[None, :, None]
           + _neumann_eigs(nx, h)[None, None, :]) * Dc
    c = scipy.fft.dctn(u0, type=2, norm="ortho")
    want = scipy.fft.idctn(c * (1 + 0.5 * tau * lam) / (1 - 0.5 * tau * lam), type=2, norm="ortho")
    assert _rel(got, want) <= 1e-12


@pytest.mark.parametrize("scheme", ["rosenbrock", "expeuler"])
def test_pure_reaction_is_the_scalar_trapezoidal_rule(scheme):
    """D = 0: every voxel is the scalar linearised trapezoidal rule
    (1 - tau c/2) u' = (1 + tau c/2) u + tau f, c = rho(1 - 2u), f = rho u^2
    (folded) or c = 0, f = rho u (1 - u)."""
    shape = (3, 4, 5)
    u = 0.05 + 0.9 * phantom.uniform(9, 1, 60).reshape(shape)
    rho, tau = 0.025, 7.3
    P = oracle.Problem(np.zeros(shape), rho=rho, scheme=scheme)
    got, _ = cn.cn_step(P, u, tau)
    if scheme == "rosenbrock":
        c, f = rho * (1 - 2 * u), rho * u * u
    else:
        c, f = np.zeros(shape), rho * u * (1 - u)
    want = ((1 + 0.5 * tau * c) * u + tau * f) / (1 - 0.5 * tau * c)
    assert _rel(got, want) <= 1e-15


def test_pure_diffusion_conserves_mass_and_never_grows_the_two_norm():
    """rho = 0, conservative: column sums of L vanish (mass kept), and for the
    symmetric negative semi-definite L the trapezoidal rule is A-stable, so
    ||u||_2 does not grow, even for steps far beyond the explicit limit."""
    D, u0 = phantom.case(12, seed=2, noise=0.1)
    P = oracle.Problem(D, rho=0.0, op="conservative", scheme="rosenbrock")
    u = u0.copy()
    for tau in (7.3, 7.3, 500.0, 5000.0):
        v, _ = cn.cn_step(P, u, tau)
        assert abs(v.sum() - u.sum()) <= 1e-12 * u.sum()
        assert np.linalg.norm(v) <= np.linalg.norm(u) * (1 + 1e-14)
        u = v


def test_system_matrix_is_symmetric_positive_definite():
    """Conservative operator, folded reaction with tau rho < 2: I - tau/2 A_n is
    symmetric and positive definite (what the GPU's conjugate gradients need)."""
    D, u0 = phantom.case((4, 5, 6), seed=5, noise=0.1)
    P = oracle.Problem(D, rho=0.025, op="conservative", scheme="rosenbrock")
    A = cn.assemble_A(P, u0).toarray()
    M = np.eye(A.shape[0]) - 0.5 * 7.3 * A
    assert np.array_equal(M, M.T)
    assert np.linalg.eigvalsh(M).min() > 0.5


def test_sparse_assembly_matches_the_matrix_free_operator():
    D, u0 = phantom.case((5, 6, 7), seed=6, noise=0.1)
    for op in ("conservative", "literal"):
        P = oracle.Problem(D, rho=0.025, op=op, scheme="rosenbrock")
        v = phantom.uniform(3, 3, D.size).reshape(D.shape) - 0.5
        A = cn.assemble_A(P, u0)
        assert np.abs(A @ v.ravel() - P.apply_A(u0, v).ravel()).max() <= 1e-15


def test_second_order_in_tau_for_linear_diffusion():
    """rho = 0: against the exact exp(T L) u0 (one oracle exponential step, whose
    truncation is below 1e-17), the error falls by 4 per halving of tau."""
    D, u0 = phantom.case(10, seed=6, noise=0.1)
    P = oracle.Problem(D, rho=0.0, op="conservative", scheme="expeuler")
    T = 60.0
    exact, _ = P.run(u0, T, 1)
    errs = []
    for k in (4, 8, 16, 32):
        u = cn.cn_run(P, u0, T / k, k)
        errs.append(np.abs(u - exact).max())
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert all(abs(o - 2.0) < 0.1 for o in orders[1:]), orders


def test_iterative_and_direct_solves_agree():
    """The CG branch (large grids) and the direct branch give the same step."""
    D, u0 = phantom.case(16, seed=7, noise=0.1)
    P = oracle.Problem(D, rho=0.025)
    direct, _ = cn.cn_step(P, u0, 7.3)
    keep = cn.DIRECT_MAX
    try:
        cn.DIRECT_MAX = 0
        iterative, iters = cn.cn_step(P, u0, 7.3)
    finally:
        cn.DIRECT_MAX = keep
    assert iters > 0
    assert _rel(iterative, direct) <= 1e-12
