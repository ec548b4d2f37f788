"""Pins of the oracle's discrete adjoint (reverse mode through its own step loops)
against central finite differences of the oracle's forward map.  CPU only."""
import numpy as np
import pytest

import oracle
from paper_2402_02273_gb300 import phantom

EPS = 1e-6


def _loss(P, u0, tau, K, tgt):
    uK, _ = P.run(u0, tau, K)
    return 0.5 * np.sum((uK - tgt) ** 2), uK


@pytest.mark.parametrize("op", ["conservative", "literal"])
@pytest.mark.parametrize("scheme", ["rosenbrock", "expeuler"])
def test_adjoint_gradients_match_central_differences(op, scheme):
    D, u0 = phantom.case((6, 7, 8), seed=3, noise=0.1)
    D[D == 0] = 0.05
    rho, tau, K = 0.025, 7.3, 3
    mk = lambda Dv=D, r=rho: oracle.Problem(Dv, op=op, scheme=scheme, rho=r)
    P = mk()
    tgt = 0.5 * phantom.uniform(5, 5, D.size).reshape(D.shape)
    J0, uK = _loss(P, u0, tau, K, tgt)
    ubar0, g_rho, g_ds = oracle.vjp(P, u0, tau, K, uK - tgt)
    fd_rho = (_loss(mk(r=rho + EPS), u0, tau, K, tgt)[0] - _loss(mk(r=rho - EPS), u0, tau, K, tgt)[0]) / (2 * EPS)
    fd_ds = (_loss(mk(Dv=D * (1 + EPS)), u0, tau, K, tgt)[0]
             - _loss(mk(Dv=D * (1 - EPS)), u0, tau, K, tgt)[0]) / (2 * EPS)
    v = phantom.uniform(6, 6, D.size).reshape(D.shape) - 0.5
    fd_u = (_loss(P, u0 + EPS * v, tau, K, tgt)[0] - _loss(P, u0 - EPS * v, tau, K, tgt)[0]) / (2 * EPS)
    assert g_rho == pytest.approx(fd_rho, rel=1e-7)
    assert g_ds == pytest.approx(fd_ds, rel=1e-7)
    assert np.sum(ubar0 * v) == pytest.approx(fd_u, rel=1e-7)


def test_adjoint_of_pure_diffusion_is_transpose_of_the_step():
    """rho = 0: the step is the linear map u -> exp(tau L) u, so the adjoint of a
    unit cotangent e_q is row q of that map's matrix.  The literal operator is
    not symmetric, so row and column differ and a transposition mistake fails."""
    D, _ = phantom.case((4, 4, 5), seed=1, noise=0.1)
    D[D == 0] = 0.08
    P = oracle.Problem(D, rho=0.0, op="literal", scheme="rosenbrock")
    n = D.size
    M = np.zeros((n, n))
    for q in range(n):
        e = np.zeros(n)
        e[q] = 1.0
        M[:, q] = P.run(e.reshape(D.shape), 7.3, 1)[0].ravel()
    for q in (0, 7, n - 1):
        e = np.zeros(n)
        e[q] = 1.0
        ub, _, _ = oracle.vjp(P, np.zeros(D.shape), 7.3, 1, e.reshape(D.shape))
        assert np.abs(ub.ravel() - M[q, :]).max() <= 1e-13 * np.abs(M).max()
