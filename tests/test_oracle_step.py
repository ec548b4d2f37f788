"""Pins of the oracle's exponential-integrator step (Sec. 2.2) against library
routines, closed forms and invariants.  CPU only."""
import json
import math
import os

import numpy as np
import pytest
import scipy.fft
import scipy.linalg

import oracle
from oracle import multinomial
from paper_2402_02273_gb300 import phantom

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _dense(P, un):
    n = P.D.size
    A = np.zeros((n, n))
    for q in range(n):
        e = np.zeros(n)
        e[q] = 1.0
        A[:, q] = P.apply_A(un, e).ravel()
    return A


def _phi1(z):
    z = np.asarray(z, dtype=np.float64)
    out = np.ones_like(z)
    nz = z != 0
    out[nz] = np.expm1(z[nz]) / z[nz]
    return out


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("shape", [(4, 4, 4), (3, 4, 5), (1, 6, 6), (8, 1, 1)])
@pytest.mark.parametrize("op", ["conservative", "literal"])
@pytest.mark.parametrize("scheme", ["rosenbrock", "expeuler"])
def test_phi1_action_equals_expm_of_augmented_matrix(shape, op, scheme):
    """exp([[tau A, tau b], [0, 0]]) [0; 1] = [tau phi1(tau A) b; 1] (Sec. 2.2), via scipy."""
    lab = phantom.head_labels(shape, seed=4)
    D = phantom.diffusion_field(lab, seed=4, noise=0.1)
    D[D == 0] = 0.05  # keep the operator non-trivial on tiny grids
    u = 0.9 * phantom.uniform(9, 1, D.size).reshape(shape)
    P = oracle.Problem(D, op=op, scheme=scheme, rho=0.025)
    tau = 7.3
    A = _dense(P, u)
    b = P.residual(u)
    n = D.size
    M = np.zeros((n + 1, n + 1))
    M[:n, :n] = tau * A
    M[:n, n] = tau * b.ravel()
    want = scipy.linalg.expm(M)[:n, n]
    got, s, m = P.phi1_action(u, b, tau)
    assert s >= 1 and m >= 8
    assert _rel(got.ravel(), want) <= 1e-13


def test_phi1_action_equals_eigendecomposition_symmetric():
    D, u0 = phantom.case((5, 6, 4), seed=5, noise=0.1)
    D[D == 0] = 0.02
    P = oracle.Problem(D, op="conservative", scheme="expeuler")
    A = _dense(P, u0)
    lam, V = np.linalg.eigh(A)
    tau = 7.3
    b = P.residual(u0).ravel()
    want = V @ (tau * _phi1(tau * lam) * (V.T @ b))
    got, _, _ = P.phi1_action(u0, b.reshape(D.shape), tau)
    assert _rel(got.ravel(), want) <= 1e-13


def _neumann_eigs(N, h):
    k = np.arange(N)
    return -(4.0 / h ** 2) * np.sin(np.pi * k / (2 * N)) ** 2


@pytest.mark.parametrize("op,factor", [("conservative", 1.0), ("literal", 2.0)])
@pytest.mark.parametrize("shape", [(16, 16, 16), (6, 10, 14)])
def test_constant_D_pure_diffusion_matches_cosine_modes(op, factor, shape):
    """Constant D, rho = 0: one step is exp(tau L) u, diagonal in DCT-II modes with
    1D eigenvalues -(4D/h^2) sin^2(pi k / 2N) (doubled for the printed operator)."""
    Dc, h, tau = 0.13, 1.0, 7.3
    D = np.full(shape, Dc)
    _, u0 = phantom.case(shape, seed=0)
    P = oracle.Problem(D, h=h, rho=0.0, op=op, scheme="expeuler")
    got, _ = P.run(u0, tau, 1)
    nz, ny, nx = shape
    lam = (_neumann_eigs(nz, h)[:, None, None] + _neumann_eigs(ny, h)[None, :, None]
           + _neumann_eigs(nx, h)[None, None, :]) * Dc * factor
    c = scipy.fft.dctn(u0, type=2, norm="ortho")
    want = scipy.fft.idctn(c * np.exp(tau * lam), type=2, norm="ortho")
    assert _rel(got, want) <= 1e-12


def test_pure_diffusion_conserves_mass_conservative_only():
    D, u0 = phantom.case(16, seed=1, noise=0.1)
    Pc = oracle.Problem(D, rho=0.0, op="conservative", scheme="rosenbrock")
    u, st = Pc.run(u0, 7.3, 5)
    assert abs(u.sum() - u0.sum()) <= 1e-13 * u0.sum()
    assert abs(st[-1]["mass"] - u.sum()) <= 1e-13 * u0.sum()
    Pl = oracle.Problem(D, rho=0.0, op="literal", scheme="rosenbrock")
    ul, _ = Pl.run(u0, 7.3, 5)
    assert abs(ul.sum() - u0.sum()) > 1e-6 * u0.sum()


@pytest.mark.parametrize("scheme", ["rosenbrock", "expeuler"])
def test_pure_reaction_matches_scalar_closed_form(scheme):
    """D = 0: each voxel follows u + tau phi1(tau c) rho u (1-u), c = rho(1-2u) or 0."""
    shape = (3, 4, 5)
    u = phantom.uniform(2, 2, 60).reshape(shape)
    rho, tau = 0.025, 7.3
    P = oracle.Problem(np.zeros(shape), rho=rho, scheme=scheme)
    got, _ = P.run(u, tau, 1)
    c = rho * (1 - 2 * u) if scheme == "rosenbrock" else np.zeros(shape)
    want = u + tau * _phi1(tau * c) * rho * u * (1 - u)
    assert np.abs(got - want).max() <= 2e-16


@pytest.mark.parametrize("op", ["conservative", "literal"])
def test_density_stays_in_unit_interval(op):
    D, u0 = phantom.case(16, seed=3, noise=0.1)
    u0 = np.minimum(1.0, u0 * 1.25)  # peak 1.0 at the seed
    P = oracle.Problem(D, op=op, scheme="rosenbrock", rho=0.025)
    states, st = P.run(u0, 7.3, 10, every=True)
    for u in states:
        assert u.min() >= -1e-14 and u.max() <= 1 + 1e-14
    assert min(x["umin"] for x in st) >= -1e-14


@pytest.mark.parametrize("shape", [(6, 5, 7), (1, 1, 9), (4, 3, 1)])
def test_step_records_are_min_max_and_sum_of_the_returned_state(shape):
    """The per-step record (tumour mass, Sec. 3.5, and the extremes of u) is a
    plain reduction of the state the step returns: umin and umax equal numpy's
    min and max exactly, the mass its sum up to summation order.  The fields sit
    strictly inside (0, 1), and their extremes lie in planes other than the
    first, so neither a 0 / 1 start value nor a reduction over one plane nor a
    swapped comparison can pass."""
    n = shape[0] * shape[1] * shape[2]
    u0 = (0.2 + 0.6 * phantom.uniform(11, 3, n)).reshape(shape)
    D = 0.05 * phantom.uniform(11, 4, n).reshape(shape)
    for scheme in ("rosenbrock", "expeuler"):
        P = oracle.Problem(D, rho=0.025, op="conservative", scheme=scheme)
        states, st = P.run(u0, 7.3, 3, every=True)
        for t in range(3):
            u = states[t + 1]
            assert st[t]["umin"] == u.min() and st[t]["umax"] == u.max()
            assert st[t]["umin"] > 0.1 and st[t]["umax"] < 0.95
            assert abs(st[t]["mass"] - u.sum()) <= 1e-14 * u.sum()
    # extremes planted in the last and a middle plane of a pure-reaction step
    # (D = 0): the step is monotone per voxel, so they stay where they were put
    u1 = np.full(shape, 0.5)
    u1.reshape(-1)[n - 1] = 0.3
    u1.reshape(-1)[n // 2] = 0.7
    P = oracle.Problem(np.zeros(shape), rho=0.025)
    u, st = P.run(u1, 7.3, 1)
    assert np.argmin(u) == n - 1 and np.argmax(u) == n // 2
    assert st[0]["umin"] == u.min() and st[0]["umax"] == u.max()


def _order(errs):
    return [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


@pytest.mark.parametrize("scheme,order", [("rosenbrock", 2.0), ("expeuler", 1.0)])
def test_temporal_convergence_order(scheme, order):
    """Halving tau: exponential Rosenbrock-Euler converges with order 2 (exact Jacobian
    folded into A), exponential Euler with order 1 (Sec. 1 calls the method first order)."""
    D, u0 = phantom.case(10, seed=6, noise=0.1)
    rho, T = 0.05, 80.0
    P = oracle.Problem(D, op="conservative", scheme=scheme, rho=rho)
    ref, _ = P.run(u0, T / 1024, 1024)
    errs = []
    for k in (8, 16, 32, 64):
        u, _ = P.run(u0, T / k, k)
        errs.append(np.abs(u - ref).max())
    orders = _order(errs)
    assert all(abs(o - order) < 0.15 for o in orders[1:]), orders


def test_front_speed_matches_fisher_kpp():
    """A pulled Fisher-KPP front moves at 2 sqrt(D rho) (Sec. 2); the slab is 1 x 1 x N."""
    N, Dc, rho, tau = 420, 0.13, 0.025, 5.0
    D = np.full((1, 1, N), Dc)
    u0 = np.zeros((1, 1, N))
    u0[0, 0, :3] = 1.0
    P = oracle.Problem(D, rho=rho, op="conservative", scheme="rosenbrock")
    states, _ = P.run(u0, tau, 600, every=True)

    def front(u):
        v = u.ravel()
        i = int(np.argmax(v < 0.5))
        return i - 1 + (v[i - 1] - 0.5) / (v[i - 1] - v[i])

    t1, t2 = 200, 600  # steps: 1000 and 3000 days
    speed = (front(states[t2]) - front(states[t1])) / ((t2 - t1) * tau)
    v_star = 2 * math.sqrt(Dc * rho)
    # Bramson's logarithmic delay, x(t) = v t - 3/(2 lambda) ln t, lambda = sqrt(rho/D)
    v_bramson = v_star - 1.5 * math.sqrt(Dc / rho) * math.log(t2 / t1) / ((t2 - t1) * tau)
    assert abs(speed - v_bramson) <= 0.03 * v_star, (speed, v_bramson, v_star)


def test_paper_front_speed_arithmetic():
    g = json.load(open(os.path.join(GOLDEN, "paper_parameters.json")))
    f3 = g["front_speed_3d"]
    Dhat = f3["p_w"] * g["D_w"] + f3["p_g"] * g["D_g"]
    assert round(2 * math.sqrt(Dhat * g["rho"]), f3["printed_digits"]) == f3["printed"]
    f2 = g["front_speed_2d"]
    Dhat2 = f2["p_w"] * g["D_w"] + f2["p_g"] * g["D_g"]
    # reading A13: the printed 2D figure is sqrt(D_hat rho) = 0.0487 cut to three
    # digits; 2 sqrt(D_hat rho) would be 0.097
    assert math.floor(math.sqrt(Dhat2 * g["rho"]) * 1000) / 1000 == f2["printed"]
    assert abs(2 * math.sqrt(Dhat2 * g["rho"]) - f2["printed"]) > 0.04
    assert (g["T"] - g["t0"]) / g["K"] == pytest.approx(33.5)
    m3 = g["measured_speed_3d"]
    # 45 / 825 = 0.0545, printed cut (not rounded) to 0.054
    assert math.floor(m3["growth_mm"] / (m3["t_end"] - m3["t_start"]) * 1000) / 1000 == m3["printed"]


def test_multinomial_form_equals_sequential_product_small_norm():
    """Sec. 2.2's multinomial expansion of (P_0+...+P_m)^s equals the factor-by-factor
    product in exact arithmetic; in FP64 they agree for a small norm."""
    D, u0 = phantom.case((3, 4, 4), seed=7, noise=0.1)
    D[D == 0] = 0.03
    P = oracle.Problem(D, op="conservative", scheme="rosenbrock")
    b = P.residual(u0)
    tau = 2.0
    s, m = 3, 7
    got = multinomial.phi1_action(P, u0, b, tau, s, m)
    # the same polynomial evaluated factor by factor with a fixed m
    x = np.zeros(D.shape)
    h = tau / s
    for _ in range(s):
        term, acc, a = x.copy(), x.copy(), 1.0
        for j in range(1, m + 1):
            term = (h / j) * (P.apply_A(u0, term) + b * a)
            a = 0.0
            acc += term
        x = acc
    assert _rel(got, x) <= 1e-13
    # and both approximate the exact action
    exact, _, _ = P.phi1_action(u0, b, tau)
    assert _rel(got, exact) <= 1e-6


def test_multinomial_coefficients_are_taylor_power():
    """sum over compositions = coefficients of (sum_t x^t / t!)^s."""
    s, m = 4, 5
    c = multinomial.power_coefficients(s, m)
    base = np.array([1.0 / math.factorial(t) for t in range(m + 1)])
    poly = np.array([1.0])
    for _ in range(s):
        poly = np.convolve(poly, base)
    assert np.allclose(c, poly, rtol=1e-14, atol=0)


def test_multinomial_form_loses_accuracy_for_large_norm():
    """Expanding in monomials undoes the scaling: for beta ~ 20 the FP64 result of the
    multinomial form is far less accurate than the sequential product (reading A8)."""
    D, u0 = phantom.case((3, 4, 4), seed=7, noise=0.1)
    D[D == 0] = 0.6
    P = oracle.Problem(D, op="conservative", scheme="rosenbrock")
    b = P.residual(u0)
    tau = 7.3
    beta = tau * P.norm_inf_A(u0)
    assert beta > 15
    s = int(math.ceil(beta / 2.0))
    m = 6
    exact, _, _ = P.phi1_action(u0, b, tau)
    got_multi = multinomial.phi1_action(P, u0, b, tau, s, m)
    x = np.zeros(D.shape)
    h = tau / s
    for _ in range(s):
        term, acc, a = x.copy(), x.copy(), 1.0
        for j in range(1, m + 1):
            term = (h / j) * (P.apply_A(u0, term) + b * a)
            a = 0.0
            acc += term
        x = acc
    err_seq = _rel(x, exact)
    err_multi = _rel(got_multi, exact)
    assert err_multi > 100 * err_seq, (err_multi, err_seq)


def test_schedule_refinement_does_not_move_result():
    D, u0 = phantom.case(12, seed=8, noise=0.1)
    P = oracle.Problem(D, op="literal", scheme="rosenbrock")
    a, _ = P.run(u0, 7.3, 2, theta=0.5)
    b, _ = P.run(u0, 7.3, 2, theta=0.2)
    assert _rel(a, b) <= 1e-14
