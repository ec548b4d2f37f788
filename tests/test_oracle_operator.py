"""Pins of the oracle's spatial operator (Sec. 2.1) against the paper's matrix and
against properties of the mathematics.  CPU only."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2402_02273_gb300 import phantom

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _random_D(shape, seed, zero_frac=0.0):
    u = phantom.uniform(seed, 7, int(np.prod(shape))).reshape(shape)
    D = (0.01 + 0.2 * u).astype(np.float32).astype(np.float64)
    if zero_frac:
        z = phantom.uniform(seed, 8, D.size).reshape(shape) < zero_frac
        D[z] = 0.0
    return D


def _dense(P, un):
    """Dense matrix of the oracle's matrix-free operator, column by column."""
    n = P.D.size
    A = np.zeros((n, n))
    for q in range(n):
        e = np.zeros(n)
        e[q] = 1.0
        A[:, q] = P.apply_A(un, e).ravel()
    return A


def _amatrix_literal(D, h, c=None):
    """Dense h^-2 * (eq. Amatrix) assembled in the test from the paper's entry table,
    with the zero-flux reading: entries that point outside the box are dropped and
    the diagonal keeps only the kept neighbours' share."""
    nz, ny, nx = D.shape
    n = D.size
    A = np.zeros((n, n))
    idx = lambda i, j, k: i + nx * (j + ny * k)
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                p = idx(i, j, k)
                Dp = D[k, j, i]
                for (di, dj, dk), ext, co in (((1, 0, 0), nx, i), ((0, 1, 0), ny, j), ((0, 0, 1), nz, k)):
                    if co + 1 < ext:
                        q = idx(i + di, j + dj, k + dk)
                        Dq = D[k + dk, j + dj, i + di]
                        A[p, q] += Dp + Dq      # D_ijk and D_{i+1,j,k} entries
                        A[p, p] -= Dp + Dq
                    if co > 0:
                        q = idx(i - di, j - dj, k - dk)
                        A[p, q] += 2 * Dp      # 2 D_ijk entry
                        A[p, p] -= 2 * Dp
    A /= h * h
    if c is not None:
        A[np.diag_indices(n)] += c.ravel()
    return A


def _flux_conservative(D, h):
    """Dense div(D grad .) with harmonic-mean faces, assembled face by face."""
    nz, ny, nx = D.shape
    n = D.size
    A = np.zeros((n, n))
    idx = lambda i, j, k: i + nx * (j + ny * k)
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                for (di, dj, dk), ext, co in (((1, 0, 0), nx, i), ((0, 1, 0), ny, j), ((0, 0, 1), nz, k)):
                    if co + 1 < ext:
                        p, q = idx(i, j, k), idx(i + di, j + dj, k + dk)
                        a, b = D[k, j, i], D[k + dk, j + dj, i + di]
                        w = 0.0 if a == 0 or b == 0 else 2 * a * b / (a + b)
                        # one face, flux leaves p and enters q
                        A[p, q] += w
                        A[q, p] += w
                        A[p, p] -= w
                        A[q, q] -= w
    return A / (h * h)


def test_interior_row_matches_printed_amatrix():
    spec = json.load(open(os.path.join(GOLDEN, "amatrix_stencil.json")))
    D = _random_D((5, 5, 5), 3)
    h = 0.7
    P = oracle.Problem(D, h=h, op="literal", scheme="expeuler")
    un = np.zeros_like(D)
    i = j = k = 2
    p = i + 5 * (j + 5 * k)
    vars_ = np.array([D[k, j, i], D[k, j, i + 1], D[k, j + 1, i], D[k + 1, j, i]])
    row = P.row_A(un, p)
    names = ["centre", "minus_x", "plus_x", "minus_y", "plus_y", "minus_z", "plus_z"]
    for col, name in enumerate(names):
        want = np.dot(spec["entries"][name], vars_) / h ** 2
        assert row[col] == pytest.approx(want, rel=1e-15, abs=1e-15), name


@pytest.mark.parametrize("shape", [(4, 4, 4), (3, 5, 6), (1, 1, 7), (2, 1, 1)])
def test_literal_matrix_free_equals_assembled_amatrix(shape):
    D = _random_D(shape, 11, zero_frac=0.2)
    u = phantom.uniform(5, 1, D.size).reshape(shape)
    for scheme in ("expeuler", "rosenbrock"):
        P = oracle.Problem(D, h=1.3, rho=0.05, op="literal", scheme=scheme)
        c = None if scheme == "expeuler" else 0.05 * (1 - 2 * u)
        want = _amatrix_literal(D, 1.3, c)
        got = _dense(P, u)
        assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()


@pytest.mark.parametrize("shape", [(4, 4, 4), (3, 5, 6), (1, 1, 7)])
def test_conservative_matrix_free_equals_face_assembly(shape):
    D = _random_D(shape, 12, zero_frac=0.2)
    P = oracle.Problem(D, h=0.9, op="conservative", scheme="expeuler")
    want = _flux_conservative(D, 0.9)
    got = _dense(P, np.zeros(shape))
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()


@pytest.mark.parametrize("op", ["conservative", "literal"])
def test_rows_sum_to_zero_and_dense_rows_match(op):
    D = _random_D((4, 5, 3), 13, zero_frac=0.3)
    P = oracle.Problem(D, op=op, scheme="expeuler")
    A = _dense(P, np.zeros(D.shape))
    assert np.abs(A.sum(axis=1)).max() <= 1e-15 * np.abs(A).max() * 8
    # oracle_row_A lists the same entries as the dense matrix
    nz, ny, nx = D.shape
    for p in range(D.size):
        e = P.row_A(np.zeros(D.shape), p)
        assert e[0] == pytest.approx(A[p, p], abs=1e-15)
        assert np.sum(np.abs(e[1:])) == pytest.approx(np.sum(np.abs(A[p])) - abs(A[p, p]), abs=1e-14)
    # norm bound is the largest absolute row sum
    assert P.norm_inf_A(np.zeros(D.shape)) == pytest.approx(np.abs(A).sum(axis=1).max(), rel=1e-14)


def test_conservative_is_symmetric_and_conserves():
    D = _random_D((5, 4, 4), 14, zero_frac=0.2)
    A = _dense(oracle.Problem(D, op="conservative", scheme="expeuler"), np.zeros(D.shape))
    assert np.abs(A - A.T).max() <= 1e-15 * np.abs(A).max()
    assert np.abs(A.sum(axis=0)).max() <= 1e-14 * np.abs(A).max()


def test_literal_does_not_conserve_for_variable_D():
    # Reading A1: the printed operator is not in divergence form; its column sums
    # differ from zero when D varies, so the pure-diffusion step changes the mass.
    D = _random_D((5, 4, 4), 15)
    A = _dense(oracle.Problem(D, op="literal", scheme="expeuler"), np.zeros(D.shape))
    assert np.abs(A.sum(axis=0)).max() > 1e-3 * np.abs(A).max()
    assert np.abs(A - A.T).max() > 1e-3 * np.abs(A).max()


def test_constant_D_literal_is_twice_conservative():
    D = np.full((4, 3, 5), 0.13)
    Al = _dense(oracle.Problem(D, op="literal", scheme="expeuler"), np.zeros(D.shape))
    Ac = _dense(oracle.Problem(D, op="conservative", scheme="expeuler"), np.zeros(D.shape))
    assert np.abs(Al - 2 * Ac).max() <= 1e-15


def test_air_voxels_exchange_nothing_conservative():
    D = _random_D((4, 4, 4), 16)
    D[1:3, 1:3, 1:3] = 0.0
    A = _dense(oracle.Problem(D, op="conservative", scheme="expeuler"), np.zeros(D.shape))
    air = np.flatnonzero(D.ravel() == 0)
    assert np.all(A[air] == 0) and np.all(A[:, air] == 0)


def test_folded_reaction_gives_same_residual():
    # eq. F: rho u (1 - u) = rho (1 - 2u) u + rho u^2, so both schemes share b.
    D, u0 = phantom.case(12, seed=2, noise=0.1)
    Pr = oracle.Problem(D, op="conservative", scheme="rosenbrock")
    Pe = oracle.Problem(D, op="conservative", scheme="expeuler")
    br, be = Pr.residual(u0), Pe.residual(u0)
    direct = Pe.apply_L(u0) + 0.025 * u0 * (1 - u0)
    assert np.abs(br - be).max() <= 1e-16
    assert np.abs(be - direct).max() <= 1e-17
    # and the folded diagonal is rho (1 - 2 u^n)
    v = phantom.uniform(3, 3, D.size).reshape(D.shape)
    diff = Pr.apply_A(u0, v) - Pe.apply_A(u0, v)
    assert np.abs(diff - 0.025 * (1 - 2 * u0) * v).max() <= 1e-16
