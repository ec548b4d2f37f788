"""Crank-Nicolson step of Sec. 2.3, the paper's comparison method (plain FP64).

TEST INFRASTRUCTURE ONLY: used by the test suite and the benchmark's CPU
baseline; the product library never imports it.

The printed scheme drops u^t from the right-hand side and flips the sign of
the implicit term; read as the standard trapezoidal rule on the same
linearised system as the exponential step (u' = A_n u + f_n, A_n and f_n as in
Sec. 2.1 with the scheme's reaction treatment):

    (I - tau/2 A_n) u^{n+1} = (I + tau/2 A_n) u^n + tau f_n .

A_n comes from the oracle's own row entries (oracle_row_A, every voxel in
one call), assembled into a sparse matrix; the linear system is solved by a
sparse direct factorisation (scipy's SuperLU) up to 2^18 voxels and by
conjugate gradients to a relative residual of 1e-14 beyond (the conservative
operator makes I - tau/2 A_n symmetric positive definite for tau rho < 2).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse
import scipy.sparse.linalg

DIRECT_MAX = 1 << 18


def assemble_A(P, un) -> scipy.sparse.csr_matrix:
    """A_n of the problem at state un as an n x n sparse matrix."""
    nz, ny, nx = P.shape
    n = nx * ny * nz
    e = P.rows_A(un)
    p = np.arange(n)
    i = p % nx
    j = (p // nx) % ny
    k = p // (nx * ny)
    rows, cols, vals = [p], [p], [e[:, 0]]
    # off-diagonals: -x, +x, -y, +y, -z, +z
    for q, (ok, off) in enumerate([(i > 0, -1), (i + 1 < nx, 1), (j > 0, -nx), (j + 1 < ny, nx),
                                   (k > 0, -nx * ny), (k + 1 < nz, nx * ny)]):
        rows.append(p[ok])
        cols.append(p[ok] + off)
        vals.append(e[ok, q + 1])
    return scipy.sparse.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                                   shape=(n, n))


def f_of(P, u):
    """f_n: rho u^2 where rho(1 - 2u) is folded into A_n, else rho u (1 - u)."""
    if P.scheme == "rosenbrock":
        return P.rho * u * u
    return P.rho * u * (1.0 - u)


def cn_step(P, u, tau):
    """u^{n+1} from u^n by one Crank-Nicolson step; returns (u^{n+1}, solver iterations or 0)."""
    un = np.ascontiguousarray(u, dtype=np.float64).reshape(P.shape)
    v = un.ravel()
    A = assemble_A(P, un)
    n = v.size
    M = (scipy.sparse.identity(n, format="csr") - 0.5 * tau * A).tocsc()
    rhs = v + 0.5 * tau * (A @ v) + tau * f_of(P, v)
    if n <= DIRECT_MAX:
        x = scipy.sparse.linalg.spsolve(M, rhs)
        return x.reshape(P.shape), 0
    count = [0]

    def cb(_):
        count[0] += 1

    x, info = scipy.sparse.linalg.cg(M.tocsr(), rhs, x0=v, rtol=1e-14, atol=0.0, maxiter=10000, callback=cb)
    if info != 0:
        raise RuntimeError(f"conjugate gradients did not converge ({info})")
    return x.reshape(P.shape), count[0]


def cn_run(P, u0, tau, nsteps, every=False):
    """nsteps Crank-Nicolson steps from u0; returns u^K or, with every=True, [u^0 .. u^K]."""
    u = np.array(u0, dtype=np.float64).reshape(P.shape)
    states = [u.copy()] if every else None
    for _ in range(nsteps):
        u, _ = cn_step(P, u, tau)
        if every:
            states.append(u.copy())
    return states if every else u
