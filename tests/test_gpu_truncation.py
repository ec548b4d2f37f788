"""The device-side a-posteriori truncation estimate of a step (Sec. 2.2: the
Taylor series of each sub-step is cut after m terms).  The residual launch
reduces max|b| and max|u^n| on the device; the stats launch evaluates
est = C(s, m) max|b| / max|u^n| and flags ET_FLAG_TRUNCATION above the
tolerance.  Checked here against the same quantity formed on the host from the
oracle's residual of the state before the step, with C written out from the
bound in include/et.h; a schedule forced too short is flagged, the library's
own schedules are not.  GPU only."""
import math

import numpy as np
import pytest

import oracle
from paper_2402_02273_gb300 import phantom

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2402_02273_gb300 as et
    et.load()
    return et, torch


def _factor(tau, rmax, rho, scheme, s, m, shift=True):
    """C of the estimate: tau e^{2 tau rho'} theta^m / m! (1 + beta/(m+1)) / (1 - theta/(m+1))."""
    rho_c = rho * (1 + 2e-3) if scheme == "rosenbrock" else 0.0
    nu = rmax + rho_c if shift else 2 * rmax + rho_c
    beta = tau * nu
    theta = beta / s
    if theta >= m + 1:
        return math.inf
    return (tau * math.exp(2 * tau * rho_c) * theta ** m / math.factorial(m) * (1 + beta / (m + 1))
            / (1 - theta / (m + 1)))


@pytest.mark.parametrize("precision", ["f64", "df64", "f32"])
@pytest.mark.parametrize("op,scheme", [("conservative", "rosenbrock"), ("literal", "expeuler")])
def test_estimate_matches_host_bound_with_oracle_residual(env, precision, op, scheme):
    et, torch = env
    D, u0 = phantom.case((20, 18, 24), seed=3, noise=0.1)
    tau, rho, nsteps = 7.3, 0.025, 3
    g = et.Grid(D.shape, precision=precision)
    g.set_coeffs(torch.from_numpy(D).cuda(), rho=rho, op=op, scheme=scheme)
    u = torch.from_numpy(u0.copy()).cuda()
    g.run(u, tau, nsteps)
    rec = g.sync_info()
    est = g.truncation()
    # the state before the last step, from the oracle (parity 1e-10 / 1e-5)
    P = oracle.Problem(D, rho=rho, op=op, scheme=scheme)
    states, _ = P.run(u0, tau, nsteps, every=True)
    un = states[nsteps - 1]
    b = P.residual(un)
    s, m, _, _ = g.schedule(tau)
    want = _factor(tau, g.rmax(), rho, scheme, s, m) * np.abs(b).max() / np.abs(un).max()
    tol_rel = 1e-9 if precision == "f64" else 1e-5
    assert est == pytest.approx(want, rel=tol_rel)
    assert est <= (1e-7 if precision == "f32" else 1e-13)
    assert not rec["flags"] & et.ET_FLAG_TRUNCATION


@pytest.mark.parametrize("precision", ["f64", "df64", "f32"])
def test_schedule_forced_too_short_is_flagged(env, precision):
    et, torch = env
    D, u0 = phantom.case((16, 16, 16), seed=4, noise=0.1)
    g = et.Grid(D.shape, precision=precision)
    # theta ~ 1.6 per sub-step: a sixth-degree polynomial is far from the
    # tolerance, yet close enough that u stays in [0, 1]
    g.set_coeffs(torch.from_numpy(D).cuda(), force_s=4, force_m=6)
    u = torch.from_numpy(u0.copy()).cuda()
    g.run(u, 7.3, 2)
    rec = g.sync_info()  # informational: no error status
    assert rec["flags"] & et.ET_FLAG_TRUNCATION
    assert g.truncation() > 1e-6
    # the library's own schedule on the same grid: no flag
    g.set_coeffs(torch.from_numpy(D).cuda())
    u = torch.from_numpy(u0.copy()).cuda()
    g.run(u, 7.3, 2)
    rec = g.sync_info()
    assert not rec["flags"] & et.ET_FLAG_TRUNCATION


def test_batched_estimate_flags_only_the_short_schedules(env):
    """Batched form: every grid's stats launch evaluates its own estimate."""
    et, torch = env
    shapes = [(12, 10, 16), (9, 14, 20)]
    cases = [phantom.case(sh, seed=30 + i, noise=0.1) for i, sh in enumerate(shapes)]
    D = torch.from_numpy(np.concatenate([c[0].ravel() for c in cases])).cuda()
    u0 = np.concatenate([c[1].ravel() for c in cases])
    B = et.Batch(shapes)
    B.set_coeffs(D, [0.025, 0.025], force_s=4, force_m=5)
    u = torch.from_numpy(u0.copy()).cuda()
    B.run(u, 7.3, 2)
    recs = B.sync_info()
    assert all(r["flags"] & et.ET_FLAG_TRUNCATION for r in recs)
    B.set_coeffs(D, [0.025, 0.025])
    u = torch.from_numpy(u0.copy()).cuda()
    B.run(u, 7.3, 2)
    recs = B.sync_info()
    assert not any(r["flags"] & et.ET_FLAG_TRUNCATION for r in recs)
