"""Crank-Nicolson steps on the GPU (Sec. 2.3, the paper's comparison method):
matrix-free conjugate gradients in FP64 against the oracle's sparse solve of
the same step, element by element, every step.  Tolerance 1e-10 relative (max
and L2 norms) with the solve converged to rtol 1e-13.  GPU only."""
import numpy as np
import pytest

import oracle
from oracle import cn
from paper_2402_02273_gb300 import phantom

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2402_02273_gb300 as et
    et.load()
    return et, torch


def _errs(got, want):
    return (np.abs(got - want).max() / np.abs(want).max(),
            np.linalg.norm((got - want).ravel()) / np.linalg.norm(want.ravel()))


def _gpu_states(et, torch, D, u0, tau, nsteps, rtol=1e-13, scheme="rosenbrock", rho=0.025, **opts):
    g = et.Grid(D.shape)
    g.set_coeffs(torch.from_numpy(D.copy()).cuda(), rho=rho, scheme=scheme, **opts)
    u = torch.from_numpy(u0.copy()).cuda()
    states, recs = [], []
    for _ in range(nsteps):
        g.cn_run(u, tau, 1, rtol=rtol)
        recs.append(g.sync_info())
        states.append(u.cpu().numpy().reshape(D.shape).copy())
    return g, states, recs


@pytest.mark.parametrize("scheme", ["rosenbrock", "expeuler"])
@pytest.mark.parametrize("shape", [(32, 32, 32), (20, 18, 37), (1, 5, 70), (9, 1, 1)])
def test_cn_steps_match_oracle_every_step(env, scheme, shape):
    et, torch = env
    D, u0 = phantom.case(shape, seed=11, noise=0.1)
    if not np.any(u0 > 0.1):
        u0 = np.zeros(shape)
        u0.reshape(-1)[u0.size // 2] = 0.8
    tau, nsteps = 7.3, 5
    P = oracle.Problem(D, rho=0.025, op="conservative", scheme=scheme)
    want = cn.cn_run(P, u0, tau, nsteps, every=True)
    g, got, recs = _gpu_states(et, torch, D, u0, tau, nsteps, scheme=scheme)
    cap = g.cn_iteration_cap(tau, 1e-13)
    for t in range(nsteps):
        e_max, e_l2 = _errs(got[t], want[t + 1])
        assert e_max <= TOL and e_l2 <= TOL, (t, e_max, e_l2)
        assert recs[t]["s"] == 0 and 0 < recs[t]["m"] <= cap
        assert recs[t]["mass"] == pytest.approx(want[t + 1].sum(), rel=1e-12)


def test_run_graph_and_direct_launches_agree_bitwise(env):
    et, torch = env
    D, u0 = phantom.case(24, seed=12, noise=0.1)
    outs = []
    for use_graph in (True, False):
        g = et.Grid(D.shape)
        g.set_coeffs(torch.from_numpy(D).cuda(), use_graph=use_graph)
        u = torch.from_numpy(u0.copy()).cuda()
        info = g.info_buffer(4)
        g.cn_run(u, 7.3, 4, info=info)
        g.sync_info()
        recs = g.decode_info(info)
        outs.append((u.cpu().numpy(), recs["m"].copy()))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])
    # a second run replays the captured step
    g = et.Grid(D.shape)
    g.set_coeffs(torch.from_numpy(D).cuda())
    u = torch.from_numpy(u0.copy()).cuda()
    g.cn_run(u, 7.3, 2)
    g.cn_run(u, 7.3, 2)
    g.sync_info()
    assert np.array_equal(u.cpu().numpy(), outs[0][0])


def test_full_size_128cubed_first_steps_match_oracle(env):
    """The 128^3 bench grid, three steps against the oracle (conjugate gradients
    in the oracle too at this size, to 1e-14)."""
    et, torch = env
    D, u0 = phantom.case(128, seed=0, noise=0.1)
    P = oracle.Problem(D, rho=0.025)
    want = cn.cn_run(P, u0, 7.3, 3, every=True)
    _, got, recs = _gpu_states(et, torch, D, u0, 7.3, 3)
    for t in range(3):
        e_max, e_l2 = _errs(got[t], want[t + 1])
        assert e_max <= TOL and e_l2 <= TOL, (t, e_max, e_l2)
    print("128^3 CN iterations per step:", [r["m"] for r in recs])


def test_cn_errors_are_reported(env):
    et, torch = env
    D, u0 = phantom.case(16, seed=13, noise=0.1)
    Dd = torch.from_numpy(D).cuda()
    u = torch.from_numpy(u0.copy()).cuda()
    g = et.Grid(D.shape)
    g.set_coeffs(Dd, op="literal")
    with pytest.raises(et.EtError) as ex:
        g.cn_run(u, 7.3, 1)
    assert ex.value.status == et.ET_ERR_UNSUPPORTED
    g32 = et.Grid(D.shape, precision="f32")
    g32.set_coeffs(Dd)
    with pytest.raises(et.EtError) as ex:
        g32.cn_run(u, 7.3, 1)
    assert ex.value.status == et.ET_ERR_UNSUPPORTED
    g.set_coeffs(Dd, rho=0.5)
    with pytest.raises(et.EtError) as ex:
        g.cn_run(u, 7.3, 1)  # tau rho = 3.65: I - tau/2 A may be indefinite
    assert ex.value.status == et.ET_ERR_ARG
    g.set_coeffs(Dd)
    for bad in (0.0, 1.0, float("nan")):
        with pytest.raises(et.EtError) as ex:
            g.cn_run(u, 7.3, 1, rtol=bad)
        assert ex.value.status == et.ET_ERR_ARG
    # a cap far below what the tolerance needs: flagged, reported as numeric
    g.cn_run(u, 7.3, 1, rtol=1e-13, max_iter=2)
    with pytest.raises(et.EtError) as ex:
        g.sync_info()
    assert ex.value.status == et.ET_ERR_NUMERIC
    assert "iteration cap" in str(ex.value)
