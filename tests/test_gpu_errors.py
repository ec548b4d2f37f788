"""Error statuses of the C ABI on a GPU: misuse and bad data are reported, never
faulted.  Bad data is planted on the host (negative D, NaN, out-of-range u)."""
import ctypes

import numpy as np
import pytest

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


def test_step_before_coeffs_is_a_state_error(env):
    et, torch = env
    g = et.Grid((4, 4, 4))
    u = torch.zeros(64, dtype=torch.float64, device="cuda")
    with pytest.raises(et.EtError) as ex:
        g.step(u, 1.0)
    assert ex.value.status == et.ET_ERR_STATE


def test_bad_D_is_a_numeric_error(env):
    et, torch = env
    g = et.Grid((4, 5, 6))
    D = np.full((4, 5, 6), 0.1)
    D[1, 2, 3] = -0.5
    with pytest.raises(et.EtError) as ex:
        g.set_coeffs(torch.from_numpy(D).cuda())
    assert ex.value.status == et.ET_ERR_NUMERIC
    D[1, 2, 3] = np.nan
    with pytest.raises(et.EtError) as ex:
        g.set_coeffs(torch.from_numpy(D).cuda())
    assert ex.value.status == et.ET_ERR_NUMERIC
    D[1, 2, 3] = 0.1
    g.set_coeffs(torch.from_numpy(D).cuda())  # recovers


def test_bad_arguments(env):
    et, torch = env
    g = et.Grid((4, 4, 4))
    g.set_coeffs(torch.full((64,), 0.1, dtype=torch.float64, device="cuda"))
    u = torch.zeros(64, dtype=torch.float64, device="cuda")
    for tau in (0.0, -1.0, float("inf"), float("nan")):
        with pytest.raises(et.EtError) as ex:
            g.step(u, tau)
        assert ex.value.status == et.ET_ERR_ARG
    with pytest.raises(et.EtError):
        g.run(u, 1.0, 0)
    lib = et.load()
    assert lib.et_step(g.handle, u.data_ptr() + 4, 1.0, None) == et.ET_ERR_ARG  # misaligned
    assert lib.et_set_coeffs(g.handle, u.data_ptr(), -1.0, 0, 0, None) == et.ET_ERR_ARG
    assert lib.et_set_coeffs(g.handle, u.data_ptr(), 0.1, 9, 0, None) == et.ET_ERR_ARG
    with pytest.raises(et.EtError):
        g.set_coeffs(torch.zeros(63, dtype=torch.float64, device="cuda"))
    # workspace too small
    ws = torch.empty(1024, dtype=torch.uint8, device="cuda")
    h = ctypes.c_void_p()
    assert lib.et_create_grid(64, 64, 64, 1.0, 0, (ws.data_ptr() + 255) // 256 * 256, 512, None,
                              ctypes.byref(h)) == et.ET_ERR_ARG


def test_nonfinite_and_out_of_range_density_are_flagged(env):
    et, torch = env
    D, u0 = phantom.case(16, seed=1)
    g = et.Grid(D.shape)
    g.set_coeffs(torch.from_numpy(D).cuda())
    bad = u0.copy()
    bad[3, 4, 5] = np.nan
    u = torch.from_numpy(bad).cuda()
    g.step(u, 7.3)
    with pytest.raises(et.EtError) as ex:
        g.sync_info()
    assert ex.value.status == et.ET_ERR_NUMERIC
    g.sync_info()  # flags were cleared
    over = u0.copy()
    over[8, 8, 8] = 1.5
    u = torch.from_numpy(over).cuda()
    g.step(u, 7.3)
    with pytest.raises(et.EtError) as ex:
        g.sync_info()
    assert "outside" in str(ex.value)
    # the exponential-Euler scheme makes no range assumption
    g.set_coeffs(torch.from_numpy(D).cuda(), scheme="expeuler")
    u = torch.from_numpy(over).cuda()
    g.step(u, 7.3)
    g.sync_info()
    # host path reports the same way
    g.set_coeffs(torch.from_numpy(D).cuda())
    with pytest.raises(et.EtError):
        g.run_host(over.copy(), 7.3, 2)


@pytest.mark.parametrize("precision,use_graph", [("f32", True), ("df64", True), ("df64", False)])
def test_bounded_wait_that_runs_out_reports_timeout(env, precision, use_graph):
    """The two-term kernel's bounded waits: with the test hook on, every block
    first waits 200 us on a device barrier that nothing completes; the wait runs
    out, the block lets its copies in flight land and stops, and the run reports
    ET_ERR_TIMEOUT.  The context stays usable: the same grid then runs without
    the hook and matches the oracle.  Two sub-steps, so that the FP32 chain
    has running-sum pairs, which take the TMA-fed kernel (its Horner pairs run
    on the four-voxel two-term kernel, which has no waits)."""
    import oracle
    et, torch = env
    shape = (12, 16, 32)  # rows of 32 voxels: TMA-eligible in both forms
    D, u0 = phantom.case(shape, seed=5, noise=0.1)
    Dd = torch.from_numpy(D).cuda()
    g = et.Grid(shape, precision=precision)
    g.set_coeffs(Dd, two_terms=True, timeout_probe_us=200, use_graph=use_graph, force_s=2)
    u = torch.from_numpy(u0.copy()).cuda()
    g.run(u, 7.3, 2)
    with pytest.raises(et.EtError) as ex:
        g.sync_info()
    assert ex.value.status == et.ET_ERR_TIMEOUT
    assert "wait ran out" in str(ex.value)
    g.sync_info()  # the flag was cleared by the failing sync
    g.set_coeffs(Dd, two_terms=True, use_graph=use_graph, force_s=2)
    u = torch.from_numpy(u0.copy()).cuda()
    g.run(u, 7.3, 2)
    g.sync_info()
    want, _ = oracle.Problem(D).run(u0, 7.3, 2)
    got = u.cpu().numpy().reshape(shape)
    tol = 1e-5 if precision == "f32" else 1e-10
    assert np.abs(got - want).max() <= tol * np.abs(want).max()


def test_bounded_wait_that_runs_out_reports_timeout_batched(env):
    """The same hook on the batched TMA-fed two-term kernel (DF64, a two-term
    variant, two sub-steps: its Horner pairs take the vector kernel, which has
    no waits, its running-sum pairs the TMA-fed one)."""
    import oracle
    et, torch = env
    shapes = [(8, 16, 32), (10, 8, 16)]
    cases = [phantom.case(sh, seed=20 + i, noise=0.1) for i, sh in enumerate(shapes)]
    D = torch.from_numpy(np.concatenate([c[0].ravel() for c in cases])).cuda()
    u0 = np.concatenate([c[1].ravel() for c in cases])
    b = et.Batch(shapes, precision="df64")
    b.set_coeffs(D, 0.025, timeout_probe_us=200, force_s=2)
    b.set_variant(0)  # the first half of the variants launch two terms at a time
    u = torch.from_numpy(u0.copy()).cuda()
    b.run(u, 7.3, 2)
    with pytest.raises(et.EtError) as ex:
        b.sync_info()
    assert ex.value.status == et.ET_ERR_TIMEOUT
    b.set_coeffs(D, 0.025, force_s=2)
    b.set_variant(0)
    u = torch.from_numpy(u0.copy()).cuda()
    b.run(u, 7.3, 2)
    b.sync_info()
    for i, (Di, ui) in enumerate(cases):
        want, _ = oracle.Problem(Di).run(ui, 7.3, 2)
        got = b.split(u)[i].cpu().numpy()
        assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()


def test_timeout_probe_option_is_range_checked(env):
    et, torch = env
    g = et.Grid((4, 4, 8), precision="f32")
    D = torch.full((128,), 0.1, dtype=torch.float64, device="cuda")
    for bad in (-1, 1000001):
        with pytest.raises(et.EtError) as ex:
            g.set_coeffs(D, timeout_probe_us=bad)
        assert ex.value.status == et.ET_ERR_ARG
