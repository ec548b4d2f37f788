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
