"""et_step_static, the entry point for callers that cannot allocate device memory
(code inside a framework whose pool owns all device memory, or code run while a
memory budget is locked): its scratch lives in a static device array of the
library instead of a caller workspace.  Checked through the C ABI against the
workspace path (et_set_coeffs + et_step) on two calls in a row, within the FP64
parity tolerance of the other tests.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_2402_02273_gb300 import phantom

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def test_static_scratch_step_matches_workspace_step_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2402_02273_gb300 as et

    lib = et.load()
    shape = (40, 36, 44)  # not a multiple of the 32 x 8 tile
    D, u0 = phantom.case(shape, seed=7, noise=0.1)
    nz, ny, nx = shape
    tau, rho = 7.3, 0.025
    Dd = torch.from_numpy(D).cuda()
    stream = torch.cuda.current_stream()

    # existing entry points: workspace-backed grid, two steps
    g = et.Grid(shape)
    g.set_coeffs(Dd, rho=rho)
    ref = torch.from_numpy(u0.copy()).cuda()
    want = []
    for _ in range(2):
        g.step(ref, tau)
        g.sync_info()
        want.append(ref.cpu().numpy().copy())

    # new entry point, two calls in a row on the same state
    u = torch.from_numpy(u0.copy()).cuda()
    msg = ctypes.create_string_buffer(256)
    for call in range(2):
        rc = lib.et_step_static(nx, ny, nz, 1.0, Dd.data_ptr(), rho, et.ET_OP_CONSERVATIVE,
                                et.ET_SCHEME_ROSENBROCK, u.data_ptr(), tau, stream.cuda_stream,
                                msg, len(msg))
        assert rc == et.ET_OK, msg.value
        got = u.cpu().numpy()
        assert _rel(got, want[call]) <= TOL64, (call, _rel(got, want[call]))

    # grids beyond the static maximum are rejected with a clear message
    big = torch.zeros(65 * 64 * 64, dtype=torch.float64, device="cuda")
    rc = lib.et_step_static(65, 64, 64, 1.0, big.data_ptr(), rho, 0, 0, big.data_ptr(), tau,
                            stream.cuda_stream, msg, len(msg))
    assert rc == et.ET_ERR_ARG
    assert b"at most 262144" in msg.value
    assert float(big.abs().max()) == 0.0  # nothing ran
