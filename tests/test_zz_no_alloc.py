"""et_step_static, the entry point for callers that cannot allocate device memory
(code inside a framework whose pool owns all device memory, or code run while a
memory budget is locked): its scratch lives in a static device array of the
library instead of a caller workspace.  Checked through the C ABI against the
workspace path (et_set_coeffs + et_step) and against the FP64 oracle, on two
calls in a row, within the FP64 parity tolerance of the other tests, for both
operators and both schemes.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2402_02273_gb300 import phantom

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
OPS = {"conservative": 0, "literal": 1}
SCHEMES = {"rosenbrock": 0, "expeuler": 1}


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("op", list(OPS))
@pytest.mark.parametrize("scheme", list(SCHEMES))
def test_static_scratch_step_matches_workspace_step_and_oracle_twice(torch_cuda, op, scheme):
    torch = torch_cuda
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
    g.set_coeffs(Dd, rho=rho, op=op, scheme=scheme)
    ref = torch.from_numpy(u0.copy()).cuda()
    want = []
    for _ in range(2):
        g.step(ref, tau)
        g.sync_info()
        want.append(ref.cpu().numpy().copy())
    exact, _ = oracle.Problem(D, rho=rho, op=op, scheme=scheme).run(u0, tau, 2, every=True)

    # new entry point, two calls in a row on the same state
    u = torch.from_numpy(u0.copy()).cuda()
    msg = ctypes.create_string_buffer(256)
    for call in range(2):
        rc = lib.et_step_static(nx, ny, nz, 1.0, Dd.data_ptr(), rho, OPS[op], SCHEMES[scheme],
                                u.data_ptr(), tau, stream.cuda_stream, msg, len(msg))
        assert rc == et.ET_OK, msg.value
        got = u.cpu().numpy()
        assert _rel(got, want[call]) <= TOL64, (call, _rel(got, want[call]))
        assert _rel(got, exact[call + 1]) <= TOL64, (call, _rel(got, exact[call + 1]))


def test_static_scratch_step_rejects_grids_beyond_its_limits(torch_cuda):
    torch = torch_cuda
    import paper_2402_02273_gb300 as et

    lib = et.load()
    stream = torch.cuda.current_stream()
    msg = ctypes.create_string_buffer(256)
    tau, rho = 7.3, 0.025
    # more voxels than the static array holds
    big = torch.zeros(65 * 64 * 64, dtype=torch.float64, device="cuda")
    rc = lib.et_step_static(65, 64, 64, 1.0, big.data_ptr(), rho, 0, 0, big.data_ptr(), tau,
                            stream.cuda_stream, msg, len(msg))
    assert rc == et.ET_ERR_ARG
    assert b"at most 262144" in msg.value
    assert float(big.abs().max()) == 0.0  # nothing ran
    # few enough voxels and blocks, but a z extent no launch can have
    col = torch.zeros(65536, dtype=torch.float64, device="cuda")
    rc = lib.et_step_static(1, 1, 65536, 1.0, col.data_ptr(), rho, 0, 0, col.data_ptr(), tau,
                            stream.cuda_stream, msg, len(msg))
    assert rc == et.ET_ERR_ARG
    assert b"nz = 65536 exceeds 65535" in msg.value
    assert float(col.abs().max()) == 0.0
