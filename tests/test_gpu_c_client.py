"""The C ABI from a plain C program (tests/c_client/et_client.c, built with
gcc against include/et.h, libet.so and the CUDA runtime): the same steps as
through the Python binding, bitwise.  GPU only."""
import os
import shutil
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def client(tmp_path_factory):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2402_02273_gb300 as et
    et.load()
    lib = et.library_path()
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("no C compiler")
    out = tmp_path_factory.mktemp("c_client") / "et_client"
    libdir = os.path.dirname(lib)
    cmd = [gcc, "-O2", "-std=c11", os.path.join(HERE, "c_client", "et_client.c"), "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(cuda, "include"), lib, "-L", os.path.join(cuda, "lib64"), "-lcudart",
           "-Wl,-rpath," + libdir, "-Wl,-rpath," + os.path.join(cuda, "lib64"), "-o", str(out)]
    subprocess.run(cmd, check=True)
    return str(out)


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_c_client_matches_python_binding(client, tmp_path, precision):
    import torch
    import paper_2402_02273_gb300 as et
    nx, ny, nz, nsteps = 36, 20, 17, 3
    res = tmp_path / "out.bin"
    subprocess.run([client, str(nx), str(ny), str(nz), str(nsteps), str(precision), str(res)], check=True)
    data = np.fromfile(res, dtype=np.float64)
    u_c, tail = data[:-5].reshape(nz, ny, nx), data[-5:]
    # the same problem through the Python binding
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    d2 = (i - 0.5 * (nx - 1)) ** 2 + (j - 0.5 * (ny - 1)) ** 2 + (k - 0.5 * (nz - 1)) ** 2
    r = 0.45 * min(nx, ny, nz)
    D = np.where(d2 < 0.36 * r * r, 0.13, np.where(d2 < r * r, 0.013, 0.0))
    u0 = np.where(d2 < 4.0, 0.8, 0.0)
    g = et.Grid((nz, ny, nx), precision={0: "f64", 1: "f32", 2: "df64"}[precision])
    g.set_coeffs(torch.from_numpy(D).cuda(), rho=0.025)
    u = torch.from_numpy(u0.copy()).cuda()
    g.run(u, 7.3, nsteps)
    rec = g.sync_info()
    assert np.array_equal(u.cpu().numpy().reshape(nz, ny, nx), u_c)
    assert tail[0] == rec["mass"] and (int(tail[3]), int(tail[4])) == (rec["s"], rec["m"])
