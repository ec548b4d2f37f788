"""GB300 exponential-integrator library for the Fisher-Kolmogorov tumour model.

Thin ctypes binding over the C ABI of include/et.h (libet.so, built from
csrc/ by build.py).  Every function of the ABI is exposed under its own name
(`et_create_grid`, `et_set_coeffs`, `et_step`, `et_run`, ...) taking plain
integers for pointers; `Grid` wraps them for torch device tensors and
streams.  All arithmetic of the step runs in the CUDA kernels of libet.so;
this module only marshals arguments.  If the library cannot be loaded, every
call raises: there is no CPU fallback.

Method (arXiv 2402.02273, Sec. 2.2): u <- u + tau phi1(tau A)(A u + f(u)),
with tau phi1(tau A) b evaluated through exp(tau B) v_1 of the augmented
matrix B, s sub-steps of m Taylor terms each.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

__all__ = ["Grid", "EtError", "load", "OPS", "SCHEMES", "PRECISIONS", "STEP_INFO_DTYPE"]

ET_OK, ET_ERR_ARG, ET_ERR_STATE, ET_ERR_CUDA, ET_ERR_NUMERIC, ET_ERR_TIMEOUT, ET_ERR_UNSUPPORTED = range(7)
ET_F64, ET_F32, ET_DF64 = 0, 1, 2
ET_OP_CONSERVATIVE, ET_OP_LITERAL = 0, 1
ET_SCHEME_ROSENBROCK, ET_SCHEME_EXPEULER = 0, 1
ET_FLAG_NONFINITE, ET_FLAG_RANGE_IN, ET_FLAG_D_INVALID, ET_FLAG_TIMEOUT, ET_FLAG_TRUNCATION, ET_FLAG_CG_CAP = (
    1, 2, 4, 8, 16, 32)

PRECISIONS = {"f64": ET_F64, "f32": ET_F32, "df64": ET_DF64}
OPS = {"conservative": ET_OP_CONSERVATIVE, "literal": ET_OP_LITERAL}
SCHEMES = {"rosenbrock": ET_SCHEME_ROSENBROCK, "expeuler": ET_SCHEME_EXPEULER}


class et_options(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("theta_max", ctypes.c_double), ("shift", ctypes.c_int),
                ("force_s", ctypes.c_int), ("force_m", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("single_terms", ctypes.c_int), ("timeout_probe_us", ctypes.c_int), ("every_row", ctypes.c_int)]


class et_step_info(ctypes.Structure):
    _fields_ = [("umin", ctypes.c_double), ("umax", ctypes.c_double), ("mass", ctypes.c_double),
                ("s", ctypes.c_int), ("m", ctypes.c_int), ("flags", ctypes.c_uint),
                ("step", ctypes.c_uint)]


STEP_INFO_DTYPE = np.dtype([("umin", "<f8"), ("umax", "<f8"), ("mass", "<f8"), ("s", "<i4"),
                            ("m", "<i4"), ("flags", "<u4"), ("step", "<u4")])
assert STEP_INFO_DTYPE.itemsize == ctypes.sizeof(et_step_info) == 40

_VP = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_SIGS = {
    "et_version": ([], _I),
    "et_status_string": ([_I], ctypes.c_char_p),
    "et_last_error": ([_VP], ctypes.c_char_p),
    "et_workspace_bytes": ([_I, _I, _I, _I], ctypes.c_size_t),
    "et_create_grid": ([_I, _I, _I, _D, _I, _VP, ctypes.c_size_t, _VP, ctypes.POINTER(_VP)], _I),
    "et_set_coeffs": ([_VP, _VP, _D, _I, _I, ctypes.POINTER(et_options)], _I),
    "et_set_coeffs_host": ([_VP, _VP, _D, _I, _I, ctypes.POINTER(et_options)], _I),
    "et_step": ([_VP, _VP, _D, _VP], _I),
    "et_run": ([_VP, _VP, _D, _I, _VP], _I),
    "et_run_host": ([_VP, _VP, _D, _I, _VP], _I),
    "et_sync_info": ([_VP, ctypes.POINTER(et_step_info)], _I),
    "et_get_schedule": ([_VP, _D, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_D),
                         ctypes.POINTER(_D)], _I),
    "et_select_schedule": ([_D, _D, _D, _I, _I, ctypes.POINTER(et_options), ctypes.POINTER(_I),
                            ctypes.POINTER(_I), ctypes.POINTER(_D), ctypes.POINTER(_D)], _I),
    "et_set_stream": ([_VP, _VP], _I),
    "et_enable_timing": ([_VP, _I], _I),
    "et_get_timing": ([_VP, ctypes.POINTER(_D), ctypes.POINTER(ctypes.c_longlong),
                       ctypes.POINTER(ctypes.c_longlong)], _I),
    "et_get_info": ([_VP, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_size_t),
                     ctypes.POINTER(_D)], _I),
    "et_destroy": ([_VP], None),
    "et_vjp_workspace_bytes": ([_VP, _D, _I, _I], ctypes.c_size_t),
    "et_vjp": ([_VP, _VP, _D, _I, _I, _VP, _VP, ctypes.POINTER(_D), ctypes.POINTER(_D), _VP, ctypes.c_size_t], _I),
    "et_run_checkpointed": ([_VP, _VP, _D, _I, _I, _VP, ctypes.c_size_t], _I),
    "et_vjp_checkpointed": ([_VP, _D, _I, _I, _VP, _VP, ctypes.POINTER(_D), ctypes.POINTER(_D), _VP,
                             ctypes.c_size_t], _I),
    "et_batch_workspace_bytes": ([_I, _VP, _I], ctypes.c_size_t),
    "et_batch_create": ([_I, _VP, _D, _I, _VP, ctypes.c_size_t, _VP, ctypes.POINTER(_VP)], _I),
    "et_batch_set_coeffs": ([_VP, _VP, _VP, _I, _I, ctypes.POINTER(et_options)], _I),
    "et_batch_run": ([_VP, _VP, _D, _I, _VP], _I),
    "et_batch_autotune": ([_VP, _D, ctypes.POINTER(_I), _VP], _I),
    "et_batch_variant_count": ([_I], _I),
    "et_batch_set_variant": ([_VP, _I], _I),
    "et_batch_sync_info": ([_VP, _VP], _I),
    "et_batch_get_schedule": ([_VP, _D, _VP, _VP], _I),
    "et_batch_get_zero_rows": ([_VP, _VP, ctypes.POINTER(ctypes.c_longlong)], _I),
    "et_batch_set_stream": ([_VP, _VP], _I),
    "et_batch_last_error": ([_VP], ctypes.c_char_p),
    "et_batch_destroy": ([_VP], None),
    "et_step_static": ([_I, _I, _I, _D, _VP, _D, _I, _I, _VP, _D, _VP, ctypes.c_char_p, ctypes.c_size_t], _I),
    "et_probe_alu_scratch_bytes": ([], ctypes.c_size_t),
    "et_probe_alu": ([_VP, ctypes.c_size_t, _VP, ctypes.POINTER(_D), ctypes.POINTER(_D)], _I),
    "et_get_truncation": ([_VP, ctypes.POINTER(_D)], _I),
    "et_get_zero_rows": ([_VP, ctypes.POINTER(ctypes.c_longlong)], _I),
    "et_set_coeffs_scaled": ([_VP, _VP, _D, _D, _I, _I, _VP], _I),
    "et_cn_run": ([_VP, _VP, _D, _I, _D, _I, _VP], _I),
    "et_cn_iteration_cap": ([_VP, _D, _D], _I),
    "et_probe_stream": ([_VP, _VP, ctypes.c_size_t, _I, _I, _VP, ctypes.POINTER(_D)], _I),
}

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_stale: bool = True):
    """Load libet.so (compiling it with nvcc first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_stale else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library {path} is missing; run build()")
            lib = ctypes.CDLL(path)
            for name, (args, res) in _SIGS.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def __getattr__(name):
    # et_* names resolve to the raw C functions
    if name in _SIGS:
        return getattr(load(), name)
    raise AttributeError(name)


class EtError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} [status {status}]")
        self.status = status


def _check(rc: int, handle=None):
    if rc != ET_OK:
        lib = load()
        msg = lib.et_last_error(handle).decode(errors="replace")
        raise EtError(rc, msg or lib.et_status_string(rc).decode())


def make_options(tol=0.0, theta_max=0.0, shift=-1, force_s=0, force_m=0, use_graph=True, single_terms=False,
                 two_terms=False, timeout_probe_us=0, every_row=False):
    """et_options; single_terms / two_terms force one / two Taylor terms per
    launch (default: the form's own choice); timeout_probe_us is the test hook
    of the two-term kernel's bounded waits; every_row evaluates the whole
    stencil in rows without off-diagonal entries too."""
    if single_terms and two_terms:
        raise ValueError("single_terms and two_terms exclude each other")
    return et_options(float(tol), float(theta_max), int(shift), int(force_s), int(force_m),
                      1 if use_graph else -1, 1 if single_terms else (-1 if two_terms else 0),
                      int(timeout_probe_us), 1 if every_row else 0)


def select_schedule(tau, rmax, rho, scheme="rosenbrock", precision="f64", **opts):
    """Host-only (s, m, mu, theta) selector of the library (no GPU needed)."""
    lib = load()
    o = make_options(**opts)
    s, m, mu, th = _I(), _I(), _D(), _D()
    rc = lib.et_select_schedule(float(tau), float(rmax), float(rho), SCHEMES[scheme],
                                PRECISIONS[precision], ctypes.byref(o), ctypes.byref(s),
                                ctypes.byref(m), ctypes.byref(mu), ctypes.byref(th))
    _check(rc)
    return s.value, m.value, mu.value, th.value


class Grid:
    """A voxel grid on the current CUDA device with its workspace.

    Parameters: shape (nz, ny, nx) (x fastest, as numpy / torch C-order),
    h voxel width, precision "f64", "f32" or "df64", stream a torch.cuda.Stream (or
    None for the current stream).  Workspace memory is a torch uint8 tensor
    owned by this object.
    """

    def __init__(self, shape, h=1.0, precision="f64", stream=None, device=None):
        import torch

        self._torch = torch
        self.lib = load()
        nz, ny, nx = (int(v) for v in shape)
        self.shape = (nz, ny, nx)
        self.n = nx * ny * nz
        self.precision = precision
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        nbytes = self.lib.et_workspace_bytes(nx, ny, nz, PRECISIONS[precision])
        if nbytes == 0:
            raise EtError(ET_ERR_ARG, f"invalid grid {shape}")
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream()
            self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
            base = self.workspace.data_ptr()
            self._ws_ptr = (base + 255) // 256 * 256
            handle = _VP()
            rc = self.lib.et_create_grid(nx, ny, nz, float(h), PRECISIONS[precision], self._ws_ptr,
                                         nbytes, self.stream.cuda_stream, ctypes.byref(handle))
            _check(rc, None)
        self.handle = handle
        self.h = h

    def _chk(self, rc):
        _check(rc, self.handle)

    def close(self):
        if getattr(self, "handle", None):
            self.lib.et_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev_f64(self, t, name):
        torch = self._torch
        if not isinstance(t, torch.Tensor) or t.device != self.device or t.dtype != torch.float64 \
                or not t.is_contiguous() or t.numel() != self.n:
            raise EtError(ET_ERR_ARG, f"{name} must be a contiguous float64 tensor of {self.n} "
                                      f"elements on {self.device}")
        return t.data_ptr()

    def set_coeffs(self, D, rho=0.025, op="conservative", scheme="rosenbrock", dscale=None, **opts):
        """D: float64 device tensor (n values) or a numpy array (copied through the host
        path).  dscale: the field is read as dscale * D (device tensors only)."""
        o = make_options(**opts)
        self.options = o
        if dscale is not None:
            rc = self.lib.et_set_coeffs_scaled(self.handle, self._dev_f64(D, "D"), float(dscale), float(rho),
                                               OPS[op], SCHEMES[scheme], ctypes.byref(o))
        elif isinstance(D, np.ndarray):
            Dh = np.ascontiguousarray(D, dtype=np.float64)
            if Dh.size != self.n:
                raise EtError(ET_ERR_ARG, "D has the wrong size")
            rc = self.lib.et_set_coeffs_host(self.handle, Dh.ctypes.data, float(rho), OPS[op],
                                             SCHEMES[scheme], ctypes.byref(o))
        else:
            rc = self.lib.et_set_coeffs(self.handle, self._dev_f64(D, "D"), float(rho), OPS[op],
                                        SCHEMES[scheme], ctypes.byref(o))
        self._chk(rc)
        self.rho, self.op, self.scheme = rho, op, scheme

    def step(self, u, tau, info=None):
        self._chk(self.lib.et_step(self.handle, self._dev_f64(u, "u"), float(tau),
                                   None if info is None else info.data_ptr()))

    def run(self, u, tau, nsteps, info=None):
        """nsteps steps in place on the device tensor u; info: uint8 device tensor of
        40 * nsteps bytes (see info_buffer) or None."""
        self._chk(self.lib.et_run(self.handle, self._dev_f64(u, "u"), float(tau), int(nsteps),
                                  None if info is None else info.data_ptr()))

    def run_host(self, u_host: np.ndarray, tau, nsteps):
        """Copies u_host (float64 numpy, contiguous; pinned helps) in, runs, copies it back."""
        if not (isinstance(u_host, np.ndarray) and u_host.dtype == np.float64 and
                u_host.flags.c_contiguous and u_host.size == self.n):
            raise EtError(ET_ERR_ARG, "u_host must be a contiguous float64 array of n values")
        rec = et_step_info()
        self._chk(self.lib.et_run_host(self.handle, u_host.ctypes.data, float(tau), int(nsteps),
                                       ctypes.byref(rec)))
        return _rec_dict(rec)

    def info_buffer(self, nsteps):
        return self._torch.zeros(40 * int(nsteps), dtype=self._torch.uint8, device=self.device)

    @staticmethod
    def decode_info(buf):
        return np.frombuffer(buf.cpu().numpy().tobytes(), dtype=STEP_INFO_DTYPE)

    def sync_info(self):
        rec = et_step_info()
        self._chk(self.lib.et_sync_info(self.handle, ctypes.byref(rec)))
        return _rec_dict(rec)

    def schedule(self, tau):
        s, m, mu, th = _I(), _I(), _D(), _D()
        self._chk(self.lib.et_get_schedule(self.handle, float(tau), ctypes.byref(s), ctypes.byref(m),
                                           ctypes.byref(mu), ctypes.byref(th)))
        return s.value, m.value, mu.value, th.value

    def cn_run(self, u, tau, nsteps, rtol=1e-12, max_iter=0, info=None):
        """nsteps Crank-Nicolson steps (Sec. 2.3) of u in place, by conjugate gradients."""
        self._chk(self.lib.et_cn_run(self.handle, self._dev_f64(u, "u"), float(tau), int(nsteps), float(rtol),
                                     int(max_iter), None if info is None else info.data_ptr()))

    def cn_iteration_cap(self, tau, rtol=1e-12):
        return int(self.lib.et_cn_iteration_cap(self.handle, float(tau), float(rtol)))

    def zero_row_voxels(self):
        """Voxels in warp rows without off-diagonal entries (their terms skip the stencil)."""
        v = ctypes.c_longlong()
        self._chk(self.lib.et_get_zero_rows(self.handle, ctypes.byref(v)))
        return v.value

    def truncation(self):
        """A-posteriori truncation estimate of the latest step (relative to max|u^n|)."""
        est = _D()
        self._chk(self.lib.et_get_truncation(self.handle, ctypes.byref(est)))
        return est.value

    def rmax(self):
        n, ws, r = ctypes.c_longlong(), ctypes.c_size_t(), _D()
        self._chk(self.lib.et_get_info(self.handle, ctypes.byref(n), ctypes.byref(ws), ctypes.byref(r)))
        return r.value

    def enable_timing(self, on=True):
        self._chk(self.lib.et_enable_timing(self.handle, 1 if on else 0))

    def timing(self):
        ms, tl, ol = _D(), ctypes.c_longlong(), ctypes.c_longlong()
        self._chk(self.lib.et_get_timing(self.handle, ctypes.byref(ms), ctypes.byref(tl), ctypes.byref(ol)))
        return ms.value, tl.value, ol.value

    def vjp(self, u0, tau, nsteps, ubar_final, checkpoint_every=10):
        """Reverse mode through nsteps steps from u0 (device tensors, float64):
        returns (dJ/du0, dJ/drho, d/ds J(s D) at s = 1) for the cotangent
        ubar_final = dJ/du^K.  Uses a temporary device workspace."""
        torch = self._torch
        nbytes = self.lib.et_vjp_workspace_bytes(self.handle, float(tau), int(nsteps), int(checkpoint_every))
        if nbytes == 0:
            raise EtError(ET_ERR_STATE, "no adjoint workspace size (coefficients set? tau valid?)")
        ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        ws_ptr = (ws.data_ptr() + 255) // 256 * 256
        ubar0 = torch.empty_like(u0)
        g_rho, g_ds = _D(), _D()
        self._chk(self.lib.et_vjp(self.handle, self._dev_f64(u0, "u0"), float(tau), int(nsteps),
                                  int(checkpoint_every), self._dev_f64(ubar_final, "ubar_final"),
                                  self._dev_f64(ubar0, "ubar0"), ctypes.byref(g_rho), ctypes.byref(g_ds),
                                  ws_ptr, nbytes))
        return ubar0, g_rho.value, g_ds.value

    def adjoint_workspace(self, tau, nsteps, checkpoint_every=10):
        """A device buffer for et_run_checkpointed / et_vjp_checkpointed: (tensor, aligned pointer, bytes)."""
        torch = self._torch
        nbytes = self.lib.et_vjp_workspace_bytes(self.handle, float(tau), int(nsteps), int(checkpoint_every))
        if nbytes == 0:
            raise EtError(ET_ERR_STATE, "no adjoint workspace size (coefficients set? tau valid?)")
        ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        return ws, (ws.data_ptr() + 255) // 256 * 256, nbytes

    def run_checkpointed(self, u, tau, nsteps, checkpoint_every=10, workspace=None):
        """et_run keeping checkpoints for a later vjp_checkpointed; returns the workspace."""
        ws = workspace if workspace is not None else self.adjoint_workspace(tau, nsteps, checkpoint_every)
        self._chk(self.lib.et_run_checkpointed(self.handle, self._dev_f64(u, "u"), float(tau), int(nsteps),
                                               int(checkpoint_every), ws[1], ws[2]))
        return ws

    def vjp_checkpointed(self, workspace, tau, nsteps, ubar_final, checkpoint_every=10):
        """Reverse pass from the checkpoints of run_checkpointed: (dJ/du0, dJ/drho, d/ds J(s D))."""
        ubar0 = self._torch.empty_like(ubar_final)
        g_rho, g_ds = _D(), _D()
        self._chk(self.lib.et_vjp_checkpointed(self.handle, float(tau), int(nsteps), int(checkpoint_every),
                                               self._dev_f64(ubar_final, "ubar_final"), self._dev_f64(ubar0, "ubar0"),
                                               ctypes.byref(g_rho), ctypes.byref(g_ds), workspace[1], workspace[2]))
        return ubar0, g_rho.value, g_ds.value

    def set_stream(self, stream):
        self.stream = stream
        self._chk(self.lib.et_set_stream(self.handle, stream.cuda_stream))


def probe_alu(stream=None):
    """Measured (FP64, FP32) FMA throughput of the current device in TFLOP/s."""
    import torch
    lib = load()
    nbytes = lib.et_probe_alu_scratch_bytes()
    buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    st = stream if stream is not None else torch.cuda.current_stream()
    f64, f32 = _D(), _D()
    _check(lib.et_probe_alu(buf.data_ptr(), nbytes, st.cuda_stream, ctypes.byref(f64), ctypes.byref(f32)))
    return f64.value, f32.value


def probe_stream(nbytes, nin=1, reps=50, stream=None):
    """Best read + write bandwidth (GB/s) of the library's streaming probe:
    nin input buffers and one output of nbytes each (inside the L2: the L2
    roofline; far beyond it: the HBM roofline)."""
    import torch
    lib = load()
    nbytes = int(nbytes) // 16 * 16
    src = torch.ones(nin * nbytes // 4, dtype=torch.float32, device="cuda")
    dst = torch.empty(nbytes // 4, dtype=torch.float32, device="cuda")
    st = stream if stream is not None else torch.cuda.current_stream()
    gbs = _D()
    _check(lib.et_probe_stream(src.data_ptr(), dst.data_ptr(), nbytes, int(nin), int(reps), st.cuda_stream,
                               ctypes.byref(gbs)))
    return gbs.value


class Batch:
    """Many grids of different sizes advanced together (the et_batch_* ABI).

    shapes: list of (nz, ny, nx); fields (D, u) are the grids' arrays flattened
    and concatenated in order (float64 CUDA tensors of sum(n_i) values).
    """

    def __init__(self, shapes, h=1.0, precision="f64", stream=None, device=None):
        import torch

        self._torch = torch
        self.lib = load()
        self.shapes = [tuple(int(v) for v in sh) for sh in shapes]
        self.count = len(self.shapes)
        dims = []
        for nz, ny, nx in self.shapes:
            dims += [nx, ny, nz]
        self._dims = (ctypes.c_int * len(dims))(*dims)
        self.sizes = [nx * ny * nz for nz, ny, nx in self.shapes]
        self.offsets = np.concatenate([[0], np.cumsum(self.sizes)]).astype(np.int64)
        self.n = int(self.offsets[-1])
        self.precision = precision
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        nbytes = self.lib.et_batch_workspace_bytes(self.count, self._dims, PRECISIONS[precision])
        if nbytes == 0:
            raise EtError(ET_ERR_ARG, "invalid batch")
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream()
            self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
            ws = (self.workspace.data_ptr() + 255) // 256 * 256
            handle = _VP()
            rc = self.lib.et_batch_create(self.count, self._dims, float(h), PRECISIONS[precision], ws, nbytes,
                                          self.stream.cuda_stream, ctypes.byref(handle))
            if rc != ET_OK:
                raise EtError(rc, self.lib.et_batch_last_error(None).decode())
        self.handle = handle

    def _chk(self, rc):
        if rc != ET_OK:
            raise EtError(rc, self.lib.et_batch_last_error(self.handle).decode())

    def close(self):
        if getattr(self, "handle", None):
            self.lib.et_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev(self, t, name):
        torch = self._torch
        if not isinstance(t, torch.Tensor) or t.device != self.device or t.dtype != torch.float64 \
                or not t.is_contiguous() or t.numel() != self.n:
            raise EtError(ET_ERR_ARG, f"{name} must be a contiguous float64 tensor of {self.n} values")
        return t.data_ptr()

    def set_coeffs(self, D, rho, op="conservative", scheme="rosenbrock", **opts):
        r = np.ascontiguousarray(np.broadcast_to(np.asarray(rho, dtype=np.float64), (self.count,)))
        self._rho = r
        o = make_options(**opts)
        self._chk(self.lib.et_batch_set_coeffs(self.handle, self._dev(D, "D"), r.ctypes.data, OPS[op],
                                               SCHEMES[scheme], ctypes.byref(o)))

    def run(self, u, tau, nsteps, info=None):
        self._chk(self.lib.et_batch_run(self.handle, self._dev(u, "u"), float(tau), int(nsteps),
                                        None if info is None else info.data_ptr()))

    def info_buffer(self, nsteps):
        return self._torch.zeros(40 * int(nsteps) * self.count, dtype=self._torch.uint8, device=self.device)

    def autotune(self, tau):
        nv = self.lib.et_batch_variant_count(PRECISIONS[self.precision])
        us = (ctypes.c_double * nv)()
        v = _I()
        self._chk(self.lib.et_batch_autotune(self.handle, float(tau), ctypes.byref(v), us))
        return v.value, list(us)

    def set_variant(self, v):
        self._chk(self.lib.et_batch_set_variant(self.handle, int(v)))

    def sync_info(self):
        recs = (et_step_info * self.count)()
        self._chk(self.lib.et_batch_sync_info(self.handle, recs))
        return [_rec_dict(r) for r in recs]

    def schedule(self, tau):
        s = (ctypes.c_int * self.count)()
        m = (ctypes.c_int * self.count)()
        self._chk(self.lib.et_batch_get_schedule(self.handle, float(tau), s, m))
        return list(s), list(m)

    def zero_row_voxels(self):
        """Per grid, the voxels in warp rows without off-diagonal entries."""
        v = (ctypes.c_longlong * self.count)()
        self._chk(self.lib.et_batch_get_zero_rows(self.handle, v, None))
        return list(v)

    def split(self, t):
        """Views of a concatenated tensor, one per grid, shaped (nz, ny, nx)."""
        return [t[self.offsets[i]:self.offsets[i + 1]].view(self.shapes[i]) for i in range(self.count)]


def _rec_dict(rec):
    return {"umin": rec.umin, "umax": rec.umax, "mass": rec.mass, "s": rec.s, "m": rec.m,
            "flags": rec.flags, "step": rec.step}


def tumour_run(u0, rho, dscale, D0, tau, nsteps, grid=None, checkpoint_every=10, **coeff_opts):
    """u^K = step^K(u0) with D = dscale * D0, differentiable in u0, rho and dscale.

    u0: float64 CUDA tensor (n values); rho, dscale: 0-d float64 tensors (or
    floats); D0: float64 CUDA tensor of per-voxel diffusion.  The backward pass
    is the library's discrete adjoint, checkpointed every `checkpoint_every`
    steps (the forward run keeps the checkpoints: et_run_checkpointed, then
    et_vjp_checkpointed); the schedule (s, m, mu) is frozen at the forward
    values.  `grid`: a Grid of the right shape (created if None).
    """
    import torch

    class _TumourRun(torch.autograd.Function):
        @staticmethod
        def forward(ctx, u0_, rho_, dscale_):
            g = grid if grid is not None else Grid(D0.shape)
            r = float(rho_)
            ds = float(dscale_)
            g.set_coeffs(D0, rho=r, dscale=ds, **coeff_opts)
            u = u0_.detach().clone().contiguous()
            # the forward run keeps the checkpoints the backward pass starts from
            ctx.ws = g.run_checkpointed(u, tau, nsteps, checkpoint_every)
            g.sync_info()
            ctx.g, ctx.ds = g, ds
            ctx.devs = (rho_.device, dscale_.device)
            return u

        @staticmethod
        def backward(ctx, ubar):
            ubar0, g_rho, g_ds = ctx.g.vjp_checkpointed(ctx.ws, tau, nsteps, ubar.contiguous(), checkpoint_every)
            ctx.ws = None
            # D = dscale D0:  dJ/d dscale = (1 / dscale) d/ds J(s D) at s = 1
            return (ubar0, torch.tensor(g_rho, dtype=torch.float64, device=ctx.devs[0]),
                    torch.tensor(g_ds / ctx.ds, dtype=torch.float64, device=ctx.devs[1]))

    as_t = lambda v: v if isinstance(v, torch.Tensor) else torch.tensor(float(v), dtype=torch.float64)
    return _TumourRun.apply(u0, as_t(rho), as_t(dscale))
