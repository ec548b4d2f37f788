"""The C-ABI library builds, loads and exports what include/et.h declares; host-only
logic (argument checks, workspace sizing, the (s, m) selector) works without a GPU."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import paper_2402_02273_gb300 as et

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "et.h")).read()
    return sorted(set(re.findall(r"ET_API[^;(]*?\b(et_\w+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = et.load()
    names = _declared()
    assert len(names) >= 18
    for name in names:
        assert hasattr(lib, name), name
    # and the binding wraps each of them under the same name
    for name in names:
        assert name in et._SIGS, name


def test_version_and_status_strings():
    lib = et.load()
    assert lib.et_version() == 100
    assert lib.et_status_string(0) == b"ok"
    assert b"argument" in lib.et_status_string(1)


def test_workspace_sizing():
    lib = et.load()
    assert lib.et_workspace_bytes(0, 4, 4, 0) == 0
    assert lib.et_workspace_bytes(4, -1, 4, 0) == 0
    assert lib.et_workspace_bytes(4, 4, 4, 7) == 0
    a = lib.et_workspace_bytes(32, 32, 32, 0)
    b = lib.et_workspace_bytes(64, 32, 32, 0)
    assert a > 11 * 8 * 32 ** 3 and b > a
    assert lib.et_workspace_bytes(32, 32, 32, 1) > 0
    # 128^3 FP64: 5 coefficient fields, 6 vectors and a staging field
    big = lib.et_workspace_bytes(128, 128, 128, 0)
    assert 12 * 8 * 128 ** 3 <= big <= 13 * 8 * 128 ** 3
    assert lib.et_workspace_bytes(2048, 1024, 1024, 0) == 0  # 2^31 voxels


def test_create_rejects_bad_arguments_without_touching_the_gpu():
    lib = et.load()
    h = ctypes.c_void_p()
    assert lib.et_create_grid(4, 4, 4, 1.0, 0, 256, 10 ** 9, None, None) == et.ET_ERR_ARG
    assert lib.et_create_grid(0, 4, 4, 1.0, 0, 256, 10 ** 9, None, ctypes.byref(h)) == et.ET_ERR_ARG
    assert not h.value
    assert b"empty" in lib.et_last_error(None)
    assert lib.et_create_grid(4, 4, 4, 0.0, 0, 256, 10 ** 9, None, ctypes.byref(h)) == et.ET_ERR_ARG
    assert lib.et_create_grid(4, 4, 4, float("nan"), 0, 256, 10 ** 9, None, ctypes.byref(h)) == et.ET_ERR_ARG
    assert lib.et_create_grid(4, 4, 4, 1.0, 0, None, 10 ** 9, None, ctypes.byref(h)) == et.ET_ERR_ARG
    assert lib.et_create_grid(4, 4, 4, 1.0, 0, 100, 10 ** 9, None, ctypes.byref(h)) == et.ET_ERR_ARG
    assert b"aligned" in lib.et_last_error(None)
    assert lib.et_create_grid(4, 4, 4, 1.0, 0, 256, 16, None, ctypes.byref(h)) == et.ET_ERR_ARG
    assert b"needed" in lib.et_last_error(None)
    assert lib.et_create_grid(4, 4, 4, 1.0, 5, 256, 10 ** 9, None, ctypes.byref(h)) == et.ET_ERR_ARG
    # NULL handles are rejected by every entry point
    assert lib.et_step(None, None, 1.0, None) == et.ET_ERR_ARG
    assert lib.et_run(None, None, 1.0, 1, None) == et.ET_ERR_ARG
    assert lib.et_sync_info(None, None) == et.ET_ERR_ARG
    lib.et_destroy(None)


def test_selector_basic_properties():
    # 128^3 phantom: rmax ~ 6 * 0.143 = 0.858 / day, tau = 7.3 days
    s, m, mu, th = et.select_schedule(7.3, 0.858, 0.025)
    assert mu == pytest.approx(-0.858)
    assert s >= 1 and m >= 2 and th <= 7.0 + 1e-12
    assert th == pytest.approx(7.3 * (0.858 + 0.025 * 1.002) / s)
    s0, m0, mu0, th0 = et.select_schedule(7.3, 0.858, 0.025, shift=0)
    assert mu0 == 0.0 and s0 * m0 > s * m  # the shift halves the norm
    # tighter tolerance never needs fewer terms
    s2, m2, _, _ = et.select_schedule(7.3, 0.858, 0.025, tol=1e-15)
    assert s2 * m2 >= s * m
    # with the shift the e^{mu h} factor cancels the growth of the partial sums,
    # so FP32 takes one long sub-step; without it theta stays small for rounding
    s3, m3, _, th3 = et.select_schedule(7.3, 0.858, 0.025, precision="f32")
    assert s3 == 1 and m3 < m
    s4, m4, _, th4 = et.select_schedule(7.3, 0.858, 0.025, precision="f32", shift=0)
    assert th4 <= 1.5 + 1e-12 and s4 * m4 > 2 * s3 * m3
    assert et.select_schedule(7.3, 0.858, 0.025, precision="df64")[:2] == (s, m)
    # forced values pass through
    assert et.select_schedule(7.3, 0.858, 0.025, force_s=3, force_m=9)[:2] == (3, 9)
    # degenerate operator: D = 0 and exponential Euler -> A = 0, one short sub-step
    assert et.select_schedule(7.3, 0.0, 0.025, scheme="expeuler")[:2] == (1, 2)
    with pytest.raises(et.EtError):
        et.select_schedule(-1.0, 0.858, 0.025)
    with pytest.raises(et.EtError):
        et.select_schedule(7.3, 0.858, 0.025, tol=1e-300, theta_max=0.001)


def _shifted_recurrence(A, b, tau, s, m, mu):
    """Model of the GPU's scaled recurrence in numpy (dense A): see et_kernels.cu."""
    n = len(b)
    At = A - mu * np.eye(n)
    h = tau / s
    gamma = math.exp(mu * h)
    y = np.zeros(n)
    ak = 1.0
    for k in range(s):
        z = y.copy()
        acc = y.copy()
        g = 1.0
        pw = 1.0
        for j in range(m):
            z = At @ z + ak * pw * b
            g *= h / (j + 1)
            acc = acc + g * z
            pw *= -mu
        y = gamma * acc
        ak = gamma * ak * sum((-mu * h) ** j / math.factorial(j) for j in range(m + 1))
    return y


@pytest.mark.parametrize("shift", [1, 0])
@pytest.mark.parametrize("op", ["conservative", "literal"])
def test_selected_schedule_meets_tolerance_on_dense_model(shift, op):
    """The selector's (s, m) with the shifted, scaled recurrence reproduces
    tau phi1(tau A) b from the oracle to the requested tolerance."""
    import oracle
    from paper_2402_02273_gb300 import phantom

    D, u0 = phantom.case((6, 7, 5), seed=2, noise=0.1)
    D[D == 0] = 0.1
    P = oracle.Problem(D, op=op, scheme="rosenbrock")
    n = D.size
    A = np.zeros((n, n))
    for q in range(n):
        e = np.zeros(n)
        e[q] = 1.0
        A[:, q] = P.apply_A(u0, e).ravel()
    # row sums of L only (the reaction diagonal is not part of rmax)
    L = A - np.diag(0.025 * (1 - 2 * u0.ravel()))
    rmax = max(np.abs(L[p]).sum() - abs(L[p, p]) for p in range(n))
    b = P.residual(u0).ravel()
    tau = 7.3
    s, m, mu, th = et.select_schedule(tau, rmax, 0.025, shift=shift, tol=1e-13)
    got = _shifted_recurrence(A, b, tau, s, m, mu)
    want, _, _ = P.phi1_action(u0, b.reshape(D.shape), tau)
    assert np.abs(got - want.ravel()).max() <= 1e-13 * max(1.0, np.abs(u0).max())


def test_terms_per_launch_option():
    """single_terms / two_terms map to the et_options field (1 / -1, 0 = the
    form's own choice) and exclude each other."""
    assert et.make_options().single_terms == 0
    assert et.make_options(single_terms=True).single_terms == 1
    assert et.make_options(two_terms=True).single_terms == -1
    with pytest.raises(ValueError):
        et.make_options(single_terms=True, two_terms=True)


def test_bench_launch_mix_and_kernel_choice():
    """The bench's bookkeeping: launches and algorithmic bytes of a chain with
    and without pairs, and the kernel each form runs at a grid size."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    # s = 1, m = 31: 30 Horner terms, one launch each or fifteen pairs
    nl, nb, nf = bench.launch_mix("f32", 1, 31, False)
    assert nl == 30 and nb == 30 * bench.HORNER_BYTES["f32"] and nf == 30 * bench.HORNER_FLOPS["f32"]
    nl, nb, nf = bench.launch_mix("f32", 1, 31, True)
    assert nl == 15 and nb == 15 * bench.HORNER_BYTES["f32"] and nf == 30 * bench.HORNER_FLOPS["f32"]
    # s = 2, m = 5: 4 Horner terms then 5 running-sum terms (2 pairs + 1 single)
    nl, nb, _ = bench.launch_mix("df64", 2, 5, True)
    assert nl == 2 + 3 and nb == 2 * bench.HORNER_BYTES["df64"] + 3 * bench.TERM_BYTES["df64"]
    assert bench.term_kernel_of("f64", False, 128 ** 3) == ("term_kernel_f64", False)
    assert bench.term_kernel_of("df64", False, 128 ** 3) == ("term2_kernel", True)
    assert bench.term_kernel_of("df64", True, 128 ** 3) == ("term_kernel_df64", False)
    assert bench.term_kernel_of("f32", False, 128 ** 3) == ("term_quad_kernel", False)
    assert bench.term_kernel_of("f32", False, 160 ** 3) == ("term2_quad_kernel", True)
    assert bench.term_kernel_of("f32", False, 192 ** 3) == ("term2_quad_kernel", True)
    assert bench.term_kernel_of("f32", True, 192 ** 3) == ("term_quad_kernel", False)
    # rows without off-diagonal entries: z, the diagonal and b in, z out
    # (4 values per voxel), 3 flops; a share f of them scales in linearly
    nl, nb, nf = bench.launch_mix("f64", 1, 3, False, zero_frac=0.25)
    assert nl == 2
    assert nb == pytest.approx(2 * (0.75 * bench.HORNER_BYTES["f64"] + 0.25 * 32))
    assert nf == pytest.approx(2 * (0.75 * bench.HORNER_FLOPS["f64"] + 0.25 * 3))
    _, nb, _ = bench.launch_mix("df64", 1, 3, False, zero_frac=1.0)
    assert nb == pytest.approx(2 * 32)
    assert "term2_kernel" not in bench.ZERO_ROW_KERNELS and "term_kernel_df64" in bench.ZERO_ROW_KERNELS
    # a kernel whose loads skip zero rows but which evaluates every product
    nl, nb, nf = bench.launch_mix("f32", 1, 3, True, zero_frac=1.0, zero_flops=False)
    assert nl == 1 and nb == pytest.approx(16) and nf == pytest.approx(2 * bench.HORNER_FLOPS["f32"])
    assert "term2_quad_kernel" not in bench.ZERO_ROW_KERNELS


def test_bench_traffic_table_names_existing_sources():
    """Every steady-state traffic entry of the bench names a kernel whose source
    file exists and carries a 12-digit SHA-256 prefix; an entry whose prefix
    no longer matches its file reports no traffic (null) instead of a stale
    figure."""
    import importlib.util
    import re
    spec = importlib.util.spec_from_file_location("bench_mod2", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    for (prec, kernel, grid), (per_voxel, sha) in bench.TERM_TRAFFIC.items():
        assert prec in ("f64", "f32", "df64") and per_voxel > 0
        assert re.fullmatch(r"[0-9a-f]{12}", sha)
        assert bench.source_sha(kernel) is not None, kernel
        if bench.source_sha(kernel) == sha:
            assert bench.term_traffic(prec, kernel, grid, 1000) == pytest.approx(per_voxel * 1000)
    assert bench.term_traffic("f64", "no_such_kernel", 128, 1000) is None
