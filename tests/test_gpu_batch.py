"""Batched form (et_batch_*) through the C ABI (GPU only).

Many grids of uneven sizes, each with its own D, rho and (s, m), advance in
one CUDA graph of batched launches.  Every grid of the batch must match the
FP64 oracle run on that grid alone (1e-10 relative, FP64 and DF64 forms) and
the single-grid path (et_run) on the same grid: bitwise where the batched
kernel runs the same per-voxel arithmetic, else within 1e-13 relative."""
import numpy as np
import pytest

import oracle
from zero_rows import zero_row_voxels
from paper_2402_02273_gb300 import phantom

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TAU = 7.3


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def et_mod():
    import paper_2402_02273_gb300 as et
    et.load()
    return et


# Ragged grids: x not a multiple of 32, y not a multiple of 8, nz of 1 and odd
# counts, a grid smaller than one tile, and a grid without diffusion.
SHAPES = [(20, 17, 33), (9, 40, 31), (24, 24, 24), (1, 1, 5), (12, 8, 70), (7, 13, 3)]
RHOS = [0.025, 0.05, 0.01, 0.03, 0.02, 0.04]
DSCALE = [1.0, 2.0, 0.5, 1.0, 1.5, 0.0]


def _mixed_batch():
    Ds, us = [], []
    for i, sh in enumerate(SHAPES):
        D, u0 = phantom.case(sh, seed=i, noise=0.1)
        D = D * DSCALE[i]
        if not np.any(u0 > 0.1):  # tiny grids: seed the middle voxel
            u0 = np.zeros(sh)
            u0.reshape(-1)[u0.size // 2] = 0.8
        Ds.append(D)
        us.append(u0)
    return Ds, us


def _concat(torch, arrays):
    return torch.from_numpy(np.concatenate([a.reshape(-1) for a in arrays])).cuda()


def _errs(got, want):
    scale = np.abs(want).max()
    return (np.abs(got - want).max() / scale,
            np.linalg.norm((got - want).ravel()) / np.linalg.norm(want.ravel()))


def _batch_run(et, torch, shapes, Ds, us, rhos, nsteps, precision="f64", variant=None, op="conservative",
               scheme="rosenbrock", info=False, **opts):
    B = et.Batch(shapes, precision=precision)
    B.set_coeffs(_concat(torch, Ds), rhos, op=op, scheme=scheme, **opts)
    if variant is not None:
        B.set_variant(variant)
    u = _concat(torch, us)
    buf = B.info_buffer(nsteps) if info else None
    B.run(u, TAU, nsteps, info=buf)
    recs = B.sync_info()
    out = [x.cpu().numpy().copy() for x in B.split(u)]
    return B, out, recs, buf


def _single_run(et, torch, D, u0, rho, nsteps, precision="f64", op="conservative", scheme="rosenbrock", **opts):
    g = et.Grid(D.shape, precision=precision)
    g.set_coeffs(torch.from_numpy(D.copy()).cuda(), rho=rho, op=op, scheme=scheme, **opts)
    u = torch.from_numpy(u0.copy()).cuda()
    g.run(u, TAU, nsteps)
    return u.cpu().numpy().reshape(D.shape), g.sync_info()


def _variants(et, precision):
    return range(et.load().et_batch_variant_count(et.PRECISIONS[precision]))


@pytest.mark.parametrize("precision", ["f64", "df64"])
def test_mixed_batch_matches_oracle_every_variant(et_mod, torch_cuda, precision):
    Ds, us = _mixed_batch()
    nsteps = 4
    want = []
    for i, sh in enumerate(SHAPES):
        P = oracle.Problem(Ds[i], rho=RHOS[i])
        want.append(P.run(us[i], TAU, nsteps)[0])
    for v in _variants(et_mod, precision):
        _, got, recs, _ = _batch_run(et_mod, torch_cuda, SHAPES, Ds, us, RHOS, nsteps, precision, variant=v)
        for i in range(len(SHAPES)):
            e_max, e_l2 = _errs(got[i], want[i])
            assert e_max <= TOL64 and e_l2 <= TOL64, (precision, v, i, e_max, e_l2)
            assert recs[i]["step"] == nsteps - 1
            assert recs[i]["mass"] == pytest.approx(want[i].sum(), rel=1e-12)


@pytest.mark.parametrize("op,scheme", [("literal", "rosenbrock"), ("conservative", "expeuler")])
def test_mixed_batch_operator_and_scheme_readings(et_mod, torch_cuda, op, scheme):
    Ds, us = _mixed_batch()
    nsteps = 3
    _, got, _, _ = _batch_run(et_mod, torch_cuda, SHAPES, Ds, us, RHOS, nsteps, op=op, scheme=scheme)
    for i in range(len(SHAPES)):
        P = oracle.Problem(Ds[i], rho=RHOS[i], op=op, scheme=scheme)
        e_max, e_l2 = _errs(got[i], P.run(us[i], TAU, nsteps)[0])
        assert e_max <= TOL64 and e_l2 <= TOL64, (op, scheme, i, e_max, e_l2)


@pytest.mark.parametrize("precision", ["f64", "df64", "f32"])
def test_batch_matches_single_grid_path(et_mod, torch_cuda, precision):
    """Variant 0 of FP64 runs the single-grid kernel's per-voxel code (bitwise);
    the other variants and forms agree to their own rounding."""
    Ds, us = _mixed_batch()
    nsteps = 5
    single = [_single_run(et_mod, torch_cuda, Ds[i], us[i], RHOS[i], nsteps, precision)[0]
              for i in range(len(SHAPES))]
    tol = 1e-13 if precision != "f32" else 1e-5
    for v in _variants(et_mod, precision):
        _, got, _, _ = _batch_run(et_mod, torch_cuda, SHAPES, Ds, us, RHOS, nsteps, precision, variant=v)
        for i in range(len(SHAPES)):
            if precision == "f64" and v == 0:
                assert np.array_equal(got[i], single[i]), (v, i)
            else:
                e_max, _ = _errs(got[i], single[i])
                assert e_max <= tol, (precision, v, i, e_max)


def test_batch_step_records_and_schedules(et_mod, torch_cuda):
    Ds, us = _mixed_batch()
    nsteps = 6
    B, got, last, buf = _batch_run(et_mod, torch_cuda, SHAPES, Ds, us, RHOS, nsteps, info=True)
    s_list, m_list = B.schedule(TAU)
    recs = buf.cpu().numpy().view(np.uint8)
    C = len(SHAPES)
    for i in range(C):
        states, ost = oracle.Problem(Ds[i], rho=RHOS[i]).run(us[i], TAU, nsteps, every=True)
        for t in range(nsteps):
            r = _decode(et_mod, recs, t * C + i)
            assert r["step"] == t
            assert (r["s"], r["m"]) == (s_list[i], m_list[i])
            assert r["mass"] == pytest.approx(states[t + 1].sum(), rel=1e-12)
            assert r["umax"] == pytest.approx(states[t + 1].max(), rel=1e-10)
        assert last[i]["step"] == nsteps - 1
        # every grid has its own schedule: the single-grid selector gives the same (s, m)
        g = et_mod.Grid(Ds[i].shape)
        g.set_coeffs(torch_cuda.from_numpy(Ds[i].copy()).cuda(), rho=RHOS[i])
        assert g.schedule(TAU)[:2] == (s_list[i], m_list[i])


def _decode(et, raw, idx):
    rec = et.et_step_info.from_buffer_copy(raw[40 * idx:40 * (idx + 1)].tobytes())
    return {"mass": rec.mass, "umin": rec.umin, "umax": rec.umax, "s": rec.s, "m": rec.m,
            "flags": rec.flags, "step": rec.step}


def test_autotune_and_graph_reuse(et_mod, torch_cuda):
    torch = torch_cuda
    Ds, us = _mixed_batch()
    B = et_mod.Batch(SHAPES)
    B.set_coeffs(_concat(torch, Ds), RHOS)
    v, times = B.autotune(TAU)
    assert 0 <= v < len(times)
    assert all(t > 0 for t in times)
    assert times[v] == min(times)  # FP64: one-term variants only
    # FP32: the fastest one-term variant, with two-term launches when those are faster
    Bf = et_mod.Batch(SHAPES, precision="f32")
    Bf.set_coeffs(_concat(torch, Ds), RHOS)
    vf, tf = Bf.autotune(TAU)
    nsv = len(tf) // 2
    single = min(range(nsv, 2 * nsv), key=lambda q: tf[q])
    assert vf == (single - nsv if min(tf[:nsv]) < tf[single] else single)
    u = _concat(torch, us)
    B.run(u, TAU, 2)
    B.run(u, TAU, 2)  # replays the captured graph
    u2 = _concat(torch, us)
    B.run(u2, TAU, 4)
    torch.cuda.synchronize()
    assert torch.equal(u, u2)


def test_full_size_batch_instances_match_oracle(et_mod, torch_cuda):
    """Eight instances of the many-patient workload (n in {96..160}, own rho,
    D scale and 1-3 seed blobs), two steps, in the launch configuration the
    benchmark times (autotuned variant, CUDA graph); every voxel vs the oracle."""
    cases = [phantom.batch_case(i) for i in range(8)]
    shapes = [c["D"].shape for c in cases]
    nsteps = 2
    B, got, recs, _ = _batch_run(et_mod, torch_cuda, shapes, [c["D"] for c in cases], [c["u0"] for c in cases],
                                 [c["rho"] for c in cases], nsteps)
    for i, c in enumerate(cases):
        want = oracle.Problem(c["D"], rho=c["rho"]).run(c["u0"], TAU, nsteps)[0]
        e_max, e_l2 = _errs(got[i], want)
        assert e_max <= TOL64 and e_l2 <= TOL64, (i, c["n"], e_max, e_l2)


def test_batch_errors(et_mod, torch_cuda):
    torch = torch_cuda
    et = et_mod
    with pytest.raises(et.EtError):
        et.Batch([])
    with pytest.raises(et.EtError):
        et.Batch([(4, 0, 4)])
    Ds, us = _mixed_batch()
    B = et.Batch(SHAPES)
    with pytest.raises(et.EtError) as ei:
        B.run(_concat(torch, us), TAU, 1)
    assert ei.value.status == et.ET_ERR_STATE
    bad = [d.copy() for d in Ds]
    bad[2].reshape(-1)[5] = -1.0
    with pytest.raises(et.EtError) as ei:
        B.set_coeffs(_concat(torch, bad), RHOS)
    assert ei.value.status == et.ET_ERR_NUMERIC
    with pytest.raises(et.EtError):
        B.set_coeffs(_concat(torch, Ds), [0.02, -1.0, 0.02, 0.02, 0.02, 0.02])
    B.set_coeffs(_concat(torch, Ds), RHOS)
    with pytest.raises(et.EtError):
        B.run(_concat(torch, us)[:-1], TAU, 1)
    with pytest.raises(et.EtError):
        B.run(_concat(torch, us), -1.0, 1)
    with pytest.raises(et.EtError):
        B.set_variant(99)
    # a density outside [0, 1] is flagged on the host after the run
    hot = [u.copy() for u in us]
    hot[0].reshape(-1)[0] = 3.0
    u = _concat(torch, hot)
    B.run(u, TAU, 1)
    with pytest.raises(et.EtError) as ei:
        B.sync_info()
    assert ei.value.status == et.ET_ERR_NUMERIC


def test_batch_forced_schedule_and_option_checks(et_mod, torch_cuda):
    torch = torch_cuda
    Ds, us = _mixed_batch()
    nsteps = 2
    _, got, recs, _ = _batch_run(et_mod, torch_cuda, SHAPES, Ds, us, RHOS, nsteps, force_s=3, force_m=5)
    for i in range(len(SHAPES)):
        assert (recs[i]["s"], recs[i]["m"]) == (3, 5)
        # the same forced polynomial on the single-grid path
        want, rec = _single_run(et_mod, torch_cuda, Ds[i], us[i], RHOS[i], nsteps, force_s=3, force_m=5)
        assert (rec["s"], rec["m"]) == (3, 5)
        assert np.array_equal(got[i], want) or _errs(got[i], want)[0] <= 1e-13, i
    B = et_mod.Batch(SHAPES)
    with pytest.raises(et_mod.EtError):
        B.set_coeffs(_concat(torch, Ds), RHOS, force_m=1)


# Grids whose rows are 16-byte multiples in both FP32 and DF64 and whose
# fields stay 16-byte aligned in the concatenated layout: every grid can take
# the two-term launches (nz = 70 spans two column segments).
PAIR_SHAPES = [(70, 20, 36), (16, 9, 64), (33, 40, 40), (5, 3, 8)]
PAIR_RHOS = [0.025, 0.04, 0.015, 0.03]


@pytest.mark.parametrize("precision", ["f32", "df64"])
def test_two_term_batch_matches_single_grids(et_mod, torch_cuda, precision):
    Ds, us = [], []
    for i, sh in enumerate(PAIR_SHAPES):
        D, u0 = phantom.case(sh, seed=20 + i, noise=0.1)
        if not np.any(u0 > 0.1):
            u0 = np.zeros(sh)
            u0.reshape(-1)[u0.size // 2] = 0.8
        Ds.append(D)
        us.append(u0)
    nsteps = 3
    nvar = et_mod.load().et_batch_variant_count(et_mod.PRECISIONS[precision])
    for v in range(nvar // 2):  # the two-term variants
        B, got, recs, _ = _batch_run(et_mod, torch_cuda, PAIR_SHAPES, Ds, us, PAIR_RHOS, nsteps, precision,
                                     variant=v)
        for i in range(len(PAIR_SHAPES)):
            want, rec = _single_run(et_mod, torch_cuda, Ds[i], us[i], PAIR_RHOS[i], nsteps, precision)
            # the same pair-arithmetic residual and per-voxel term arithmetic
            assert np.array_equal(got[i], want), (v, i, np.abs(got[i] - want).max())
            if precision == "df64":
                ref = oracle.Problem(Ds[i], rho=PAIR_RHOS[i]).run(us[i], TAU, nsteps)[0]
                e_max, e_l2 = _errs(got[i], ref)
                assert e_max <= TOL64 and e_l2 <= TOL64, (v, i, e_max, e_l2)


@pytest.mark.parametrize("precision", ["f64", "df64", "f32"])
@pytest.mark.parametrize("op,scheme", [("conservative", "rosenbrock"), ("literal", "expeuler")])
def test_batch_zero_row_skip_matches_every_row_bitwise(et_mod, torch_cuda, precision, op, scheme):
    """The batched FP64 one-tile-per-block kernel and the DF64 kernels (one
    term per launch: warp rows marked per grid by et_batch_set_coeffs; two
    terms per launch: voxels whose six weights are zero) skip the products
    of rows without off-diagonal entries, and so do the residuals (FP32 and
    DF64: the pair-arithmetic one).  Every variant gives, bit for bit,
    the state of the same batch with every product evaluated
    (options.every_row) and, for FP64 variant 0, the single-grid path's.  Rows
    of 44 and 100 voxels end in a partial warp row; the last grid has D = 0."""
    torch = torch_cuda
    shapes = [(40, 36, 44), (9, 30, 100), (6, 7, 256), (7, 13, 3)]
    rhos = [0.025, 0.04, 0.015, 0.03]
    Ds, us = [], []
    for i, sh in enumerate(shapes):
        D, u0 = phantom.case(sh, seed=20 + i, noise=0.1)
        Ds.append(D * (0.0 if i == 3 else 1.0))
        us.append(u0 if np.any(u0 > 0.1) else np.full(sh, 0.3))
    nsteps = 3
    for v in _variants(et_mod, precision):
        B, skip, _, _ = _batch_run(et_mod, torch, shapes, Ds, us, rhos, nsteps, precision, variant=v, op=op,
                                   scheme=scheme)
        assert B.zero_row_voxels() == [zero_row_voxels(D, op) for D in Ds]
        _, full, _, _ = _batch_run(et_mod, torch, shapes, Ds, us, rhos, nsteps, precision, variant=v, op=op,
                                   scheme=scheme, every_row=True)
        for i in range(len(shapes)):
            assert np.array_equal(skip[i], full[i]), (precision, v, i)
    if precision == "f64":
        _, got, _, _ = _batch_run(et_mod, torch, shapes, Ds, us, rhos, nsteps, precision, variant=0, op=op,
                                  scheme=scheme)
        for i in range(len(shapes)):
            want = _single_run(et_mod, torch, Ds[i], us[i], rhos[i], nsteps, precision, op=op, scheme=scheme,
                               single_terms=True)[0]
            assert np.array_equal(got[i].reshape(shapes[i]), want), i
