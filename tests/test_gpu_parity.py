"""CUDA path vs the FP64 oracle, element by element, through the C ABI (GPU only).

Tolerance (FP64 kernels): max |u_gpu - u_oracle| <= 1e-10 * max|u_oracle| and the
same for the L2 norm, after every step.  FP32 kernels: errors are reported and
bounded by 1e-5 relative (their own arithmetic limit, not a parity claim)."""

import numpy as np
import pytest

import oracle
from zero_rows import zero_row_voxels as _zero_row_voxels
from paper_2402_02273_gb300 import phantom

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


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


def _errs(got, want):
    scale = np.abs(want).max()
    return (np.abs(got - want).max() / scale,
            np.linalg.norm((got - want).ravel()) / np.linalg.norm(want.ravel()))


def _gpu_states(et, torch, D, u0, tau, nsteps, precision="f64", op="conservative",
                scheme="rosenbrock", rho=0.025, **opts):
    """Runs nsteps single steps; returns the states after every step and the records."""
    g = et.Grid(D.shape, precision=precision)
    g.set_coeffs(torch.from_numpy(D.copy()).cuda(), rho=rho, op=op, scheme=scheme, **opts)
    u = torch.from_numpy(u0.copy()).cuda()
    states, recs = [], []
    for _ in range(nsteps):
        g.step(u, tau)
        recs.append(g.sync_info())
        states.append(u.cpu().numpy().reshape(D.shape).copy())
    return g, states, recs


def _compare_every_step(et, torch, D, u0, tau, nsteps, tol, **kw):
    rho = kw.get("rho", 0.025)
    P = oracle.Problem(D, rho=rho, op=kw.get("op", "conservative"), scheme=kw.get("scheme", "rosenbrock"))
    want, ost = P.run(u0, tau, nsteps, every=True)
    _, got, recs = _gpu_states(et, torch, D, u0, tau, nsteps, **kw)
    worst = 0.0
    for t in range(nsteps):
        e_max, e_l2 = _errs(got[t], want[t + 1])
        worst = max(worst, e_max, e_l2)
        assert e_max <= tol and e_l2 <= tol, (t, e_max, e_l2)
        assert recs[t]["mass"] == pytest.approx(ost[t]["mass"], rel=max(tol, 1e-12), abs=1e-300)
        assert recs[t]["umax"] == pytest.approx(ost[t]["umax"], rel=max(tol, 1e-12))
        assert recs[t]["umin"] == pytest.approx(ost[t]["umin"], abs=max(tol, 1e-12))
    return worst


FP64_FORMS = ["f64", "df64"]  # both held to the FP64 parity tolerance


@pytest.mark.parametrize("precision", FP64_FORMS)
def test_32cubed_10_steps(et_mod, torch_cuda, precision):
    """32^3 phantom, h = 1, tau = 7.3 d, 10 steps (white-matter D = 0.065)."""
    D, u0 = phantom.case(32, seed=0, d_white=0.065)
    _compare_every_step(et_mod, torch_cuda, D, u0, 7.3, 10, TOL64, precision=precision)


@pytest.mark.parametrize("precision", FP64_FORMS)
@pytest.mark.parametrize("op", ["conservative", "literal"])
@pytest.mark.parametrize("scheme", ["rosenbrock", "expeuler"])
def test_operator_and_scheme_readings(et_mod, torch_cuda, op, scheme, precision):
    D, u0 = phantom.case(24, seed=1, noise=0.1)
    _compare_every_step(et_mod, torch_cuda, D, u0, 7.3, 4, TOL64, op=op, scheme=scheme,
                        precision=precision)


@pytest.mark.parametrize("precision", FP64_FORMS)
@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 5, 1), (7, 1, 1), (1, 1, 45), (5, 17, 33),
                                   (9, 8, 40), (3, 70, 2)])
def test_ragged_and_degenerate_shapes(et_mod, torch_cuda, shape, precision):
    """Sizes that are not multiples of the 32 x 8 x 4 tile, lines, single voxels."""
    D = (0.01 + 0.2 * phantom.uniform(4, 7, int(np.prod(shape)))).reshape(shape)
    D = D.astype(np.float32).astype(np.float64)
    u0 = 0.9 * phantom.uniform(4, 8, D.size).reshape(shape)
    _compare_every_step(et_mod, torch_cuda, D, u0, 7.3, 3, TOL64, precision=precision)


@pytest.mark.parametrize("precision", FP64_FORMS)
@pytest.mark.parametrize("shift", [0, 1])
def test_unshifted_and_forced_schedules(et_mod, torch_cuda, shift, precision):
    D, u0 = phantom.case(20, seed=2, noise=0.1)
    _compare_every_step(et_mod, torch_cuda, D, u0, 7.3, 3, TOL64, shift=shift, precision=precision)
    # forced sub-stepping with many short sub-steps also matches
    _compare_every_step(et_mod, torch_cuda, D, u0, 7.3, 2, TOL64, shift=shift, force_s=5, force_m=14,
                        precision=precision)


def _run_states(et, torch, D, u0, tau, nsteps, precision, **kw):
    g = et.Grid(D.shape, precision=precision)
    opts = {k: v for k, v in kw.items() if k not in ("rho", "op", "scheme")}
    g.set_coeffs(torch.from_numpy(D.copy()).cuda(), rho=kw.get("rho", 0.025), op=kw.get("op", "conservative"),
                 scheme=kw.get("scheme", "rosenbrock"), **opts)
    u = torch.from_numpy(u0.copy()).cuda()
    g.run(u, tau, nsteps)
    rec = g.sync_info()
    rec["term_launches"] = g.timing()[1]
    return u.cpu().numpy().reshape(D.shape), rec


@pytest.mark.parametrize("precision", ["f32", "df64"])
@pytest.mark.parametrize("op,scheme", [("conservative", "rosenbrock"), ("literal", "rosenbrock"),
                                       ("conservative", "expeuler")])
@pytest.mark.parametrize("shape", [(5, 17, 33), (9, 8, 40), (1, 1, 45), (3, 70, 2), (40, 12, 36), (7, 19, 68),
                                   (33, 9, 64), (2, 3, 8), (6, 5, 4), (4, 9, 132), (6, 40, 128), (11, 23, 160),
                                   (5, 31, 96)])
@pytest.mark.parametrize("sched", [{}, {"force_s": 3, "force_m": 5}, {"force_s": 2, "force_m": 4},
                                   {"force_s": 1, "force_m": 2}])
def test_term_pairs_match_single_terms_bitwise(et_mod, torch_cuda, precision, op, scheme, shape, sched):
    """Two terms per launch (TMA-fed, on-chip first term) against one term per
    launch: the per-voxel arithmetic is the same, so the results are identical.
    Rows of a 16-byte multiple take the pair kernel (fewer launches), others run
    one term per launch.  The schedules cover odd and even term counts per
    sub-step, a lone trailing term, s = 1 (the pair finishes the step) and m = 2
    (no pair); the shapes cover ragged y and z, several x tiles and z segments.
    FP32 single terms on rows of a multiple of 4 voxels run the four-voxel
    kernel (rows of one quad, rows longer than a warp's 32 quads, rows split
    between blocks), so this also checks it against the two-term kernels.  FP32
    Horner pairs on such rows take the four-voxel two-term kernel (full-width
    tiles; the last three shapes have several tiles in y), running-sum pairs
    the TMA-fed one."""
    D = (0.01 + 0.2 * phantom.uniform(5, 7, int(np.prod(shape)))).reshape(shape)
    D = D.astype(np.float32).astype(np.float64)
    u0 = 0.9 * phantom.uniform(5, 8, D.size).reshape(shape)
    kw = dict(op=op, scheme=scheme, **sched)
    fused, rf = _run_states(et_mod, torch_cuda, D, u0, 7.3, 3, precision, two_terms=True, **kw)
    single, rs = _run_states(et_mod, torch_cuda, D, u0, 7.3, 3, precision, single_terms=True, **kw)
    assert (rf["s"], rf["m"]) == (rs["s"], rs["m"])
    # pairs run where TMA can address the rows, except the literal DF64 stage,
    # whose shared memory admits one block per SM (one-term launches are faster)
    eligible = (shape[2] * (4 if precision == "f32" else 8)) % 16 == 0
    eligible = eligible and not (op == "literal" and precision == "df64")
    if eligible and rf["m"] >= 3:
        assert rf["term_launches"] < rs["term_launches"]
    else:
        assert rf["term_launches"] <= rs["term_launches"]
    assert np.array_equal(fused, single), np.abs(fused - single).max()


@pytest.mark.parametrize("precision", FP64_FORMS)
def test_no_diffusion_and_no_growth_edge_cases(et_mod, torch_cuda, precision):
    shape = (6, 9, 35)
    pr = {"precision": precision}
    u0 = phantom.uniform(5, 1, int(np.prod(shape))).reshape(shape)
    # D = 0 everywhere: the pure-reaction closed form per voxel
    _compare_every_step(et_mod, torch_cuda, np.zeros(shape), u0, 7.3, 2, TOL64, **pr)
    _compare_every_step(et_mod, torch_cuda, np.zeros(shape), u0, 7.3, 2, TOL64, scheme="expeuler", **pr)
    # rho = 0: pure diffusion
    D, v0 = phantom.case(shape, seed=5, noise=0.1)
    _compare_every_step(et_mod, torch_cuda, D, v0, 7.3, 2, TOL64, rho=0.0, **pr)
    # u = 0 stays 0
    _, got, recs = _gpu_states(et_mod, torch_cuda, D, np.zeros(shape), 7.3, 2, **pr)
    assert np.all(got[-1] == 0) and recs[-1]["mass"] == 0


@pytest.mark.parametrize("shift", [1, 0])
def test_fp32_terms_error_is_reported_and_small(et_mod, torch_cuda, shift):
    D, u0 = phantom.case(32, seed=0, noise=0.1)
    P = oracle.Problem(D)
    want, _ = P.run(u0, 7.3, 10, every=True)
    _, got, recs = _gpu_states(et_mod, torch_cuda, D, u0, 7.3, 10, precision="f32", shift=shift)
    worst = 0.0
    for t in range(10):
        e_max, e_l2 = _errs(got[t], want[t + 1])
        worst = max(worst, e_max)
        assert e_max <= 1e-5 and e_l2 <= 1e-5, (t, e_max, e_l2)
        assert abs(recs[t]["mass"] - want[t + 1].sum()) <= 1e-5 * want[t + 1].sum()
    print(f"FP32 terms (shift={shift}): worst max-norm error over 10 steps {worst:.2e}")


def test_run_graph_direct_and_host_paths_agree_bitwise(et_mod, torch_cuda):
    torch = torch_cuda
    D, u0 = phantom.case(40, seed=3, noise=0.1)
    outs = []
    for use_graph in (True, False):
        g = et_mod.Grid(D.shape)
        g.set_coeffs(torch.from_numpy(D).cuda(), use_graph=use_graph)
        u = torch.from_numpy(u0.copy()).cuda()
        info = g.info_buffer(5)
        g.run(u, 7.3, 5, info)
        rec = g.sync_info()
        outs.append(u.cpu().numpy())
        recs = g.decode_info(info)
        assert list(recs["step"]) == [0, 1, 2, 3, 4]
        assert recs["mass"][-1] == rec["mass"]
        # a second identical run is bitwise identical (deterministic reductions)
        u2 = torch.from_numpy(u0.copy()).cuda()
        g.run(u2, 7.3, 5, info)
        g.sync_info()
        assert np.array_equal(u2.cpu().numpy(), outs[-1])
    assert np.array_equal(outs[0], outs[1])
    g = et_mod.Grid(D.shape)
    g.set_coeffs(D)  # host D path
    uh = u0.copy()
    rec = g.run_host(uh, 7.3, 5)
    assert np.array_equal(uh, outs[0].reshape(D.shape))
    assert rec["step"] == 4


@pytest.mark.parametrize("precision", ["f64", "df64", "f32"])
def test_new_coefficients_after_a_captured_run(et_mod, torch_cuda, precision):
    """et_set_coeffs keeps the grid's captured runs; a later run replays one
    only if every coefficient scalar it holds is unchanged.  A new D with the
    same bound rmax replays the graph (which reads the new weights), a new rho
    or a D with another bound captures a new one: every result equals that of
    a fresh grid with the same coefficients."""
    torch = torch_cuda
    D, u0 = phantom.case(40, seed=3, noise=0.1)
    g = et_mod.Grid(D.shape, precision=precision)
    g.set_coeffs(torch.from_numpy(D).cuda())
    r0 = g.rmax()
    # a D that differs at one tissue voxel but keeps the bound
    D_same = None
    for q in np.flatnonzero(D.ravel() > 0)[::97]:
        cand = D.copy()
        cand.reshape(-1)[q] *= 0.5
        g.set_coeffs(torch.from_numpy(cand).cuda())
        if g.rmax() == r0:
            D_same = cand
            break
    assert D_same is not None
    cases = [(D, 0.025), (D_same, 0.025), (D_same, 0.03), (D * 1.5, 0.03), (D, 0.025)]
    for Dc, rho in cases:
        g.set_coeffs(torch.from_numpy(Dc).cuda(), rho=rho)
        u = torch.from_numpy(u0.copy()).cuda()
        g.run(u, 7.3, 3)
        g.sync_info()
        fresh = et_mod.Grid(D.shape, precision=precision)
        fresh.set_coeffs(torch.from_numpy(Dc).cuda(), rho=rho)
        v = torch.from_numpy(u0.copy()).cuda()
        fresh.run(v, 7.3, 3)
        fresh.sync_info()
        assert torch.equal(u, v), (rho, float((u - v).abs().max()))


@pytest.mark.parametrize("precision", ["f32", "df64"])
def test_state_without_16_byte_alignment(et_mod, torch_cuda, precision):
    """A state u that is 8- but not 16-byte aligned (a view one element into a
    buffer) cannot take the vector kernels' 16-byte accesses: its steps run the
    one-voxel kernels, with identical results."""
    torch = torch_cuda
    D, u0 = phantom.case(24, seed=5, noise=0.1)
    outs = []
    for offset in (0, 1):
        g = et_mod.Grid(D.shape, precision=precision)
        g.set_coeffs(torch.from_numpy(D).cuda())
        buf = torch.zeros(u0.size + 2, dtype=torch.float64, device="cuda")
        u = buf[offset:offset + u0.size]
        assert (u.data_ptr() % 16 == 0) == (offset == 0)
        u.copy_(torch.from_numpy(u0.ravel()))
        g.run(u, 7.3, 3)
        g.sync_info()
        outs.append(u.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


@pytest.fixture(scope="module")
def oracle_128_three_steps():
    D, u0 = phantom.case(128, seed=0, noise=0.1)
    want, ost = oracle.Problem(D).run(u0, 7.3, 3)
    return D, u0, want, ost


@pytest.mark.parametrize("precision", FP64_FORMS)
def test_full_size_128cubed_first_steps_match_oracle(et_mod, torch_cuda, oracle_128_three_steps,
                                                     precision):
    """The bench workload (128^3, per-voxel D noise 10 %, tau = 7.3 d), first 3 steps
    element by element against the oracle, in the graph-replayed et_run path."""
    torch = torch_cuda
    D, u0, want, ost = oracle_128_three_steps
    g = et_mod.Grid(D.shape, precision=precision)
    g.set_coeffs(torch.from_numpy(D).cuda())
    u = torch.from_numpy(u0.copy()).cuda()
    info = g.info_buffer(3)
    g.run(u, 7.3, 3, info)
    g.sync_info()
    e_max, e_l2 = _errs(u.cpu().numpy().reshape(D.shape), want)
    assert e_max <= TOL64 and e_l2 <= TOL64, (e_max, e_l2)
    recs = g.decode_info(info)
    for t in range(3):
        assert recs["mass"][t] == pytest.approx(ost[t]["mass"], rel=1e-12)


def test_full_size_128cubed_100_steps_properties(et_mod, torch_cuda):
    """Full bench run (100 steps): density stays in [0, 1], the tumour mass grows
    monotonically, records agree with the field, and with rho = 0 the conservative
    operator keeps the mass to 1e-12 over all 100 steps."""
    torch = torch_cuda
    D, u0 = phantom.case(128, seed=0, noise=0.1)
    g = et_mod.Grid(D.shape)
    g.set_coeffs(torch.from_numpy(D).cuda())
    u = torch.from_numpy(u0.copy()).cuda()
    info = g.info_buffer(100)
    g.run(u, 7.3, 100, info)
    g.sync_info()
    recs = g.decode_info(info)
    uf = u.cpu().numpy()
    assert uf.min() >= -1e-12 and uf.max() <= 1 + 1e-12
    assert np.all(np.diff(recs["mass"]) > 0)
    assert recs["mass"][-1] == pytest.approx(uf.sum(), rel=1e-12)
    g.set_coeffs(torch.from_numpy(D).cuda(), rho=0.0)
    v = torch.from_numpy(u0.copy()).cuda()
    g.run(v, 7.3, 100, info)
    g.sync_info()
    assert v.sum().item() == pytest.approx(u0.sum(), rel=1e-12)


@pytest.fixture(scope="module")
def oracle_128_hundred_steps():
    D, u0 = phantom.case(128, seed=0, noise=0.1)
    states, ost = oracle.Problem(D).run(u0, 7.3, 100, every=True)
    return D, u0, states, ost


@pytest.mark.parametrize("precision", ["f64", "df64", "f32"])
def test_full_size_128cubed_100_steps_match_oracle(et_mod, torch_cuda, oracle_128_hundred_steps, precision):
    """The whole bench run, every step against the oracle: FP64 forms to 1e-10; the
    FP32 form's per-step max, L2 and mass errors are printed and bounded by 1e-5."""
    torch = torch_cuda
    D, u0, want, ost = oracle_128_hundred_steps
    g = et_mod.Grid(D.shape, precision=precision)
    g.set_coeffs(torch.from_numpy(D).cuda())
    u = torch.from_numpy(u0.copy()).cuda()
    tol = TOL64 if precision != "f32" else 1e-5
    worst = [0.0, 0.0, 0.0]
    for t in range(100):
        g.step(u, 7.3)
        rec = g.sync_info()
        got = u.cpu().numpy().reshape(D.shape)
        e_max, e_l2 = _errs(got, want[t + 1])
        e_mass = abs(rec["mass"] - ost[t]["mass"]) / ost[t]["mass"]
        worst = [max(worst[0], e_max), max(worst[1], e_l2), max(worst[2], e_mass)]
        if precision == "f32" and t % 10 == 9:
            print(f"f32 step {t + 1}: max {e_max:.2e} L2 {e_l2:.2e} mass {e_mass:.2e}")
        assert e_max <= tol and e_l2 <= tol and e_mass <= tol, (t, e_max, e_l2, e_mass)
    print(f"128^3 x 100 steps {precision}: worst max {worst[0]:.2e}, L2 {worst[1]:.2e}, "
          f"mass {worst[2]:.2e}")


@pytest.mark.parametrize("precision", FP64_FORMS + ["f32"])
@pytest.mark.parametrize("op,scheme", [("conservative", "rosenbrock"), ("literal", "expeuler")])
@pytest.mark.parametrize("shape", [(40, 36, 44), (9, 30, 100), (6, 7, 256)])
def test_zero_row_skip_matches_full_stencil_bitwise(et_mod, torch_cuda, precision, op, scheme, shape):
    """The one-term FP64 and DF64 kernels skip the stencil in warp rows
    without off-diagonal entries (D = 0 around them).  The count matches the
    one formed from D on the host, and the state equals, bit for bit, the one
    of the same run with every product evaluated (options.every_row); FP64
    also equals the batched form's one-tile-per-block variant, which skips the
    same rows.  One term per launch in every form; rows of 44 and 100 voxels
    end in a partial warp row, FP32 rows of a multiple of 4 voxels run the
    four-voxel kernel (which evaluates every row)."""
    torch = torch_cuda
    D, u0 = phantom.case(shape, seed=9, noise=0.1)
    Dd = torch.from_numpy(D).cuda()
    states = []
    for every_row in (False, True):
        g = et_mod.Grid(shape, precision=precision)
        g.set_coeffs(Dd, op=op, scheme=scheme, single_terms=True, every_row=every_row)
        zr = g.zero_row_voxels()
        assert zr == _zero_row_voxels(D, op)
        assert 0 < zr < D.size
        u = torch.from_numpy(u0.copy()).cuda()
        g.run(u, 7.3, 3)
        g.sync_info()
        states.append(u)
    assert torch.equal(states[0], states[1])
    if precision == "f64":
        B = et_mod.Batch([shape])
        B.set_coeffs(Dd, [0.025], op=op, scheme=scheme)
        B.set_variant(0)
        v = torch.from_numpy(u0.copy()).cuda()
        B.run(v, 7.3, 3)
        B.sync_info()
        assert torch.equal(states[0], v)


@pytest.mark.parametrize("precision", ["df64", "f32"])
@pytest.mark.parametrize("op,scheme", [("conservative", "rosenbrock"), ("literal", "expeuler")])
@pytest.mark.parametrize("shape", [(40, 36, 44), (9, 30, 100)])
@pytest.mark.parametrize("force_s", [0, 2])
def test_two_term_zero_voxel_skip_matches_every_product_bitwise(et_mod, torch_cuda, precision, op, scheme, shape,
                                                                force_s):
    """Two terms per launch: the TMA-fed DF64 kernel evaluates dt z + beta b
    alone at voxels whose six off-diagonal weights are zero (first and second
    term, halo voxels included).  Its states equal, bit for bit, those of the
    same runs with every product evaluated (options.every_row) and those of
    one term per launch; with s = 2 the running-sum pairs of the second
    sub-step run too.  FP32 (every voxel evaluated) is checked the same way."""
    torch = torch_cuda
    D, u0 = phantom.case(shape, seed=13, noise=0.1)
    Dd = torch.from_numpy(D).cuda()
    states = []
    for every_row, single in ((False, False), (True, False), (False, True)):
        g = et_mod.Grid(shape, precision=precision)
        g.set_coeffs(Dd, op=op, scheme=scheme, every_row=every_row, single_terms=single, two_terms=not single,
                     force_s=force_s, force_m=9 if force_s else 0)
        u = torch.from_numpy(u0.copy()).cuda()
        g.run(u, 7.3, 3)
        g.sync_info()
        states.append(u)
    assert torch.equal(states[0], states[1])
    assert torch.equal(states[0], states[2])
