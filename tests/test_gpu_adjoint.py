"""The GPU adjoint (et_vjp, discrete reverse mode with checkpointing) against the
oracle's own adjoint, against central finite differences of the GPU forward map,
and through torch.autograd.  GPU only."""
import numpy as np
import pytest

import oracle
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


def _problem(shape, seed=3):
    D, u0 = phantom.case(shape, seed=seed, noise=0.1)
    tgt = 0.5 * phantom.uniform(seed, 11, D.size).reshape(shape)
    return D, u0, tgt


@pytest.mark.parametrize("op", ["conservative", "literal"])
@pytest.mark.parametrize("scheme", ["rosenbrock", "expeuler"])
def test_vjp_matches_oracle_adjoint(env, op, scheme):
    et, torch = env
    shape, tau, K = (18, 20, 22), 7.3, 4
    D, u0, tgt = _problem(shape)
    P = oracle.Problem(D, op=op, scheme=scheme)
    uK, _ = P.run(u0, tau, K)
    o_ub, o_rho, o_ds = oracle.vjp(P, u0, tau, K, uK - tgt)
    g = et.Grid(shape)
    g.set_coeffs(torch.from_numpy(D).cuda(), op=op, scheme=scheme)
    u0d = torch.from_numpy(u0.copy()).cuda()
    ubarK = torch.from_numpy((uK - tgt).copy()).cuda()
    ub, g_rho, g_ds = g.vjp(u0d, tau, K, ubarK, checkpoint_every=3)
    ub = ub.cpu().numpy().reshape(shape)
    assert np.abs(ub - o_ub).max() <= 1e-9 * np.abs(o_ub).max()
    assert g_rho == pytest.approx(o_rho, rel=1e-9)
    assert g_ds == pytest.approx(o_ds, rel=1e-9)


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("op", ["conservative", "literal"])
def test_zero_row_skip_leaves_the_gradient_unchanged(env, precision, op):
    """The reverse terms of the conservative operator skip the transpose
    products of rows without off-diagonal entries (a symmetric operator's
    empty row is an empty column); the forward chains skip them as well.  The
    gradients equal those with every product evaluated (options.every_row)
    bit for bit; the literal operator, whose transpose is not empty there,
    is checked the same way."""
    et, torch = env
    shape, tau, K = (12, 30, 44), 7.3, 4
    D, u0, tgt = _problem(shape, seed=6)
    got = []
    for every_row in (False, True):
        g = et.Grid(shape, precision=precision)
        g.set_coeffs(torch.from_numpy(D).cuda(), op=op, every_row=every_row)
        assert g.zero_row_voxels() > 0
        got.append(g.vjp(torch.from_numpy(u0.copy()).cuda(), tau, K, torch.from_numpy(tgt.copy()).cuda(),
                         checkpoint_every=2))
    assert torch.equal(got[0][0], got[1][0]) and got[0][1] == got[1][1] and got[0][2] == got[1][2]


def test_checkpoint_spacing_does_not_change_the_gradient(env):
    et, torch = env
    shape, tau, K = (16, 16, 16), 7.3, 7
    D, u0, tgt = _problem(shape, seed=5)
    g = et.Grid(shape)
    g.set_coeffs(torch.from_numpy(D).cuda())
    u0d = torch.from_numpy(u0.copy()).cuda()
    ubarK = torch.from_numpy(tgt.copy()).cuda()
    ref = g.vjp(u0d, tau, K, ubarK, checkpoint_every=1)
    for ck in (2, 3, 7, 50):
        got = g.vjp(u0d, tau, K, ubarK, checkpoint_every=ck)
        assert torch.equal(got[0], ref[0]) and got[1] == ref[1] and got[2] == ref[2]


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_checkpointed_forward_and_reverse_equal_vjp(env, precision):
    """et_run_checkpointed + et_vjp_checkpointed (one forward pass shared with
    the caller's run) give et_run's state and et_vjp's gradients bitwise."""
    et, torch = env
    shape, tau, K, ck = (20, 18, 24), 7.3, 7, 3
    D, u0, tgt = _problem(shape, seed=9)
    g = et.Grid(shape, precision=precision)
    g.set_coeffs(torch.from_numpy(D).cuda())
    u0d = torch.from_numpy(u0.copy()).cuda()
    u_run = u0d.clone()
    g.run(u_run, tau, K)
    u_ck = u0d.clone()
    ws = g.run_checkpointed(u_ck, tau, K, ck)
    torch.cuda.synchronize()
    assert torch.equal(u_run, u_ck)
    ubarK = (u_ck - torch.from_numpy(tgt.copy()).cuda()).contiguous()
    ref = g.vjp(u0d, tau, K, ubarK, checkpoint_every=ck)
    got = g.vjp_checkpointed(ws, tau, K, ubarK, checkpoint_every=ck)
    assert torch.equal(got[0], ref[0]) and got[1] == ref[1] and got[2] == ref[2]


def test_fp32_adjoint_error_is_small(env):
    et, torch = env
    shape, tau, K = (18, 20, 22), 7.3, 4
    D, u0, tgt = _problem(shape)
    P = oracle.Problem(D)
    uK, _ = P.run(u0, tau, K)
    o_ub, o_rho, o_ds = oracle.vjp(P, u0, tau, K, uK - tgt)
    g = et.Grid(shape, precision="f32")
    g.set_coeffs(torch.from_numpy(D).cuda())
    ub, g_rho, g_ds = g.vjp(torch.from_numpy(u0.copy()).cuda(), tau, K,
                            torch.from_numpy((uK - tgt).copy()).cuda(), checkpoint_every=2)
    ub = ub.cpu().numpy().reshape(shape)
    err = np.abs(ub - o_ub).max() / np.abs(o_ub).max()
    print(f"FP32 adjoint vs oracle: u0 {err:.2e}, rho {abs(g_rho / o_rho - 1):.2e}, "
          f"D scale {abs(g_ds / o_ds - 1):.2e}")
    assert err <= 1e-4
    assert g_rho == pytest.approx(o_rho, rel=1e-4)
    assert g_ds == pytest.approx(o_ds, rel=1e-4)


@pytest.mark.parametrize("sched", [{}, {"force_s": 2, "force_m": 5}, {"force_s": 3, "force_m": 4}])
def test_fp32_recorded_pairs_equal_single_terms(env, sched):
    """On TMA-eligible rows the FP32 adjoint can record its forward chains with
    the two-term kernel (storing both terms); the gradients equal those of the
    one-term recording (the four-voxel kernel, the default) bitwise, and stay
    within the FP32 bound of the oracle's."""
    et, torch = env
    shape, tau, K = (18, 20, 24), 7.3, 4
    D, u0, tgt = _problem(shape, seed=4)
    P = oracle.Problem(D)
    uK, _ = P.run(u0, tau, K)
    o_ub, o_rho, o_ds = oracle.vjp(P, u0, tau, K, uK - tgt)
    got = []
    for two in (True, False):
        g = et.Grid(shape, precision="f32")
        g.set_coeffs(torch.from_numpy(D).cuda(), two_terms=two, **sched)
        got.append(g.vjp(torch.from_numpy(u0.copy()).cuda(), tau, K,
                         torch.from_numpy((uK - tgt).copy()).cuda(), checkpoint_every=2))
    assert torch.equal(got[0][0], got[1][0]) and got[0][1] == got[1][1] and got[0][2] == got[1][2]
    if not sched:
        ub = got[0][0].cpu().numpy().reshape(shape)
        assert np.abs(ub - o_ub).max() <= 1e-4 * np.abs(o_ub).max()
        assert got[0][1] == pytest.approx(o_rho, rel=1e-4)
        assert got[0][2] == pytest.approx(o_ds, rel=1e-4)


def test_128cubed_50_steps_against_central_differences(env):
    """128^3, 50 steps, checkpoints every 10; target from the forward model with
    rho x 1.1, D scale x 1.1 and the seed shifted by 2 voxels; gradients in rho, the D
    scale and a random direction of u0 against central differences (eps 1e-6)."""
    et, torch = env
    shape, tau, K = (128, 128, 128), 7.3, 50
    D, u0 = phantom.case(shape, seed=0, noise=0.1)
    cx, cy, cz = phantom.seed_centre(shape)
    u0_tgt = phantom.gaussian_blob(shape, (cx + 2.0, cy, cz))
    Dd = torch.from_numpy(D).cuda()
    g = et.Grid(shape)

    def forward(u_init, rho, ds):
        g.set_coeffs(Dd * ds, rho=rho)
        u = torch.from_numpy(np.ascontiguousarray(u_init)).cuda() if isinstance(u_init, np.ndarray) else u_init.clone()
        g.run(u, tau, K)
        g.sync_info()
        return u

    tgt = forward(u0_tgt, 0.025 * 1.1, 1.1)
    loss = lambda u: 0.5 * float(((u - tgt) ** 2).sum())
    rho, ds = 0.025, 1.0
    uK = forward(u0, rho, ds)
    g.set_coeffs(Dd, rho=rho)
    u0d = torch.from_numpy(u0.copy()).cuda()
    ub, g_rho, g_ds = g.vjp(u0d, tau, K, uK - tgt, checkpoint_every=10)
    eps = 1e-6
    fd_rho = (loss(forward(u0, rho + eps, ds)) - loss(forward(u0, rho - eps, ds))) / (2 * eps)
    fd_ds = (loss(forward(u0, rho, ds + eps)) - loss(forward(u0, rho, ds - eps))) / (2 * eps)
    v = phantom.uniform(9, 9, D.size).reshape(shape) - 0.5
    v *= (u0 > 1e-3)  # a direction inside the seed
    fd_u = (loss(forward(u0 + eps * v, rho, ds)) - loss(forward(u0 - eps * v, rho, ds))) / (2 * eps)
    ad_u = float((ub.cpu() * torch.from_numpy(v)).sum())
    print(f"128^3 x 50: rho {g_rho:.6e} vs fd {fd_rho:.6e}; D scale {g_ds:.6e} vs {fd_ds:.6e}; "
          f"u0 dir {ad_u:.6e} vs {fd_u:.6e}")
    assert g_rho == pytest.approx(fd_rho, rel=1e-5)
    assert g_ds == pytest.approx(fd_ds, rel=1e-5)
    assert ad_u == pytest.approx(fd_u, rel=1e-5)
    # the FP32 adjoint of the FP32 forward, checked against these FP64 gradients
    gf = et.Grid(shape, precision="f32")
    gf.set_coeffs(Dd, rho=rho)
    uf = u0d.clone()
    gf.run(uf, tau, K)
    ubf, f_rho, f_ds = gf.vjp(u0d, tau, K, (uf - tgt).contiguous(), checkpoint_every=10)
    f_u = float((ubf.cpu() * torch.from_numpy(v)).sum())
    print(f"FP32 adjoint at 128^3 x 50: rho {abs(f_rho / g_rho - 1):.2e}, D scale {abs(f_ds / g_ds - 1):.2e}, "
          f"u0 dir {abs(f_u / ad_u - 1):.2e} relative to FP64")
    assert f_rho == pytest.approx(g_rho, rel=1e-4)
    assert f_ds == pytest.approx(g_ds, rel=1e-4)
    assert f_u == pytest.approx(ad_u, rel=1e-4)


def test_autograd_function_gradients(env):
    et, torch = env
    shape, tau, K = (10, 11, 12), 7.3, 3
    D, u0, tgt = _problem(shape, seed=8)
    D0 = torch.from_numpy(D).cuda()
    u0d = torch.from_numpy(u0.copy()).cuda().requires_grad_(True)
    rho = torch.tensor(0.03, dtype=torch.float64, requires_grad=True)
    ds = torch.tensor(1.2, dtype=torch.float64, requires_grad=True)
    tg = torch.from_numpy(tgt.copy()).cuda()
    uK = et.tumour_run(u0d, rho, ds, D0, tau, K, checkpoint_every=2)
    loss = 0.5 * ((uK - tg) ** 2).sum()
    loss.backward()
    # the oracle's gradient at the same point (D = 1.2 D0, rho = 0.03)
    P = oracle.Problem(1.2 * D, rho=0.03)
    oK, _ = P.run(u0, tau, K)
    o_ub, o_rho, o_ds = oracle.vjp(P, u0, tau, K, oK - tgt)
    assert np.abs(u0d.grad.cpu().numpy() - o_ub).max() <= 1e-9 * np.abs(o_ub).max()
    assert rho.grad.item() == pytest.approx(o_rho, rel=1e-9)
    assert ds.grad.item() == pytest.approx(o_ds / 1.2, rel=1e-9)


def test_scaled_coefficients_equal_a_scaled_field_bitwise():
    """et_set_coeffs_scaled reads dscale * D in the coefficient kernel: the same
    weights, and so the same run, as et_set_coeffs on the field scaled in FP64
    beforehand (the autograd function uses it for its D scale)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2402_02273_gb300 as et
    D, u0 = phantom.case((14, 12, 20), seed=8, noise=0.1)
    Dd = torch.from_numpy(D).cuda()
    outs = []
    for scaled in (True, False):
        g = et.Grid(D.shape)
        if scaled:
            g.set_coeffs(Dd, dscale=1.7)
        else:
            g.set_coeffs(Dd * 1.7)
        u = torch.from_numpy(u0.copy()).cuda()
        g.run(u, 7.3, 3)
        g.sync_info()
        outs.append((u.cpu().numpy(), g.rmax()))
    assert np.array_equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1]
    g = et.Grid(D.shape)
    with pytest.raises(et.EtError) as ex:
        g.set_coeffs(Dd, dscale=-1.0)
    assert ex.value.status == et.ET_ERR_ARG
