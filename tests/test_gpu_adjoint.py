"""Log-domain forward and the adjoint kernel against the FP64 oracle.

Forward: log-beliefs within 1e-5 relative (per node, as for the linear path).
Gradient: elementwise dL/d log g, dL/df(d), dL/dfbar against torch autograd of
the FP64 dense forward, and dL/d alpha, fbar, beta against central finite
differences in FP64, within 1e-4 * max(1, |reference|)."""
import numpy as np
import pytest

from oracle import gradient, grid
from paper_1010_0012_gb300 import workload as wl
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu
GRAD_TOL = 1e-4


def _close(got, ref, tol=GRAD_TOL):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return np.all(np.abs(got - ref) <= tol * np.maximum(1.0, np.abs(ref)))


@pytest.mark.parametrize("M,T,schedule", [(16, 2, "sync"), (17, 1, "sync"), (64, 3, "sync"), (32, 4, "redblack")])
def test_log_forward_matches_oracle(M, T, schedule):
    cfg = wl.small_config("lg", 19, 11, M, T, alpha=0.9, structure="planar", seed=M)
    st, g, _ = H.stereo_inputs(cfg)
    tab, fbar = wl.pair_table_f32(cfg.alpha, T)
    H.check_sum_case(g, tab, T, fbar, 7, schedule, log=True)


def _gpu_grad(cost, d_gt, alpha, fbar, beta, T, K, every, on_torch_stream=False, params_on_gpu=False):
    import torch
    from paper_1010_0012_gb300 import autograd, bp
    Hh, W, M = cost.shape
    G = bp.BPGrid(W, Hh, M, bp.BP_F32, stream=torch.cuda.current_stream() if on_torch_stream else None)
    pdev = "cuda" if params_on_gpu else "cpu"
    a = torch.tensor(alpha, dtype=torch.float32, device=pdev, requires_grad=True)
    fb = torch.tensor(fbar, dtype=torch.float32, device=pdev, requires_grad=True)
    b = torch.tensor(beta, dtype=torch.float32, device="cuda", requires_grad=True)
    cost_t = torch.from_numpy(np.ascontiguousarray(cost, dtype=np.float32)).cuda()
    loss = autograd.stereo_nll(cost_t, d_gt, a, fb, b, T, K, G, every)
    loss.backward()
    out = {"loss": float(loss.detach()), "d_alpha": float(a.grad), "d_fbar": float(fb.grad), "d_beta": float(b.grad)}
    G.close()
    return out


def test_adjoint_elementwise_against_fp64_autograd():
    import torch
    from paper_1010_0012_gb300 import autograd, bp
    cfg = wl.small_config("ad", 12, 9, 16, 2, alpha=1.0, structure="planar", seed=5)
    st = wl.make_stereo(cfg)
    T, K, beta = cfg.T, 6, 0.1
    d = np.arange(-T, T + 1)
    table = np.exp(-cfg.alpha * np.abs(d)).astype(np.float32)
    fbar = float(np.float32(np.exp(-cfg.alpha * T)))
    logg = (-beta * st.cost.astype(np.float64)).astype(np.float32)
    ref = gradient.reference_gradient_table(-logg.astype(np.float64) / beta, st.d_gt, table.astype(np.float64),
                                            fbar, beta, T, K)
    G = bp.BPGrid(cfg.W, cfg.H, cfg.M, bp.BP_F32)
    lg = torch.from_numpy(logg).cuda().requires_grad_(True)
    tab = torch.from_numpy(table).requires_grad_(True)
    fb = torch.tensor(fbar, dtype=torch.float32, requires_grad=True)
    logb = autograd.log_beliefs(lg, tab, fb, G, T, K, every=2)
    idx = torch.as_tensor(st.d_gt, dtype=torch.long, device="cuda")[..., None]
    loss = -torch.gather(logb, -1, idx).sum()
    loss.backward()
    assert abs(float(loss.detach()) - ref["loss"]) <= 1e-5 * abs(ref["loss"])
    assert _close(lg.grad.cpu().numpy(), ref["d_logg"])
    assert _close(tab.grad.numpy(), ref["d_table"])
    assert _close(float(fb.grad), ref["d_fbar"])
    G.close()


@pytest.mark.parametrize("every", [1, 4, 13])
def test_checkpoint_interval_does_not_change_the_gradient(every):
    cfg = wl.small_config("ck", 14, 10, 32, 3, alpha=0.7, structure="planar", seed=9)
    st = wl.make_stereo(cfg)
    base = _gpu_grad(st.cost, st.d_gt, 0.7, float(np.exp(-0.7 * 3)), 0.1, 3, 13, 13)
    got = _gpu_grad(st.cost, st.d_gt, 0.7, float(np.exp(-0.7 * 3)), 0.1, 3, 13, every)
    for k in base:
        assert got[k] == base[k], (k, got[k], base[k])


@pytest.mark.parametrize("W,Hh,K", [(96, 96, 30), (256, 256, 30)])
def test_parameter_gradients_against_finite_differences(W, Hh, K):
    """The 256 x 256, M = 64, T = 3, 30-iteration workload (checkpoint every 5)
    and a reduced grid with the same recipe."""
    base = wl.CONFIGS["grid256_m64_grad"]
    import dataclasses
    cfg = dataclasses.replace(base, W=W, H=Hh)
    st = wl.make_stereo(cfg)
    alpha, beta, T = cfg.alpha, cfg.beta, cfg.T
    fbar = float(np.exp(-alpha * T))
    # both sides see the same float32-rounded parameters
    alpha32, fbar32, beta32 = (float(np.float32(v)) for v in (alpha, fbar, beta))
    gpu = _gpu_grad(st.cost, st.d_gt, alpha32, fbar32, beta32, T, K, 5)
    fd = gradient.finite_difference(st.cost.astype(np.float64), st.d_gt, alpha32, fbar32, beta32, T, K)
    errs = {k: abs(gpu[k] - fd[k]) / max(1.0, abs(fd[k])) for k in ("d_alpha", "d_fbar", "d_beta")}
    assert all(e <= GRAD_TOL for e in errs.values()), (errs, gpu, fd)


def test_backward_without_recorded_forward_is_a_state_error():
    import torch
    from paper_1010_0012_gb300 import bp
    G = bp.BPGrid(6, 5, 16, bp.BP_F32)
    G.set_unary(torch.ones((5, 6, 16), device="cuda"))
    tab, fbar = wl.pair_table_f32(1.0, 2)
    G.set_potential(tab, 2, fbar)
    G.reset()
    G.iterate(3, bp.BP_SUM | bp.BP_LOG)
    with pytest.raises(bp.BPError) as ei:
        bp.bp_backward(G.h, torch.zeros((5, 6, 16), device="cuda"), torch.zeros((5, 6, 16), device="cuda"), 5)
    assert ei.value.status == bp.BP_ERR_STATE
    G.close()


def test_ill_conditioned_beta_gradient_stays_at_the_fp32_floor():
    """On 40 x 32 cells of the same workload, dL/d beta = sum_i,x dL/d log g_i(x)
    (-cost_i(x)) is the small difference of large terms (sum of |terms| is
    ~3400 times the result), so FP32 rounding carried through 30 iterations,
    not the method, sets its accuracy.  The bar there: the error stays below
    2^-24 * K * sum |dL/d log g * cost| (each per-node term accurate to K
    rounding steps), with alpha and fbar still within 1e-4."""
    import dataclasses
    cfg = dataclasses.replace(wl.CONFIGS["grid256_m64_grad"], W=40, H=32)
    st = wl.make_stereo(cfg)
    alpha, beta, T, K = cfg.alpha, cfg.beta, cfg.T, 30
    a32, f32, b32 = (float(np.float32(v)) for v in (alpha, float(np.exp(-alpha * T)), beta))
    gpu = _gpu_grad(st.cost, st.d_gt, a32, f32, b32, T, K, 5)
    fd = gradient.finite_difference(st.cost.astype(np.float64), st.d_gt, a32, f32, b32, T, K)
    ref = gradient.reference_gradient(st.cost.astype(np.float64), st.d_gt, a32, f32, b32, T, K)
    floor = 2.0 ** -24 * K * float(np.sum(np.abs(ref["d_logg"] * st.cost)))
    assert abs(gpu["d_beta"] - fd["d_beta"]) <= floor
    for k in ("d_alpha", "d_fbar"):
        assert abs(gpu[k] - fd[k]) <= GRAD_TOL * max(1.0, abs(fd[k]))


def test_grid_on_torch_stream_gives_the_same_gradient():
    """A grid created on torch's current stream skips the host synchronisation
    between the library's forward and torch's next operations; the gradient
    must be the same bit for bit."""
    import dataclasses
    cfg = dataclasses.replace(wl.CONFIGS["grid256_m64_grad"], W=48, H=40)
    st = wl.make_stereo(cfg)
    args = (st.cost, st.d_gt, 0.9, float(np.float32(np.exp(-0.9 * cfg.T))), 0.1, cfg.T, 12, 4)
    a = _gpu_grad(*args)
    b = _gpu_grad(*args, on_torch_stream=True)
    assert a == b


def test_parameters_on_the_gpu_give_the_same_gradient():
    """With the table f(d) and fbar on the GPU the backward takes the
    device-output reverse pass (bp_backward_device: no host wait).  Given the
    same parameter values, the gradients wrt log g, f(d) and fbar must equal
    the host path's bit for bit, on the handle's own stream and on torch's."""
    import dataclasses
    import torch
    from paper_1010_0012_gb300 import autograd, bp
    cfg = dataclasses.replace(wl.CONFIGS["grid256_m64_grad"], W=48, H=40)
    st = wl.make_stereo(cfg)
    T, K = cfg.T, 12
    logg0 = torch.from_numpy((-0.1 * st.cost).astype(np.float32)).cuda()
    tab = np.exp(-0.9 * np.abs(np.arange(-T, T + 1))).astype(np.float32)
    fbar = np.float32(np.exp(-0.9 * (T + 1)))
    wts = torch.from_numpy(np.random.default_rng(3).standard_normal(logg0.shape).astype(np.float32)).cuda()
    outs = []
    for dev, torch_stream in (("cpu", False), ("cuda", False), ("cuda", True)):
        G = bp.BPGrid(cfg.W, cfg.H, cfg.M, bp.BP_F32, stream=torch.cuda.current_stream() if torch_stream else None)
        lg = logg0.clone().requires_grad_(True)
        tab_t = torch.tensor(tab, device=dev, requires_grad=True)
        fb_t = torch.tensor(fbar, device=dev, requires_grad=True)
        logb = autograd.log_beliefs(lg, tab_t, fb_t, G, T, K, 4)
        (logb * wts).sum().backward()
        outs.append((lg.grad.cpu().numpy(), tab_t.grad.cpu().numpy(), float(fb_t.grad)))
        G.close()
    for o in outs[1:]:
        np.testing.assert_array_equal(o[0], outs[0][0])
        np.testing.assert_array_equal(o[1], outs[0][1])
        assert o[2] == outs[0][2]


@pytest.mark.parametrize("M,T,K", [(16, 3, 7), (8, 9, 5), (16, 2, 0)])
def test_backward_device_equals_backward(M, T, K):
    """bp_backward_device writes the same float64 parameter gradients as
    bp_backward, including the zero entries of |d| > M - 1 (T = 9 > 7) and a
    recorded run of no iterations, and the same dL/d log g."""
    import torch
    from paper_1010_0012_gb300 import bp
    rng = np.random.default_rng(M + T + K)
    W, Hh = 9, 7
    logg = torch.from_numpy(rng.uniform(-3.0, 0.0, (Hh, W, M)).astype(np.float32)).cuda()
    tab = np.exp(-0.7 * np.abs(np.arange(-T, T + 1))).astype(np.float32)
    fbar = float(np.float32(np.exp(-0.7 * (T + 1))))
    dlogb = torch.from_numpy(rng.standard_normal((Hh, W, M)).astype(np.float32)).cuda()
    outs = []
    for device_out in (False, True):
        G = bp.BPGrid(W, Hh, M, bp.BP_F32)
        bp.bp_set_unary_log(G.h, logg)
        bp.bp_set_potential(G.h, tab, T, fbar, bp.BP_F32)
        bp.bp_set_checkpoint_interval(G.h, 3)
        G.reset()
        bp.bp_iterate(G.h, K, bp.BP_SUM | bp.BP_LOG | bp.BP_RECORD, bp.BP_SYNC)
        logb = torch.empty_like(logg)
        bp.bp_beliefs(G.h, logb)
        dlogg = torch.empty_like(logg)
        if device_out:
            dt = torch.full((2 * T + 1,), 7.0, dtype=torch.float64, device="cuda")
            df = torch.full((1,), 7.0, dtype=torch.float64, device="cuda")
            bp.bp_backward_device(G.h, dlogb, dlogg, dt, df)
            G.sync()
            dtab, dfbar = dt.cpu().numpy(), float(df.cpu()[0])
        else:
            dtab, dfbar = bp.bp_backward(G.h, dlogb, dlogg, 2 * T + 1)
        outs.append((np.asarray(dtab), dfbar, dlogg.cpu().numpy()))
        G.close()
    (t0, f0, g0), (t1, f1, g1) = outs
    np.testing.assert_array_equal(t0, t1)
    assert f0 == f1
    np.testing.assert_array_equal(g0, g1)
    if T > M - 1:
        assert np.all(t1[:T - (M - 1)] == 0) and np.all(t1[T + M:] == 0)
