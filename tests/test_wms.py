"""Learned weighted min-sum BP: training kernels through the C ABI.

The forward of the training path (T iterations, no early stop, every message stored) must equal
the oracle's weighted BP bit for bit; the hand-written backward must match central finite
differences of the loss computed with the FP64 oracle forward, along random directions and on
the coordinates with the largest gradient.
"""
import numpy as np
import pytest

import oracle
from tests import frames as fr

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

from paper_1609_09358_gb300 import api, build, wms  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    api.load()


def _setup(N, K, crc, B, T, ebn0, seed):
    ocode = fr.oracle_code(N, K, crc)
    code = fr.api_code(ocode)
    pay, llr = fr.frames(ocode, ebn0, B, seed=seed)
    u = np.stack([oracle.build_u(p, ocode) for p in pay])
    sign = (1.0 - 2.0 * u[:, ocode.info_idx]).astype(np.float64)
    rng = np.random.default_rng(seed)
    w = rng.uniform(0.7, 1.3, (T, 2, ocode.n, N)).astype(np.float32)
    return ocode, code, llr, sign, w


@pytest.mark.parametrize("N,K,crc,T", [(128, 64, 8, 5), (1024, 512, 16, 3), (256, 128, 16, 20)])
def test_wms_forward_bit_exact(N, K, crc, T):
    ocode, code, llr, _, w = _setup(N, K, crc, 9, T, 1.5, 31 + N)
    ref = oracle.bp_decode(llr, ocode, T, 20.0, "f32", early_stop=False, w=w)
    out = torch.empty((9, N), dtype=torch.float32, device="cuda")
    ws = torch.empty(api.wms_workspace_bytes(code, 9, T), dtype=torch.uint8, device="cuda")
    api.wms_forward(code, torch.from_numpy(llr).cuda(), T, 20.0, torch.from_numpy(w).cuda(), out, ws)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), ref["llr_u"])


def test_wms_backward_matches_oracle_gradient():
    """wms_backward against the oracle's reverse sweep on the same FP32 forward (the subgradient
    branches match exactly); the oracle's gradient is itself pinned to central differences."""
    T, B = 4, 12
    ocode, code, llr, _, w = _setup(128, 64, 8, B, T, 2.0, 5)
    rng = np.random.default_rng(3)
    dy = (rng.normal(size=(B, 128)) * (1 - ocode.frozen)).astype(np.float32)
    ws = torch.empty(api.wms_workspace_bytes(code, B, T), dtype=torch.uint8, device="cuda")
    out = torch.empty((B, 128), dtype=torch.float32, device="cuda")
    llr_d, w_d = torch.from_numpy(llr).cuda(), torch.from_numpy(w).cuda()
    gw = torch.empty_like(w_d)
    api.wms_forward(code, llr_d, T, 20.0, w_d, out, ws)
    api.wms_backward(code, llr_d, T, 20.0, w_d, torch.from_numpy(dy).cuda(), gw, ws)
    torch.cuda.synchronize()
    ref = oracle.wms_grad(llr, ocode, T, 20.0, w, dy.astype(np.float64), "f32")
    got = gw.double().cpu().numpy()
    assert np.abs(ref).max() > 0
    assert np.allclose(got, ref, rtol=1e-4, atol=1e-5 * np.abs(ref).max())


def test_wms_all_iterations_forward_and_backward():
    """Per-iteration outputs: iteration t's LLR(u) equals the oracle's weighted BP run for t + 1
    iterations (bit for bit), and the backward of a loss over every iteration equals the oracle's
    reverse sweep of the same loss."""
    T, B = 5, 10
    ocode, code, llr, _, w = _setup(128, 64, 8, B, T, 2.0, 6)
    ws = torch.empty(api.wms_workspace_bytes(code, B, T), dtype=torch.uint8, device="cuda")
    out = torch.empty((T, B, 128), dtype=torch.float32, device="cuda")
    llr_d, w_d = torch.from_numpy(llr).cuda(), torch.from_numpy(w).cuda()
    api.wms_forward(code, llr_d, T, 20.0, w_d, out, ws)
    rng = np.random.default_rng(8)
    dy = (rng.normal(size=(T, B, 128)) * (1 - ocode.frozen)).astype(np.float32)
    gw = torch.empty_like(w_d)
    api.wms_backward(code, llr_d, T, 20.0, w_d, torch.from_numpy(dy).cuda(), gw, ws)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for t in range(T):
        ref = oracle.bp_decode(llr, ocode, t + 1, 20.0, "f32", early_stop=False, w=w)
        assert np.array_equal(got[t], ref["llr_u"]), t
    ref_g = oracle.wms_grad(llr, ocode, T, 20.0, w, dy.astype(np.float64), "f32", all_iters=True)
    g = gw.double().cpu().numpy()
    assert np.abs(ref_g).max() > 0
    assert np.allclose(g, ref_g, rtol=1e-4, atol=1e-5 * np.abs(ref_g).max())


def test_wms_autograd_matches_finite_differences():
    """The torch.autograd wrapper: per-coordinate central differences of the BCE loss through the
    FP64 oracle forward, on the coordinates with the largest gradient."""
    T, B = 4, 12
    ocode, code, llr, sign, w = _setup(128, 64, 8, B, T, 2.0, 5)
    w_t = torch.from_numpy(w).cuda().requires_grad_(True)
    y = wms.wms_llr_u(w_t, torch.from_numpy(llr).cuda(), code, T, 20.0)
    loss = wms.bce_loss(y, torch.from_numpy(sign).float().cuda(), torch.as_tensor(ocode.info_idx).long().cuda())
    loss.backward()
    g = w_t.grad.double().cpu().numpy()

    def loss64(ww):
        yy = oracle.bp_decode(llr, ocode, T, 20.0, "f64", early_stop=False, w=ww, llr_u_double=True)["llr_u_f64"]
        return float(np.mean(np.logaddexp(0.0, -sign * yy[:, ocode.info_idx])))

    h, agree = 1e-5, 0
    flat = np.argsort(-np.abs(g).ravel())[:8]
    for idx in flat:
        wp, wm = w.copy(), w.copy()
        wp.flat[idx] += h
        wm.flat[idx] -= h
        fd = (loss64(wp) - loss64(wm)) / (float(wp.flat[idx]) - float(wm.flat[idx]))
        agree += abs(fd - g.flat[idx]) <= 1e-2 * abs(g.flat[idx]) + 1e-7
    assert agree >= 7, agree  # a perturbation may straddle a min/clip kink


@pytest.mark.parametrize("all_iters", [False, True])
def test_wms_training_reduces_loss(all_iters):
    code = fr.api_code(fr.oracle_code(128, 64, 8))
    w, hist = wms.train(code, T=5, steps=40, batch=512, lr=1e-2, log_every=10, all_iters=all_iters)
    assert hist[-1][1] < hist[0][1], hist
    assert torch.isfinite(w).all()
