"""Learned weighted min-sum BP: per-edge, per-iteration scale factors trained by gradient descent.

The weighted BP multiplies every g term of the BP update (Sec. II-B) by a learned scale
w[t][dir][s-1][node] (dir 0: R message, 1: L message; node: the output node).  Forward and backward
are the hand-written CUDA kernels behind `wms_forward` / `wms_backward` of the C ABI; this module
only wires them into torch.autograd, draws training frames with the library's generator (Eb/N0
uniform per frame), and runs an optimiser.  Inference with trained weights goes through
`bp_decode` / `hybrid_decode` (wms_scales), with CRC early stop and CA-SCL as fallback.
"""
from __future__ import annotations

import math
import os

import torch

from . import api


class WMSFunction(torch.autograd.Function):
    """LLR(u) of T weighted BP iterations, [B][N] after the last iteration or [T][B][N] after every
    iteration (all_iters); gradient w.r.t. the weights [T][2][n][N]."""

    @staticmethod
    def forward(ctx, w, llr, code, T, llr_max, all_iters=False):
        B, N = llr.shape
        ws = torch.empty(api.wms_workspace_bytes(code, B, T), dtype=torch.uint8, device=llr.device)
        out = torch.empty((T, B, N) if all_iters else (B, N), dtype=torch.float32, device=llr.device)
        w = w.detach().contiguous()
        api.wms_forward(code, llr, T, llr_max, w, out, ws)
        ctx.save_for_backward(w, llr)
        ctx.ws, ctx.code, ctx.T, ctx.llr_max = ws, code, T, llr_max
        return out

    @staticmethod
    def backward(ctx, grad_out):
        w, llr = ctx.saved_tensors
        grad_w = torch.empty_like(w)
        api.wms_backward(ctx.code, llr, ctx.T, ctx.llr_max, w, grad_out.contiguous(), grad_w, ctx.ws)
        ctx.ws = None
        return grad_w, None, None, None, None, None


def wms_llr_u(w, llr, code: api.PolarCode, T: int, llr_max: float = 20.0, all_iters: bool = False):
    return WMSFunction.apply(w, llr, code, T, llr_max, all_iters)


def bce_loss(llr_u, u_info_sign, info_idx):
    """Mean binary cross-entropy of the information bits: softplus(-s * LLR) with s = 1 - 2u.
    llr_u [B][N], or [T][B][N] for the mean over iterations (the per-iteration loss)."""
    y = llr_u[..., info_idx]
    return torch.nn.functional.softplus(-u_info_sign * y).mean()


class FrameSource:
    """Seeded training batches from the library's generator kernels (Eb/N0 uniform per frame)."""

    def __init__(self, code: api.PolarCode, batch: int, ebn0_range=(1.0, 4.0), seed: int = 1609093583,
                 device="cuda"):
        self.code, self.B, self.lo, self.hi, self.seed = code, batch, ebn0_range[0], ebn0_range[1], seed
        self.dev = torch.device(device)
        self.gen = torch.Generator(device=self.dev)
        self.gen.manual_seed(seed)
        self.payload = torch.empty((batch, code.row_bytes), dtype=torch.uint8, device=self.dev)
        self.cw = torch.empty((batch, code.N // 8), dtype=torch.uint8, device=self.dev)
        self.llr = torch.empty((batch, code.N), dtype=torch.float32, device=self.dev)
        self.frame = 0
        self.info = torch.as_tensor(code.info_idx, dtype=torch.long, device=self.dev)

    def next(self):
        c = self.code
        api.polar_random_payload(self.B, c.P, self.seed, self.frame, self.payload)
        api.polar_encode(c, self.payload, self.cw)
        ebn0 = self.lo + (self.hi - self.lo) * torch.rand(self.B, generator=self.gen, device=self.dev)
        sig = torch.sqrt(1.0 / (2.0 * (c.P / c.N) * torch.pow(10.0, ebn0 / 10.0))).float().contiguous()
        api.polar_awgn_llr(self.cw, c.N, 1.0, self.seed, self.frame, self.llr, sigma_per_frame=sig)
        self.frame += self.B
        # bits of the information positions: x = u G, u = x G; read u back from the codeword
        bits = self.cw.unsqueeze(-1).bitwise_right_shift(torch.arange(8, device=self.dev, dtype=torch.uint8))
        x = (bits & 1).reshape(self.B, c.N)
        u = polar_transform_bits(x)
        sign = 1.0 - 2.0 * u[:, self.info].float()
        return self.llr, sign


def polar_transform_bits(x):
    """u = x G over GF(2) for a [B][N] 0/1 tensor (G is an involution); used for training labels."""
    u = x.clone()
    N = u.shape[1]
    d = 1
    while d < N:
        v = u.view(u.shape[0], N // (2 * d), 2, d)
        v[:, :, 0, :] ^= v[:, :, 1, :]
        d *= 2
    return u


def train(code: api.PolarCode, T: int = 20, steps: int = 300, batch: int = 4096, lr: float = 3e-3,
          ebn0_range=(1.0, 4.0), llr_max: float = 20.0, seed: int = 1609093583, log_every: int = 50,
          w0=None, device="cuda", all_iters: bool = False, w_max: float = 4.0):
    """Adam on the BCE of the information bits of LLR(u) after T iterations (all_iters: the mean
    of the BCE after every iteration, which rewards early convergence), each step followed by a
    projection of the scales onto [0, w_max]; returns (w, history).  With w_max = 1 the decoders
    take their unit-scale form (no clip of the scaled term; half2 frame pairs on one iteration)."""
    torch.manual_seed(seed)
    n, N = code.n, code.N
    w = (torch.ones((T, 2, n, N), dtype=torch.float32, device=device) if w0 is None else w0.clone().to(device))
    w.requires_grad_(True)
    opt = torch.optim.Adam([w], lr=lr)
    src = FrameSource(code, batch, ebn0_range, seed, device)
    hist = []
    for step in range(steps):
        llr, sign = src.next()
        y = wms_llr_u(w, llr, code, T, llr_max, all_iters)
        loss = bce_loss(y, sign, src.info)
        opt.zero_grad(set_to_none=True)
        loss.backward()
        opt.step()
        with torch.no_grad():
            w.clamp_(0.0, w_max)
        if step % log_every == 0 or step == steps - 1:
            hist.append((step, float(loss.item())))
    return w.detach(), hist


def save(path: str, w, code: api.PolarCode, T: int, meta: dict | None = None) -> None:
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    torch.save({"w": w.cpu(), "N": code.N, "K": code.K, "crc_len": code.crc_len, "T": T,
                "frozen": torch.as_tensor(code.frozen), "meta": meta or {}}, path)


def load(path: str, device="cuda"):
    d = torch.load(path, map_location="cpu")
    code = api.PolarCode(d["N"], d["K"], d["crc_len"], d["frozen"].numpy())
    return d["w"].to(device), code, d["T"], d.get("meta", {})


def sigma_of(ebn0_db: float, rate: float) -> float:
    return math.sqrt(1.0 / (2.0 * rate * 10.0 ** (ebn0_db / 10.0)))


# ------------------------------------------------------------------------ evaluation
def evaluate_point(code: api.PolarCode, ebn0_db: float, frames: int, variants: dict, L: int = 8, seed: int = 1609093584,
                   device="cuda") -> dict:
    """Hybrid decoding of the same seeded frames with each variant; variants maps a name to
    (max_iters, precision, weights or None).  Returns FER, BER, CA-SCL fallback rate and the
    decoding time of each."""
    P, N = code.P, code.N
    dev = torch.device(device)
    payload = torch.empty((frames, code.row_bytes), dtype=torch.uint8, device=dev)
    cw = torch.empty((frames, N // 8), dtype=torch.uint8, device=dev)
    llr = torch.empty((frames, N), dtype=torch.float32, device=dev)
    api.polar_random_payload(frames, P, seed, 0, payload)
    api.polar_encode(code, payload, cw)
    api.polar_awgn_llr(cw, N, sigma_of(ebn0_db, P / N), seed, 0, llr)
    dec = api.Decoder(code, frames, L, device=dev)
    out = {}
    for name, (imax, prec, w) in variants.items():
        M = 32.0 if prec == api.POLAR_FP16 else 20.0
        if w is not None:
            w = api.PreparedScales(code, w, prec)
        dec.hybrid(llr, imax, M, prec, w)  # warm-up (code tables, first launch)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        dec.hybrid(llr, imax, M, prec, w)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        ferr = (dec.bits != payload).any(dim=1)
        popc = torch.tensor([bin(v).count("1") for v in range(256)], dtype=torch.int64, device=dev)
        nbit = int(popc[(dec.bits ^ payload).long()].sum().item())
        out[name] = {"fer": float(ferr.float().mean().item()),
                     "ber": nbit / (frames * P),
                     "fallback_rate": float((dec.status != api.FRAME_BP_OK).float().mean().item()),
                     "avg_bp_iters": float(dec.iters.float().mean().item()),
                     "ms": ms, "gbit_s": P * frames / (ms * 1e-3) / 1e9}
    return out


def main(argv=None):
    import argparse
    import json
    ap = argparse.ArgumentParser(description="learned weighted min-sum BP: train / evaluate")
    sub = ap.add_subparsers(dest="cmd", required=True)
    tr = sub.add_parser("train")
    tr.add_argument("--N", type=int, default=1024)
    tr.add_argument("--K", type=int, default=512)
    tr.add_argument("--crc", type=int, default=16)
    tr.add_argument("--T", type=int, default=20)
    tr.add_argument("--steps", type=int, default=1500)
    tr.add_argument("--batch", type=int, default=4096)
    tr.add_argument("--lr", type=float, default=3e-2)
    tr.add_argument("--all-iters", action="store_true", help="loss = mean BCE after every iteration")
    tr.add_argument("--init", type=float, default=1.0, help="initial value of every scale")
    tr.add_argument("--max-scale", type=float, default=1.0, help="scales are projected onto [0, max-scale]")
    tr.add_argument("--out", required=True)
    ev = sub.add_parser("eval")
    ev.add_argument("--weights", required=True)
    ev.add_argument("--ebn0", type=float, nargs="+", default=[1.0, 1.5, 2.0, 2.5, 3.0])
    ev.add_argument("--frames", type=int, default=100_000)
    ev.add_argument("--L", type=int, default=8)
    a = ap.parse_args(argv)
    if a.cmd == "train":
        code = api.make_code(a.N, a.K, a.crc)
        w0 = torch.full((a.T, 2, code.n, code.N), a.init, dtype=torch.float32)
        w, hist = train(code, T=a.T, steps=a.steps, batch=a.batch, lr=a.lr, w0=w0, all_iters=a.all_iters,
                        w_max=a.max_scale)
        save(a.out, w, code, a.T, {"steps": a.steps, "batch": a.batch, "lr": a.lr, "ebn0_range": [1.0, 4.0],
                                   "all_iters": a.all_iters, "init": a.init, "max_scale": a.max_scale,
                                   "loss_history": hist})
        print(json.dumps({"saved": a.out, "loss_first": hist[0][1], "loss_last": hist[-1][1]}))
    else:
        w, code, T, _ = load(a.weights)
        # i200 with learned weights: the learned scales in the first T iterations, plain after them
        variants = {"plain_fp32_i200": (200, api.POLAR_FP32, None), "plain_fp32_i20": (T, api.POLAR_FP32, None),
                    "learned_fp32_i20": (T, api.POLAR_FP32, w), "learned_fp16_i20": (T, api.POLAR_FP16, w),
                    "plain_fp16_i20": (T, api.POLAR_FP16, None), "plain_fp16_i200": (200, api.POLAR_FP16, None),
                    "learned_fp16_i200": (200, api.POLAR_FP16, w)}
        for e in a.ebn0:
            r = evaluate_point(code, e, a.frames, variants, a.L)
            print(json.dumps({"ebn0_db": e, "frames": a.frames, **r}), flush=True)


if __name__ == "__main__":
    main()
