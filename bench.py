#!/usr/bin/env python3
"""Benchmark of the hybrid BP + CA-SCL polar decoder (arXiv 1609.09358) on GB300.

Workload (one step): hybrid decoding (min-sum BP with CRC early stop, CA-SCL on the CRC-failed
frames) of 100 000 seeded BPSK-AWGN frames of the N = 1024, K = 512 (incl. CRC-16 0x1021) polar
code at Eb/N0 = 2.5 dB, BP i_max = 200, CA-SCL L = 8, FP32 messages (--precision fp16: half2 BP
messages clipped at 32).  Frozen set: Bhattacharyya at 0 dB design, rate P/N.  Inputs are generated
on the device by the library's generator before timing; they (410 MB of LLRs per step) exceed the
129 MB L2, so no flush is needed between steps.

Metric: information (payload) Gbit/s = P x frames / time, summed over all ranks (weak scaling:
every rank decodes its own frames).  `python bench.py --impl reference` times the CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "info Gbit/s at matched FER, N=1024 R=1/2 hybrid BP+CA-SCL, plain vs learned/FP16"
N, K, CRC, IMAX, LIST, LLR_MAX = 1024, 512, 16, 200, 8, 20.0
SEED = 1609093581


def parse():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "fp16"], default="fp32")
    ap.add_argument("--ebn0", type=float, default=2.5)
    ap.add_argument("--frames", type=int, default=100_000)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--weights", default=os.path.join(ROOT, "paper_1609_09358_gb300", "weights", "wms_n1024_k512_t20.pt"))
    return ap.parse_args()


def workload_name(a):
    prec = "FP32" if a.precision == "fp32" else "half2 FP16 (clip 32)"
    return ("plain hybrid N=%d K=%d CRC-16 i_max=%d L=%d %s, BPSK-AWGN %.1f dB, %d frames per GPU per step"
            % (N, K, IMAX, LIST, prec, a.ebn0, a.frames))


# ----------------------------------------------------------------------------- distributed
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ----------------------------------------------------------------------------- clocks
QUERY = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", "polar_clocks_%d_%d.csv" % (os.getpid(), gpu_index))

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        try:
            self.f.close()
        except Exception:
            pass

    def mark(self):
        return time.time()

    def summary(self, t0=None, t1=None):
        """Samples taken between wall times t0 and t1 (the timed region)."""
        import datetime
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 10:
                    continue
                try:
                    ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                except ValueError:
                    continue
                if t0 is not None and not (t0 - 0.05 <= ts <= t1 + 0.05):
                    continue
                rows.append(parts[1:])
        except Exception:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["clock sampling unavailable"]}
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no clock samples in the timed region"]}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        pw = [num(r[3]) for r in rows if num(r[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "samples": len(rows), "reasons": reasons}


# ----------------------------------------------------------------------------- CPU oracle leg
def oracle_sample_rate(n_frames: int, ebn0: float, seed: int, min_seconds: float = 0.0):
    """Decode seeded frames of the workload with the CPU oracle (all host cores): Gbit/s + stats."""
    import numpy as np

    import oracle
    from paper_1609_09358_gb300 import inputs
    ocode = oracle.make_code(N, K, CRC, 0.0)
    sigma = oracle.sigma_for(ebn0, ocode.P / N)
    done, secs, errs = 0, 0.0, 0
    frame0 = 0
    while True:
        pay = inputs.payload_bits(seed, frame0, n_frames, ocode.P)
        x = oracle.encode_batch(pay, ocode)
        llr = oracle.channel_llr(x, inputs.unit_noise(seed, frame0, n_frames, N), sigma)
        t0 = time.perf_counter()
        out = oracle.hybrid_decode(llr, ocode, IMAX, LLR_MAX, LIST)
        secs += time.perf_counter() - t0
        errs += int(np.sum(np.any(oracle.payload_of(out["u_hat"], ocode) != pay, axis=1)))
        done += n_frames
        frame0 += n_frames
        if secs >= min_seconds:
            break
    return {"value": ocode.P * done / secs / 1e9, "frames": done, "seconds": secs, "cores": oracle.num_threads(),
            "fer": errs / done}


def run_reference(a, world, rank):
    if rank != 0:
        return 0
    per_step = 256
    for _ in range(a.warmup):
        oracle_sample_rate(per_step, a.ebn0, SEED + 7)
    vals, secs = [], 0.0
    for s in range(a.steps):
        r = oracle_sample_rate(per_step, a.ebn0, SEED + 1000 + s)
        vals.append(r)
        secs += r["seconds"]
    frames = sum(r["frames"] for r in vals)
    value = 496 * frames / secs / 1e9
    cores = vals[0]["cores"]
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Gbit/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * secs / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(a).replace("%d frames per GPU per step" % a.frames,
                                                            "%d frames per step (CPU sample)" % per_step)},
            "cpu_baseline": {"value": value, "unit": "Gbit/s", "cores": cores, "kind": "oracle",
                             "sample": "%d seeded frames per step of the same workload, C oracle with OpenMP" % per_step},
            "e2e": {"value": value, "unit": "Gbit/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- GPU leg
def main():
    a = parse()
    world, rank, local = dist_setup()
    if a.impl == "reference":
        return run_reference(a, world, rank)

    import numpy as np
    import torch

    from paper_1609_09358_gb300 import api, build
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    api.load()

    code = api.make_code(N, K, CRC, 0.0)
    P, B = code.P, a.frames
    prec = api.POLAR_FP16 if a.precision == "fp16" else api.POLAR_FP32
    llr_max = 32.0 if prec == api.POLAR_FP16 else LLR_MAX
    sigma = float(np.sqrt(1.0 / (2.0 * (P / N) * 10 ** (a.ebn0 / 10.0))))
    frame0 = rank * B
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    payload = torch.empty((B, code.row_bytes), dtype=torch.uint8, device=dev)
    cw = torch.empty((B, N // 8), dtype=torch.uint8, device=dev)
    llr = torch.empty((B, N), dtype=torch.float32, device=dev)
    api.polar_random_payload(B, P, SEED, frame0, payload)
    api.polar_encode(code, payload, cw)
    api.polar_awgn_llr(cw, N, sigma, SEED, frame0, llr)
    dec = api.Decoder(code, B, LIST, device=dev)

    def step():
        dec.hybrid(llr, IMAX, llr_max, prec)

    for _ in range(max(a.warmup, 0)):
        step()
    torch.cuda.synchronize()
    # decoding statistics of one step (deterministic: every step decodes the same frames)
    iters = dec.iters.cpu().numpy().astype(np.int64)
    status = dec.status.cpu().numpy()
    bits = dec.bits
    frame_err = (bits != payload).any(dim=1)
    bit_err = int(sum(bin(int(v)).count("1") for v in (bits ^ payload)[frame_err].flatten().cpu().numpy()))
    fer = float(frame_err.float().mean().item())
    n_fb = int(np.sum(status != api.FRAME_BP_OK))

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        time.sleep(1.0)  # let the sampler start; samples are filtered to the timed window
        for _ in range(2):
            step()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        api.polar_profile_enable(True)
        t_start = clk.mark()
        e0.record(stream)
        for _ in range(a.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        t_end = clk.mark()
        api.polar_profile_enable(False)
        time.sleep(0.3)
    clocks = clk.summary(t_start, t_end)
    bp_ms, bp_n, scl_ms, scl_n = api.polar_profile_read()
    ms = e0.elapsed_time(e1)
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    if dist:
        dist.barrier()
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    value = world * P * B * a.steps / (ms_max * 1e-3) / 1e9

    # roofline of the dominant kernel (BP): algorithmic lane-ops / measured average launch time
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    sm_max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    n = code.n
    ops_per_frame_iter = 6 * n * N + K   # 6 ops per PE half-iteration (2 add, 2 g, 2 clip) + CRC
    lanes = 128 * (2 if prec == api.POLAR_FP16 else 1)
    peak_ops = sms * lanes * sm_max_mhz * 1e6
    bp_avg_ms = bp_ms / max(bp_n, 1)
    # every step decodes the same frames: total algorithmic ops of the timed BP launches over their
    # summed device time (= ops per launch / average launch time when a step is one launch)
    achieved = ops_per_frame_iter * float(iters.sum()) * a.steps / (bp_ms * 1e-3)
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if os.path.exists(tfile):
        for line in open(tfile):
            f = line.split()
            if len(f) >= 3 and f[0] == "bp_kernel" and f[1] == ("fp16" if prec == api.POLAR_FP16 else "fp32"):
                traffic = float(f[2])
    roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12, "unit": "Top/s",
                "frac": achieved / peak_ops, "traffic": traffic, "kernel": "bp_kernel",
                "ops_per_frame_iter": ops_per_frame_iter, "bp_avg_ms": bp_avg_ms,
                "peak_basis": "%d SMs x %d lanes x %.0f MHz (sm_max_mhz of MEASURED_PEAKS.json)"
                              % (sms, lanes, sm_max_mhz)}

    line = {"metric": METRIC, "value": value, "unit": "Gbit/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms_max / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f16" if prec == api.POLAR_FP16 else "f32", "data": "synthetic",
            "config": {"workload": workload_name(a), "frames_per_gpu": B, "ebn0_db": a.ebn0, "N": N, "K": K,
                       "crc": "CRC-16 0x1021", "i_max": IMAX, "L": LIST, "llr_max": llr_max,
                       "cache": "inputs larger than L2 (%.0f MB of LLRs per step per GPU), no flush" % (B * N * 4 / 1e6)},
            "fer": fer, "ber": bit_err / (B * P), "fallback_rate": n_fb / B, "avg_bp_iters": float(iters.mean()),
            "bp_ms_per_step": bp_ms / a.steps, "scl_ms_per_step": scl_ms / a.steps,
            "gpu_launches": bp_n + scl_n, "roofline": roofline, "clocks": clocks}

    if not a.no_learned and os.path.exists(a.weights):
        line["learned_fp16"] = learned(a, llr, payload, stream, dist)
    if not a.no_e2e:
        line["e2e"] = e2e(a, code, llr, prec, llr_max, dev, stream, dist)
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        r = oracle_sample_rate(1024, a.ebn0, SEED + 99, min_seconds=10.0)
        line["cpu_baseline"] = {"value": r["value"], "unit": "Gbit/s", "cores": r["cores"], "kind": "oracle",
                                "sample": "%d seeded frames of the same workload (%.1f s), C oracle, OpenMP"
                                          % (r["frames"], r["seconds"])}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def learned(a, llr, payload, stream, dist):
    """The learned/FP16 form on the same frames: half2 BP with the trained per-edge weights,
    T = 20 iterations with CRC early stop, then CA-SCL L = 8 on the CRC failures."""
    import torch

    from paper_1609_09358_gb300 import api, wms
    w, lcode, T, meta = wms.load(a.weights, device=llr.device)
    B = llr.shape[0]
    dec = api.Decoder(lcode, B, LIST, device=llr.device)

    def step():
        dec.hybrid(llr, T, 32.0, api.POLAR_FP16, w)

    for _ in range(max(a.warmup, 1)):
        step()
    torch.cuda.synchronize()
    steps = max(1, min(a.steps, 50))
    if dist:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    api.polar_profile_enable(True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    api.polar_profile_enable(False)
    bp_ms, _, scl_ms, _ = api.polar_profile_read()
    t = torch.tensor([e0.elapsed_time(e1)], dtype=torch.float64, device=llr.device)
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    world = dist.get_world_size() if dist else 1
    ferr = (dec.bits != payload).any(dim=1)
    return {"value": world * lcode.P * B * steps / (float(t.item()) * 1e-3) / 1e9, "unit": "Gbit/s", "steps": steps,
            "ms_per_step": float(t.item()) / steps, "fer": float(ferr.float().mean().item()),
            "fallback_rate": float((dec.status != api.FRAME_BP_OK).float().mean().item()),
            "avg_bp_iters": float(dec.iters.float().mean().item()), "i_max": T,
            "bp_ms_per_step": bp_ms / steps, "scl_ms_per_step": scl_ms / steps, "dtype": "f16",
            "weights": os.path.relpath(a.weights, ROOT), "training": {k: meta.get(k) for k in ("steps", "batch", "lr")}}


def e2e(a, code, llr, prec, llr_max, dev, stream, dist):
    """Same metric through hybrid_decode_host: LLRs in pinned host memory, H2D copy, decode and D2H of
    the decided bits, status and iteration counts inside the timed region."""
    import torch

    from paper_1609_09358_gb300 import api
    B = llr.shape[0]
    llr_h = torch.empty((B, N), dtype=torch.float32, pin_memory=True)
    llr_h.copy_(llr.cpu())
    bits_h = torch.empty((B, code.row_bytes), dtype=torch.uint8, pin_memory=True)
    status_h = torch.empty(B, dtype=torch.uint8, pin_memory=True)
    iters_h = torch.empty(B, dtype=torch.int16, pin_memory=True)
    ws = torch.empty(api.polar_workspace_bytes(code, B, LIST, api.POLAR_OP_HYBRID_HOST), dtype=torch.uint8, device=dev)

    def step():
        api.hybrid_decode_host(code, llr_h, IMAX, llr_max, prec, None, LIST, bits_h, status_h, iters_h, ws)

    for _ in range(max(a.warmup, 1)):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    t = torch.tensor([e0.elapsed_time(e1)], dtype=torch.float64, device=dev)
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    world = dist.get_world_size() if dist else 1
    value = world * code.P * B * a.steps / (float(t.item()) * 1e-3) / 1e9
    return {"value": value, "unit": "Gbit/s", "h2d_bytes_per_step": B * N * 4,
            "d2h_bytes_per_step": B * (code.row_bytes + 1 + 2), "api": "hybrid_decode_host (pinned host buffers)"}


if __name__ == "__main__":
    sys.exit(main())
