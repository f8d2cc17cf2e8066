"""Half2 and learned BP against the FP64 oracle: LLR deviation and error rates.

With early stop disabled (POLAR_FIXED_ITERS, exactly T iterations on both sides) the final LLR(u)
of the GPU's half2 BP -- plain and with the learned scales -- is compared with the oracle's
weighted BP in binary64 on the same frames: the maximum and mean absolute deviation and the
agreement of the hard decisions.  The hybrid decoder in half2 is compared with the oracle's
binary64 hybrid on the frame error rate of a seeded sample.  The numbers are printed (run with
-s to see them) and bounded loosely; they are not a parity check (binary16 rounding makes the
trajectories differ), they quantify it.
"""
import json
import os

import numpy as np
import pytest

import oracle
from tests import frames as fr

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

from paper_1609_09358_gb300 import api, build, wms  # noqa: E402

WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1609_09358_gb300",
                       "weights", "wms_n1024_k512_t20.pt")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    api.load()


def gpu_llr_u(ocode, llr, T, precision, w=None):
    code = fr.api_code(ocode)
    B, N = llr.shape
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    bits = torch.zeros((B, code.row_bytes), dtype=torch.uint8, device="cuda")
    status = torch.zeros(B, dtype=torch.uint8, device="cuda")
    iters = torch.zeros(B, dtype=torch.int16, device="cuda")
    lu = torch.zeros((B, N), dtype=torch.float32, device="cuda")
    M = 32.0 if precision == api.POLAR_FP16 else 20.0
    api.bp_decode(code, dev(llr), T, M, precision | api.POLAR_FIXED_ITERS, None if w is None else dev(w), bits, status,
                  iters, lu)
    torch.cuda.synchronize()
    assert (iters.cpu().numpy() == T).all()
    return lu.cpu().numpy().astype(np.float64)


def deviation(ocode, llr, T, precision, w=None):
    """Deviation of LLR(u) on the information positions after exactly T iterations, over all
    frames and over the frames whose binary64 run meets the CRC within the T iterations (stable).
    Without the CRC stop, frames keep iterating; where they oscillate, rounding differences flip
    min choices and the trajectories part -- in FP32 as well as in binary16 -- so long runs are
    reported, short ones bounded."""
    M = 32.0 if precision == api.POLAR_FP16 else 20.0
    ref = oracle.bp_decode(llr, ocode, T, M, "f64", early_stop=False, w=w, llr_u_double=True)["llr_u_f64"]
    stop = oracle.bp_decode(llr, ocode, T, M, "f64", early_stop=True, w=w, want_llr=False)
    stable = stop["status"] == 1
    got = gpu_llr_u(ocode, llr, T, precision, w)
    info = ocode.info_idx
    out = {"frames": int(len(llr)), "stable": int(stable.sum())}
    for name, sel in (("all", np.ones(len(llr), bool)), ("stable", stable)):
        if not sel.any():
            continue
        d = np.abs(got[sel][:, info] - ref[sel][:, info])
        agree = np.mean((got[sel][:, info] < 0) == (ref[sel][:, info] < 0))
        out[name] = {"max_abs_dev": float(d.max()), "mean_abs_dev": float(d.mean()),
                     "hard_decision_agreement": float(agree)}
    return out


@pytest.mark.parametrize("N,K,crc", [(128, 64, 8), (1024, 512, 16)])
def test_half2_llr_deviation_vs_f64(N, K, crc):
    ocode = fr.oracle_code(N, K, crc)
    _, llr = fr.frames(ocode, 2.5, 64, seed=4242 + N)
    rep = {"N": N, "K": K, "ebn0_db": 2.5}
    for T in (5, 20):
        rep["T%d" % T] = {"fp16_vs_f64": deviation(ocode, llr, T, api.POLAR_FP16),
                          "fp32_vs_f64": deviation(ocode, llr, T, api.POLAR_FP32)}
    print(json.dumps(rep))
    r32, r16 = rep["T5"]["fp32_vs_f64"], rep["T5"]["fp16_vs_f64"]
    # FP32 differs from binary64 by rounding only; binary16 (11-bit significand) more
    assert r32["all"]["max_abs_dev"] < 0.05 and r32["all"]["hard_decision_agreement"] > 0.999
    assert r16["stable"]["max_abs_dev"] < 4.0 and r16["stable"]["mean_abs_dev"] < 0.2
    assert r16["stable"]["hard_decision_agreement"] > 0.999


def test_learned_half2_llr_deviation_vs_f64():
    if not os.path.exists(WEIGHTS):
        pytest.skip("no trained weights")
    w, code, T, _ = wms.load(WEIGHTS, device="cpu")
    w = w.numpy().astype(np.float32)
    ocode = oracle.Code(code.N, code.K, code.crc_len, oracle.CRC_POLYS[code.crc_len], code.frozen.astype(np.uint8),
                        np.nonzero(code.frozen == 0)[0].astype(np.int32))
    _, llr = fr.frames(ocode, 2.5, 64, seed=4343)
    rep = {"N": code.N, "ebn0_db": 2.5}
    for TT in (5, T):
        rep["T%d" % TT] = {"learned_fp16_vs_learned_f64": deviation(ocode, llr, TT, api.POLAR_FP16, w),
                           "learned_fp32_vs_learned_f64": deviation(ocode, llr, TT, api.POLAR_FP32, w)}
    print(json.dumps(rep))
    r16 = rep["T5"]["learned_fp16_vs_learned_f64"]
    assert r16["stable"]["mean_abs_dev"] < 0.2 and r16["stable"]["hard_decision_agreement"] > 0.999


def test_half2_hybrid_fer_vs_f64_hybrid():
    """Frame errors of the half2 hybrid and the binary64 oracle hybrid on the same 600 frames at
    1.5 dB (N = 1024, i_max = 60, L = 8): the counts must agree within the sampling noise."""
    ocode = fr.oracle_code(1024, 512, 16)
    pay, llr = fr.frames(ocode, 1.5, 600, seed=4444)
    ref = oracle.hybrid_decode(llr, ocode, 60, 32.0, 8, precision="f64")
    e64 = int(np.sum(np.any(oracle.payload_of(ref["u_hat"], ocode) != pay, axis=1)))
    code = fr.api_code(ocode)
    dec = api.Decoder(code, len(llr), 8)
    bits, status, _ = dec.hybrid(torch.from_numpy(llr).cuda(), 60, 32.0, api.POLAR_FP16)
    torch.cuda.synchronize()
    e16 = int(np.sum(np.any(api.unpack_bits(bits.cpu().numpy(), ocode.P) != pay, axis=1)))
    print(json.dumps({"frames": len(llr), "ebn0_db": 1.5, "fer_f64_hybrid": e64 / len(llr),
                      "fer_fp16_hybrid": e16 / len(llr)}))
    assert abs(e16 - e64) <= 3 * np.sqrt(max(e64, 1)) + 3
