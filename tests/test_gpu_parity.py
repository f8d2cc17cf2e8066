"""GPU parity: the CUDA decoder through the C ABI against the CPU oracle, element by element.

FP32 BP, SCL and hybrid are compared bit-exactly (decided bits, per-frame status and iteration
counts, and the output LLRs as float32 values); the half-precision BP bit-exactly against the
oracle's binary16 emulation.  Inputs are seeded frames built on the CPU (tests/frames.py).  Batch
sizes are chosen so that the CTA grid has a ragged tail (B not a multiple of the frames per CTA).
"""
import numpy as np
import pytest

import oracle
from tests import frames as fr

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

from paper_1609_09358_gb300 import api, build  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    api.load()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run_bp(ocode, llr, max_iters, llr_max, precision=api.POLAR_FP32, w=None, want_llr=True):
    code = fr.api_code(ocode)
    B, N = llr.shape
    bits = torch.zeros((B, code.row_bytes), dtype=torch.uint8, device="cuda")
    status = torch.zeros(B, dtype=torch.uint8, device="cuda")
    iters = torch.zeros(B, dtype=torch.int16, device="cuda")
    lu = torch.zeros((B, N), dtype=torch.float32, device="cuda") if want_llr else None
    lx = torch.zeros((B, N), dtype=torch.float32, device="cuda") if want_llr else None
    w = None if w is None else (w if isinstance(w, api.PreparedScales) else dev(w))
    api.bp_decode(code, dev(llr), max_iters, llr_max, precision, w, bits, status, iters, lu, lx)
    torch.cuda.synchronize()
    out = {"bits": api.unpack_bits(bits.cpu().numpy(), ocode.P), "status": status.cpu().numpy(),
           "iters": iters.cpu().numpy().astype(np.int32)}
    if want_llr:
        out["llr_u"] = lu.cpu().numpy()
        out["llr_x"] = lx.cpu().numpy()
    return out


def assert_bp_equal(got, ref, ocode, with_llr=True):
    assert np.array_equal(got["iters"], ref["iters"]), np.nonzero(got["iters"] != ref["iters"])[0][:10]
    assert np.array_equal(got["status"], ref["status"])
    assert np.array_equal(got["bits"], oracle.payload_of(ref["u_hat"], ocode))
    if with_llr:
        assert np.array_equal(got["llr_u"], ref["llr_u"]), np.max(np.abs(got["llr_u"] - ref["llr_u"]))
        assert np.array_equal(got["llr_x"], ref["llr_x"]), np.max(np.abs(got["llr_x"] - ref["llr_x"]))


BP_CASES = [
    # N, K, crc, Eb/N0, B, max_iters
    (128, 64, 8, 2.5, 203, 50),
    (128, 64, 8, 0.5, 61, 50),
    (256, 128, 16, 2.0, 97, 60),
    (512, 256, 16, 2.0, 45, 60),
    (1024, 512, 16, 2.5, 37, 200),
    (1024, 512, 16, 1.0, 12, 200),
    (2048, 1024, 24, 1.5, 9, 80),
    (1024, 512, 24, 2.0, 19, 100),   # CRC-24: the syndrome columns unpacked
    (1024, 768, 16, 3.0, 21, 100),
    (256, 64, 16, 1.0, 33, 40),
    (4096, 2048, 16, 2.0, 7, 50),    # the paper's length: one 512-thread frame group per SM
    (4096, 2048, 16, 1.0, 3, 50),
]


@pytest.mark.parametrize("N,K,crc,ebn0,B,imax", BP_CASES)
def test_bp_fp32_bit_exact(N, K, crc, ebn0, B, imax):
    ocode = fr.oracle_code(N, K, crc)
    _, llr = fr.frames(ocode, ebn0, B, seed=1000 + N + K)
    ref = oracle.bp_decode(llr, ocode, imax, 20.0, "f32")
    got = run_bp(ocode, llr, imax, 20.0)
    assert_bp_equal(got, ref, ocode)


@pytest.mark.parametrize("N,K,crc,ebn0,B,imax", [c for c in BP_CASES if c[0] <= 1024][:6] + [(2048, 1024, 24, 1.5, 9, 80),
                                                                                              (4096, 2048, 16, 2.0, 9, 50)])
def test_bp_fp16_bit_exact_vs_binary16_emulation(N, K, crc, ebn0, B, imax):
    ocode = fr.oracle_code(N, K, crc)
    _, llr = fr.frames(ocode, ebn0, B, seed=2000 + N + K)
    ref = oracle.bp_decode(llr, ocode, imax, 32.0, "f16")
    got = run_bp(ocode, llr, imax, 32.0, api.POLAR_FP16)
    assert_bp_equal(got, ref, ocode)


@pytest.mark.parametrize("precision", ["f32", "f16"])
@pytest.mark.parametrize("N,K,crc,B", [(2048, 1024, 24, 1400), (4096, 2048, 16, 700)])
def test_bp_refill_long_codes_bit_exact(N, K, crc, B, precision):
    """Several frames per frame group at N = 2048 and 4096 (more frames than the persistent grid
    holds), so every group refills: the channel column these kernels keep in shared memory is
    rewritten per frame (per half of a half2 register), and every output must still equal the
    oracle's."""
    ocode = fr.oracle_code(N, K, crc)
    _, llr = fr.frames(ocode, 3.0, B, seed=4700 + N)
    m = 20.0 if precision == "f32" else 32.0
    ref = oracle.bp_decode(llr, ocode, 50, m, precision)
    flag = api.POLAR_FP32 if precision == "f32" else api.POLAR_FP16
    got = run_bp(ocode, llr, 50, m, flag)
    assert_bp_equal(got, ref, ocode)


@pytest.mark.parametrize("N,K,crc,B", [(512, 256, 16, 40), (1024, 512, 16, 33), (1024, 512, 24, 17),
                                       (2048, 1024, 24, 9), (4096, 2048, 16, 5)])
@pytest.mark.parametrize("precision", ["f32", "f16"])
def test_bp_fixed_iterations_bit_exact(N, K, crc, B, precision):
    """Exactly T iterations whatever the CRC says (POLAR_FIXED_ITERS): every output after the
    last one equals the oracle's BP without early stop.  With FP32 frames over several warps the
    kernels read an iteration's stop decision one exchange later (after the next iteration's first
    stages), and the 16-node plans (N = 1024, FP32 at 4096) exchange columns in three groups: both
    must leave the T-th iteration's messages as they are."""
    T = 7
    ocode = fr.oracle_code(N, K, crc)
    _, llr = fr.frames(ocode, 2.0, B, seed=4100 + N + K)
    m = 20.0 if precision == "f32" else 32.0
    ref = oracle.bp_decode(llr, ocode, T, m, precision, early_stop=False)
    flag = api.POLAR_FP32 if precision == "f32" else api.POLAR_FP16
    got = run_bp(ocode, llr, T, m, flag | api.POLAR_FIXED_ITERS)
    assert np.all(got["iters"] == T)
    assert_bp_equal(got, ref, ocode)


@pytest.mark.parametrize("N,K,crc", [(128, 64, 8), (256, 128, 16), (512, 256, 16), (1024, 512, 16),
                                     (2048, 1024, 24)])
@pytest.mark.parametrize("precision", ["f32", "f16"])
def test_bp_weighted_bit_exact(N, K, crc, precision):
    ocode = fr.oracle_code(N, K, crc)
    _, llr = fr.frames(ocode, 1.5, 19, seed=3000 + N)
    rng = np.random.default_rng(N)
    T = 6
    w = rng.uniform(0.5, 1.5, (T, 2, ocode.n, N)).astype(np.float32)
    M = 20.0 if precision == "f32" else 32.0
    ref = oracle.bp_decode(llr, ocode, 10, M, precision, w=w)
    got = run_bp(ocode, llr, 10, M, api.POLAR_FP32 if precision == "f32" else api.POLAR_FP16, w=w)
    assert_bp_equal(got, ref, ocode)


@pytest.mark.parametrize("precision", ["f32", "f16"])
def test_hybrid_prepared_weights_reused(precision):
    """Weights prepared once (wms_prepare) and passed to two hybrid decodes of different batches:
    each equals the oracle's weighted hybrid; iterations past the learned ones run unweighted."""
    ocode = fr.oracle_code(256, 128, 16)
    code = fr.api_code(ocode)
    rng = np.random.default_rng(77)
    T = 4
    w = rng.uniform(0.6, 1.4, (T, 2, ocode.n, 256)).astype(np.float32)
    prec = api.POLAR_FP32 if precision == "f32" else api.POLAR_FP16
    M = 20.0 if precision == "f32" else 32.0
    pw = api.PreparedScales(code, dev(w), prec)
    for seed, B in ((41, 67), (42, 30)):
        _, llr = fr.frames(ocode, 1.5, B, seed=seed)
        # oracle hybrid: weighted BP in the message precision, FP32 CA-SCL on its failures
        ref = oracle.bp_decode(llr, ocode, 12, M, precision, w=w, want_llr=False)
        u_ref, st_ref = ref["u_hat"].copy(), ref["status"].copy()
        failed = np.nonzero(st_ref != api.FRAME_BP_OK)[0]
        assert 0 < len(failed) < B
        scl = oracle.scl_decode(llr[failed], ocode, 4, "f32")
        u_ref[failed] = scl["u_hat"]
        st_ref[failed] = scl["status"]  # FRAME_SCL_OK / FRAME_SCL_CRC_FAIL
        dec = api.Decoder(code, B, 4)
        bits, status, iters = dec.hybrid(dev(llr), 12, M, prec, pw)
        torch.cuda.synchronize()
        assert np.array_equal(iters.cpu().numpy().astype(np.int32), ref["iters"])
        assert np.array_equal(status.cpu().numpy(), st_ref)
        assert np.array_equal(api.unpack_bits(bits.cpu().numpy(), ocode.P), oracle.payload_of(u_ref, ocode))
    other = api.POLAR_FP16 if prec == api.POLAR_FP32 else api.POLAR_FP32
    with pytest.raises(api.PolarError):
        dec.hybrid(dev(llr), 12, M, other, pw)


@pytest.mark.parametrize("N,K,crc,B", [(128, 64, 8, 203), (256, 128, 16, 97), (512, 256, 16, 45),
                                     (1024, 512, 16, 37), (2048, 1024, 24, 13)])
def test_bp_unit_scales_aligned_pairs_bit_exact(N, K, crc, B):
    """Learned scales within [0, 1] (POLAR_WMS_UNIT) with max_iters <= T: the half2 decoder keeps
    both frames of a register on the same iteration and skips the clip of the scaled term; every
    frame still equals the oracle's weighted binary16 BP (bits, status, iterations, LLR(u), LLR(x)),
    whichever frame shares its register; an odd B leaves one register half empty."""
    ocode = fr.oracle_code(N, K, crc)
    code = fr.api_code(ocode)
    _, llr = fr.frames(ocode, 2.5, B, seed=3100 + N)
    rng = np.random.default_rng(N + 1)
    T = 12
    w = rng.uniform(0.75, 1.0, (T, 2, ocode.n, N)).astype(np.float32)
    w[0, 0, 0, :4] = 1.0
    w[1, 1, 0, :4] = 0.0
    pw = api.PreparedScales(code, dev(w), api.POLAR_FP16)
    assert pw.unit
    for imax in (T, 7):
        ref = oracle.bp_decode(llr, ocode, imax, 32.0, "f16", w=w)
        assert 0 < np.sum(ref["status"] == api.FRAME_BP_OK) < B
        got = run_bp(ocode, llr, imax, 32.0, api.POLAR_FP16, w=pw)
        assert_bp_equal(got, ref, ocode)
        fixed = run_bp(ocode, llr, imax, 32.0, api.POLAR_FP16 | api.POLAR_FIXED_ITERS, w=pw)
        assert_bp_equal(fixed, oracle.bp_decode(llr, ocode, imax, 32.0, "f16", early_stop=False, w=w), ocode)


@pytest.mark.parametrize("N,K,crc,B,L", [(256, 128, 16, 301, 4), (1024, 512, 16, 150, 8)])
def test_hybrid_unit_scales_aligned_pairs_bit_exact(N, K, crc, B, L):
    """The hybrid with learned scales in [0, 1], half2 BP with i_max = T (the aligned-pair form):
    BP results as the oracle's weighted binary16 BP, CA-SCL on exactly its failures."""
    ocode = fr.oracle_code(N, K, crc)
    code = fr.api_code(ocode)
    _, llr = fr.frames(ocode, 2.5, B, seed=3200 + N)
    rng = np.random.default_rng(N + 2)
    T = 10
    w = rng.uniform(0.75, 1.0, (T, 2, ocode.n, N)).astype(np.float32)
    pw = api.PreparedScales(code, dev(w), api.POLAR_FP16)
    ref = oracle.bp_decode(llr, ocode, T, 32.0, "f16", w=w, want_llr=False)
    u_ref, st_ref = ref["u_hat"].copy(), ref["status"].copy()
    failed = np.nonzero(st_ref != api.FRAME_BP_OK)[0]
    assert 0 < len(failed) < B
    scl = oracle.scl_decode(llr[failed], ocode, L, "f32")
    u_ref[failed] = scl["u_hat"]
    st_ref[failed] = scl["status"]
    dec = api.Decoder(code, B, L)
    bits, status, iters = dec.hybrid(dev(llr), T, 32.0, api.POLAR_FP16, pw)
    torch.cuda.synchronize()
    assert np.array_equal(iters.cpu().numpy().astype(np.int32), ref["iters"])
    assert np.array_equal(status.cpu().numpy(), st_ref)
    assert np.array_equal(api.unpack_bits(bits.cpu().numpy(), ocode.P), oracle.payload_of(u_ref, ocode))


@pytest.mark.parametrize("N,K,crc,L,frac", [(256, 128, 16, 4, 0.5), (1024, 512, 16, 8, 0.25), (1024, 512, 16, 16, 0.5),
                                         (2048, 1024, 24, 32, 0.3), (128, 64, 8, 2, 0.9)])
def test_decision_aided_scl_and_hybrid_bit_exact(N, K, crc, L, frac):
    """Decision-aided CA-SCL (the most reliable information positions decided without branching):
    scl_decode and the hybrid decoder against the oracle with the same mask."""
    import dataclasses
    ocode0 = fr.oracle_code(N, K, crc)
    code0 = fr.api_code(ocode0)
    mask = api.decided_mask(code0, int(frac * K))
    ocode = dataclasses.replace(ocode0, decided=mask)
    code = api.PolarCode(N, K, crc, ocode0.frozen.copy(), ocode0.crc_poly, decided=mask)
    _, llr = fr.frames(ocode, 1.0, 45, seed=7070 + N + L)
    ref = oracle.scl_decode(llr, ocode, L, "f32")
    dec = api.Decoder(code, 45, L)
    bits, status = dec.scl(dev(llr))
    torch.cuda.synchronize()
    assert np.array_equal(status.cpu().numpy(), ref["status"])
    assert np.array_equal(api.unpack_bits(bits.cpu().numpy(), ocode.P), oracle.payload_of(ref["u_hat"], ocode))
    href = oracle.hybrid_decode(llr, ocode, 30, 20.0, L, precision="f32")
    bits, status, iters = dec.hybrid(dev(llr), 30, 20.0)
    torch.cuda.synchronize()
    assert np.array_equal(status.cpu().numpy(), href["status"])
    assert np.array_equal(iters.cpu().numpy().astype(np.int32), href["iters"])
    assert np.array_equal(api.unpack_bits(bits.cpu().numpy(), ocode.P), oracle.payload_of(href["u_hat"], ocode))


@pytest.mark.parametrize("N,K", [(256, 128), (1024, 512), (4096, 2048)])
@pytest.mark.parametrize("precision", ["f32", "f16"])
def test_bp_edge_inputs(N, K, precision):
    """NaN reads as an erasure, +-inf clips, max_iters = 1, a single frame; at N = 1024 and 4096
    also through the kernels that keep the channel column in shared memory and (FP32) read the
    stop decision one exchange late."""
    ocode = fr.oracle_code(N, K, 16)
    _, llr = fr.frames(ocode, 2.0, 5, seed=5)
    llr[0, :7] = np.nan
    llr[1, ::3] = np.inf
    llr[2, ::5] = -np.inf
    llr[3] = 0.0
    m = 20.0 if precision == "f32" else 32.0
    flag = api.POLAR_FP32 if precision == "f32" else api.POLAR_FP16
    for imax in (1, 25):
        ref = oracle.bp_decode(llr, ocode, imax, m, precision)
        got = run_bp(ocode, llr, imax, m, flag)
        assert_bp_equal(got, ref, ocode)
    ref = oracle.bp_decode(llr[:1], ocode, 25, m, precision)
    assert_bp_equal(run_bp(ocode, llr[:1], 25, m, flag), ref, ocode)


def test_bp_degenerate_codes():
    """No CRC (the check is void, BP stops after one iteration), K = N (nothing frozen), P = 0."""
    for N, K, crc in [(128, 64, 0), (128, 128, 16), (256, 16, 16)]:
        frozen, info, _ = oracle.construct(N, K, 0.0, 0.5)
        ocode = oracle.Code(N, K, crc, oracle.CRC_POLYS[crc], frozen, info)
        rng = np.random.default_rng(N + K)
        llr = rng.normal(1.0, 2.0, (13, N)).astype(np.float32)
        ref = oracle.bp_decode(llr, ocode, 20, 20.0, "f32")
        got = run_bp(ocode, llr, 20, 20.0)
        assert_bp_equal(got, ref, ocode)


def run_scl(ocode, llr, L):
    code = fr.api_code(ocode)
    B = llr.shape[0]
    bits = torch.zeros((B, code.row_bytes), dtype=torch.uint8, device="cuda")
    status = torch.zeros(B, dtype=torch.uint8, device="cuda")
    ws = torch.zeros(max(api.polar_workspace_bytes(code, B, L, api.POLAR_OP_SCL), 256), dtype=torch.uint8,
                     device="cuda")
    api.scl_decode(code, dev(llr), L, bits, status, ws)
    torch.cuda.synchronize()
    return api.unpack_bits(bits.cpu().numpy(), ocode.P), status.cpu().numpy()


def _wilson(k, n, z=1.959963984540054):
    p = k / n
    c = (p + z * z / (2 * n)) / (1 + z * z / n)
    h = z * np.sqrt(p * (1 - p) / n + z * z / (4 * n * n)) / (1 + z * z / n)
    return c - h, c + h


def test_scl_fer_non_increasing_in_list_size():
    """A statistical property of CA-SCL: a larger list does not raise the frame-error rate.  On the
    same 6000 frames (N = 512, K = 256, CRC-16, 1.5 dB) the errors for L = 1, 2, ..., 32 must not
    grow beyond the 95% Wilson interval of the previous list size, and L = 32 must beat SC (L = 1)
    outright.  (CRC false accepts grow with L, but at about L / 2^16 per frame they stay far below
    these error rates.)"""
    ocode = fr.oracle_code(512, 256, 16)
    pay, llr = fr.frames_large(ocode, 1.5, 6000, seed=9100)
    errs = []
    for L in (1, 2, 4, 8, 16, 32):
        bits, _ = run_scl(ocode, llr, L)
        errs.append(int(np.sum(np.any(bits != pay, axis=1))))
    n = llr.shape[0]
    for a, b in zip(errs, errs[1:]):
        assert b / n <= _wilson(a, n)[1], errs
    assert _wilson(errs[-1], n)[1] < _wilson(errs[0], n)[0], errs


SCL_CASES = [
    # N, K, crc, Eb/N0, B, L
    (128, 64, 8, 1.0, 50, 4),
    (128, 64, 8, 1.0, 30, 1),
    (128, 64, 8, 0.0, 30, 32),
    (256, 128, 16, 1.0, 24, 8),
    (256, 128, 16, 1.0, 12, 2),
    (512, 256, 16, 1.0, 10, 16),
    (1024, 512, 16, 1.0, 12, 8),
    (2048, 1024, 24, 1.0, 4, 8),
    (4096, 2048, 16, 1.5, 3, 32),   # the paper's configuration
    (4096, 2048, 16, 1.5, 5, 8),
]


@pytest.mark.parametrize("N,K,crc,ebn0,B,L", SCL_CASES)
def test_scl_bit_exact(N, K, crc, ebn0, B, L):
    ocode = fr.oracle_code(N, K, crc)
    _, llr = fr.frames(ocode, ebn0, B, seed=4000 + N + L)
    ref = oracle.scl_decode(llr, ocode, L, "f32")
    bits, status = run_scl(ocode, llr, L)
    assert np.array_equal(status, ref["status"])
    assert np.array_equal(bits, oracle.payload_of(ref["u_hat"], ocode))


def test_scl_global_scratch_path():
    """L = 32 at N = 2048 keeps the list's LLR arrays in the device workspace."""
    ocode = fr.oracle_code(2048, 1024, 24)
    _, llr = fr.frames(ocode, 1.0, 3, seed=77)
    ref = oracle.scl_decode(llr, ocode, 32, "f32")
    bits, status = run_scl(ocode, llr, 32)
    assert np.array_equal(status, ref["status"])
    assert np.array_equal(bits, oracle.payload_of(ref["u_hat"], ocode))


@pytest.mark.parametrize("L,B", [(32, 2500), (16, 2500), (32, 40), (16, 7)])
def test_scl_few_and_many_frames(L, B):
    """With at most one frame per CTA of the persistent grid, a CTA's warps share each frame's
    upper-level updates; with more frames every warp decodes its own.  Both forms are bit-exact
    (2 500 frames exceed every grid this launch can have; 40 and 7 do not)."""
    ocode = fr.oracle_code(128, 64, 8)
    _, llr = fr.frames(ocode, 0.5, B, seed=91 + B + L)
    ref = oracle.scl_decode(llr, ocode, L, "f32")
    bits, status = run_scl(ocode, llr, L)
    assert np.array_equal(status, ref["status"])
    assert np.array_equal(bits, oracle.payload_of(ref["u_hat"], ocode))


def run_hybrid(ocode, llr, imax, L, llr_max=20.0, precision=api.POLAR_FP32):
    code = fr.api_code(ocode)
    B = llr.shape[0]
    dec = api.Decoder(code, B, L)
    dec.hybrid(dev(llr), imax, llr_max, precision)
    torch.cuda.synchronize()
    nfb = api.polar_hybrid_fallback_count(dec.workspace)
    return (api.unpack_bits(dec.bits.cpu().numpy(), ocode.P), dec.status.cpu().numpy(),
            dec.iters.cpu().numpy().astype(np.int32), nfb)


@pytest.mark.parametrize("ebn0", [1.5, 2.0])
def test_hybrid_fer_matches_scl_alone(ebn0):
    """Sec. IV: the hybrid decodes as well as CA-SCL alone.  On the same 20 000 frames (N = 1024,
    K = 512, CRC-16, L = 8, i_max = 200) the two frame-error rates' 95% Wilson intervals overlap.
    (BP tests the CRC after every iteration, so a few frames it gets wrong pass the CRC: the
    hybrid's rate can only be a little higher.)"""
    ocode = fr.oracle_code(1024, 512, 16)
    pay, llr = fr.frames_large(ocode, ebn0, 20000, seed=9300 + int(10 * ebn0))
    bh, _, _, _ = run_hybrid(ocode, llr, 200, 8)
    bs, _ = run_scl(ocode, llr, 8)
    n = llr.shape[0]
    eh = int(np.sum(np.any(bh != pay, axis=1)))
    es = int(np.sum(np.any(bs != pay, axis=1)))
    lo_h, hi_h = _wilson(eh, n)
    lo_s, hi_s = _wilson(es, n)
    assert lo_h <= hi_s and lo_s <= hi_h, (eh, es)


@pytest.mark.parametrize("N,K,crc,ebn0,B,imax,L", [
    (128, 64, 8, 2.5, 1000, 50, 4),   # the small plain-hybrid workload in full
    (128, 64, 8, 1.0, 300, 50, 4),
    (1024, 512, 16, 2.0, 160, 200, 8),
    (1024, 512, 16, 1.0, 24, 30, 8),
    (512, 256, 16, 1.5, 70, 40, 16),
    (4096, 2048, 16, 1.5, 12, 50, 32),  # the paper's configuration, min-sum BP
])
def test_hybrid_bit_exact(N, K, crc, ebn0, B, imax, L):
    ocode = fr.oracle_code(N, K, crc)
    _, llr = fr.frames(ocode, ebn0, B, seed=5000 + N)
    ref = oracle.hybrid_decode(llr, ocode, imax, 20.0, L, precision="f32")
    bits, status, iters, nfb = run_hybrid(ocode, llr, imax, L)
    assert np.array_equal(iters, ref["iters"])
    assert np.array_equal(status, ref["status"])
    assert np.array_equal(bits, oracle.payload_of(ref["u_hat"], ocode))
    assert nfb == int(np.sum(ref["status"] != oracle.BP_OK))


def _non_finite_frames(ocode, B, seed):
    """Low-SNR frames (BP often fails) with NaN, +-inf and huge values planted: frame 0 a NaN
    run, frame 1 infinities of both signs, frame 2 opposite infinities at j and j + N/2 (their
    top-level g adds inf and -inf), frame 3 a noiseless codeword given as +-inf, the others a few
    NaN, infinite or huge values."""
    pay, llr = fr.frames(ocode, 1.5, B, seed=seed)
    xs = oracle.encode_batch(pay, ocode)
    N = ocode.N
    rng = np.random.default_rng(seed)
    llr[0, 5:40] = np.nan
    llr[1, ::7] = np.inf
    llr[1, 3::11] = -np.inf
    llr[2, 10:20] = np.inf
    llr[2, N // 2 + 10:N // 2 + 20] = -np.inf
    pay = np.zeros((1, ocode.P), np.uint8)
    pay[0, ::3] = 1
    x = oracle.encode_batch(pay, ocode)[0]
    llr[3] = np.where(x == 1, -np.inf, np.inf)
    for b in range(4, B):
        # NaN, or a huge value or an infinity with the sign of the sent bit
        pos = np.nonzero(rng.random(N) < 0.03)[0]
        mag = rng.choice(np.array([np.nan, np.inf, 3e38, 1e31], np.float32), len(pos))
        llr[b, pos] = np.where(xs[b, pos] == 1, -mag, mag)
    return llr


@pytest.mark.parametrize("N,K,crc,B,L", [(256, 128, 16, 24, 8), (1024, 512, 16, 12, 8), (2048, 1024, 24, 6, 32)])
def test_scl_and_hybrid_non_finite_inputs(N, K, crc, B, L):
    """CA-SCL reads NaN as an erasure and saturates +-inf at +-2^100, bit-exactly like the oracle,
    alone and as the hybrid's fallback for frames whose BP fails."""
    ocode = fr.oracle_code(N, K, crc)
    llr = _non_finite_frames(ocode, B, 9100 + N)
    ref = oracle.scl_decode(llr, ocode, L, "f32")
    bits, status = run_scl(ocode, llr, L)
    assert np.array_equal(status, ref["status"])
    assert np.array_equal(bits, oracle.payload_of(ref["u_hat"], ocode))
    href = oracle.hybrid_decode(llr, ocode, 30, 20.0, L, precision="f32")
    assert np.sum(href["status"] != oracle.BP_OK) >= B // 2
    hbits, hstatus, hiters, nfb = run_hybrid(ocode, llr, 30, L)
    assert np.array_equal(hiters, href["iters"])
    assert np.array_equal(hstatus, href["status"])
    assert np.array_equal(hbits, oracle.payload_of(href["u_hat"], ocode))
    assert nfb == int(np.sum(href["status"] != oracle.BP_OK))


def test_hybrid_full_size_sampled():
    """The production workload as the benchmark launches it (N = 1024, K = 512, CRC-16, 1e5 frames,
    i_max = 200, L = 8, 2.5 dB): every frame's status and the decoded bits of a random sample plus
    every SCL frame are compared with the oracle, which decodes those frames one by one."""
    ocode = fr.oracle_code(1024, 512, 16)
    B = 100_000
    pay, llr = fr.frames_large(ocode, 2.5, B, seed=1609093582)
    bits, status, iters, nfb = run_hybrid(ocode, llr, 200, 8)
    rng = np.random.default_rng(0)
    fb = np.nonzero(status != oracle.BP_OK)[0]
    sample = np.unique(np.concatenate([rng.choice(B, 200, replace=False), fb[:200]]))
    ref = oracle.hybrid_decode(llr[sample], ocode, 200, 20.0, 8, precision="f32")
    assert np.array_equal(iters[sample], ref["iters"])
    assert np.array_equal(status[sample], ref["status"])
    assert np.array_equal(bits[sample], oracle.payload_of(ref["u_hat"], ocode))
    assert nfb == len(fb)
    # properties that hold at any size: BP_OK frames pass the CRC, statuses are valid
    assert set(np.unique(status)) <= {1, 2, 3}
    ok = status == oracle.BP_OK
    assert np.all(iters[ok] >= 1) and np.all(iters[~ok] == 200)


@pytest.mark.parametrize("form", ["half2", "learned"])
def test_half2_and_learned_full_size_sampled(form):
    """The default workload's half2 forms as the benchmark launches them (N = 1024, K = 512, 1e5
    frames, 2.5 dB, L = 8): plain half2 BP with i_max = 200, and the learned form with the shipped
    scales (all in [0, 1]) and i_max = T = 20, i.e. the aligned-pair kernel.  Every status is valid;
    a random sample plus CA-SCL frames equal the oracle's binary16 (weighted) BP followed by its
    CA-SCL, frame by frame."""
    import os
    from paper_1609_09358_gb300 import wms
    ocode = fr.oracle_code(1024, 512, 16)
    code = fr.api_code(ocode)
    B = 100_000
    _, llr = fr.frames_large(ocode, 2.5, B, seed=1609093586)
    w_np, pw, imax = None, None, 200
    if form == "learned":
        wfile = os.path.join(os.path.dirname(api.__file__), "weights", "wms_n1024_k512_t20.pt")
        w, wcode, imax, _ = wms.load(wfile, device="cuda")
        assert np.array_equal(wcode.frozen, ocode.frozen)
        pw = api.PreparedScales(code, w, api.POLAR_FP16)
        assert pw.unit
        w_np = w.cpu().numpy()
    dec = api.Decoder(code, B, L=8)
    dec.hybrid(torch.from_numpy(llr).cuda(), imax, 32.0, api.POLAR_FP16, pw)
    torch.cuda.synchronize()
    status = dec.status.cpu().numpy()
    iters = dec.iters.cpu().numpy().astype(np.int32)
    assert set(np.unique(status)) <= {1, 2, 3}
    rng = np.random.default_rng(11)
    fb = np.nonzero(status != oracle.BP_OK)[0]
    sample = np.unique(np.concatenate([rng.choice(B, 150, replace=False), fb[:100]]))
    rows = llr[sample]
    bp = oracle.bp_decode(rows, ocode, imax, 32.0, "f16", w=w_np, want_llr=False)
    u, st = bp["u_hat"].copy(), bp["status"].copy()
    failed = st != oracle.BP_OK
    if failed.any():
        scl = oracle.scl_decode(rows[failed], ocode, 8, "f32")
        u[failed], st[failed] = scl["u_hat"], scl["status"]
    assert np.array_equal(iters[sample], bp["iters"])
    assert np.array_equal(status[sample], st)
    assert np.array_equal(api.unpack_bits(dec.bits.cpu().numpy()[sample], ocode.P), oracle.payload_of(u, ocode))
    assert np.all(iters[status == oracle.BP_OK] >= 1) and np.all(iters[status != oracle.BP_OK] == imax)


def test_encoder_bit_exact():
    for N, K, crc in [(128, 64, 8), (256, 100, 16), (1024, 512, 16), (2048, 1024, 24), (512, 24, 24), (4096, 2048, 16)]:
        ocode = fr.oracle_code(N, K, crc, design_rate=K / N)
        code = fr.api_code(ocode)
        from paper_1609_09358_gb300 import inputs
        pay = inputs.payload_bits(9, 0, 67, ocode.P)
        x_ref = oracle.encode_batch(pay, ocode)
        cw = torch.zeros((67, N // 8), dtype=torch.uint8, device="cuda")
        api.polar_encode(code, dev(api.pack_bits(pay)), cw)
        torch.cuda.synchronize()
        assert np.array_equal(api.unpack_bits(cw.cpu().numpy(), N), x_ref)


def test_generators_match_cpu_stream():
    from paper_1609_09358_gb300 import inputs
    B, P, N = 37, 496, 1024
    pay = torch.zeros((B, (P + 7) // 8), dtype=torch.uint8, device="cuda")
    api.polar_random_payload(B, P, 1234, 77, pay)
    torch.cuda.synchronize()
    assert np.array_equal(api.unpack_bits(pay.cpu().numpy(), P), inputs.payload_bits(1234, 77, B, P))
    x = np.random.default_rng(1).integers(0, 2, (B, N), dtype=np.uint8)
    llr = torch.zeros((B, N), dtype=torch.float32, device="cuda")
    sigma = 0.8
    api.polar_awgn_llr(dev(api.pack_bits(x)), N, sigma, 99, 5, llr)
    torch.cuda.synchronize()
    z = inputs.unit_noise(99, 5, B, N)
    ref = 2.0 * ((1.0 - 2.0 * x) + sigma * z) / sigma ** 2
    assert np.allclose(llr.cpu().numpy(), ref, rtol=1e-4, atol=1e-4)


def test_hybrid_host_buffers_match_device_path():
    """hybrid_decode_host over several chunks (and a ragged last chunk) equals hybrid_decode."""
    ocode = fr.oracle_code(128, 64, 8)
    code = fr.api_code(ocode)
    B = 70_001
    _, llr = fr.frames_large(ocode, 1.5, B, seed=88)
    dec = api.Decoder(code, B, 4)
    dec.hybrid(dev(llr), 50, 20.0)
    torch.cuda.synchronize()
    bits_h = torch.zeros((B, code.row_bytes), dtype=torch.uint8).pin_memory()
    status_h = torch.zeros(B, dtype=torch.uint8).pin_memory()
    iters_h = torch.zeros(B, dtype=torch.int16).pin_memory()
    ws = torch.zeros(api.polar_workspace_bytes(code, B, 4, api.POLAR_OP_HYBRID_HOST), dtype=torch.uint8,
                     device="cuda")
    api.hybrid_decode_host(code, torch.from_numpy(llr).pin_memory(), 50, 20.0, api.POLAR_FP32, None, 4, bits_h,
                           status_h, iters_h, ws)
    torch.cuda.synchronize()
    assert np.array_equal(bits_h.numpy(), dec.bits.cpu().numpy())
    assert np.array_equal(status_h.numpy(), dec.status.cpu().numpy())
    assert np.array_equal(iters_h.numpy(), dec.iters.cpu().numpy())


def test_profiling_hooks_count_launches():
    ocode = fr.oracle_code(256, 128, 16)
    code = fr.api_code(ocode)
    _, llr = fr.frames(ocode, 1.0, 64, seed=3)
    dec = api.Decoder(code, 64, 8)
    api.polar_profile_enable(True)
    for _ in range(3):
        dec.hybrid(dev(llr), 20, 20.0)
    api.polar_profile_enable(False)
    bp_ms, bp_n, scl_ms, scl_n = api.polar_profile_read()
    assert bp_n == 3 and scl_n == 3 and bp_ms > 0 and scl_ms > 0
    assert api.polar_profile_read()[1] == 0


def test_hybrid_multi_chunk_every_frame():
    """A batch of several hybrid chunks (BP chunks on two streams, CA-SCL of each chunk
    concurrent with later BP chunks), at an Eb/N0 where a large share of frames falls back: every
    frame is compared with the oracle."""
    ocode = fr.oracle_code(128, 64, 8)
    B = 40_000
    _, llr = fr.frames_large(ocode, 1.0, B, seed=606)
    ref = oracle.hybrid_decode(llr, ocode, 30, 20.0, 4, precision="f32")
    bits, status, iters, nfb = run_hybrid(ocode, llr, 30, 4)
    assert nfb == int(np.sum(ref["status"] != oracle.BP_OK)) > 1000
    assert np.array_equal(iters, ref["iters"])
    assert np.array_equal(status, ref["status"])
    assert np.array_equal(bits, oracle.payload_of(ref["u_hat"], ocode))


def test_stress_batch_full_size_sampled():
    """The fallback-heavy stress workload's batch as the benchmark launches it (N = 2048, K = 1024,
    CRC-24, 1.5 dB, 2^16 frames, learned half2 BP with the trained 20-iteration scales, then CA-SCL
    L = 32): the status of every frame is valid and the decoded bits, status and iterations of a
    sample (random frames and CA-SCL frames) equal the oracle's half-precision weighted BP followed
    by its CA-SCL, frame by frame."""
    import os
    from paper_1609_09358_gb300 import wms
    wfile = os.path.join(os.path.dirname(api.__file__), "weights", "wms_n2048_k1024_t20.pt")
    if not os.path.exists(wfile):
        pytest.skip("no trained weights for N = 2048")
    w, code, T, _ = wms.load(wfile, device="cuda")
    ocode = fr.oracle_code(2048, 1024, 24)
    assert np.array_equal(ocode.frozen, code.frozen)
    B = 1 << 16
    _, llr = fr.frames_large(ocode, 1.5, B, seed=1609093577)
    pw = api.PreparedScales(code, w, api.POLAR_FP16)
    dec = api.Decoder(code, B, L=32)
    dec.hybrid(torch.from_numpy(llr).cuda(), T, 32.0, api.POLAR_FP16, pw)
    torch.cuda.synchronize()
    status = dec.status.cpu().numpy()
    iters = dec.iters.cpu().numpy().astype(np.int32)
    assert set(np.unique(status)) <= {1, 2, 3}
    rng = np.random.default_rng(5)
    fb = np.nonzero(status != oracle.BP_OK)[0]
    ok = np.nonzero(status == oracle.BP_OK)[0]
    sample = np.unique(np.concatenate([rng.choice(B, 12, replace=False), fb[:6], ok[:6]]))
    rows = llr[sample]
    bp = oracle.bp_decode(rows, ocode, T, 32.0, "f16", w=w.cpu().numpy(), want_llr=False)
    u, st = bp["u_hat"].copy(), bp["status"].copy()
    failed = st != oracle.BP_OK
    if failed.any():
        scl = oracle.scl_decode(rows[failed], ocode, 32, "f32")
        u[failed], st[failed] = scl["u_hat"], scl["status"]
    assert np.array_equal(iters[sample], bp["iters"])
    assert np.array_equal(status[sample], st)
    assert np.array_equal(api.unpack_bits(dec.bits.cpu().numpy()[sample], ocode.P), oracle.payload_of(u, ocode))
