"""BP variants of Sec. II-B through the C ABI against the CPU oracle.

The re-encoding stop (min-sum g): bit-exact -- decided bits, status, iteration counts and output
LLRs of bp_decode, and the hybrid's bits, status and iterations.  Inputs are seeded frames built on
the CPU (tests/frames.py), batch sizes with a ragged tail of the CTA grid.
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


def run_bp(ocode, llr, max_iters, precision):
    code = fr.api_code(ocode)
    B, N = llr.shape
    bits = torch.zeros((B, code.row_bytes), dtype=torch.uint8, device="cuda")
    status = torch.zeros(B, dtype=torch.uint8, device="cuda")
    iters = torch.zeros(B, dtype=torch.int16, device="cuda")
    lu = torch.zeros((B, N), dtype=torch.float32, device="cuda")
    lx = torch.zeros((B, N), dtype=torch.float32, device="cuda")
    api.bp_decode(code, dev(llr), max_iters, 20.0, precision, None, bits, status, iters, lu, lx)
    torch.cuda.synchronize()
    return {"bits": api.unpack_bits(bits.cpu().numpy(), ocode.P), "status": status.cpu().numpy(),
            "iters": iters.cpu().numpy().astype(np.int32), "llr_u": lu.cpu().numpy(), "llr_x": lx.cpu().numpy()}


def run_hybrid(ocode, llr, imax, L, precision):
    code = fr.api_code(ocode)
    dec = api.Decoder(code, llr.shape[0], L)
    dec.hybrid(dev(llr), imax, 20.0, precision)
    torch.cuda.synchronize()
    return (api.unpack_bits(dec.bits.cpu().numpy(), ocode.P), dec.status.cpu().numpy(),
            dec.iters.cpu().numpy().astype(np.int32))


REENC = api.POLAR_FP32 | api.POLAR_STOP_REENCODE


@pytest.mark.parametrize("N,K,crc,ebn0,B,imax", [
    (128, 64, 8, 2.0, 203, 50),
    (256, 128, 16, 2.0, 97, 60),
    (512, 256, 16, 1.5, 45, 60),
    (1024, 512, 16, 2.5, 37, 200),
    (1024, 512, 16, 1.0, 12, 100),
    (2048, 1024, 24, 2.0, 9, 80),
    (4096, 2048, 16, 2.0, 5, 50),
])
def test_reencoding_stop_bit_exact(N, K, crc, ebn0, B, imax):
    ocode = fr.oracle_code(N, K, crc)
    _, llr = fr.frames(ocode, ebn0, B, seed=7000 + N)
    ref = oracle.bp_decode(llr, ocode, imax, 20.0, "f32", stop="reencode")
    got = run_bp(ocode, llr, imax, REENC)
    assert np.array_equal(got["iters"], ref["iters"]), np.nonzero(got["iters"] != ref["iters"])[0][:10]
    assert np.array_equal(got["status"], ref["status"])
    assert np.array_equal(got["bits"], oracle.payload_of(ref["u_hat"], ocode))
    assert np.array_equal(got["llr_u"], ref["llr_u"])
    assert np.array_equal(got["llr_x"], ref["llr_x"])


@pytest.mark.parametrize("N,K,crc,ebn0,B,imax,L", [(128, 64, 8, 1.5, 300, 50, 4), (1024, 512, 16, 2.0, 120, 200, 8)])
def test_reencoding_stop_hybrid_bit_exact(N, K, crc, ebn0, B, imax, L):
    ocode = fr.oracle_code(N, K, crc)
    _, llr = fr.frames(ocode, ebn0, B, seed=7100 + N)
    ref = oracle.hybrid_decode(llr, ocode, imax, 20.0, L, precision="f32", stop="reencode")
    bits, status, iters = run_hybrid(ocode, llr, imax, L, REENC)
    assert np.array_equal(iters, ref["iters"])
    assert np.array_equal(status, ref["status"])
    assert np.array_equal(bits, oracle.payload_of(ref["u_hat"], ocode))
    assert np.any(status != oracle.BP_OK)


@pytest.mark.parametrize("N,K,crc,ebn0,B,imax,L,chunk", [
    (128, 64, 8, 1.5, 3001, 50, 4, 256),       # 12 chunks, ragged last chunk, many CA-SCL launches
    (1024, 512, 16, 2.0, 1500, 200, 8, 700),   # chunk not a multiple of the frames per CTA
    (2048, 1024, 24, 2.0, 300, 60, 16, 4096),  # one chunk
])
def test_host_scheduled_equals_hybrid(N, K, crc, ebn0, B, imax, L, chunk):
    """The host-scheduled form of Fig. 3 decodes every frame exactly as hybrid_decode (BP, then
    CA-SCL on the CRC failures), whatever the chunking; a sample is checked against the oracle."""
    ocode = fr.oracle_code(N, K, crc)
    code = fr.api_code(ocode)
    _, llr = fr.frames(ocode, ebn0, B, seed=7200 + N)
    dec = api.Decoder(code, B, L)
    llr_d = dev(llr)
    dec.hybrid(llr_d, imax, 20.0, api.POLAR_FP32)
    torch.cuda.synchronize()
    want = [t.cpu().numpy().copy() for t in (dec.bits, dec.status, dec.iters)]
    for t in (dec.bits, dec.status, dec.iters):
        t.zero_()
    dec.scheduled(llr_d, imax, 20.0, api.POLAR_FP32, chunk=chunk)
    torch.cuda.synchronize()
    got = [t.cpu().numpy() for t in (dec.bits, dec.status, dec.iters)]
    for w, g in zip(want, got):
        assert np.array_equal(w, g)
    assert np.any(got[1] != oracle.BP_OK) and np.any(got[1] == oracle.BP_OK)
    sample = np.unique(np.concatenate([np.arange(0, B, max(1, B // 40)), np.nonzero(got[1] != oracle.BP_OK)[0][:20]]))
    ref = oracle.hybrid_decode(llr[sample], ocode, imax, 20.0, L, precision="f32")
    assert np.array_equal(got[1][sample], ref["status"])
    assert np.array_equal(got[2][sample].astype(np.int32), ref["iters"])
    assert np.array_equal(api.unpack_bits(got[0][sample], ocode.P), oracle.payload_of(ref["u_hat"], ocode))


EXACT = api.POLAR_FP32 | api.POLAR_G_EXACT


@pytest.mark.parametrize("N,K,crc,ebn0,B", [(128, 64, 8, 2.0, 64), (1024, 512, 16, 2.0, 24), (2048, 1024, 24, 1.5, 8),
                                            (4096, 2048, 16, 1.5, 4)])
@pytest.mark.parametrize("T", [1, 3, 5])
def test_exact_g_llrs_within_tolerance(N, K, crc, ebn0, B, T):
    """The exact PE function: the kernel evaluates its two correction terms with the fast
    exponential and logarithm, so each update carries an absolute error of at most about 2e-6
    (those functions' error plus one binary32 rounding of values up to LLR_max = 20), and an LLR after
    T iterations is reached through about 2 n T updates of 1-Lipschitz operations: the kernel's
    LLR(u) and LLR(x) after exactly T iterations are within 4e-6 n T of the oracle's FP64
    evaluation, and the hard decisions of the information bits agree wherever the oracle's LLR is
    farther than that from zero."""
    ocode = fr.oracle_code(N, K, crc)
    _, llr = fr.frames(ocode, ebn0, B, seed=7300 + N)
    ref = oracle.bp_decode(llr, ocode, T, 20.0, "f64", early_stop=False, g="exact")
    got = run_bp(ocode, llr, T, EXACT | api.POLAR_FIXED_ITERS)
    tol = 4e-6 * ocode.n * T
    assert np.max(np.abs(got["llr_u"] - ref["llr_u"])) <= tol
    assert np.max(np.abs(got["llr_x"] - ref["llr_x"])) <= tol
    info = ocode.info_idx
    sure = np.abs(ref["llr_u"][:, info]) > tol
    assert np.array_equal((got["llr_u"][:, info] < 0)[sure], (ref["llr_u"][:, info] < 0)[sure])
    assert np.all(got["iters"] == T)


@pytest.mark.parametrize("N,K,crc,ebn0,B,imax,L,stop", [(128, 64, 8, 1.5, 600, 50, 4, "crc"),
                                                        (1024, 512, 16, 2.0, 200, 200, 8, "crc"),
                                                        (1024, 512, 16, 2.0, 200, 200, 8, "reencode")])
def test_exact_g_hybrid_agrees_with_oracle(N, K, crc, ebn0, B, imax, L, stop):
    """Hybrid decoding with the exact PE function: since BP is iterated to a CRC (or re-encoding)
    decision, rounding-level differences can move a frame's stopping iteration, so frames are
    compared as outcomes: at least 95% of frames decode to the same bits with the same status as the
    oracle's FP64 hybrid, and the two frame-error counts differ by at most max(2, 1% of B)."""
    ocode = fr.oracle_code(N, K, crc)
    pay, llr = fr.frames(ocode, ebn0, B, seed=7400 + N)
    ref = oracle.hybrid_decode(llr, ocode, imax, 20.0, L, precision="f64", stop=stop, g="exact")
    flags = EXACT | (api.POLAR_STOP_REENCODE if stop == "reencode" else 0)
    bits, status, iters = run_hybrid(ocode, llr, imax, L, flags)
    rb = oracle.payload_of(ref["u_hat"], ocode)
    same = np.all(bits == rb, axis=1) & (status == ref["status"])
    assert same.mean() >= 0.95, same.mean()
    fe_gpu = int(np.sum(np.any(bits != pay, axis=1)))
    fe_ref = int(np.sum(np.any(rb != pay, axis=1)))
    assert abs(fe_gpu - fe_ref) <= max(2, B // 100), (fe_gpu, fe_ref)
