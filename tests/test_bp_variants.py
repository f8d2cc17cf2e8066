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


# Largest error of one evaluation of the kernels' exact PE function against the function itself at
# the same binary32 inputs: the fast exponential (relative error about 2^-22, on values <= 1) and
# logarithm (absolute error about 2^-22 on its argument range here) contribute a few 1e-7 each to
# ln(p / q); the Newton quotient 1e-8; the final fused add rounds a result of magnitude < 32 to
# binary32 (half an ulp, <= 9.5e-7).  test_exact_pe_function_per_update_error measures it.
EPS_G = 2e-6
U32 = 2.0 ** -24  # relative rounding error of a binary32 addition (round to nearest)


def _g_exact64(x, y):
    """The exact PE function of Sec. II-B in binary64."""
    return np.log((1.0 + np.exp(x + y)) / (np.exp(x) + np.exp(y)))


def test_exact_pe_function_per_update_error():
    """Each evaluation of the exact PE function by the kernels (the scalar form and the packed pair
    form the FP32 BP kernels use, through polar_pe_eval) is within EPS_G of the function evaluated in
    binary64 at the same inputs, over the whole range the decoder feeds it (first argument a clipped
    message, |a| <= 20; second a sum of two, |b| <= 40; a dense grid plus near-zero and edge values),
    and the two forms agree bit for bit."""
    a1 = np.concatenate([np.linspace(-20, 20, 1601), [-1e-30, 0.0, 1e-30, 1e-6, -1e-6]]).astype(np.float32)
    b1 = np.concatenate([np.linspace(-40, 40, 3201), [-1e-30, 0.0, 1e-30, 1e-6, -1e-6, 19.999998]]).astype(np.float32)
    a, b = (v.ravel() for v in np.meshgrid(a1, b1, indexing="ij"))
    ad, bd = dev(a), dev(b)
    out = {}
    for op in (api.POLAR_PE_EXACT, api.POLAR_PE_EXACT_PACKED, api.POLAR_PE_MINSUM):
        o = torch.empty_like(ad)
        api.polar_pe_eval(op, ad, bd, o)
        torch.cuda.synchronize()
        out[op] = o.cpu().numpy()
    ref = _g_exact64(a.astype(np.float64), b.astype(np.float64))
    err = np.abs(out[api.POLAR_PE_EXACT].astype(np.float64) - ref)
    assert err.max() <= EPS_G, (err.max(), a[err.argmax()], b[err.argmax()])
    assert np.array_equal(out[api.POLAR_PE_EXACT].view(np.uint32), out[api.POLAR_PE_EXACT_PACKED].view(np.uint32))
    ms = np.sign(a) * np.sign(b) * np.minimum(np.abs(a), np.abs(b))
    assert np.array_equal(out[api.POLAR_PE_MINSUM], ms.astype(np.float32))


def _dsup(x, ex, y, ey):
    """Largest |dg/dx| = |sinh y| / (cosh x + cosh y) over |x' - x| <= ex, |y' - y| <= ey: the
    derivative falls with |x| and grows with |y|, so it is taken at |x| - ex (not below 0) and
    |y| + ey; written with exponentials of non-positive arguments only."""
    ax = np.maximum(np.abs(x) - ex, 0.0)
    ay = np.abs(y) + ey
    with np.errstate(over="ignore"):
        return (1.0 - np.exp(-2.0 * ay)) / (np.exp(ax - ay) + np.exp(-ax - ay) + 1.0 + np.exp(-2.0 * ay))


def _bp_exact_bounds(llr32, ocode, T, M=20.0):
    """LLR(u), LLR(x) after T iterations of BP with the exact PE function in binary64 (the oracle's
    schedule: the R sweep, then the L sweep, every message clipped to [-M, M]) and, element by
    element, a bound on how far a binary32 decoder can be from them when each of its PE functions is
    within EPS_G of the exact one at its own inputs and each addition rounds to nearest.  The bound
    is carried through every update, counting the fan-in of errors: by the mean value theorem
    |g(x', y') - g(x, y)| <= D_x |x' - x| + D_y |y' - y| with D the largest partial derivatives over
    the inputs' error boxes (_dsup); an addition adds its operands' bounds and its rounding error;
    a clip does not increase a difference."""
    B, N = llr32.shape
    n = ocode.n
    L = np.zeros((n + 2, B, N))
    R = np.zeros((n + 2, B, N))
    EL, ER = np.zeros_like(L), np.zeros_like(R)
    L[n + 1] = np.clip(llr32.astype(np.float64), -M, M)
    R[1] = np.where(ocode.frozen.astype(bool), M, 0.0)[None, :]

    def ge(x, ex, y, ey):
        return np.clip(_g_exact64(x, y), -M, M), _dsup(x, ex, y, ey) * ex + _dsup(y, ey, x, ex) * ey + EPS_G

    def add(x, ex, y, ey):
        v = x + y
        return v, ex + ey + U32 * (np.abs(v) + ex + ey)

    idx = np.arange(N)
    for _ in range(T):
        for sweep in ("R", "L"):
            stages = range(1, n + 1) if sweep == "R" else range(n, 0, -1)
            for s in stages:
                d = 1 << (s - 1)
                jA = idx[(idx & d) == 0]
                jB = jA + d
                a1, ea1, a2, ea2 = R[s][:, jA], ER[s][:, jA], R[s][:, jB], ER[s][:, jB]
                l1, el1, l2, el2 = L[s + 1][:, jA], EL[s + 1][:, jA], L[s + 1][:, jB], EL[s + 1][:, jB]
                y, ey = add(l2, el2, a2, ea2)
                if sweep == "R":
                    o1, e1 = ge(a1, ea1, y, ey)
                    o2, e2 = add(*ge(a1, ea1, l1, el1), a2, ea2)
                    R[s + 1][:, jA], ER[s + 1][:, jA] = o1, e1
                    R[s + 1][:, jB], ER[s + 1][:, jB] = np.clip(o2, -M, M), e2
                else:
                    o1, e1 = ge(l1, el1, y, ey)
                    o2, e2 = add(*ge(a1, ea1, l1, el1), l2, el2)
                    L[s][:, jA], EL[s][:, jA] = o1, e1
                    L[s][:, jB], EL[s][:, jB] = np.clip(o2, -M, M), e2
    return add(L[1], EL[1], R[1], ER[1]), add(L[n + 1], EL[n + 1], R[n + 1], ER[n + 1])


@pytest.mark.parametrize("N,K,crc,ebn0,B", [(128, 64, 8, 2.0, 64), (1024, 512, 16, 2.0, 24), (2048, 1024, 24, 1.5, 8),
                                            (4096, 2048, 16, 1.5, 4)])
@pytest.mark.parametrize("T", [1, 2, 3])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_exact_g_llrs_within_propagated_bound(N, K, crc, ebn0, B, T, seed):
    """BP with the exact PE function after exactly T iterations: every LLR(u) and LLR(x) of the
    kernel lies within the element's propagated error bound (_bp_exact_bounds) of binary64 BP, and
    the hard decisions of the information bits agree wherever the binary64 LLR is farther from zero
    than its bound.  The binary64 replica that carries the bounds equals the oracle's binary64 BP.
    The bound is worst-case (errors that add along every path of the graph), so it grows quickly
    with the iterations (median about 1e-3 at T = 3): the first iterations are checked here, the
    decoding outcome of full runs by the hybrid tests below."""
    ocode = fr.oracle_code(N, K, crc)
    _, llr = fr.frames(ocode, ebn0, B, seed=7300 + N + 1000 * seed)
    (u, eu), (x, ex) = _bp_exact_bounds(llr, ocode, T)
    ref = oracle.bp_decode(llr, ocode, T, 20.0, "f64", early_stop=False, g="exact", llr_u_double=True)
    assert np.max(np.abs(u - ref["llr_u_f64"])) <= 1e-9
    assert np.max(np.abs(x - ref["llr_x"].astype(np.float64))) <= 4e-6  # the oracle returns LLR(x) in binary32
    got = run_bp(ocode, llr, T, EXACT | api.POLAR_FIXED_ITERS)
    du = np.abs(got["llr_u"].astype(np.float64) - u)
    dx = np.abs(got["llr_x"].astype(np.float64) - x)
    assert np.all(du <= eu + 1e-9), (np.max(du - eu), np.max(du / eu))
    assert np.all(dx <= ex + 1e-9), (np.max(dx - ex), np.max(dx / ex))
    info = ocode.info_idx
    sure = np.abs(u[:, info]) > eu[:, info]
    assert np.array_equal((got["llr_u"][:, info] < 0)[sure], (u[:, info] < 0)[sure])
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


@pytest.mark.parametrize("stop", ["crc", "reencode"])
def test_paper_configuration_hybrid_end_to_end(stop):
    """The paper's own decoder (Sec. II-B exact PE function with LLR_max = 20, Sec. III hybrid with
    i_max = 50 and CA-SCL L = 32) on its code length N = 4096, R = 1/2 (K = 2048 incl. CRC-16), at
    1.5 dB where about a quarter of the frames fall back to CA-SCL: per-frame outcomes against the
    oracle's FP64 hybrid.  As in the N <= 1024 test, a rounding-level difference may move a frame's stopping
    iteration, so outcomes (bits and status) are compared: all but at most one of the 32 frames
    identical, the frame-error counts within 2, and every frame the two sides both send to CA-SCL
    decoded to the same bits."""
    ocode = fr.oracle_code(4096, 2048, 16)
    B = 32
    pay, llr = fr.frames(ocode, 1.5, B, seed=7500)
    ref = oracle.hybrid_decode(llr, ocode, 50, 20.0, 32, precision="f64", stop=stop, g="exact")
    flags = EXACT | (api.POLAR_STOP_REENCODE if stop == "reencode" else 0)
    bits, status, iters = run_hybrid(ocode, llr, 50, 32, flags)
    rb = oracle.payload_of(ref["u_hat"], ocode)
    same = np.all(bits == rb, axis=1) & (status == ref["status"])
    assert int(np.sum(~same)) <= 1, np.nonzero(~same)[0]
    both_scl = (status != oracle.BP_OK) & (ref["status"] != oracle.BP_OK)
    assert np.any(both_scl) and np.any(status == oracle.BP_OK)
    assert np.array_equal(bits[both_scl], rb[both_scl])
    fe_gpu = int(np.sum(np.any(bits != pay, axis=1)))
    fe_ref = int(np.sum(np.any(rb != pay, axis=1)))
    assert abs(fe_gpu - fe_ref) <= 2, (fe_gpu, fe_ref)
