"""CPU oracle for the hybrid BP + CA-SCL polar decoder (arXiv 1609.09358).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It is a plain, slow reference written from the paper
(Sec. II encoder and construction, Sec. II-A CA-SCL, Sec. II-B BP, Sec. III hybrid rule) in C,
compiled with ``gcc -O2 -ffp-contract=off`` and loaded through ctypes.  It shares no code with the
CUDA decoder in ``paper_1609_09358_gb300``; neither imports the other.

Parity pins: tests/test_oracle_pins.py.  Every oracle function is pinned there against something
other than itself (the paper's Fig. 1 worked example, catalogue CRC check values, closed forms,
brute-force ML, invariants).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = [os.path.join(_HERE, "polar_oracle.c"), os.path.join(_HERE, "polar_oracle_decoders.inc")]
_lock = threading.Lock()
_lib = None

# per-frame status codes of the hybrid decoder (same meaning as the library's)
BP_OK, SCL_OK, SCL_CRC_FAIL, BP_FAIL = 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (plain gcc, no GPU headers)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in _SRC)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    tmp = _SO + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-o", tmp, _SRC[0], "-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _SO)
    return _SO


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
        return _lib


_u8p = ctypes.POINTER(ctypes.c_uint8)
_i32p = ctypes.POINTER(ctypes.c_int32)
_f32p = ctypes.POINTER(ctypes.c_float)
_f64p = ctypes.POINTER(ctypes.c_double)
_c_int, _c_uint, _c_double = ctypes.c_int, ctypes.c_uint, ctypes.c_double


def _declare(L):
    L.or_bhattacharyya_lnz.argtypes = [_c_int, _c_int, _c_double]
    L.or_bhattacharyya_lnz.restype = _c_double
    L.or_construct.argtypes = [_c_int, _c_int, _c_double, _c_double, _u8p, _i32p, _f64p]
    L.or_poly_mod.argtypes = [_u8p, _c_int, _c_uint, _c_int, _u8p]
    L.or_crc.argtypes = [_u8p, _c_int, _c_uint, _c_int, _u8p]
    L.or_crc_check.argtypes = [_u8p, _c_int, _c_uint, _c_int]
    L.or_generator_entry.argtypes = [_c_int, _c_int]
    L.or_polar_transform.argtypes = [_u8p, _c_int, _u8p]
    L.or_encode_circuit.argtypes = [_u8p, _c_int, _u8p]
    L.or_build_u.argtypes = [_u8p, _c_int, _c_int, _i32p, _c_uint, _c_int, _u8p]
    L.or_encode_batch.argtypes = [_u8p, _c_int, _c_int, _c_int, _i32p, _c_uint, _c_int, _u8p]
    L.or_channel_llr.argtypes = [_u8p, _f64p, ctypes.c_longlong, _c_double, _f32p]
    L.or_round_half.argtypes = [ctypes.c_float]
    L.or_round_half.restype = ctypes.c_float
    L.or_ml_decode.argtypes = [_f64p, _c_int, _c_int, _i32p, _u8p]
    L.or_ml_decode.restype = _c_double
    L.or_set_num_threads.argtypes = [_c_int]
    L.or_num_threads.restype = _c_int
    for sfx in ("f32", "f64", "f16"):
        getattr(L, "or_bp_decode_batch_" + sfx).argtypes = [
            _f32p, _c_int, _c_int, _u8p, _i32p, _c_int, _c_uint, _c_int, _c_int, _c_double, _c_int,
            _f32p, _c_int, _u8p, _u8p, _i32p, _f32p, _f32p, _f64p]
    for sfx in ("f32", "f64"):
        getattr(L, "or_wms_grad_" + sfx).argtypes = [_f32p, _c_int, _u8p, _c_int, _c_double, _f32p, _f64p, _c_int,
                                                     _f64p]
        getattr(L, "or_sc_decode_" + sfx).argtypes = [_f32p, _c_int, _u8p, _u8p]
        getattr(L, "or_sc_bit_llr_" + sfx).argtypes = [_f32p, _c_int, _u8p, _c_int]
        getattr(L, "or_sc_bit_llr_" + sfx).restype = _c_double
        getattr(L, "or_scl_decode_" + sfx).argtypes = [
            _f32p, _c_int, _u8p, _u8p, _i32p, _c_int, _c_uint, _c_int, _c_int, _u8p, _f64p, _u8p, _f64p,
            _i32p]
        getattr(L, "or_scl_decode_batch_" + sfx).argtypes = [
            _f32p, _c_int, _c_int, _u8p, _u8p, _i32p, _c_int, _c_uint, _c_int, _c_int, _u8p, _u8p, _f64p]
        getattr(L, "or_hybrid_decode_batch_" + sfx).argtypes = [
            _f32p, _c_int, _c_int, _u8p, _u8p, _i32p, _c_int, _c_uint, _c_int, _c_int, _c_double, _c_int,
            _c_int, _f32p, _c_int, _u8p, _u8p, _i32p]
    for sfx in ("f32", "f64", "f16"):
        getattr(L, "or_pe_g_exact_" + sfx).argtypes = [_c_double, _c_double]
        getattr(L, "or_pe_g_exact_" + sfx).restype = _c_double


# BP mode bits of the C library (or_bp_decode): stopping rule and PE function (Sec. II-B)
BP_CRC_STOP, BP_REENC_STOP, BP_G_EXACT = 1, 2, 4


def bp_mode(early_stop: bool = True, stop: str = "crc", g: str = "minsum") -> int:
    """Mode bits: stop "crc" (the CRC of u, the paper's rule) or "reencode" (HD(LLR(x)) equals the
    re-encoded HD(LLR(u))); g "minsum" or "exact"."""
    if stop not in ("crc", "reencode") or g not in ("minsum", "exact"):
        raise ValueError("stop in {crc, reencode}, g in {minsum, exact}")
    m = (BP_CRC_STOP if stop == "crc" else BP_REENC_STOP) if early_stop else 0
    return m | (BP_G_EXACT if g == "exact" else 0)


def pe_g_exact(a: float, b: float, precision: str = "f64") -> float:
    """The exact PE function g(a, b) of Sec. II-B as the BP of the given precision evaluates it."""
    return float(getattr(lib(), "or_pe_g_exact_" + precision)(a, b))


def _dec(code):
    """The decision-aided mask of a code as a contiguous uint8 array, or None."""
    return None if code.decided is None else np.ascontiguousarray(code.decided, dtype=np.uint8)


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def _u8(a):
    return np.ascontiguousarray(a, dtype=np.uint8)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


@dataclass
class Code:
    """A polar code: length N, K non-frozen positions (c of them CRC), CRC generator."""
    N: int
    K: int
    crc_len: int
    crc_poly: int
    frozen: np.ndarray    # uint8 [N], 1 = frozen
    info_idx: np.ndarray  # int32 [K], ascending
    # uint8 [N] or None: information positions CA-SCL decides without branching (decision aiding)
    decided: Optional[np.ndarray] = None

    @property
    def n(self) -> int:
        return self.N.bit_length() - 1

    @property
    def P(self) -> int:
        return self.K - self.crc_len


CRC_POLYS = {0: 0x0, 8: 0x07, 16: 0x1021, 24: 0x864CFB}


def set_threads(n: int) -> None:
    lib().or_set_num_threads(int(n))


def num_threads() -> int:
    return int(lib().or_num_threads())


# ---------------------------------------------------------------- construction / CRC / encoder
def bhattacharyya_lnz(n: int, i: int, lnz0: float) -> float:
    return float(lib().or_bhattacharyya_lnz(n, i, lnz0))


def construct(N: int, K: int, design_ebn0_db: float, design_rate: float):
    frozen = np.zeros(N, np.uint8)
    info = np.zeros(K, np.int32)
    lnz = np.zeros(N, np.float64)
    rc = lib().or_construct(N, K, design_ebn0_db, design_rate, _p(frozen, _u8p), _p(info, _i32p),
                            _p(lnz, _f64p))
    if rc != 0:
        raise ValueError("bad construction arguments")
    return frozen, info, lnz


def make_code(N: int, K: int, crc_len: int, design_ebn0_db: float = 0.0, design_rate=None) -> Code:
    """Code with a Bhattacharyya frozen set at the design point; design rate = payload rate."""
    if design_rate is None:
        design_rate = (K - crc_len) / N
    frozen, info, _ = construct(N, K, design_ebn0_db, design_rate)
    return Code(N, K, crc_len, CRC_POLYS[crc_len], frozen, info)


def poly_mod(m, poly: int, c: int) -> np.ndarray:
    m = _u8(m)
    out = np.zeros(max(c, 1), np.uint8)
    lib().or_poly_mod(_p(m, _u8p), len(m), poly, c, _p(out, _u8p))
    return out[:c]


def crc(msg, poly: int, c: int) -> np.ndarray:
    msg = _u8(msg)
    out = np.zeros(max(c, 1), np.uint8)
    lib().or_crc(_p(msg, _u8p), len(msg), poly, c, _p(out, _u8p))
    return out[:c]


def crc_check(bits, poly: int, c: int) -> bool:
    bits = _u8(bits)
    return bool(lib().or_crc_check(_p(bits, _u8p), len(bits), poly, c))


def generator_entry(i: int, j: int) -> int:
    return int(lib().or_generator_entry(i, j))


def polar_transform(u) -> np.ndarray:
    u = _u8(u)
    x = np.zeros_like(u)
    lib().or_polar_transform(_p(u, _u8p), len(u), _p(x, _u8p))
    return x


def encode_circuit(u) -> np.ndarray:
    u = _u8(u)
    x = np.zeros_like(u)
    lib().or_encode_circuit(_p(u, _u8p), len(u), _p(x, _u8p))
    return x


def build_u(payload, code: Code) -> np.ndarray:
    payload = _u8(payload)
    u = np.zeros(code.N, np.uint8)
    lib().or_build_u(_p(payload, _u8p), code.N, code.K, _p(code.info_idx, _i32p), code.crc_poly,
                     code.crc_len, _p(u, _u8p))
    return u


def encode_batch(payload, code: Code) -> np.ndarray:
    """payload uint8 [B][P] (one byte per bit) -> codeword uint8 [B][N] (matrix definition)."""
    payload = _u8(payload)
    B = payload.shape[0] if payload.ndim == 2 else payload.size // max(code.P, 1)
    payload = payload.reshape(B, code.P)
    x = np.zeros((B, code.N), np.uint8)
    lib().or_encode_batch(_p(payload, _u8p), B, code.N, code.K, _p(code.info_idx, _i32p),
                          code.crc_poly, code.crc_len, _p(x, _u8p))
    return x


def channel_llr(x, noise, sigma: float) -> np.ndarray:
    x = _u8(x)
    noise = np.ascontiguousarray(noise, dtype=np.float64)
    assert noise.shape == x.shape
    out = np.zeros(x.shape, np.float32)
    lib().or_channel_llr(_p(x, _u8p), _p(noise, _f64p), x.size, sigma, _p(out, _f32p))
    return out


def sigma_for(ebn0_db: float, rate: float) -> float:
    """Noise standard deviation for BPSK at Eb/N0 and code rate R: sigma^2 = 1 / (2 R Eb/N0)."""
    return float(np.sqrt(1.0 / (2.0 * rate * 10.0 ** (ebn0_db / 10.0))))


def round_half(x: float) -> float:
    return float(lib().or_round_half(float(x)))


# ---------------------------------------------------------------- decoders
def bp_decode(llr, code: Code, max_iters: int, llr_max: float, precision: str = "f32",
              early_stop: bool = True, w=None, want_llr: bool = True, llr_u_double: bool = False,
              stop: str = "crc", g: str = "minsum") -> dict:
    """BP with early stop on a batch llr float32 [B][N] (Sec. II-B): min-sum or exact g, CRC or
    re-encoding stop (bp_mode)."""
    llr = _f32(llr).reshape(-1, code.N)
    B, N = llr.shape
    u = np.zeros((B, N), np.uint8)
    st = np.zeros(B, np.uint8)
    it = np.zeros(B, np.int32)
    lu = np.zeros((B, N), np.float32) if want_llr else None
    lx = np.zeros((B, N), np.float32) if want_llr else None
    lud = np.zeros((B, N), np.float64) if llr_u_double else None
    w_iters = 0
    if w is not None:
        w = _f32(w)
        w_iters = w.shape[0]
        assert w.shape == (w_iters, 2, code.n, N)  # iterations past w_iters run unweighted
    getattr(lib(), "or_bp_decode_batch_" + precision)(
        _p(llr, _f32p), B, N, _p(code.frozen, _u8p), _p(code.info_idx, _i32p), code.K,
        code.crc_poly, code.crc_len, max_iters, llr_max, bp_mode(early_stop, stop, g), _p(w, _f32p), w_iters,
        _p(u, _u8p), _p(st, _u8p), _p(it, _i32p), _p(lu, _f32p), _p(lx, _f32p), _p(lud, _f64p))
    return {"u_hat": u, "status": st, "iters": it, "llr_u": lu, "llr_x": lx, "llr_u_f64": lud}


def wms_grad(llr, code: Code, T: int, llr_max: float, w, dy, precision: str = "f64",
             all_iters: bool = False) -> np.ndarray:
    """d/dw of sum_b sum_i dy[b][i] LLR(u_i) after T weighted BP iterations (no early stop); with
    all_iters, dy is [T][B][N] and the loss sums over the LLR(u) of every iteration."""
    llr = _f32(llr).reshape(-1, code.N)
    B = llr.shape[0]
    dy = np.asarray(dy, dtype=np.float64)
    dy = dy.reshape(T, B, code.N) if all_iters else dy.reshape(1, B, code.N)
    w = _f32(w)
    g = np.zeros(w.shape, np.float64)
    fn = getattr(lib(), "or_wms_grad_" + precision)
    for b in range(B):
        row = np.ascontiguousarray(llr[b])
        dyb = np.ascontiguousarray(dy[:, b, :])
        fn(_p(row, _f32p), code.N, _p(code.frozen, _u8p), T, llr_max, _p(w, _f32p), _p(dyb, _f64p),
           1 if all_iters else 0, _p(g, _f64p))
    return g


def sc_decode(llr, code: Code, precision: str = "f32") -> np.ndarray:
    llr = _f32(llr).reshape(-1, code.N)
    out = np.zeros(llr.shape, np.uint8)
    fn = getattr(lib(), "or_sc_decode_" + precision)
    for b in range(llr.shape[0]):
        row = np.ascontiguousarray(llr[b])
        o = np.zeros(code.N, np.uint8)
        fn(_p(row, _f32p), code.N, _p(code.frozen, _u8p), _p(o, _u8p))
        out[b] = o
    return out


def sc_bit_llr(llr_row, u, i: int, precision: str = "f64") -> float:
    """SC LLR of bit i given the decided prefix u[0..i-1] (Sec. II-A recursion)."""
    row = _f32(llr_row)
    u = _u8(u)
    return float(getattr(lib(), "or_sc_bit_llr_" + precision)(_p(row, _f32p), len(row), _p(u, _u8p), i))


def scl_decode(llr, code: Code, L: int, precision: str = "f32") -> dict:
    llr = _f32(llr).reshape(-1, code.N)
    B, N = llr.shape
    u = np.zeros((B, N), np.uint8)
    st = np.zeros(B, np.uint8)
    pm = np.zeros(B, np.float64)
    getattr(lib(), "or_scl_decode_batch_" + precision)(
        _p(llr, _f32p), B, N, _p(code.frozen, _u8p), _p(_dec(code), _u8p), _p(code.info_idx, _i32p), code.K,
        code.crc_poly, code.crc_len, L, _p(u, _u8p), _p(st, _u8p), _p(pm, _f64p))
    return {"u_hat": u, "status": st, "pm": pm}


def scl_list(llr_row, code: Code, L: int, precision: str = "f32"):
    """Final list of one frame: (list_u [A][N], list_pm [A], chosen u, crc_ok)."""
    row = _f32(llr_row).reshape(code.N)
    lu = np.zeros((L, code.N), np.uint8)
    lpm = np.zeros(L, np.float64)
    u = np.zeros(code.N, np.uint8)
    pm = np.zeros(1, np.float64)
    na = np.zeros(1, np.int32)
    ok = getattr(lib(), "or_scl_decode_" + precision)(
        _p(row, _f32p), code.N, _p(code.frozen, _u8p), _p(_dec(code), _u8p), _p(code.info_idx, _i32p), code.K,
        code.crc_poly, code.crc_len, L, _p(u, _u8p), _p(pm, _f64p), _p(lu, _u8p), _p(lpm, _f64p),
        _p(na, _i32p))
    a = int(na[0])
    return lu[:a], lpm[:a], u, bool(ok)


def hybrid_decode(llr, code: Code, max_iters: int, llr_max: float, L: int, w=None,
                  precision: str = "f32", stop: str = "crc", g: str = "minsum") -> dict:
    """Sec. III hybrid: BP with CRC stop (or the re-encoding stop), CA-SCL on the frames whose CRC
    fails when BP stops."""
    llr = _f32(llr).reshape(-1, code.N)
    B, N = llr.shape
    u = np.zeros((B, N), np.uint8)
    st = np.zeros(B, np.uint8)
    it = np.zeros(B, np.int32)
    w_iters = 0
    if w is not None:
        w = _f32(w)
        w_iters = w.shape[0]
    getattr(lib(), "or_hybrid_decode_batch_" + precision)(
        _p(llr, _f32p), B, N, _p(code.frozen, _u8p), _p(_dec(code), _u8p), _p(code.info_idx, _i32p), code.K,
        code.crc_poly, code.crc_len, max_iters, llr_max, bp_mode(True, stop, g), L, _p(w, _f32p), w_iters,
        _p(u, _u8p),
        _p(st, _u8p), _p(it, _i32p))
    return {"u_hat": u, "status": st, "iters": it}


def ml_decode(llr_row, code: Code):
    """Brute force over all 2^K information words (K <= 20)."""
    row = np.ascontiguousarray(llr_row, dtype=np.float64).reshape(code.N)
    u = np.zeros(code.N, np.uint8)
    d = lib().or_ml_decode(_p(row, _f64p), code.N, code.K, _p(code.info_idx, _i32p), _p(u, _u8p))
    return u, float(d)


def payload_of(u_hat, code: Code) -> np.ndarray:
    """Payload bits [B][P] (one byte per bit) read from decided u vectors [B][N]."""
    u_hat = np.asarray(u_hat).reshape(-1, code.N)
    return u_hat[:, code.info_idx[: code.P]]
