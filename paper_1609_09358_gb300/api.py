"""Thin ctypes binding of the C ABI in include/polar_gb300.h (same names, argument marshalling only).

Device buffers are torch CUDA tensors; every call is queued on the current torch stream.  All
decoding runs in the CUDA kernels of libpolar_gb300.so: if the library is missing, the first call
raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpolar_gb300.so")

POLAR_OK = 0
POLAR_FP32, POLAR_FP16 = 0, 1
POLAR_FIXED_ITERS = 0x100  # bp_decode: OR into precision to run exactly max_iters iterations
# BP variants of Sec. II-B (OR into precision; FP32 messages, no learned weights): the exact PE
# function instead of min-sum, and the re-encoding stop (HD(LLR(x)) = HD(LLR(u)) G) instead of the CRC
POLAR_G_EXACT = 0x200
POLAR_STOP_REENCODE = 0x400
# learned scales all within [-1, 1] (set by the binding for such PreparedScales): no clip of the
# scaled term, and the half2 frames of a register kept on the same iteration when max_iters <= T
POLAR_WMS_UNIT = 0x800
_MSG = 0xFF  # message-type part of precision
POLAR_OP_BP, POLAR_OP_SCL, POLAR_OP_HYBRID, POLAR_OP_HYBRID_HOST, POLAR_OP_HYBRID_SCHED = 0, 1, 2, 3, 4
POLAR_SCHED_BP_STREAMS = 3
FRAME_BP_OK, FRAME_SCL_OK, FRAME_SCL_CRC_FAIL, FRAME_BP_FAIL = 1, 2, 3, 4
CRC_POLYS = {0: 0x0, 8: 0x07, 16: 0x1021, 24: 0x864CFB}

_lib = None


class PolarError(RuntimeError):
    pass


class _PolarCode(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("K", ctypes.c_int32), ("crc_len", ctypes.c_int32),
                ("crc_poly", ctypes.c_uint32), ("frozen", ctypes.POINTER(ctypes.c_uint8)),
                ("scl_decided", ctypes.POINTER(ctypes.c_uint8))]


_vp, _i32, _u64, _f32, _f64, _sz = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint64, ctypes.c_float,
                                    ctypes.c_double, ctypes.c_size_t)
_CP = ctypes.POINTER(_PolarCode)

# name -> (restype, argtypes); every exported symbol of the header
SIGNATURES = {
    "polar_construct": (ctypes.c_int, [_i32, _i32, _f64, _f64, _vp, _vp]),
    "polar_reliability": (ctypes.c_int, [_i32, _f64, _f64, _vp]),
    "polar_encode": (ctypes.c_int, [_CP, _vp, _i32, _vp, _vp]),
    "polar_random_payload": (ctypes.c_int, [_i32, _i32, _u64, _u64, _vp, _vp]),
    "polar_awgn_llr": (ctypes.c_int, [_vp, _i32, _i32, _f32, _vp, _u64, _u64, _vp, _vp]),
    "wms_prepared_bytes": (_sz, [_CP, _i32, _i32]),
    "wms_prepare": (ctypes.c_int, [_CP, _vp, _i32, _i32, _vp, _sz, _vp]),
    "wms_workspace_bytes": (_sz, [_CP, _i32, _i32]),
    "wms_forward": (ctypes.c_int, [_CP, _vp, _i32, _i32, _f32, _vp, _i32, _vp, _vp, _sz, _vp]),
    "wms_backward": (ctypes.c_int, [_CP, _vp, _i32, _i32, _f32, _vp, _i32, _vp, _vp, _vp, _sz, _vp]),
    "bp_decode": (ctypes.c_int, [_CP, _vp, _i32, _i32, _f32, _i32, _vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _sz,
                                 _vp]),
    "scl_decode": (ctypes.c_int, [_CP, _vp, _i32, _i32, _vp, _vp, _vp, _sz, _vp]),
    "hybrid_decode": (ctypes.c_int, [_CP, _vp, _i32, _i32, _f32, _i32, _vp, _i32, _i32, _vp, _vp, _vp, _vp, _sz,
                                     _vp]),
    "hybrid_decode_host": (ctypes.c_int, [_CP, _vp, _i32, _i32, _f32, _i32, _vp, _i32, _i32, _vp, _vp, _vp, _vp,
                                          _sz, _vp]),
    "hybrid_decode_noalloc": (ctypes.c_int, [_CP, _vp, _i32, _i32, _f32, _i32, _vp, _i32, _i32, _vp, _vp, _vp,
                                             _vp]),
    "hybrid_decode_scheduled": (ctypes.c_int, [_CP, _vp, _i32, _i32, _f32, _i32, _vp, _i32, _i32, _i32, _vp, _vp,
                                               _vp, _vp, _sz, _vp]),
    "polar_mixed_workspace_bytes": (_sz, [_CP, _i32, _i32, _i32]),
    "hybrid_decode_mixed": (ctypes.c_int, [_CP, _i32, _vp, _vp, _vp, _i32, _i32, _f32, _i32, _i32, _vp, _i32, _vp, _vp,
                                           _vp, _sz, _vp]),
    "polar_mixed_autotune": (ctypes.c_int, [_CP, _i32, _vp, _vp, _vp, _i32, _i32, _f32, _i32, _vp, _i32, _vp, _vp,
                                            _vp, _sz, _vp, ctypes.POINTER(_i32), ctypes.POINTER(_f32),
                                            ctypes.POINTER(_f32)]),
    "polar_mixed_set_plan": (ctypes.c_int, [_i32, _i32, _i32]),
    "polar_profile_enable": (ctypes.c_int, [_i32]),
    "polar_profile_read": (ctypes.c_int, [ctypes.POINTER(_f64), ctypes.POINTER(_i32), ctypes.POINTER(_f64),
                                          ctypes.POINTER(_i32)]),
    "polar_workspace_bytes": (_sz, [_CP, _i32, _i32, _i32]),
    "polar_hybrid_fallback_count": (ctypes.c_int, [_vp, ctypes.POINTER(_i32), _vp]),
    "polar_last_error": (ctypes.c_char_p, []),
    "polar_pe_eval": (ctypes.c_int, [_i32, _vp, _vp, _vp, _i32, _vp]),
    "polar_pipe_rate_scratch_bytes": (_sz, []),
    "polar_pipe_rate": (ctypes.c_int, [_i32, _i32, _vp, _sz, ctypes.POINTER(_f64), _vp]),
}


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Open the library (built by paper_1609_09358_gb300.build); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise PolarError("libpolar_gb300.so not built (%s): run paper_1609_09358_gb300/build.py" % path)
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(rc: int, what: str) -> None:
    if rc != POLAR_OK:
        raise PolarError("%s failed (%d): %s" % (what, rc, load().polar_last_error().decode()))


def _ptr(t) -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise PolarError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise PolarError("expected a contiguous tensor")
    return t.data_ptr()


def _stream(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


@dataclass
class PolarCode:
    """Host description of a code; `frozen` is uint8 [N] (1 = frozen); `decided` is None or uint8
    [N], 1 on the information positions CA-SCL decides without branching (decision aiding)."""
    N: int
    K: int
    crc_len: int
    frozen: np.ndarray
    crc_poly: int = -1
    decided: np.ndarray = None
    _c: _PolarCode = field(default=None, repr=False)

    def __post_init__(self):
        if self.crc_poly < 0:
            self.crc_poly = CRC_POLYS[self.crc_len]
        self.frozen = np.ascontiguousarray(self.frozen, dtype=np.uint8)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        if self.decided is not None:
            self.decided = np.ascontiguousarray(self.decided, dtype=np.uint8)
        self._c = _PolarCode(self.N, self.K, self.crc_len, self.crc_poly, self.frozen.ctypes.data_as(u8p),
                             self.decided.ctypes.data_as(u8p) if self.decided is not None else None)

    @property
    def P(self) -> int:
        return self.K - self.crc_len

    @property
    def n(self) -> int:
        return self.N.bit_length() - 1

    @property
    def row_bytes(self) -> int:
        return (self.P + 7) // 8

    @property
    def info_idx(self) -> np.ndarray:
        return np.nonzero(self.frozen == 0)[0].astype(np.int32)

    def ref(self):
        return ctypes.byref(self._c)


def polar_construct(N: int, K: int, design_ebn0_db: float, design_rate: float):
    frozen = np.zeros(N, np.uint8)
    info = np.zeros(max(K, 1), np.int32)
    _check(load().polar_construct(N, K, design_ebn0_db, design_rate, frozen.ctypes.data, info.ctypes.data),
           "polar_construct")
    return frozen, info[:K]


def polar_reliability(N: int, design_ebn0_db: float, design_rate: float) -> np.ndarray:
    """ln Z of every bit-channel at the design point (smaller = more reliable)."""
    lnz = np.zeros(N, np.float64)
    _check(load().polar_reliability(N, design_ebn0_db, design_rate, lnz.ctypes.data), "polar_reliability")
    return lnz


def decided_mask(code: PolarCode, count: int, design_ebn0_db: float = 0.0, design_rate=None) -> np.ndarray:
    """uint8 [N]: the `count` most reliable information positions (smallest ln Z at the design
    point; ties: the larger index, as in the construction) -- CA-SCL decides them without
    branching."""
    if design_rate is None:
        design_rate = code.P / code.N
    lnz = polar_reliability(code.N, design_ebn0_db, design_rate)
    info = code.info_idx
    order = sorted(info.tolist(), key=lambda i: (lnz[i], -i))
    mask = np.zeros(code.N, np.uint8)
    mask[order[:count]] = 1
    return mask


def make_code(N: int, K: int, crc_len: int, design_ebn0_db: float = 0.0, design_rate=None) -> PolarCode:
    """Bhattacharyya construction at the design point (design rate defaults to the payload rate)."""
    if design_rate is None:
        design_rate = (K - crc_len) / N
    frozen, _ = polar_construct(N, K, design_ebn0_db, design_rate)
    return PolarCode(N, K, crc_len, frozen)


def polar_encode(code: PolarCode, payload, codeword, stream=None) -> None:
    B = payload.shape[0]
    _check(load().polar_encode(code.ref(), _ptr(payload), B, _ptr(codeword), _stream(stream)), "polar_encode")


def polar_random_payload(B: int, P: int, seed: int, frame0: int, payload, stream=None) -> None:
    _check(load().polar_random_payload(B, P, seed, frame0, _ptr(payload), _stream(stream)),
           "polar_random_payload")


def polar_awgn_llr(codeword, N: int, sigma: float, seed: int, frame0: int, llr, stream=None,
                   sigma_per_frame=None) -> None:
    B = codeword.shape[0]
    _check(load().polar_awgn_llr(_ptr(codeword), B, N, sigma, _ptr(sigma_per_frame), seed, frame0, _ptr(llr),
                                 _stream(stream)), "polar_awgn_llr")


def wms_workspace_bytes(code: PolarCode, B: int, T: int) -> int:
    return int(load().wms_workspace_bytes(code.ref(), B, T))


def _wms_all_iters(llr_u, B: int, T: int, N: int) -> int:
    """1 when llr_u (or its gradient) holds every iteration [T][B][N], 0 for the last [B][N]."""
    shape = tuple(llr_u.shape)
    if shape == (T, B, N):
        return 1
    if shape == (B, N):
        return 0
    raise PolarError("LLR(u) tensor of shape %s: expected [B][N] or [T][B][N]" % (shape,))


def wms_forward(code: PolarCode, llr, T: int, llr_max: float, w, llr_u, workspace, stream=None) -> None:
    """llr_u [B][N]: LLR(u) of the last iteration; [T][B][N]: of every iteration."""
    B = llr.shape[0]
    ws_b = workspace.numel() * workspace.element_size()
    all_iters = _wms_all_iters(llr_u, B, T, code.N)
    _check(load().wms_forward(code.ref(), _ptr(llr), B, T, llr_max, _ptr(w), all_iters, _ptr(llr_u), _ptr(workspace),
                              ws_b, _stream(stream)), "wms_forward")


def wms_backward(code: PolarCode, llr, T: int, llr_max: float, w, grad_llr_u, grad_w, workspace,
                 stream=None) -> None:
    B = llr.shape[0]
    ws_b = workspace.numel() * workspace.element_size()
    all_iters = _wms_all_iters(grad_llr_u, B, T, code.N)
    _check(load().wms_backward(code.ref(), _ptr(llr), B, T, llr_max, _ptr(w), all_iters, _ptr(grad_llr_u),
                               _ptr(grad_w), _ptr(workspace), ws_b, _stream(stream)), "wms_backward")


def polar_workspace_bytes(code: PolarCode, B: int, L: int, op: int) -> int:
    return int(load().polar_workspace_bytes(code.ref(), B, L, op))


def wms_prepared_bytes(code: PolarCode, wms_iters: int, precision: int) -> int:
    return int(load().wms_prepared_bytes(code.ref(), wms_iters, precision))


def wms_prepare(code: PolarCode, w, precision: int, prepared, stream=None) -> None:
    """w: CUDA float32 [T][2][n][N] -> `prepared` (CUDA uint8 tensor of wms_prepared_bytes)."""
    nb = prepared.numel() * prepared.element_size()
    _check(load().wms_prepare(code.ref(), _ptr(w), int(w.shape[0]), precision, _ptr(prepared), nb, _stream(stream)),
           "wms_prepare")


class PreparedScales:
    """Learned weights rewritten once into the decoder's layout and precision (wms_prepare);
    pass as `wms_scales` to the decoding calls of the same block length and precision.  `unit`:
    whether every scale lies in [-1, 1] (None: read from w once, here); decoding calls with such
    scales pass POLAR_WMS_UNIT."""

    def __init__(self, code: PolarCode, w, precision: int, stream=None, unit=None):
        import torch
        if tuple(w.shape[1:]) != (2, code.n, code.N) or w.dtype != torch.float32 or not w.is_cuda:
            raise PolarError("weights must be a CUDA float32 tensor [T][2][n][N]")
        self.N, self.iters, self.precision = code.N, int(w.shape[0]), precision
        self.unit = bool(w.abs().max().item() <= 1.0) if unit is None else bool(unit)
        self.buf = torch.empty(wms_prepared_bytes(code, self.iters, precision), dtype=torch.uint8, device=w.device)
        self._w = w.contiguous()  # read by the queued prepare kernel
        wms_prepare(code, self._w, precision, self.buf, stream)


def _scales(code: PolarCode, wms_scales, precision: int, stream):
    """(pointer, iterations, keep-alive, precision flags) of the wms_scales argument of a decoding
    call: None, a PreparedScales of this length and precision, or natural-layout weights prepared
    for this call; POLAR_WMS_UNIT is added for scales within [-1, 1]."""
    if wms_scales is None:
        return None, 0, None, precision
    msg = precision & _MSG
    if not isinstance(wms_scales, PreparedScales):
        wms_scales = PreparedScales(code, wms_scales, msg, stream)
        if stream is not None:
            wms_scales.buf.record_stream(stream)
    if wms_scales.N != code.N or wms_scales.precision != msg:
        raise PolarError("prepared weights are for N = %d, precision %d" % (wms_scales.N, wms_scales.precision))
    if wms_scales.unit:
        precision |= POLAR_WMS_UNIT
    return wms_scales.buf.data_ptr(), wms_scales.iters, wms_scales, precision


def bp_decode(code: PolarCode, llr, max_iters: int, llr_max: float, precision: int, wms_scales, bits, status,
              iters, llr_u=None, llr_x=None, workspace=None, stream=None) -> None:
    """wms_scales: None, PreparedScales, or CUDA float32 weights [T][2][n][N] (prepared per call)."""
    B = llr.shape[0]
    wms_scales, w_iters, _keep, precision = _scales(code, wms_scales, precision, stream)
    ws_b = 0 if workspace is None else workspace.numel() * workspace.element_size()
    _check(load().bp_decode(code.ref(), _ptr(llr), B, max_iters, llr_max, precision, wms_scales, w_iters,
                            _ptr(bits), _ptr(status), _ptr(iters), _ptr(llr_u), _ptr(llr_x), _ptr(workspace), ws_b,
                            _stream(stream)), "bp_decode")


def scl_decode(code: PolarCode, llr, L: int, bits, status, workspace, stream=None) -> None:
    B = llr.shape[0]
    ws_b = workspace.numel() * workspace.element_size()
    _check(load().scl_decode(code.ref(), _ptr(llr), B, L, _ptr(bits), _ptr(status), _ptr(workspace), ws_b,
                             _stream(stream)), "scl_decode")


def hybrid_decode(code: PolarCode, llr, max_iters: int, llr_max: float, precision: int, wms_scales, L: int, bits,
                  status, iters, workspace, stream=None) -> None:
    B = llr.shape[0]
    wms_scales, w_iters, _keep, precision = _scales(code, wms_scales, precision, stream)
    ws_b = workspace.numel() * workspace.element_size()
    _check(load().hybrid_decode(code.ref(), _ptr(llr), B, max_iters, llr_max, precision, wms_scales, w_iters,
                                L, _ptr(bits), _ptr(status), _ptr(iters), _ptr(workspace), ws_b, _stream(stream)),
           "hybrid_decode")


def hybrid_decode_host(code: PolarCode, llr_host, max_iters: int, llr_max: float, precision: int, wms_scales, L: int,
                       bits_host, status_host, iters_host, workspace, stream=None) -> None:
    """Host-buffer hybrid decode: llr_host and the outputs are CPU tensors (pin them to overlap)."""
    B = llr_host.shape[0]
    for t in (llr_host, bits_host, status_host, iters_host):
        if t.is_cuda or not t.is_contiguous():
            raise PolarError("hybrid_decode_host expects contiguous host tensors")
    wms_scales, w_iters, _keep, precision = _scales(code, wms_scales, precision, stream)
    ws_b = workspace.numel() * workspace.element_size()
    _check(load().hybrid_decode_host(code.ref(), llr_host.data_ptr(), B, max_iters, llr_max, precision,
                                     wms_scales, w_iters, L, bits_host.data_ptr(), status_host.data_ptr(),
                                     iters_host.data_ptr(), _ptr(workspace), ws_b, _stream(stream)),
           "hybrid_decode_host")


def hybrid_decode_scheduled(code: PolarCode, llr, max_iters: int, llr_max: float, precision: int, wms_scales, L: int,
                            chunk: int, bits, status, iters, workspace, stream=None) -> None:
    """The host-scheduled hybrid of Fig. 3 (chunked BP launches polled by the host, CA-SCL started
    on the chunks' failures when idle); device tensors as hybrid_decode, workspace of
    POLAR_OP_HYBRID_SCHED size.  Blocks the calling thread until every BP launch has finished."""
    B = llr.shape[0]
    wms_scales, w_iters, _keep, precision = _scales(code, wms_scales, precision, stream)
    ws_b = workspace.numel() * workspace.element_size()
    _check(load().hybrid_decode_scheduled(code.ref(), _ptr(llr), B, max_iters, llr_max, precision, wms_scales,
                                          w_iters, L, chunk, _ptr(bits), _ptr(status), _ptr(iters), _ptr(workspace),
                                          ws_b, _stream(stream)),
           "hybrid_decode_scheduled")


def hybrid_decode_noalloc(code: PolarCode, llr, max_iters: int, llr_max: float, precision: int, wms_scales,
                          L: int, bits, status, iters, stream=None) -> None:
    """hybrid_decode for callers that cannot allocate device memory: no workspace argument; the
    library's static scratch array is used instead (B <= 65536 frames, CA-SCL list in shared
    memory).  Calls that overlap on the GPU race on that array."""
    B = llr.shape[0]
    wms_scales, w_iters, _keep, precision = _scales(code, wms_scales, precision, stream)
    _check(load().hybrid_decode_noalloc(code.ref(), _ptr(llr), B, max_iters, llr_max, precision, wms_scales,
                                        w_iters, L, _ptr(bits), _ptr(status), _ptr(iters), _stream(stream)),
           "hybrid_decode_noalloc")


POLAR_PE_MINSUM, POLAR_PE_EXACT, POLAR_PE_EXACT_PACKED = 0, 1, 2


def polar_pe_eval(op: int, a, b, out, stream=None) -> None:
    """out = g(a, b) elementwise with the BP kernels' PE function (CUDA float32 tensors, unclipped)."""
    n = a.numel()
    if b.numel() != n or out.numel() != n:
        raise PolarError("polar_pe_eval: a, b and out must have the same size")
    _check(load().polar_pe_eval(op, _ptr(a), _ptr(b), _ptr(out), n, _stream(stream)), "polar_pe_eval")


# issue-rate microbenchmark ops (polar_pipe_rate)
PIPE_RATE_OPS = {"min.xorsign.abs.f32": 0, "min.xorsign.abs.f16x2": 1, "add.rn.f32": 2, "add.rn.f16x2": 3,
                 "mul.rn.f16x2": 4, "min.f32": 5, "ex2.approx.ftz.f32": 6, "lg2.approx.ftz.f32": 7, "prmt.b32": 8}


def polar_pipe_rate(op: int, iters: int, scratch, stream=None) -> float:
    """Results of one lane per SM per SM clock of instruction `op` (a PIPE_RATE_OPS value);
    scratch: a CUDA byte tensor of polar_pipe_rate_scratch_bytes() bytes.  Synchronises the stream."""
    out = _f64(0.0)
    _check(load().polar_pipe_rate(op, iters, _ptr(scratch), scratch.numel() * scratch.element_size(),
                                  ctypes.byref(out), _stream(stream)), "polar_pipe_rate")
    return float(out.value)


def polar_pipe_rate_scratch_bytes() -> int:
    return int(load().polar_pipe_rate_scratch_bytes())


def polar_profile_enable(on: bool) -> None:
    _check(load().polar_profile_enable(1 if on else 0), "polar_profile_enable")


def polar_profile_read():
    """(bp_ms, bp_launches, scl_ms, scl_launches) accumulated since the last read."""
    a, b, c, d = _f64(0), _i32(0), _f64(0), _i32(0)
    _check(load().polar_profile_read(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)),
           "polar_profile_read")
    return a.value, b.value, c.value, d.value


def polar_hybrid_fallback_count(workspace, stream=None) -> int:
    out = _i32(0)
    _check(load().polar_hybrid_fallback_count(_ptr(workspace), ctypes.byref(out), _stream(stream)),
           "polar_hybrid_fallback_count")
    return int(out.value)


# ------------------------------------------------------------------------ convenience wrappers
class Decoder:
    """Owns the output and workspace tensors for one code and batch size (device memory via torch)."""

    def __init__(self, code: PolarCode, B: int, L: int = 8, device="cuda"):
        import torch
        self.code, self.B, self.L = code, B, L
        self.bits = torch.zeros((B, code.row_bytes), dtype=torch.uint8, device=device)
        self.status = torch.zeros(B, dtype=torch.uint8, device=device)
        self.iters = torch.zeros(B, dtype=torch.int16, device=device)
        ws = max(polar_workspace_bytes(code, B, L, op) for op in (POLAR_OP_HYBRID, POLAR_OP_SCL, POLAR_OP_HYBRID_SCHED))
        self.workspace = torch.zeros(max(ws, 256), dtype=torch.uint8, device=device)

    def hybrid(self, llr, max_iters: int, llr_max: float = 20.0, precision: int = POLAR_FP32, wms_scales=None,
               stream=None):
        hybrid_decode(self.code, llr, max_iters, llr_max, precision, wms_scales, self.L, self.bits, self.status,
                      self.iters, self.workspace, stream)
        return self.bits, self.status, self.iters

    def scheduled(self, llr, max_iters: int, llr_max: float = 20.0, precision: int = POLAR_FP32, wms_scales=None,
                  chunk: int = 16384, stream=None):
        hybrid_decode_scheduled(self.code, llr, max_iters, llr_max, precision, wms_scales, self.L, chunk, self.bits,
                                self.status, self.iters, self.workspace, stream)
        return self.bits, self.status, self.iters

    def bp(self, llr, max_iters: int, llr_max: float = 20.0, precision: int = POLAR_FP32, wms_scales=None,
           llr_u=None, llr_x=None, stream=None):
        bp_decode(self.code, llr, max_iters, llr_max, precision, wms_scales, self.bits, self.status, self.iters,
                  llr_u, llr_x, None, stream)
        return self.bits, self.status, self.iters

    def scl(self, llr, stream=None):
        scl_decode(self.code, llr, self.L, self.bits, self.status, self.workspace, stream)
        return self.bits, self.status


def unpack_bits(packed: np.ndarray, nbits: int) -> np.ndarray:
    """[B][ceil(nbits/8)] little-endian packed bytes -> uint8 [B][nbits], one byte per bit."""
    packed = np.asarray(packed, dtype=np.uint8).reshape(packed.shape[0], -1)
    return np.unpackbits(packed, axis=1, bitorder="little")[:, :nbits]


def pack_bits(bits: np.ndarray) -> np.ndarray:
    """uint8 [B][nbits] (one byte per bit) -> [B][ceil(nbits/8)] little-endian packed bytes."""
    bits = np.asarray(bits, dtype=np.uint8)
    return np.packbits(bits, axis=1, bitorder="little")


# ------------------------------------------------------------------------ mixed batches
def _code_array(codes):
    arr = (_PolarCode * len(codes))(*[c._c for c in codes])
    return arr


def polar_mixed_workspace_bytes(codes, B: int, L: int) -> int:
    arr = _code_array(codes)
    return int(load().polar_mixed_workspace_bytes(arr, len(codes), B, L))


def hybrid_decode_mixed(codes, code_of, llr_off, llr, max_iters: int, llr_max: float, precision: int, L: int, bits,
                        status, iters, workspace, stream=None) -> None:
    """One batch of frames of several codes; code_of int32 [B], llr_off int64 [B] (CUDA tensors)."""
    arr = _code_array(codes)
    B = code_of.shape[0]
    ws_b = workspace.numel() * workspace.element_size()
    _check(load().hybrid_decode_mixed(arr, len(codes), _ptr(code_of), _ptr(llr_off), _ptr(llr), B, max_iters,
                                      llr_max, precision, L, _ptr(bits), bits.shape[1], _ptr(status), _ptr(iters),
                                      _ptr(workspace), ws_b, _stream(stream)), "hybrid_decode_mixed")


def polar_mixed_autotune(codes, code_of, llr_off, llr, max_iters: int, llr_max: float, precision: int, bits, status,
                         iters, workspace, stream=None) -> dict:
    """{"nodes_per_thread": {N: nodes per thread chosen}, "bp_ms": BP time with the chosen plans,
    "bp_ms_default_plans": with the default plans}."""
    arr = _code_array(codes)
    B = code_of.shape[0]
    ws_b = workspace.numel() * workspace.element_size()
    chosen, best, base = (_i32 * 13)(), _f32(0), _f32(0)
    _check(load().polar_mixed_autotune(arr, len(codes), _ptr(code_of), _ptr(llr_off), _ptr(llr), B, max_iters,
                                       llr_max, precision, _ptr(bits), bits.shape[1], _ptr(status), _ptr(iters),
                                       _ptr(workspace), ws_b, _stream(stream), chosen, ctypes.byref(best),
                                       ctypes.byref(base)), "polar_mixed_autotune")
    plans = {1 << n: int(chosen[n]) for n in range(13) if chosen[n]}
    return {"nodes_per_thread": plans, "bp_ms": float(best.value), "bp_ms_default_plans": float(base.value)}


def polar_mixed_set_plan(N: int, nodes_per_thread: int, precision: int) -> None:
    _check(load().polar_mixed_set_plan(int(N).bit_length() - 1, nodes_per_thread, precision), "polar_mixed_set_plan")


class MixedDecoder:
    """Buffers and workspace for mixed batches of a fixed code set and batch size; `capture()`
    records one decode into a CUDA graph that `replay()` relaunches."""

    def __init__(self, codes, B: int, L: int = 8, device="cuda"):
        import torch
        self.codes, self.B, self.L = list(codes), B, L
        self.row = max(c.row_bytes for c in self.codes)
        self.bits = torch.zeros((B, self.row), dtype=torch.uint8, device=device)
        self.status = torch.zeros(B, dtype=torch.uint8, device=device)
        self.iters = torch.zeros(B, dtype=torch.int16, device=device)
        self.workspace = torch.zeros(polar_mixed_workspace_bytes(self.codes, B, L), dtype=torch.uint8, device=device)
        self.graph = None

    def decode(self, code_of, llr_off, llr, max_iters: int, llr_max: float = 20.0, precision: int = POLAR_FP32,
               stream=None):
        hybrid_decode_mixed(self.codes, code_of, llr_off, llr, max_iters, llr_max, precision, self.L, self.bits,
                            self.status, self.iters, self.workspace, stream)
        return self.bits, self.status, self.iters

    def autotune(self, code_of, llr_off, llr, max_iters: int, llr_max: float = 20.0, precision: int = POLAR_FP32):
        return polar_mixed_autotune(self.codes, code_of, llr_off, llr, max_iters, llr_max, precision, self.bits,
                                    self.status, self.iters, self.workspace)

    def capture(self, code_of, llr_off, llr, max_iters: int, llr_max: float = 20.0, precision: int = POLAR_FP32):
        import torch
        self.decode(code_of, llr_off, llr, max_iters, llr_max, precision)  # uploads code tables first
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                self.decode(code_of, llr_off, llr, max_iters, llr_max, precision, stream=s)
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()
        return self.bits, self.status, self.iters
