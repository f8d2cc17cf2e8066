"""hybrid_decode_noalloc: the hybrid decoder for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc -- a receive chain that must not allocate once it runs (an
allocation can synchronise the device and take unbounded time), or a plug-in whose host
application owns all device memory.  This entry point takes no workspace and uses a static device
array inside the library instead.  The test calls it through the C ABI twice in a row, on different
frames and batch sizes, and checks each call bit-exactly against hybrid_decode with a caller
workspace (the tolerance of every other FP32 parity test: exact).  It lives in its own file, named
to be collected last, and passes alone in a fresh process as well as after the other tests.
"""
import numpy as np
import pytest

from tests import frames as fr

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

from paper_1609_09358_gb300 import api, build  # noqa: E402


def _reference(code, llr_d, B, L):
    dec = api.Decoder(code, B, L)
    dec.hybrid(llr_d, 200, 20.0)
    return dec.bits, dec.status, dec.iters


def test_noalloc_matches_workspace_path_on_consecutive_calls():
    build.build()
    api.load()
    ocode = fr.oracle_code(1024, 512, 16)
    code = fr.api_code(ocode)
    L = 8
    for call, (B, seed) in enumerate([(3000, 11), (1777, 12)]):
        _, llr = fr.frames(ocode, 1.5, B, seed=seed)
        llr_d = torch.from_numpy(llr).cuda()
        bits = torch.full((B, code.row_bytes), 0xAB, dtype=torch.uint8, device="cuda")
        status = torch.zeros(B, dtype=torch.uint8, device="cuda")
        iters = torch.zeros(B, dtype=torch.int16, device="cuda")
        api.hybrid_decode_noalloc(code, llr_d, 200, 20.0, api.POLAR_FP32, None, L, bits, status, iters)
        rb, rs, ri = _reference(code, llr_d, B, L)
        torch.cuda.synchronize()
        assert int((status != api.FRAME_BP_OK).sum()) > 0, "no frame reached CA-SCL in call %d" % call
        assert torch.equal(status, rs), "status differs in call %d" % call
        assert torch.equal(iters, ri), "iterations differ in call %d" % call
        assert torch.equal(bits, rb), "decoded bits differ in call %d" % call


def test_noalloc_rejects_requests_beyond_its_static_limit():
    build.build()
    lib = api.load()
    big = fr.api_code(fr.oracle_code(2048, 1024, 24))
    x = torch.zeros((4, 2048), dtype=torch.float32, device="cuda")
    out = torch.zeros((4, 128), dtype=torch.uint8, device="cuda")
    st = torch.zeros(4, dtype=torch.uint8, device="cuda")
    it = torch.zeros(4, dtype=torch.int16, device="cuda")
    with pytest.raises(api.PolarError, match="static array"):
        api.hybrid_decode_noalloc(big, x, 10, 20.0, api.POLAR_FP32, None, 32, out, st, it)
    code = fr.api_code(fr.oracle_code(128, 64, 8))
    rc = lib.hybrid_decode_noalloc(code.ref(), x.data_ptr(), 65537, 10, 20.0, 0, None, 0, 4, out.data_ptr(),
                                   st.data_ptr(), it.data_ptr(), None)
    assert rc == -1 and "static limit" in lib.polar_last_error().decode()
