"""Mixed batches: frames of 15 codes (N = 128..2048, R = 1/4, 1/2, 3/4, CRC-16) in one call --
one persistent BP launch and one CA-SCL launch -- checked frame by frame against the oracle's
hybrid decoder with each frame's own code; FP16 against the binary16 BP emulation followed by the
FP32 CA-SCL.  Also: the autotuned plans and a CUDA-graph replay give the same results."""
import numpy as np
import pytest

import oracle
from tests import frames as fr

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

from paper_1609_09358_gb300 import api, build  # noqa: E402

NS = [128, 256, 512, 1024, 2048]
RS = [0.25, 0.5, 0.75]


def mixed_batch(B, ebn0, seed):
    ocodes = [fr.oracle_code(N, int(R * N), 16) for N in NS for R in RS]
    rng = np.random.default_rng(seed)
    code_of = rng.integers(0, len(ocodes), B).astype(np.int32)
    off = np.zeros(B, np.int64)
    sizes = np.array([ocodes[c].N for c in code_of], np.int64)
    off[1:] = np.cumsum(sizes)[:-1]
    llr = np.zeros(int(sizes.sum()), np.float32)
    for c, oc in enumerate(ocodes):
        idx = np.nonzero(code_of == c)[0]
        if len(idx):
            _, l = fr.frames(oc, ebn0, len(idx), seed=seed + 101 * c)
            for k, b in enumerate(idx):
                llr[off[b]:off[b] + oc.N] = l[k]
    return ocodes, code_of, off, llr


def reference(ocodes, code_of, off, llr, imax, L, precision):
    B = len(code_of)
    bits, status, iters = {}, np.zeros(B, np.uint8), np.zeros(B, np.int32)
    for c, oc in enumerate(ocodes):
        idx = np.nonzero(code_of == c)[0]
        if not len(idx):
            continue
        rows = np.stack([llr[off[b]:off[b] + oc.N] for b in idx])
        if precision == "f32":
            ref = oracle.hybrid_decode(rows, oc, imax, 20.0, L, precision="f32")
            u, st, it = ref["u_hat"], ref["status"], ref["iters"]
        else:
            bp = oracle.bp_decode(rows, oc, imax, 32.0, "f16", want_llr=False)
            u, st, it = bp["u_hat"].copy(), bp["status"].copy(), bp["iters"]
            failed = st != oracle.BP_OK
            if failed.any():
                scl = oracle.scl_decode(rows[failed], oc, L, "f32")
                u[failed], st[failed] = scl["u_hat"], scl["status"]
        for k, b in enumerate(idx):
            bits[b] = oracle.payload_of(u[k:k + 1], oc)[0]
        status[idx], iters[idx] = st, it
    return bits, status, iters


def check(ocodes, code_of, dbits, dstat, diter, ref):
    rbits, rstat, riter = ref
    assert np.array_equal(dstat, rstat)
    assert np.array_equal(diter, riter)
    for b in range(len(code_of)):
        P = ocodes[code_of[b]].P
        assert np.array_equal(api.unpack_bits(dbits[b:b + 1], P)[0], rbits[b]), b


@pytest.mark.parametrize("precision", ["f32", "f16"])
def test_mixed_batch_matches_oracle_per_frame(precision):
    build.build()
    ocodes, code_of, off, llr = mixed_batch(1500, 2.0, 77)
    codes = [fr.api_code(oc) for oc in ocodes]
    dec = api.MixedDecoder(codes, len(code_of), L=8)
    prec = api.POLAR_FP32 if precision == "f32" else api.POLAR_FP16
    M = 20.0 if precision == "f32" else 32.0
    args = (torch.from_numpy(code_of).cuda(), torch.from_numpy(off).cuda(), torch.from_numpy(llr).cuda())
    dec.decode(*args, 40, M, prec)
    torch.cuda.synchronize()
    ref = reference(ocodes, code_of, off, llr, 40, 8, precision)
    assert int(np.sum(ref[1] != oracle.BP_OK)) > 20
    check(ocodes, code_of, dec.bits.cpu().numpy(), dec.status.cpu().numpy(),
          dec.iters.cpu().numpy().astype(np.int32), ref)
    # the autotuner may switch the plans of N = 256 / 512 / 1024; results must not change
    tuned = dec.autotune(*args, 40, M, prec)
    assert set(tuned["nodes_per_thread"]) == {oc.N for oc in ocodes}
    assert tuned["bp_ms"] <= tuned["bp_ms_default_plans"]
    dec.decode(*args, 40, M, prec)
    torch.cuda.synchronize()
    check(ocodes, code_of, dec.bits.cpu().numpy(), dec.status.cpu().numpy(),
          dec.iters.cpu().numpy().astype(np.int32), ref)
    # every plan of every length, set by hand: the same results
    for plans in ({256: 4, 512: 4, 1024: 4}, {256: 8, 512: 8, 1024: 8}):
        for N, npt in plans.items():
            api.polar_mixed_set_plan(N, npt, prec)
        dec.decode(*args, 40, M, prec)
        torch.cuda.synchronize()
        check(ocodes, code_of, dec.bits.cpu().numpy(), dec.status.cpu().numpy(),
              dec.iters.cpu().numpy().astype(np.int32), ref)
    with pytest.raises(api.PolarError):
        api.polar_mixed_set_plan(2048, 4, prec)


def test_mixed_batch_cuda_graph_replay():
    build.build()
    ocodes, code_of, off, llr = mixed_batch(600, 2.0, 5)
    codes = [fr.api_code(oc) for oc in ocodes]
    dec = api.MixedDecoder(codes, len(code_of), L=8)
    args = (torch.from_numpy(code_of).cuda(), torch.from_numpy(off).cuda(), torch.from_numpy(llr).cuda())
    dec.capture(*args, 40, 20.0, api.POLAR_FP32)
    dec.bits.zero_()
    dec.status.zero_()
    dec.replay()
    torch.cuda.synchronize()
    ref = reference(ocodes, code_of, off, llr, 40, 8, "f32")
    check(ocodes, code_of, dec.bits.cpu().numpy(), dec.status.cpu().numpy(),
          dec.iters.cpu().numpy().astype(np.int32), ref)


def test_mixed_full_size_sampled():
    """The mixed workload at its full size and in the launch configuration the benchmark times
    (2^16 frames of the 15 codes at 2.0 dB, i_max = 200, L = 8, half2 BP, autotuned plans, CUDA
    graph replay): a random sample of frames and the first CA-SCL frames of every code are
    decoded one by one by the oracle and compared."""
    build.build()
    B = 1 << 16
    ocodes, code_of, off, llr = mixed_batch(B, 2.0, 2024)
    codes = [fr.api_code(oc) for oc in ocodes]
    dec = api.MixedDecoder(codes, B, L=8)
    args = (torch.from_numpy(code_of).cuda(), torch.from_numpy(off).cuda(), torch.from_numpy(llr).cuda())
    dec.autotune(*args, 200, 32.0, api.POLAR_FP16)
    dec.capture(*args, 200, 32.0, api.POLAR_FP16)
    dec.replay()
    torch.cuda.synchronize()
    dstat = dec.status.cpu().numpy()
    rng = np.random.default_rng(3)
    fb = np.nonzero(dstat != oracle.BP_OK)[0]
    pick = [rng.choice(B, 120, replace=False)]
    for c in range(len(ocodes)):
        pick.append(fb[code_of[fb] == c][:3])
    sample = np.unique(np.concatenate(pick))
    sub_off = np.zeros(len(sample), np.int64)
    sizes = np.array([ocodes[c].N for c in code_of[sample]], np.int64)
    sub_off[1:] = np.cumsum(sizes)[:-1]
    sub_llr = np.concatenate([llr[off[b]:off[b] + ocodes[code_of[b]].N] for b in sample])
    ref = reference(ocodes, code_of[sample], sub_off, sub_llr, 200, 8, "f16")
    check(ocodes, code_of[sample], dec.bits.cpu().numpy()[sample], dstat[sample],
          dec.iters.cpu().numpy().astype(np.int32)[sample], ref)
    assert len(fb) > 1000 and set(np.unique(dstat)) <= {1, 2, 3}
