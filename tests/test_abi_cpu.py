"""The C-ABI library: builds, loads and exports every symbol of include/polar_gb300.h; host-only
entry points (construction, argument checks) behave as documented.  No GPU needed."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_1609_09358_gb300 import api, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "polar_gb300.h")


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?(?:int|size_t|char\s*\*|void)\s*\*?\s*(\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return api.load()


def test_every_declared_symbol_is_exported(lib):
    names = header_functions()
    assert len(names) >= 10, names
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(api.SIGNATURES), set(names) ^ set(api.SIGNATURES)


@pytest.mark.parametrize("N,K,design_db", [(8, 4, 0.0), (128, 64, 0.0), (256, 100, 1.0), (1024, 512, 0.0),
                                           (2048, 1024, 0.0), (2048, 1024, -2.0), (512, 384, 3.0), (64, 1, 0.0),
                                           (64, 64, 0.0), (4096, 2048, 0.0)])
def test_construct_matches_oracle(lib, N, K, design_db):
    rate = 0.5
    f_lib, info_lib = api.polar_construct(N, K, design_db, rate)
    f_or, info_or, _ = oracle.construct(N, K, design_db, rate)
    assert np.array_equal(f_lib, f_or)
    assert np.array_equal(info_lib, info_or)


def test_argument_errors_without_gpu(lib):
    assert lib.polar_construct(100, 10, 0.0, 0.5, None, None) == -1
    assert "power of two" in lib.polar_last_error().decode()
    frozen = np.ones(100, np.uint8)
    bad = api.PolarCode(100, 0, 0, frozen)
    rc = lib.bp_decode(bad.ref(), None, 4, 10, 20.0, 0, None, 0, None, None, None, None, None, None, 0, None)
    assert rc == -1 and "N = 100" in lib.polar_last_error().decode()
    good = api.PolarCode(128, 64, 8, oracle.make_code(128, 64, 8).frozen)
    rc = lib.bp_decode(good.ref(), None, 4, 0, 20.0, 0, None, 0, None, None, None, None, None, None, 0, None)
    assert rc == -1 and "max_iters" in lib.polar_last_error().decode()
    rc = lib.hybrid_decode(good.ref(), None, 4, 10, 20.0, 0, None, 0, 3, None, None, None, None, 0, None)
    assert rc == -1
    wrongk = api.PolarCode(128, 63, 8, good.frozen)
    rc = lib.scl_decode(wrongk.ref(), None, 4, 8, None, None, None, 0, None)
    assert rc == -1 and "information positions" in lib.polar_last_error().decode()
    assert lib.polar_workspace_bytes(bad.ref(), 10, 8, 2) == 0
    assert lib.polar_workspace_bytes(good.ref(), 10, 8, 0) == 0
    assert lib.polar_workspace_bytes(good.ref(), 10, 3, 1) == 0


def test_bp_variant_flags_are_checked(lib):
    """The exact g and the re-encoding stop are FP32, unweighted, single-code variants: other uses
    are rejected before anything reaches the device."""
    good = api.PolarCode(128, 64, 8, oracle.make_code(128, 64, 8).frozen)
    for flags in (api.POLAR_G_EXACT, api.POLAR_STOP_REENCODE, api.POLAR_G_EXACT | api.POLAR_STOP_REENCODE):
        rc = lib.bp_decode(good.ref(), None, 4, 10, 20.0, api.POLAR_FP16 | flags, None, 0, None, None, None, None,
                           None, None, 0, None)
        assert rc == -1 and "POLAR_FP32" in lib.polar_last_error().decode()
        w = ctypes.c_void_p(64)  # never dereferenced: the flag check comes first
        rc = lib.hybrid_decode(good.ref(), None, 4, 10, 20.0, flags, w, 20, 8, None, None, None, None, 0, None)
        assert rc == -1 and "learned weights" in lib.polar_last_error().decode()
        codes = (api._PolarCode * 1)(good._c)
        rc = lib.hybrid_decode_mixed(codes, 1, None, None, None, 4, 10, 20.0, flags, 8, None, 16, None, None, None,
                                     0, None)
        assert rc == -1 and "mixed" in lib.polar_last_error().decode()


def test_scheduled_arguments_without_gpu(lib):
    good = api.PolarCode(128, 64, 8, oracle.make_code(128, 64, 8).frozen)
    rc = lib.hybrid_decode_scheduled(good.ref(), None, 0, 10, 20.0, 0, None, 0, 8, 255, None, None, None, None, 0,
                                     None)
    assert rc == -1 and "chunk" in lib.polar_last_error().decode()
    assert lib.polar_workspace_bytes(good.ref(), 1000, 8, api.POLAR_OP_HYBRID_SCHED) >= \
        lib.polar_workspace_bytes(good.ref(), 1000, 8, api.POLAR_OP_HYBRID)
    assert lib.polar_workspace_bytes(good.ref(), 1000, 8, 5) == 0


def test_bit_packing_roundtrip():
    rng = np.random.default_rng(0)
    b = rng.integers(0, 2, (5, 61), dtype=np.uint8)
    assert np.array_equal(api.unpack_bits(api.pack_bits(b), 61), b)


@pytest.mark.parametrize("N,design_db,rate", [(64, 0.0, 0.5), (1024, 1.0, 0.484375), (2048, -1.0, 0.25)])
def test_reliability_matches_oracle_and_construction(lib, N, design_db, rate):
    """polar_reliability equals the oracle's Bhattacharyya recursion and orders the channels as
    polar_construct does (its K most reliable are the information set)."""
    lnz = api.polar_reliability(N, design_db, rate)
    lnz0 = -rate * 10 ** (design_db / 10)
    n = N.bit_length() - 1
    ref = np.array([oracle.bhattacharyya_lnz(n, i, lnz0) for i in range(N)])
    assert np.allclose(lnz, ref, rtol=1e-12, atol=1e-300)
    K = N // 2
    frozen, _ = api.polar_construct(N, K, design_db, rate)
    order = sorted(range(N), key=lambda i: (lnz[i], -i))
    assert set(order[:K]) == set(np.nonzero(frozen == 0)[0].tolist())


def test_decided_mask_and_its_validation(lib):
    code = api.make_code(256, 128, 16)
    m = api.decided_mask(code, 40)
    assert m.sum() == 40 and not (m & code.frozen).any()
    da = api.PolarCode(256, 128, 16, code.frozen, decided=m)
    assert lib.polar_workspace_bytes(da.ref(), 10, 8, 2) > 0
    bad = m.copy()
    bad[np.nonzero(code.frozen)[0][0]] = 1
    wrong = api.PolarCode(256, 128, 16, code.frozen, decided=bad)
    assert lib.polar_workspace_bytes(wrong.ref(), 10, 8, 2) == 0
    rc = lib.scl_decode(wrong.ref(), None, 4, 8, None, None, None, 0, None)
    assert rc == -1 and "scl_decided" in lib.polar_last_error().decode()


def test_measurement_entry_points_check_arguments_without_gpu(lib):
    """polar_pe_eval, polar_pipe_rate and polar_mixed_set_plan reject bad arguments before any
    device call; polar_mixed_set_plan accepts exactly the plans the mixed kernel has."""
    assert lib.polar_pe_eval(3, None, None, None, 4, None) == -1
    assert "op" in lib.polar_last_error().decode()
    assert lib.polar_pe_eval(api.POLAR_PE_EXACT, None, None, None, -1, None) == -1
    assert lib.polar_pe_eval(api.POLAR_PE_EXACT, None, None, None, 0, None) == 0
    assert lib.polar_pe_eval(api.POLAR_PE_MINSUM, None, None, None, 8, None) == -1
    out = ctypes.c_double(0.0)
    assert lib.polar_pipe_rate(99, 16, ctypes.c_void_p(64), 1024, ctypes.byref(out), None) == -1
    assert lib.polar_pipe_rate(0, 0, ctypes.c_void_p(64), 1024, ctypes.byref(out), None) == -1
    for log2n, npt, ok in ((7, 4, True), (7, 8, False), (8, 8, True), (8, 4, True), (9, 4, True), (10, 4, True),
                           (10, 8, True), (11, 8, True), (11, 4, False), (12, 8, False)):
        assert (lib.polar_mixed_set_plan(log2n, npt, api.POLAR_FP32) == 0) == ok, (log2n, npt)
    assert lib.polar_mixed_set_plan(10, 8, 5) == -1
    for log2n, npt in ((8, 8), (9, 8), (10, 8)):  # back to the default plans
        assert lib.polar_mixed_set_plan(log2n, npt, api.POLAR_FP32) == 0
