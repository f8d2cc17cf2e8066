"""Pins of the CPU oracle against facts the paper and the mathematics fix (no GPU needed).

Each test pins one oracle function against something other than the oracle itself: the Fig. 1
worked example, catalogue CRC check values, closed forms, exhaustive enumeration, brute-force ML,
or an exact invariant of the method.  A plausible slip (a dropped term, a swapped index, a wrong
wiring direction) breaks at least one of them.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from paper_1609_09358_gb300 import inputs


def _read_golden(golden_dir, name):
    rows = []
    with open(os.path.join(golden_dir, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line)
    return rows


# ------------------------------------------------------------------------------------ encoder
def test_fig1_encoder_wiring(golden_dir):
    """Fig. 1: each output x_j of the N = 8 encoder graph XORs the listed u indices."""
    rows = _read_golden(golden_dir, "fig1_encoder_n8.txt")
    wiring = {}
    for r in rows:
        key, vals = r.split(":")
        if key.startswith("x"):
            wiring[int(key[1:])] = set(int(v) for v in vals.split())
    assert len(wiring) == 8
    for i in range(8):
        e = np.zeros(8, np.uint8)
        e[i] = 1
        for fn in (oracle.polar_transform, oracle.encode_circuit):
            x = fn(e)
            for j in range(8):
                assert x[j] == (i in wiring[j]), (fn.__name__, i, j)


def test_generator_is_kronecker_power():
    """G = F^{(x)n} with F = [[1,0],[1,1]] (Sec. II), built independently with np.kron."""
    F = np.array([[1, 0], [1, 1]], dtype=np.int64)
    G = np.array([[1]], dtype=np.int64)
    for n in range(1, 7):
        G = np.kron(G, F)
        N = 1 << n
        ours = np.array([[oracle.generator_entry(i, j) for j in range(N)] for i in range(N)])
        assert np.array_equal(ours, G), n


def test_generator_is_involution():
    """G G = I over GF(2): encoding twice returns u."""
    rng = np.random.default_rng(7)
    for n in range(1, 12):
        N = 1 << n
        for _ in range(3):
            u = rng.integers(0, 2, N, dtype=np.uint8)
            assert np.array_equal(oracle.encode_circuit(oracle.encode_circuit(u)), u)
    for n in range(1, 7):
        N = 1 << n
        G = np.array([[oracle.generator_entry(i, j) for j in range(N)] for i in range(N)])
        assert np.array_equal((G @ G) % 2, np.eye(N, dtype=G.dtype))


@pytest.mark.parametrize("N", [4, 64, 512, 2048])
def test_matrix_definition_matches_fig1_circuit(N):
    rng = np.random.default_rng(N)
    for _ in range(2):
        u = rng.integers(0, 2, N, dtype=np.uint8)
        assert np.array_equal(oracle.polar_transform(u), oracle.encode_circuit(u))


# ------------------------------------------------------------------------------ construction
@pytest.mark.parametrize("design_db", [0.0, -3.0, 2.0])
def test_fig1_frozen_set(golden_dir, design_db):
    """Fig. 1 marks u0, u1, u2, u4 frozen for N = 8, k = 4."""
    rows = _read_golden(golden_dir, "fig1_encoder_n8.txt")
    frozen_ref = [int(v) for r in rows if r.startswith("frozen:") for v in r.split(":")[1].split()]
    info_ref = [int(v) for r in rows if r.startswith("info:") for v in r.split(":")[1].split()]
    frozen, info, _ = oracle.construct(8, 4, design_db, 0.5)
    assert list(np.nonzero(frozen)[0]) == frozen_ref
    assert list(info) == info_ref


@pytest.mark.parametrize("eps", [0.3, 0.5])
def test_bhattacharyya_is_exact_on_bec(eps):
    """On a BEC(eps) the recursion Z -> (2Z - Z^2, Z^2) is exact: Z_i equals the erasure
    probability of bit i under genie-aided SC.  Enumerate all 2^8 erasure patterns of the
    all-zero codeword and run the oracle's SC recursion (min-sum f and g are exact on the BEC).
    This pins the index order of the construction (MSB = channel-side split) and the SC
    recursion's pairing and partial sums together."""
    n, N = 3, 8
    p_erase = np.zeros(N)
    for pattern in itertools.product([0, 1], repeat=N):
        llr = np.array([0.0 if e else 1.0 for e in pattern], dtype=np.float32)
        weight = eps ** sum(pattern) * (1 - eps) ** (N - sum(pattern))
        u = np.zeros(N, np.uint8)
        for i in range(N):
            if oracle.sc_bit_llr(llr, u, i) == 0.0:
                p_erase[i] += weight
    z = np.array([math.exp(oracle.bhattacharyya_lnz(n, i, math.log(eps))) for i in range(N)])
    assert np.allclose(z, p_erase, rtol=0, atol=1e-12), (z, p_erase)
    # the recursion order matters: the bit-reversed assignment does not fit
    rev = [int(format(i, "03b")[::-1], 2) for i in range(N)]
    assert not np.allclose(z[rev], p_erase, atol=1e-6)


def test_bhattacharyya_closed_form_and_partial_order():
    n = 10
    lnz0 = -0.5
    # all-ones index: n squarings, Z0^(2^n)
    assert oracle.bhattacharyya_lnz(n, (1 << n) - 1, lnz0) == pytest.approx(lnz0 * 2 ** n, rel=1e-15)
    lnz = np.array([oracle.bhattacharyya_lnz(n, i, lnz0) for i in range(1 << n)])
    # binary domination: setting a 0 bit of the index to 1 can only lower Z
    for i in range(1 << n):
        for b in range(n):
            if not (i >> b) & 1:
                assert lnz[i | (1 << b)] <= lnz[i] + 1e-13 * abs(lnz[i])
    assert np.all(lnz <= 0)


# ------------------------------------------------------------------------------------------ CRC
def _ascii_bits(s):
    return np.array([(ord(ch) >> (7 - k)) & 1 for ch in s for k in range(8)], np.uint8)


def test_crc_catalogue_check_values(golden_dir):
    rows = _read_golden(golden_dir, "crc_check_values.txt")
    assert len(rows) == 3
    msg = _ascii_bits("123456789")
    for r in rows:
        name, width, poly, check = r.split()
        width, poly, check = int(width), int(poly, 16), int(check, 16)
        rem = oracle.crc(msg, poly, width)
        val = int("".join(str(int(b)) for b in rem), 2)
        assert val == check, name
        assert oracle.CRC_POLYS[width] == poly


@pytest.mark.parametrize("c", [8, 16, 24])
def test_crc_linear_and_detects_single_errors(c):
    poly = oracle.CRC_POLYS[c]
    rng = np.random.default_rng(c)
    for _ in range(5):
        a = rng.integers(0, 2, 100, dtype=np.uint8)
        b = rng.integers(0, 2, 100, dtype=np.uint8)
        assert np.array_equal(oracle.crc(a ^ b, poly, c), oracle.crc(a, poly, c) ^ oracle.crc(b, poly, c))
        cw = np.concatenate([a, oracle.crc(a, poly, c)])
        assert oracle.crc_check(cw, poly, c)
        for k in rng.choice(len(cw), 10, replace=False):
            bad = cw.copy()
            bad[k] ^= 1
            assert not oracle.crc_check(bad, poly, c)


# ------------------------------------------------------------------------------- SC / SCL / ML
def _noisy_frames(code, ebn0_db, B, seed):
    pay = inputs.payload_bits(seed, 0, B, code.P)
    x = oracle.encode_batch(pay, code)
    noise = inputs.unit_noise(seed, 0, B, code.N)
    sigma = oracle.sigma_for(ebn0_db, code.P / code.N)
    return pay, x, oracle.channel_llr(x, noise, sigma)


def test_scl_with_list_one_is_sc():
    code = oracle.make_code(64, 32, 8)
    _, _, llr = _noisy_frames(code, 1.0, 40, 11)
    sc = oracle.sc_decode(llr, code)
    scl = oracle.scl_decode(llr, code, 1)
    assert np.array_equal(sc, scl["u_hat"])


@pytest.mark.parametrize("N,K", [(8, 4), (16, 5)])
def test_full_list_scl_is_ml(N, K):
    """With L >= 2^K the final list holds every codeword; with min-sum f the path metric of each
    equals its correlation discrepancy sum |llr_j| [x_j != HD(llr_j)], so the chosen path is
    the brute-force ML codeword."""
    frozen, info, _ = oracle.construct(N, K, 0.0, K / N)
    code = oracle.Code(N, K, 0, 0, frozen, info)
    rng = np.random.default_rng(N)
    L = 1 << K
    for _ in range(60):
        llr = rng.normal(1.0, 1.5, N).astype(np.float32)
        lst, pms, u, ok = oracle.scl_list(llr, code, L, "f64")
        assert ok and len(lst) == L
        seen = set()
        for up, pm in zip(lst, pms):
            x = oracle.polar_transform(up)
            d = float(np.sum(np.abs(llr.astype(np.float64)) * (x != (llr < 0))))
            assert pm == pytest.approx(d, abs=1e-9)
            seen.add(tuple(up[info]))
        assert len(seen) == L
        u_ml, d_ml = oracle.ml_decode(llr.astype(np.float64), code)
        x = oracle.polar_transform(u)
        d = float(np.sum(np.abs(llr.astype(np.float64)) * (x != (llr < 0))))
        assert d == pytest.approx(d_ml, abs=1e-9)


def test_noiseless_frames_decode_exactly():
    code = oracle.make_code(128, 64, 8)
    pay = inputs.payload_bits(3, 0, 16, code.P)
    x = oracle.encode_batch(pay, code)
    llr = (8.0 * (1.0 - 2.0 * x)).astype(np.float32)
    u_true = np.stack([oracle.build_u(p, code) for p in pay])
    assert np.array_equal(oracle.sc_decode(llr, code), u_true)
    scl = oracle.scl_decode(llr, code, 4)
    assert np.array_equal(scl["u_hat"], u_true) and np.all(scl["status"] == oracle.SCL_OK)
    bp = oracle.bp_decode(llr, code, 50, 20.0)
    assert np.array_equal(bp["u_hat"], u_true)
    assert np.all(bp["status"] == oracle.BP_OK) and np.all(bp["iters"] == 1)
    hy = oracle.hybrid_decode(llr, code, 50, 20.0, 4)
    assert np.array_equal(hy["u_hat"], u_true) and np.all(hy["status"] == oracle.BP_OK)


def test_scl_larger_list_not_worse():
    code = oracle.make_code(64, 32, 8)
    pay, _, llr = _noisy_frames(code, 1.0, 300, 5)
    errs = []
    for L in (1, 4, 16):
        u = oracle.scl_decode(llr, code, L)["u_hat"]
        errs.append(int(np.sum(np.any(oracle.payload_of(u, code) != pay, axis=1))))
    assert errs[2] <= errs[1] <= errs[0] and errs[2] < errs[0], errs


def test_scl_non_finite_channel_values():
    """SC and CA-SCL read a NaN channel value as an erasure (0) and saturate a magnitude beyond
    2^100 (+-inf included) at 2^100: decisions and metrics equal those of the frame with those
    substitutions made by hand.  A noiseless frame given as +-inf decodes exactly with metric 0,
    and every path of the final list keeps a finite metric although the wrong paths' g adds
    opposite infinities (inf - inf would be NaN)."""
    code = oracle.make_code(64, 32, 8)
    _, _, llr = _noisy_frames(code, 1.0, 16, 41)
    rng = np.random.default_rng(41)
    pos = rng.random(llr.shape) < 0.15
    sgn = np.where(rng.random(llr.shape) < 0.5, -1.0, 1.0).astype(np.float32)
    big = np.float32(2.0 ** 100)
    a_nan, a_zero = llr.copy(), llr.copy()
    a_nan[pos], a_zero[pos] = np.nan, 0.0
    a_inf, a_sat = llr.copy(), llr.copy()
    a_inf[pos], a_sat[pos] = sgn[pos] * np.inf, sgn[pos] * big
    a_inf[0, 3], a_sat[0, 3] = np.float32(3e38), big
    for x, y in ((a_nan, a_zero), (a_inf, a_sat)):
        assert np.array_equal(oracle.sc_decode(x, code), oracle.sc_decode(y, code))
        for L in (1, 4, 8):
            rx, ry = oracle.scl_decode(x, code, L), oracle.scl_decode(y, code, L)
            for k in ("u_hat", "status", "pm"):
                assert np.array_equal(rx[k], ry[k]), (L, k)
            assert np.all(np.isfinite(rx["pm"]))
    pay = inputs.payload_bits(43, 0, 4, code.P)
    xs = oracle.encode_batch(pay, code)
    for b in range(4):
        row = np.where(xs[b] == 1, -np.inf, np.inf).astype(np.float32)
        lu, lpm, u, ok = oracle.scl_list(row, code, 8)
        assert ok and np.array_equal(u, oracle.build_u(pay[b], code)) and np.all(np.isfinite(lpm))
        assert lpm.min() == 0.0 and lpm.max() > 0.0


# ------------------------------------------------------------------------------------------ BP
def _code_from(N, info):
    frozen = np.ones(N, np.uint8)
    frozen[list(info)] = 0
    return oracle.Code(N, len(info), 0, 0, frozen, np.array(sorted(info), np.int32))


def test_bp_repetition_closed_forms():
    """On repetition codes (cycle-free graphs) BP gives the exact MAP LLR, the sum of the channel
    LLRs, for the information bit and for every code bit."""
    code2 = _code_from(2, [1])
    for l0, l1 in [(1.5, -0.25), (-3.0, 2.5), (0.75, 0.5)]:
        out = oracle.bp_decode(np.array([l0, l1], np.float32), code2, 1, 20.0, early_stop=False)
        assert out["llr_u"][0, 1] == l0 + l1
        assert out["llr_x"][0, 0] == l0 + l1 and out["llr_x"][0, 1] == l0 + l1
    # N = 4, only u3 free: LLR(u3) is exact after one iteration; the code-bit LLRs need a second
    # one, since the first R sweep runs before any L message has left the channel column.
    code4 = _code_from(4, [3])
    rng = np.random.default_rng(4)
    for _ in range(20):
        lam = (rng.integers(-12, 13, 4) / 4.0).astype(np.float32)
        total = float(np.sum(lam.astype(np.float64)))
        one = oracle.bp_decode(lam, code4, 1, 20.0, early_stop=False)
        assert one["llr_u"][0, 3] == total
        two = oracle.bp_decode(lam, code4, 2, 20.0, early_stop=False)
        assert two["llr_u"][0, 3] == total
        assert np.all(two["llr_x"][0] == total)


def test_bp_first_half_frozen_free_bit():
    """N = 2 with u1 frozen: x1 carries no information about u0, so LLR(u0) = lambda_0."""
    code = _code_from(2, [0])
    out = oracle.bp_decode(np.array([-1.25, 3.0], np.float32), code, 1, 20.0, early_stop=False)
    assert out["llr_u"][0, 0] == -1.25


def _read_bp_cases(golden_dir):
    cases, cur = [], None
    for r in _read_golden(golden_dir, "bp_clip_schedule.txt"):
        f = r.split()
        if f[0] == "case":
            kv = dict(x.split("=") for x in f[2:])
            frozen = [] if kv["frozen"] == "-" else [int(v) for v in kv["frozen"].split(",")]
            cur = {"name": f[1], "N": int(kv["N"]), "frozen": frozen,
                   "llr": [float(v) for v in kv["llr"].split(",")], "iters": []}
            cases.append(cur)
        else:
            kv = dict(x.split("=") for x in f[2:])
            cur["iters"].append((int(f[1]), [float(v) for v in kv["u"].split(",")],
                                 [float(v) for v in kv["x"].split(",")]))
    return cases


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_bp_clip_and_sweep_order_hand_computed(golden_dir, precision):
    """Sec. II-B clips every computed message and the staged channel values to LLR_max = 20: on
    the hand-worked cases of tests/golden/bp_clip_schedule.txt a sum above 20 (LLR(u1) = 27 of the
    N = 2 repetition, the R sweep's 35, the staged 25) must come out clipped, and the N = 4 case's
    three iterations, whose messages change each time, fix the order of the sweeps (the R sweep
    of iteration t reads the L messages of iteration t - 1)."""
    cases = _read_bp_cases(golden_dir)
    assert [c["name"] for c in cases] == ["sum_clipped", "staging_clip", "r_sweep_clip", "schedule"]
    for c in cases:
        N = c["N"]
        code = _code_from(N, [i for i in range(N) if i not in c["frozen"]])
        lam = np.array([c["llr"]], np.float32)
        for t, u, x in c["iters"]:
            out = oracle.bp_decode(lam, code, t, 20.0, precision, early_stop=False)
            assert out["llr_u"][0].tolist() == u, (c["name"], t, out["llr_u"][0])
            assert out["llr_x"][0].tolist() == x, (c["name"], t, out["llr_x"][0])
            assert np.array_equal(out["u_hat"][0], [0 if i in c["frozen"] else int(u[i] < 0) for i in range(N)])


@pytest.mark.parametrize("precision", ["f32", "f64", "f16"])
def test_bp_weighted_update_hand_computed(golden_dir, precision):
    """The learned variant's update: each g term is scaled by w[t][dir][s-1][output node] before
    the addition and the clip, iterations past the learned ones run unweighted
    (tests/golden/bp_weighted_n2.txt, worked out by hand; every value is exact in binary16)."""
    rows = _read_golden(golden_dir, "bp_weighted_n2.txt")
    ws, want = {}, []
    for r in rows:
        f = r.split()
        kv = dict(x.split("=") for x in f[2:])
        if f[0] == "w":
            ws[int(f[1])] = ([float(v) for v in kv["R"].split(",")], [float(v) for v in kv["L"].split(",")])
        else:
            want.append((int(f[1]), [float(v) for v in kv["u"].split(",")], [float(v) for v in kv["x"].split(",")]))
    T = len(ws)
    w = np.zeros((T, 2, 1, 2), np.float32)
    for t, (wr, wl) in ws.items():
        w[t, 0, 0], w[t, 1, 0] = wr, wl
    code = _code_from(2, [1])
    lam = np.array([[15.0, 12.0]], np.float32)
    for t, u, x in want:
        out = oracle.bp_decode(lam, code, t, 20.0, precision, early_stop=False, w=w)
        assert out["llr_u"][0].tolist() == u, (t, out["llr_u"][0])
        assert out["llr_x"][0].tolist() == x, (t, out["llr_x"][0])


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_bp_channel_symmetry(precision):
    """Min-sum BP is symmetric: flipping the channel LLRs by a codeword's signs flips every
    message by the node values of that codeword, so u_hat is XOR-shifted by u, the LLRs are
    sign-flipped and (the CRC being linear) the early stop happens at the same iteration."""
    code = oracle.make_code(128, 64, 8)
    _, _, llr = _noisy_frames(code, 1.5, 32, 21)
    pay = inputs.payload_bits(99, 0, 32, code.P)
    u = np.stack([oracle.build_u(p, code) for p in pay])
    x = np.stack([oracle.polar_transform(r) for r in u])
    a = oracle.bp_decode(llr, code, 50, 20.0, precision)
    b = oracle.bp_decode(llr * (1 - 2 * x.astype(np.float32)), code, 50, 20.0, precision)
    nz = a["llr_u"] != 0
    assert np.array_equal(a["iters"], b["iters"])
    assert np.array_equal(a["status"], b["status"])
    assert np.array_equal((a["u_hat"] ^ u)[nz], b["u_hat"][nz])
    assert np.array_equal((a["llr_u"] * (1 - 2 * u.astype(np.float32))), b["llr_u"])
    assert np.array_equal((a["llr_x"] * (1 - 2 * x.astype(np.float32))), b["llr_x"])


def test_bp_weights_of_one_are_plain():
    code = oracle.make_code(64, 32, 8)
    _, _, llr = _noisy_frames(code, 1.0, 16, 8)
    w = np.ones((20, 2, code.n, code.N), np.float32)
    a = oracle.bp_decode(llr, code, 20, 20.0)
    b = oracle.bp_decode(llr, code, 20, 20.0, w=w)
    for k in ("u_hat", "status", "iters", "llr_u", "llr_x"):
        assert np.array_equal(a[k], b[k]), k


def test_round_half_matches_ieee_binary16():
    rng = np.random.default_rng(1)
    xs = np.concatenate([rng.normal(0, 10, 2000), rng.normal(0, 1e-5, 2000),
                         np.array([0.0, -0.0, 65504.0, 65519.9, 65520.0, 2.0 ** -24, 2.0 ** -25,
                                   3 * 2.0 ** -26, 1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -11])])
    xs = xs.astype(np.float32)
    for v in xs:
        with np.errstate(over="ignore"):  # 65520 rounds to infinity in binary16, as intended
            ref = float(np.float16(v))
        got = oracle.round_half(float(v))
        assert (got == ref) or (math.isinf(ref) and math.isinf(got)), (v, got, ref)


def test_half_bp_equals_fp32_when_exact():
    """With integer LLRs every half-precision sum is exact, so the FP16 BP equals the FP32 BP."""
    code = oracle.make_code(128, 64, 8)
    rng = np.random.default_rng(2)
    llr = rng.integers(-6, 7, (16, 128)).astype(np.float32)
    a = oracle.bp_decode(llr, code, 30, 32.0, "f32")
    b = oracle.bp_decode(llr, code, 30, 32.0, "f16")
    for k in ("u_hat", "status", "iters", "llr_u", "llr_x"):
        assert np.array_equal(a[k], b[k]), k


def test_hybrid_is_bp_then_scl():
    """Sec. III: frames whose CRC holds after BP keep the BP result, the others the SCL result."""
    code = oracle.make_code(128, 64, 8)
    _, _, llr = _noisy_frames(code, 1.0, 64, 31)
    bp = oracle.bp_decode(llr, code, 10, 20.0)
    scl = oracle.scl_decode(llr, code, 4)
    hy = oracle.hybrid_decode(llr, code, 10, 20.0, 4)
    ok = bp["status"] == oracle.BP_OK
    assert 0 < ok.sum() < len(ok)
    assert np.array_equal(hy["u_hat"][ok], bp["u_hat"][ok])
    assert np.array_equal(hy["u_hat"][~ok], scl["u_hat"][~ok])
    assert np.array_equal(hy["status"][~ok], scl["status"][~ok])
    assert np.array_equal(hy["iters"], bp["iters"])


# ----------------------------------------------------------------------------- input generator
def test_philox_known_answers(golden_dir):
    for r in _read_golden(golden_dir, "philox4x32_10_kat.txt"):
        v = [int(t, 16) for t in r.split()]
        out = inputs.philox4x32_10(*v[:6])
        assert [int(o) for o in out] == v[6:]


def test_input_statistics():
    z = inputs.unit_noise(5, 0, 64, 1024)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01
    b = inputs.payload_bits(5, 0, 64, 1000)
    assert abs(b.mean() - 0.5) < 0.01
    # counter-based: a frame's stream does not depend on the batch it is drawn in
    assert np.array_equal(inputs.unit_noise(5, 10, 3, 64), inputs.unit_noise(5, 0, 13, 64)[10:])


def test_scl_path_metric_is_discrepancy_for_any_list():
    """For any list size, every complete path's metric is the correlation discrepancy of its
    codeword (the same identity as in the full-list case), the final paths are distinct, and the
    output is the first CRC-passing path in metric order."""
    code = oracle.make_code(64, 32, 8)
    _, _, llr = _noisy_frames(code, 1.0, 20, 17)
    for row in llr:
        lst, pms, u, ok = oracle.scl_list(row, code, 8, "f64")
        assert len(lst) == 8 and len({tuple(p) for p in lst}) == 8
        a = np.abs(row.astype(np.float64))
        for up, pm in zip(lst, pms):
            x = oracle.polar_transform(up)
            assert pm == pytest.approx(float(np.sum(a * (x != (row < 0)))), abs=1e-9)
        passing = [k for k in np.argsort(pms, kind="stable")
                   if oracle.crc_check(lst[k][code.info_idx], code.crc_poly, code.crc_len)]
        if passing:
            assert ok and np.array_equal(u, lst[passing[0]])
        else:
            assert not ok and np.array_equal(u, lst[int(np.argmin(pms))])


@pytest.mark.parametrize("N,T", [(16, 3), (32, 2)])
def test_wms_gradient_matches_central_differences(N, T):
    """The oracle's reverse sweep of the weighted BP equals central differences of its FP64
    forward (the loss sum_i dy_i LLR(u_i) is linear in the output, so only the BP is tested)."""
    frozen, info, _ = oracle.construct(N, N // 2, 0.0, 0.5)
    code = oracle.Code(N, N // 2, 0, 0, frozen, info)
    rng = np.random.default_rng(N)
    llr = rng.normal(1.5, 2.0, (2, N)).astype(np.float32)
    w = rng.uniform(0.7, 1.3, (T, 2, code.n, N)).astype(np.float32)
    dy = rng.normal(size=(2, N))

    def f(ww):
        y = oracle.bp_decode(llr, code, T, 20.0, "f64", early_stop=False, w=ww, llr_u_double=True)["llr_u_f64"]
        return float(np.sum(dy * y))

    g = oracle.wms_grad(llr, code, T, 20.0, w, dy, "f64")
    assert np.abs(g).max() > 0
    h = 1e-6
    idx = np.argsort(-np.abs(g).ravel())[:6].tolist() + rng.choice(w.size, 6, replace=False).tolist()
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp.flat[i] += h
        wm.flat[i] -= h
        fd = (f(wp) - f(wm)) / (float(wp.flat[i]) - float(wm.flat[i]))
        assert fd == pytest.approx(g.flat[i], rel=1e-6, abs=1e-9), i
    for _ in range(3):
        v = rng.choice([-1.0, 1.0], size=w.shape)
        wp, wm = (w + h * v).astype(np.float32), (w - h * v).astype(np.float32)
        fd = f(wp) - f(wm)
        assert fd == pytest.approx(float(np.sum(g * (wp.astype(np.float64) - wm.astype(np.float64)))), rel=1e-5, abs=1e-12)


@pytest.mark.parametrize("N,T", [(16, 3), (32, 4)])
def test_wms_gradient_all_iterations_matches_central_differences(N, T):
    """Per-iteration loss sum_t sum_i dy[t][i] LLR_t(u_i), LLR_t after t + 1 iterations (each a
    separate FP64 forward of the oracle): the reverse sweep against central differences."""
    frozen, info, _ = oracle.construct(N, N // 2, 0.0, 0.5)
    code = oracle.Code(N, N // 2, 0, 0, frozen, info)
    rng = np.random.default_rng(N + T)
    llr = rng.normal(1.0, 2.0, (2, N)).astype(np.float32)
    w = rng.uniform(0.7, 1.3, (T, 2, code.n, N)).astype(np.float32)
    dy = rng.normal(size=(T, 2, N))

    def f(ww):
        tot = 0.0
        for t in range(T):
            y = oracle.bp_decode(llr, code, t + 1, 20.0, "f64", early_stop=False, w=ww, llr_u_double=True)["llr_u_f64"]
            tot += float(np.sum(dy[t] * y))
        return tot

    g = oracle.wms_grad(llr, code, T, 20.0, w, dy, "f64", all_iters=True)
    # early iterations get their own term: the gradient of iteration 0 differs from the
    # last-iteration-only loss
    g_last = oracle.wms_grad(llr, code, T, 20.0, w, dy[-1], "f64")
    assert not np.allclose(g[0], g_last[0])
    h = 1e-6
    idx = np.argsort(-np.abs(g).ravel())[:6].tolist() + rng.choice(w.size, 6, replace=False).tolist()
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp.flat[i] += h
        wm.flat[i] -= h
        fd = (f(wp) - f(wm)) / (float(wp.flat[i]) - float(wm.flat[i]))
        assert fd == pytest.approx(g.flat[i], rel=1e-6, abs=1e-9), i


# ---------------------------------------------------------------------------- decision aiding
def _da_code(N, K, crc, frac, seed):
    """The code with a random subset (fraction `frac`) of its information positions decided."""
    import dataclasses
    code = oracle.make_code(N, K, crc)
    rng = np.random.default_rng(seed)
    dec = np.zeros(N, np.uint8)
    pick = rng.choice(code.info_idx, int(frac * K), replace=False)
    dec[pick] = 1
    return dataclasses.replace(code, decided=dec)


@pytest.mark.parametrize("N,K,crc", [(64, 32, 8), (128, 64, 8)])
def test_decision_aided_list_of_one_is_sc(N, K, crc):
    """With L = 1 the list never branches, so deciding some positions by the hard decision (what
    SC does at every information position) changes nothing: CA-SCL(L = 1) = SC for any mask."""
    code = _da_code(N, K, crc, 0.5, N)
    rng = np.random.default_rng(N + 1)
    llr = rng.normal(1.0, 2.5, (20, N)).astype(np.float32)
    sc = oracle.sc_decode(llr, code)
    assert np.array_equal(oracle.scl_decode(llr, code, 1)["u_hat"], sc)


@pytest.mark.parametrize("L", [2, 4, 8])
def test_decision_aided_all_information_bits_is_sc(L):
    """Every information position decided: the list never grows past one path, for any L."""
    import dataclasses
    code = oracle.make_code(128, 64, 8)
    dec = (1 - code.frozen).astype(np.uint8)
    code = dataclasses.replace(code, decided=dec)
    rng = np.random.default_rng(L)
    llr = rng.normal(1.0, 2.5, (20, 128)).astype(np.float32)
    assert np.array_equal(oracle.scl_decode(llr, code, L)["u_hat"], oracle.sc_decode(llr, code))


def test_decision_aided_empty_mask_is_plain_and_noiseless_decodes():
    import dataclasses
    plain = oracle.make_code(128, 64, 8)
    empty = dataclasses.replace(plain, decided=np.zeros(128, np.uint8))
    rng = np.random.default_rng(9)
    llr = rng.normal(1.0, 2.5, (30, 128)).astype(np.float32)
    a, b = oracle.scl_decode(llr, plain, 4), oracle.scl_decode(llr, empty, 4)
    assert np.array_equal(a["u_hat"], b["u_hat"]) and np.array_equal(a["status"], b["status"])
    code = _da_code(128, 64, 8, 0.5, 3)
    pay = rng.integers(0, 2, (10, code.P)).astype(np.uint8)
    x = oracle.encode_batch(pay, code)
    out = oracle.scl_decode(20.0 * (1.0 - 2.0 * x.astype(np.float32)), code, 4)
    assert np.array_equal(oracle.payload_of(out["u_hat"], code), pay)
    assert (out["status"] == 2).all()


# ----------------------------------------------------- exact PE function and re-encoding stop
def _kron_G(N):
    F = np.array([[1, 0], [1, 1]], dtype=np.int64)
    G = np.array([[1]], dtype=np.int64)
    while G.shape[0] < N:
        G = np.kron(G, F)
    return G


def _tanh_rule(lams):
    """Posterior LLR of the XOR of independent bits with LLRs lams (the textbook tanh rule)."""
    return float(2.0 * np.arctanh(np.prod(np.tanh(np.asarray(lams, np.float64) / 2.0))))


def test_exact_g_is_the_tanh_rule():
    """g(a, b) = ln((1 + e^(a+b)) / (e^a + e^b)) is the LLR of the XOR of two independent bits:
    2 atanh(tanh(a/2) tanh(b/2)); symmetric, odd in each argument, |g| <= min(|a|, |b|) and the
    min-sum approximation overshoots by at most ln 2."""
    rng = np.random.default_rng(12)
    for _ in range(400):
        a, b = (float(v) for v in rng.uniform(-15, 15, 2))
        g = oracle.pe_g_exact(a, b)
        assert g == pytest.approx(_tanh_rule([a, b]), abs=1e-9)
        assert g == oracle.pe_g_exact(b, a)
        assert oracle.pe_g_exact(-a, b) == pytest.approx(-g, abs=1e-12)
        m = min(abs(a), abs(b))
        assert abs(g) <= m and m - abs(g) <= math.log(2.0) + 1e-12
        assert np.sign(g) == np.sign(a) * np.sign(b)
    assert oracle.pe_g_exact(3.0, 0.0) == 0.0
    assert oracle.pe_g_exact(-3.0, 40.0) == pytest.approx(-3.0, abs=1e-12)


@pytest.mark.parametrize("N", [8, 16, 64])
def test_bp_first_l_sweep_is_the_exact_posterior_of_u(N):
    """No frozen bit: u = x G with the x_i independent given y, so the posterior LLR of u_j is the
    tanh rule over {i : G[i][j] = 1}.  Every R message stays 0 in the first iteration, and its L
    sweep computes exactly that with the exact g, and sign product times smallest magnitude with
    the min-sum g (G from np.kron, independent of the oracle)."""
    G = _kron_G(N)
    code = _code_from(N, range(N))
    rng = np.random.default_rng(N)
    lam = np.clip(rng.normal(1.5, 2.0, (5, N)), -8, 8).astype(np.float32)
    ex = oracle.bp_decode(lam, code, 1, 20.0, "f64", early_stop=False, g="exact")
    ms = oracle.bp_decode(lam, code, 1, 20.0, "f64", early_stop=False)
    for b in range(5):
        for j in range(N):
            S = np.nonzero(G[:, j])[0]
            v = lam[b, S].astype(np.float64)
            assert ex["llr_u"][b, j] == pytest.approx(_tanh_rule(v), rel=1e-6, abs=1e-6), (b, j)
            assert ms["llr_u"][b, j] == np.float32(np.prod(np.sign(v)) * np.min(np.abs(v))), (b, j)


@pytest.mark.parametrize("N", [8, 32])
def test_bp_first_r_sweep_is_the_prior_of_x(N):
    """Zero channel LLRs: the first R sweep sees no channel information, so R[n+1] -- and LLR(x)
    after one iteration -- is the prior of x = u G from the u-side LLRs alone: the tanh rule over
    {j : G[j][i] = 1} of LLR_max (frozen u_j = 0) and 0 (free u_j)."""
    G = _kron_G(N)
    rng = np.random.default_rng(N + 1)
    for _ in range(4):
        info = sorted(rng.choice(N, size=N // 4, replace=False).tolist())
        code = _code_from(N, info)
        out = oracle.bp_decode(np.zeros((1, N), np.float32), code, 1, 20.0, "f64", early_stop=False, g="exact")
        for i in range(N):
            T = np.nonzero(G[:, i])[0]
            prior = [20.0 if code.frozen[j] else 0.0 for j in T]
            assert out["llr_x"][0, i] == pytest.approx(_tanh_rule(prior), abs=4e-6), (info, i)


@pytest.mark.parametrize("g", ["minsum", "exact"])
def test_reencoding_stop_rule(g):
    """The re-encoding stop ends BP at the first iteration t where HD(LLR(x)) = HD(LLR(u)) G (G from
    np.kron), checked on the outputs of runs of t and t - 1 iterations without early stop; the
    frame counts as decoded iff the CRC of that u holds."""
    code = oracle.make_code(64, 32, 8)
    G = _kron_G(64)
    _, _, llr = _noisy_frames(code, 2.0, 24, 31)
    imax = 25
    r = oracle.bp_decode(llr, code, imax, 20.0, "f32", stop="reencode", g=g)

    def holds(b, T):
        o = oracle.bp_decode(llr[b:b + 1], code, T, 20.0, "f32", early_stop=False, g=g)
        x = (o["u_hat"][0].astype(np.int64) @ G) % 2
        return np.array_equal(x, (o["llr_x"][0] < 0).astype(np.int64)), o

    stopped_early = 0
    for b in range(llr.shape[0]):
        t = int(r["iters"][b])
        ok, o = holds(b, t)
        assert ok or t == imax, b
        stopped_early += t < imax
        if t > 1:
            assert not holds(b, t - 1)[0], b
        assert np.array_equal(o["u_hat"][0], r["u_hat"][b])
        crc_ok = oracle.crc_check(o["u_hat"][0][code.info_idx], code.crc_poly, code.crc_len)
        assert (r["status"][b] == oracle.BP_OK) == crc_ok, b
    assert stopped_early >= 12


def test_exact_g_and_reencoding_noiseless_and_hybrid():
    """Noiseless frames decode exactly with every stop rule and g; the hybrid with either stop rule
    is BP followed by CA-SCL on exactly the frames whose CRC fails when BP stops."""
    code = oracle.make_code(128, 64, 8)
    pay = inputs.payload_bits(3, 0, 8, code.P)
    x = oracle.encode_batch(pay, code)
    llr = (8.0 * (1.0 - 2.0 * x)).astype(np.float32)
    u_true = np.stack([oracle.build_u(p, code) for p in pay])
    for stop in ("crc", "reencode"):
        for g in ("minsum", "exact"):
            bp = oracle.bp_decode(llr, code, 50, 20.0, stop=stop, g=g)
            assert np.array_equal(bp["u_hat"], u_true) and np.all(bp["status"] == oracle.BP_OK), (stop, g)
    _, _, noisy = _noisy_frames(code, 1.5, 60, 17)
    for stop in ("crc", "reencode"):
        bp = oracle.bp_decode(noisy, code, 10, 20.0, stop=stop, g="exact")
        hy = oracle.hybrid_decode(noisy, code, 10, 20.0, 4, stop=stop, g="exact")
        scl = oracle.scl_decode(noisy, code, 4)
        ok = bp["status"] == oracle.BP_OK
        assert 0 < ok.sum() < len(ok)
        assert np.array_equal(hy["iters"], bp["iters"])
        assert np.array_equal(hy["u_hat"][ok], bp["u_hat"][ok])
        assert np.array_equal(hy["u_hat"][~ok], scl["u_hat"][~ok])
