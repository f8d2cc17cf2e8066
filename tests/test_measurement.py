"""The measurement and checking entry points on the GPU: the issue-rate microbenchmark gives the
rates the roofline rests on, and polar_pe_eval's packed form handles an odd length."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

from paper_1609_09358_gb300 import api, build  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    api.load()


def test_pipe_rates_are_plausible():
    """Results of one lane per SM per clock: the comparison pipe's min.xorsign.abs at half the 128
    FP32 lanes, the special-function ex2 at twice lg2's rate; every rate within (8, 300)."""
    scratch = torch.empty(api.polar_pipe_rate_scratch_bytes(), dtype=torch.uint8, device="cuda")
    r = {name: api.polar_pipe_rate(op, 1024, scratch) for name, op in api.PIPE_RATE_OPS.items()}
    for name, v in r.items():
        assert 8.0 < v < 300.0, (name, v)
    assert 48.0 <= r["min.xorsign.abs.f32"] <= 72.0
    assert 1.6 <= r["ex2.approx.ftz.f32"] / r["lg2.approx.ftz.f32"] <= 2.4
    with pytest.raises(api.PolarError):
        api.polar_pipe_rate(0, 16, scratch[:8])


def test_pe_eval_packed_tail_and_min_sum():
    """An odd n leaves the packed form a last element without a partner: it still equals the scalar
    form; the min-sum form is sign(a) sign(b) min(|a|, |b|) exactly."""
    rng = np.random.default_rng(5)
    a = rng.uniform(-20, 20, 1001).astype(np.float32)
    b = rng.uniform(-40, 40, 1001).astype(np.float32)
    ad, bd = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    outs = {}
    for op in (api.POLAR_PE_MINSUM, api.POLAR_PE_EXACT, api.POLAR_PE_EXACT_PACKED):
        o = torch.empty_like(ad)
        api.polar_pe_eval(op, ad, bd, o)
        outs[op] = o.cpu().numpy()
    assert np.array_equal(outs[api.POLAR_PE_EXACT].view(np.uint32), outs[api.POLAR_PE_EXACT_PACKED].view(np.uint32))
    ms = (np.sign(a) * np.sign(b) * np.minimum(np.abs(a), np.abs(b))).astype(np.float32)
    assert np.array_equal(outs[api.POLAR_PE_MINSUM], ms)
