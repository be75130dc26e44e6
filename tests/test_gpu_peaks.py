"""The library's peak microbenchmarks (mf_measure_peak): each kind runs and
gives a rate within a factor of the hardware's lane counts at the clocks a
GB300 can run (FP32: 128 FMA lanes per SM, FP64: 2, at 1-2.1 GHz), and the
packed-pair FP32 kernel does the same work per FMA lane as the scalar one."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2106_10279_gb300 import api
    return torch, api


def test_peaks_are_plausible(env):
    torch, api = env
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    r = {k: api.mf_measure_peak(k, reps=3)[0] for k in ("fp32_ffma", "fp32_ffma2", "fp64_dfma", "tf32_mma")}
    lo, hi = 0.9e9, 2.2e9                       # SM clock range, Hz
    assert nsm * 128 * 2 * lo * 0.5 / 1e12 < r["fp32_ffma"] < nsm * 128 * 2 * hi / 1e12, r
    assert 0.5 < r["fp32_ffma2"] / r["fp32_ffma"] < 2.05, r
    assert nsm * 2 * 2 * lo * 0.5 / 1e12 < r["fp64_dfma"] < nsm * 2 * 2 * hi * 1.05 / 1e12, r
    assert r["tf32_mma"] > r["fp32_ffma"], r
