"""The FP64 peak probe (mm_probe_fp64_peak) runs through the C ABI and returns
rates a GB300's FP64 pipe can have; the plain FP64 product does not run
faster than the probe's MMA rate by more than timing noise."""
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_probe_rates_are_plausible():
    import paper_1106_1347_gb300 as mm
    import synthetic as S

    dfma, dmma = mm.probe_fp64_peak(40.0)
    # Nominal GB300 FP64: about 1.25 TFLOP/s; anything far outside means the probe
    # is not measuring the pipe.
    assert 0.3 < dfma < 5.0, dfma
    assert 0.3 < dmma < 5.0, dmma
    n = 2048
    dev = torch.device("cuda")
    a = torch.from_numpy(S.uniform(n, n, S.stream_seed(1, 0))).to(dev)
    b = torch.from_numpy(S.uniform(n, n, S.stream_seed(1, 1))).to(dev)
    c = mm.naive(a, b)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(3):
        mm.naive(a, b, out=c)
    e1.record()
    torch.cuda.synchronize()
    tflops = 3 * 2.0 * n ** 3 / (e0.elapsed_time(e1) * 1e-3) / 1e12
    assert tflops <= 1.05 * dmma, (tflops, dmma)


def test_probe_rejects_bad_duration():
    import paper_1106_1347_gb300 as mm

    with pytest.raises(mm.MMError):
        mm.probe_fp64_peak(0.0)
