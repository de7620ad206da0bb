"""The FP32 multiply-add throughput probe (mfadvr_probe_fma), which the bench
uses as the measured ceiling of the FMA-bound kernels."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("packed", [False, True])
def test_probe_rate_is_below_the_unit_count_bound(torch_cuda, packed):
    """The probe's rate lies between a third of and the bound from unit counts
    at a 2.2 GHz clock (above any GB300 clock): 128 FP32 lanes x 2 FLOP per SM."""
    from paper_2204_11762_gb300 import mfadvr
    torch = torch_cuda
    dev = torch.device("cuda:0")
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    bound = sms * 128 * 2 * 2.2e9 / 1e12
    sink = torch.zeros(1, device=dev)
    stream = torch.cuda.current_stream(dev)
    best = 0.0
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fmas = mfadvr.probe_fma(sink, 1024, packed=packed, stream=stream)
        e1.record(stream)
        e1.synchronize()
        best = max(best, fmas * 2 / (e0.elapsed_time(e1) / 1000.0) / 1e12)
    assert fmas > 0
    assert bound / 3 < best < bound, f"{best:.1f} TFLOP/s against a bound of {bound:.1f}"
    assert float(sink[0].item()) == 0.0  # the keep-alive store never happens


def test_probe_rejects_bad_arguments(torch_cuda):
    from paper_2204_11762_gb300 import mfadvr
    torch = torch_cuda
    sink = torch.zeros(1, device="cuda:0")
    host = torch.zeros(1)
    for args in [(sink, 0), (sink, (1 << 24) + 1), (host, 16)]:
        with pytest.raises(mfadvr.MfadvrError) as e:
            mfadvr.probe_fma(*args)
        assert e.value.status == mfadvr.EINVAL
