"""The measurement utilities behind the ALU roofline: SIMT FMA peaks (FP32, FP64, packed FP32)
and the throughput of the P(dt) kernel's register FFT alone.  They must return plausible rates
for a GB300-class device and keep their documented ordering."""
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ch():
    import paper_2205_02380_gb300 as pkg
    pkg.chasm.lib()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return pkg


def test_fma_peaks_are_plausible(ch):
    fp32, fp64 = ch.chasm.fma_peaks()
    fp32x2 = ch.chasm.fma_peak_f32x2()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    # at most 128 FP32 lanes x 2 flops x 2.2 GHz per SM; FP64 far below FP32 on this part
    assert 0.3 * sms * 128 * 2 * 1.0e9 / 1e12 < fp32 <= sms * 128 * 2 * 2.2e9 / 1e12
    assert 0.3 * fp32 < fp32x2 <= 1.2 * fp32
    assert 0.0 < fp64 < 0.5 * fp32


def test_fft_rate_is_below_the_packed_fma_ceiling(ch):
    fft = ch.chasm.fft_pk_rate()
    fp32x2 = ch.chasm.fma_peak_f32x2()
    # 388 packed instructions per pair of 32-point transforms (1600 counted flops): at most about
    # 1.03 counted flops per FMA flop
    assert 0.3 * fp32x2 < fft < 1.1 * fp32x2
