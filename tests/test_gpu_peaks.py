"""The arithmetic-peak probe (include/kin_peaks.h) on the GPU: the measured
FMA rate is a pipe throughput (it does not change when the chains run twice
as long, so launch overhead is not in it), the FP64 rate lies in the range
the GB300's FP64 units allow (2 FMA lanes per SM per clock at most), and the
FP32 pipe is far wider than the FP64 one."""
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1309_2710_gb300 import build as kbuild  # noqa: E402

kbuild.build()
from paper_1309_2710_gb300 import peaks  # noqa: E402


def test_fma_probe_measures_a_throughput():
    props = torch.cuda.get_device_properties(0)
    nsm = props.multi_processor_count
    out = {}
    for prec, iters in ((peaks.FP64, 4000), (peaks.FP32, 100000)):
        peaks.fma_rate(prec, iters // 4)  # warm up (module load, clocks)
        ms1, r1 = peaks.fma_rate(prec, iters)
        ms2, r2 = peaks.fma_rate(prec, 2 * iters)
        assert ms2 == pytest.approx(2 * ms1, rel=0.15), (prec, ms1, ms2)
        assert r2 == pytest.approx(r1, rel=0.15)
        out[prec] = max(r1, r2)
    # FP64: at most 2 FMA per SM per clock at <= 2.1 GHz, and clearly more
    # than a tenth of that
    top64 = 2 * nsm * 2.1e9
    assert 0.1 * top64 < out[peaks.FP64] <= 1.05 * top64, out
    assert out[peaks.FP32] > 16 * out[peaks.FP64], out
    print("FMA/s: FP64 %.4g, FP32 %.4g (%d SMs)" % (out[peaks.FP64], out[peaks.FP32], nsm))


def test_fma_probe_rejects_bad_arguments():
    with pytest.raises(RuntimeError):
        peaks.fma_rate(7, 10)
    with pytest.raises(RuntimeError):
        peaks.fma_rate(peaks.FP64, 10, threads=33)
    with pytest.raises(RuntimeError):
        peaks.fma_rate(peaks.FP64, 0)
