"""The FP64 arithmetic rate the FP64 mode's roofline is quoted against: a
positive rate below the device's nominal FP32 rate (FP64 on GB300 runs far
below FP32), and stable between two measurements."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2409_17299_gb300 as q  # noqa: E402


def test_fp64_peak_measurement():
    from paper_2409_17299_gb300 import build
    build.build()
    f1, ms1 = q.qed_measure_fp64_peak(1 << 14)
    f2, ms2 = q.qed_measure_fp64_peak(1 << 14)
    assert ms1 > 0 and ms2 > 0
    assert 1e10 < f1 < 1e14 and 1e10 < f2 < 1e14
    assert abs(f1 / f2 - 1) < 0.2
    with pytest.raises(q.QedError):
        q.qed_measure_fp64_peak(0)
