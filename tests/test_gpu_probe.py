"""Throughput probes behind the roofline fractions (kx_peak_probe).

The FP64 and FP32 probes time independent FMA chains on the plain pipes,
the DMMA probe FP64 tensor-core mma.sync chains.  On GB300 the FP32 pipe
is far faster than the FP64 one (the split-precision design rests on that
ratio), and every probe must report a positive rate.
"""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1401_6961_gb300 import build
    build.build()
    import paper_1401_6961_gb300 as kx
    kx.load()
    return kx


def test_probes_report_positive_rates(kx):
    f64 = kx.kx_peak_probe(0, kx.KX_FP64)
    f32 = kx.kx_peak_probe(0, kx.KX_MIXED)
    mma = kx.kx_peak_probe(0, kx.KX_PROBE_FP64_MMA)
    dw = kx.kx_peak_probe(0, kx.KX_PROBE_DW)
    print(f"FP64 FMA {f64:.0f} GFLOP/s, FP32 FMA {f32:.0f} GFLOP/s, FP64 DMMA {mma:.0f} GFLOP/s, "
          f"double-word FMA {dw:.0f} GFLOP/s")
    assert f64 > 0 and f32 > 0 and mma > 0 and dw > 0
    assert f32 > 10 * f64
    # a double-word FMA is about 15 FP32 instructions: well above the FP64 pipe on GB300
    assert f64 < dw < f32


def test_probe_rejects_unknown_kind(kx):
    with pytest.raises(kx.KxError):
        kx.kx_peak_probe(0, 4)
