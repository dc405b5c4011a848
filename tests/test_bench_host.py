"""Host-side logic of the benchmark without a GPU: the clock summary that
accompanies every bench line, the kernel names it reports, and the
workload descriptions."""
import numpy as np

import bench
import workloads as wl


def _summary(lines):
    c = bench.ClockSampler(0)
    c.lines = lines
    return c.summary()


def test_clock_summary_median_and_reasons():
    lines = ["1995, 2070, 0x0000000000000000", "2070, 2070, 0x0000000000000004",
             "2070, 2070, 0x0000000000000001", "garbage", "2040, 2070, 0x0000000000000060"]
    s = _summary(lines)
    assert s["samples"] == 4
    assert s["sm_mhz"] == 2055.0 and s["sm_max_mhz"] == 2070.0
    # gpu_idle is not a throttle reason; 0x60 = sw_thermal_slowdown | hw_thermal_slowdown
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap", "sw_thermal_slowdown"]


def test_clock_summary_without_samples():
    assert _summary([]) == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}


class _FakeKx:
    def __init__(self, variants):
        self.v = variants

    def kx_get_launch_shapes(self, ctx):
        return None, None, self.v


def test_kernel_names_follow_the_variant_of_each_stream():
    v = np.zeros(243, dtype=np.int32)
    dd = 80                                 # (dd|dd)
    assert bench.kernel_name(_FakeKx(v), None, 40) == "k_eri<1,1,1,1,double>"
    assert bench.kernel_name(_FakeKx(v), None, 81 + 40) == "k_eri<1,1,1,1,float>"
    assert bench.kernel_name(_FakeKx(v), None, dd) == "k_eri_rolled<2,2,2,2,double>"
    v[dd] = 1
    assert bench.kernel_name(_FakeKx(v), None, dd) == "k_eri_big64<2,2,2,2>"
    v[dd] = 2
    assert bench.kernel_name(_FakeKx(v), None, dd) == "k_eri_big64p<2,2,2,2>"
    assert bench.kernel_name(_FakeKx(v), None, 81 + dd) == "k_eri_big<2,2,2,2>"
    v[81 + dd] = 1
    assert bench.kernel_name(_FakeKx(v), None, 81 + dd) == "k_eri_bigp<2,2,2,2>"
    assert bench.kernel_name(_FakeKx(v), None, 162 + 40) == "k_eri<1,1,1,1,kx::dw>"


def test_workload_descriptions():
    s = wl.water64(2)
    c = bench.workload_config(s, "mixed", "water64", True, 16)
    assert c["n_fn"] == 1984 and c["n_shell"] == 1024 and c["leaf_max"] == 16
    assert c["split_threshold"] == bench.SPLIT and c["symmetric"] is True
    assert "(H2O)64" in c["workload"] and "model" not in c
    f = bench.workload_config(s, "fp64", "water64")
    assert f["split_threshold"] is None and f["leaf_max"] == 10


def test_job_rate_counts_every_rank():
    assert bench.job_rate(1, 1, 2.0) == 0.5
    assert bench.job_rate(3, 4, 2.0) == 6.0
