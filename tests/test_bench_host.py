"""Host logic of bench.py (no GPU): the committed profile the roofline's
`traffic` comes from matches the current kernel source (its digest), and the
derived FP64 peak follows the part's unit counts and the sampled clock."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_multidot_profile_matches_the_current_kernel_source():
    # a change to k_krylov.cu without a new capture makes the bench report
    # traffic = null; this test makes that visible before a run
    t = bench.traffic_from_profile("k_multidot_c3.md", "multidot", "k_krylov.cu")
    assert isinstance(t, tuple) and t[0] == "ratio"
    assert 0.95 < t[1] < 1.10


def test_traffic_is_null_for_another_source():
    assert bench.traffic_from_profile("k_multidot_c3.md", "multidot", "k_ilu.cu") is None


def test_derived_fp64_peak():
    class Props:
        multi_processor_count = 152

    class Cuda:
        @staticmethod
        def get_device_properties(i):
            return Props()

    class Torch:
        cuda = Cuda()

    peak, src = bench.fp64_peak(Torch(), {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0})
    assert abs(peak - 2 * 152 * 2070e6) < 1.0
    assert "152 SMs" in src
    peak2, _ = bench.fp64_peak(Torch(), {"sm_mhz": None, "sm_max_mhz": 1965.0})
    assert abs(peak2 - 2 * 152 * 1965e6) < 1.0
