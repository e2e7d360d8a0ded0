"""Host-side pieces of bench.py that need no GPU: the step-time fit, the choice of the K V
kernel the roofline reports, and the ncu traffic record of the chosen path's dominant kernel
(reported only while it was captured from the current sources)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_step_time_fit_recovers_a_linear_model():
    rounds = np.array([3, 4, 3, 5, 70, 3, 4, 68, 3, 4], dtype=float)
    ms = 2.7 + 1.26 * rounds
    fit = bench._fit_step_time(list(ms), list(rounds.astype(int)))
    assert abs(fit["fixed_ms"] - 2.7) < 1e-9 and abs(fit["ms_per_round"] - 1.26) < 1e-9


def test_kernel_key_follows_the_tuner():
    tab = [{"cross_term": 2}] * 16 + [{"cross_term": 1}]
    assert bench.kernel_key("fp32") == "fp32"
    assert bench.kernel_key("mixed") == "mixed_tensor"
    assert bench.kernel_key("mixed", tab, 16) == "mixed_tensor"
    assert bench.kernel_key("mixed", tab, 17) == "mixed_pipe"


def test_traffic_record_of_the_chosen_kernel_is_current():
    key = "mixed_tensor"
    rec = bench._kv_file(bench.KMV_KERNELS[key][1])
    assert rec.get("kmv_source_hash") == bench.kmv_source_hash(key), (
        "the ncu traffic record of %s was taken from other sources: re-capture it" % key)
    assert float(rec["dram_bytes_per_launch"]) > 0
