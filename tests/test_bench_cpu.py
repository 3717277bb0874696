"""Host-side pieces of the benchmark: the algorithmic bytes per launch and the
link between the training kernel's revision and its committed ncu summary
(the DRAM traffic the bench line reports is taken from that summary only
while both name the same revision)."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402


def test_algorithmic_bytes_per_unit():
    w = bench.WORKLOADS["spectral256"]  # L = 16, F = 2
    # per sample: 8 FP32 volume reads, 16 x 8 FP16x2 gathers, 16 x 8 FP32x2 gradient updates
    assert bench.kernel_bytes("train_fused_fp16", w, 0, 1) == 8 * 4 + 16 * 8 * 2 * 2 + 16 * 8 * 2 * 4 == 1568
    assert bench.kernel_bytes("adam", w, 1000, 0) == 34 * 1000
    assert bench.kernel_bytes("train_fused_fp16", w, 0, 1 << 18) == 1568 << 18


def test_training_profile_is_of_the_current_kernel_revision():
    t, src = bench.measured_traffic("train_fused_fp16", "spectral256")
    assert t is not None and t > 0, src
    assert "profiles/k_mp_train_fp16_spectral256.md" in src and "not this run" in src
    assert bench.measured_traffic("adam", "spectral256") == (None, None)
