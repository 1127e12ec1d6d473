"""Host-side bookkeeping of bench.py (no GPU): the kernel-launch counts, byte model and summary
statistics it reports."""
import numpy as np

import bench


def test_batch_launch_count_per_schedule_kind():
    sm = {"iters": np.array([100, 40, 30]), "iters_fp32": np.zeros(3, np.int64)}
    # grid loop: 7 launches of 16 iterations + the body that sees every instance done; one launch
    # per kind of small instance; kb_init_ctl + kb_init
    assert bench.batch_launches(sm, np.array([0, 1, 2]), 0) == 2 + 8 + 2
    assert bench.batch_launches(sm, np.array([0, 1, 1]), 0) == 2 + 8 + 1
    assert bench.batch_launches(sm, np.array([1, 2, 2]), 0) == 2 + 2
    mixed = {"iters": np.array([100, 40]), "iters_fp32": np.array([64, 40])}
    # two stages (FP32 64 and 0 iterations on the grid) + the hand-over's four kernels
    assert bench.batch_launches(mixed, np.array([0, 1]), 1) == 2 + 4 + (4 + 1 + 1) + (3 + 1 + 1)


def test_diff_launch_count():
    K, C = 2000, 100
    grid = np.zeros(64, np.int32)
    assert bench.diff_launches(K, C, grid) == 9 + (2 + 125 + 0 + 1 + 20 + 2) + (2 + 40 + 3)
    small = np.array([1, 2], np.int32)
    assert bench.diff_launches(K, C, small) == 9 + (2 + 0 + 2 + 1 + 20 + 2) + (2 + 40 + 3)
    mixed = np.array([0, 1], np.int32)  # both segment kernels per segment and direction
    assert bench.diff_launches(K, C, mixed) == 9 + (2 + 125 + 1 + 1 + 40 + 2) + (2 + 80 + 3)


def test_kernel_work_fp32_moves_fewer_bytes_and_no_fp64_ops():
    class LP:
        m, n, nnz = 10, 20, 50
    b64, b32 = bench.kernel_work(LP(), 8), bench.kernel_work(LP(), 4)
    for k in ("k1_rows", "k2_cols"):
        assert b32[k][0] < b64[k][0] and b32[k][1] is None and b64[k][1] > 0
    assert b64["k1_rows"][0] == 12 * 50 + 8 * 11 + 8 * 20 + 56 * 10
    # the scope table's per-iteration figure: 24 nnz + 72 (m + n) + 16
    assert b64["k1_rows"][0] + b64["k2_cols"][0] == 24 * 50 + 72 * 30 + 16
    assert b64["k1_rows"][1] == 50 + 15 * 10 and bench.kernel_work(LP(), 8, loop=False)["k1_rows"][1] == 50 + 17 * 10


def test_sgm10_is_the_shifted_geometric_mean():
    """Section 4 summarises solve times by the shifted geometric mean with shift 10."""
    assert bench.sgm10([5.0]) == 5.0
    # (t + 10) = 10 and 40: geometric mean 20, minus the shift
    assert abs(bench.sgm10([0.0, 30.0]) - 10.0) < 1e-12
    assert bench.sgm10([]) is None


def test_cpu_info_reports_model_and_core_count():
    info = bench.cpu_info()
    assert info["nproc"] >= 1 and "cpu_model" in info
