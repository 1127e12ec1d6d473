"""The allocation-free power iteration (lp_power_norm_noalloc) against the one lp_create runs.

lp_power_norm_noalloc exists for callers that must not allocate device memory (their memory
is owned by their own pool allocator, or they cannot afford the synchronisation an
allocation may cause); it keeps its scratch in a static device array.  These tests check that
it returns the same ||A||_2 estimate as the existing path (lp_create on the unscaled matrix,
reported by lp_get_info), within the tolerance of the other power-iteration tests, on two
calls in a row (the second call reuses scratch the first one left behind), and that sizes
beyond its static scratch are refused.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import paper_2507_14051_b300 as lpx
from paper_2507_14051_b300 import gen


def test_sizes_beyond_the_static_scratch_are_refused():
    with pytest.raises(lpx.LPError) as e:
        lpx.lp_power_norm_noalloc(262145, 10, 0, None, None, None)
    assert e.value.code == lpx.LP_ERR_TOO_LARGE
    assert "262144" in lpx.lp_last_error()


@pytest.mark.gpu
@pytest.mark.parametrize("make", [lambda: gen.small_lp(0), lambda: gen.miplib_like(0, 3000, 6000, 2000),
                                  lambda: gen.ragged_rows(1, 400, 900)])
def test_noalloc_power_norm_matches_lp_create(cuda_device, make):
    import torch
    lp = make()
    with lpx.Solver(lp, ruiz_iters=0, pc_enabled=0) as s:
        s.solve(0.0, 1)
        ref = s.result()["norm_A"]
    assert ref > 0.0
    rp = torch.tensor(lp.row_ptr, dtype=torch.int64, device="cuda")
    ci = torch.tensor(lp.col_idx, dtype=torch.int32, device="cuda")
    va = torch.tensor(lp.val, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        norm, steps = lpx.lp_power_norm_noalloc(lp.m, lp.n, lp.nnz, rp, ci, va, 1e-7, 10000, 0, stream)
        assert steps >= 2
        assert norm == pytest.approx(ref, rel=1e-6), (call, norm, ref)
