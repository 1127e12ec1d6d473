"""The allocation-free power iteration (lp_power_norm_noalloc).

lp_power_norm_noalloc exists for callers that must not allocate device memory: code whose
device memory is owned by its own pool allocator, or latency-critical code that cannot afford
the implicit synchronisation an allocation may cause.  It keeps all of its scratch in one
static device array.  These tests check
  * that it returns the same ||A||_2 estimate as the existing path (lp_create's power iteration
    on the unscaled matrix, reported by lp_get_info) and as the oracle's power iteration,
    within the tolerance of the other power-iteration tests, on two calls in a row (the second
    call reuses the scratch the first one left behind);
  * that a call allocates no device memory: the device's free bytes (cudaMemGetInfo) and
    torch's allocator counters are the same before and after it;
  * the iteration cap, the empty matrix, sizes beyond the static scratch, and a CSR with an
    out-of-range column index, which the kernels' own checks turn into LP_ERR_INVALID_INPUT;
  * that its source names no allocating call.
This file is collected last on purpose.
"""
import os
import re

import numpy as np
import pytest

import paper_2507_14051_b300 as lpx
from paper_2507_14051_b300 import gen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SOURCE = os.path.join(ROOT, "paper_2507_14051_b300", "csrc", "noalloc.cu")


def test_sizes_beyond_the_static_scratch_are_refused():
    with pytest.raises(lpx.LPError) as e:
        lpx.lp_power_norm_noalloc(262145, 10, 0, None, None, None)
    assert e.value.code == lpx.LP_ERR_TOO_LARGE
    assert "262144" in lpx.lp_last_error()


def test_source_names_no_allocating_call():
    with open(SOURCE) as f:
        text = f.read()
    banned = r"\b(cudaMalloc\w*|cudaFree\w*|cuMem\w*Alloc\w*|cuMemFree\w*|cudaHostAlloc|malloc|calloc|realloc|" \
             r"new\s+\w|std::vector|cudaMallocAsync|cudaMemPool\w*|cudaGraphInstantiate)\b"
    hits = re.findall(banned, text)
    assert not hits, hits


def test_wrapper_refuses_wrong_dtypes_before_the_call():
    import torch
    lp = gen.small_lp(0)
    rp = torch.tensor(lp.row_ptr, dtype=torch.int64)
    ci64 = torch.tensor(lp.col_idx, dtype=torch.int64)  # e.g. a torch sparse CSR's col_indices()
    va = torch.tensor(lp.val, dtype=torch.float64)
    with pytest.raises(ValueError, match="col_idx must have dtype"):
        lpx.lp_power_norm_noalloc(lp.m, lp.n, lp.nnz, rp, ci64, va)
    with pytest.raises(ValueError, match="row_ptr has"):
        lpx.lp_power_norm_noalloc(lp.m, lp.n, lp.nnz, rp[:-1], ci64.int(), va)


def _device_csr(lp):
    import torch
    return (torch.tensor(lp.row_ptr, dtype=torch.int64, device="cuda"),
            torch.tensor(lp.col_idx, dtype=torch.int32, device="cuda"),
            torch.tensor(lp.val, dtype=torch.float64, device="cuda"))


@pytest.mark.gpu
@pytest.mark.parametrize("make", [lambda: gen.small_lp(0), lambda: gen.miplib_like(0, 3000, 6000, 2000),
                                  lambda: gen.ragged_rows(1, 400, 900)])
def test_noalloc_power_norm_matches_lp_create_and_the_oracle(cuda_device, make):
    import torch
    import oracle
    lp = make()
    with lpx.Solver(lp, ruiz_iters=0, pc_enabled=0) as s:
        s.solve(0.0, 1)
        ref = s.result()["norm_A"]
    assert ref > 0.0
    orc, _ = oracle.power_norm(lp, tol=1e-7, max_iter=10000, seed=0)
    rp, ci, va = _device_csr(lp)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        norm, steps = lpx.lp_power_norm_noalloc(lp.m, lp.n, lp.nnz, rp, ci, va, 1e-7, 10000, 0, stream)
        assert steps >= 2
        assert norm == pytest.approx(ref, rel=1e-6), (call, norm, ref)
        assert norm == pytest.approx(orc, rel=1e-6), (call, norm, orc)


@pytest.mark.gpu
def test_noalloc_call_allocates_no_device_memory(cuda_device):
    import torch
    lp = gen.miplib_like(1, 3000, 6000, 2000)
    rp, ci, va = _device_csr(lp)
    stream = torch.cuda.current_stream().cuda_stream
    # the first call may load the library's device code (and with it the static array)
    lpx.lp_power_norm_noalloc(lp.m, lp.n, lp.nnz, rp, ci, va, 1e-7, 10000, 0, stream)
    torch.cuda.synchronize()
    stats0 = torch.cuda.memory_stats()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        lpx.lp_power_norm_noalloc(lp.m, lp.n, lp.nnz, rp, ci, va, 1e-7, 10000, 0, stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    stats1 = torch.cuda.memory_stats()
    assert free1 == free0, (free0, free1)
    for key in ("allocation.all.allocated", "segment.all.allocated", "reserved_bytes.all.allocated"):
        assert stats1.get(key, 0) == stats0.get(key, 0), key


@pytest.mark.gpu
def test_noalloc_iteration_cap_and_empty_matrix(cuda_device):
    import torch
    lp = gen.small_lp(2)
    rp, ci, va = _device_csr(lp)
    stream = torch.cuda.current_stream().cuda_stream
    norm, steps = lpx.lp_power_norm_noalloc(lp.m, lp.n, lp.nnz, rp, ci, va, 1e-7, 2, 0, stream)
    assert steps == 2 and norm > 0.0
    # 17 steps: one full batch of 16 plus one
    full, steps = lpx.lp_power_norm_noalloc(lp.m, lp.n, lp.nnz, rp, ci, va, 0.0, 17, 0, stream)
    orc, it = __import__("oracle").power_norm(lp, tol=0.0, max_iter=17, seed=0)
    assert it == steps == 17 and full == pytest.approx(orc, rel=1e-12)
    empty_rp = torch.zeros(lp.m + 1, dtype=torch.int64, device="cuda")
    assert lpx.lp_power_norm_noalloc(lp.m, lp.n, 0, empty_rp, None, None, 1e-7, 100, 0, stream) == (0.0, 0)


@pytest.mark.gpu
def test_noalloc_refuses_a_column_index_out_of_range(cuda_device):
    import torch
    lp = gen.small_lp(3)
    rp, ci, va = _device_csr(lp)
    bad = ci.clone()
    bad[lp.nnz // 2] = lp.n  # one past the last column: the kernels skip it and raise the flag
    stream = torch.cuda.current_stream().cuda_stream
    with pytest.raises(lpx.LPError) as e:
        lpx.lp_power_norm_noalloc(lp.m, lp.n, lp.nnz, rp, bad, va, 1e-7, 100, 0, stream)
    assert e.value.code == lpx.LP_ERR_INVALID_INPUT
    assert "out of range" in lpx.lp_last_error()
    # the scratch is still usable afterwards
    norm, _ = lpx.lp_power_norm_noalloc(lp.m, lp.n, lp.nnz, rp, ci, va, 1e-7, 10000, 0, stream)
    assert norm == pytest.approx(__import__("oracle").power_norm(lp)[0], rel=1e-6)
