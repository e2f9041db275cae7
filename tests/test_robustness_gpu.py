"""Failure handling and checkpoint/resume on the GPU, with faults injected on
the host only (no device fault, trap or hang):

* a configuration whose launch fails (fr_options.fault_config) is marked
  invalid, its sub-batch is re-run with the default configuration and the
  call reports FR_ERR_LAUNCH; the volume is still the oracle's and tuning
  finishes without it;
* the accumulator state saved from one context and loaded into another
  resumes the insertion: the result is bitwise that of one uninterrupted run.
"""
import numpy as np
import pytest
import torch

from oracle import gemm
from paper_1910_08498_gb300 import _lib as L
from paper_1910_08498_gb300 import inputs
from tests.helpers import TOL_F32, oracle_insert, rel_err

pytestmark = pytest.mark.gpu


def _finalize(ctx, S):
    D = S + 1
    V = torch.empty(D ** 3, dtype=torch.complex64, device="cuda")
    W = torch.empty(D ** 3, dtype=torch.float32, device="cuda")
    L.fr_finalize(ctx, V, W)
    torch.cuda.synchronize()
    return V.cpu().numpy(), W.cpu().numpy()


def test_injected_launch_failure_falls_back():
    S = 32
    # enough tuning steps (4 per insert) to measure every configuration of the space
    batches = [inputs.make_batch(S, 80, 120 + b) for b in range(20)]
    Vr, Wr, _ = oracle_insert(S, batches)
    bad = 7  # a gather configuration of the exhaustive order
    ctx = L.fr_create(S)
    try:
        L.fr_set_options(ctx, tuning=1, search=L.FR_SEARCH_EXHAUSTIVE, steps_per_insert=4,
                         fault_config=bad + 1)
        statuses = [L.fr_insert(ctx, img.cuda(), rot.cuda()) for img, rot in batches]
        torch.cuda.synchronize()
        rep = L.fr_tuning_report(ctx)
        measured = {c for c, _, _ in L.fr_tuning_measurements(ctx)}
        V, W = _finalize(ctx, S)
    finally:
        L.fr_destroy(ctx)
    assert statuses.count(L.FR_ERR_LAUNCH) == 1 and all(s in (L.FR_OK, L.FR_ERR_LAUNCH) for s in statuses)
    assert bad not in measured and rep["tuned"] == 1 and rep["best_config"] != bad
    assert rel_err(V.astype(np.complex128), Vr) <= TOL_F32
    assert rel_err(W.astype(np.float64), Wr) <= TOL_F32


def test_fault_config_out_of_range_is_rejected():
    ctx = L.fr_create(16)
    try:
        with pytest.raises(L.FrError):
            L.fr_set_options(ctx, fault_config=L.fr_num_configs() + 1)
    finally:
        L.fr_destroy(ctx)


@pytest.mark.parametrize("where", ["cpu", "cuda"])
def test_checkpoint_resume_is_bitwise(where):
    """Save after two inserts, load into a new context, insert the rest: the
    volume equals the uninterrupted one bit for bit.  Batches of 15 images:
    no brick is split over several units (a split unit takes at least 8
    images), so every voxel is summed in a fixed order."""
    S = 48
    batches = [[t.cuda() for t in inputs.make_batch(S, 15, 130 + b)] for b in range(6)]
    full = L.fr_create(S)
    first = L.fr_create(S)
    second = L.fr_create(S)
    try:
        for c in (full, first, second):
            L.fr_set_options(c, tuning=0, forced_config=-1)
        for img, rot in batches:
            L.fr_insert(full, img, rot)
        for img, rot in batches[:3]:
            L.fr_insert(first, img, rot)
        nbytes = L.fr_state_bytes(first)
        assert nbytes == 6 * 4 * (S + 1) ** 2 * (S // 2 + 1 + 1)  # x from -floor(a) = -1 to S/2
        buf = torch.empty(nbytes // 4, dtype=torch.float32, device=where)
        L.fr_state_save(first, buf)
        L.fr_state_load(second, buf)
        for img, rot in batches[3:]:
            L.fr_insert(second, img, rot)
        V1, W1 = _finalize(full, S)
        V2, W2 = _finalize(second, S)
    finally:
        for c in (full, first, second):
            L.fr_destroy(c)
    assert np.array_equal(V1, V2) and np.array_equal(W1, W2)


@pytest.mark.parametrize("family", ["scatter", "gather"])
def test_injected_allocation_failure_falls_back(family):
    """fr_options.fault_alloc = 1: the first device allocation of the insertion
    path (the scatter's scratch, or the gather's work-unit list) fails as out of
    memory; the step is redone with the default configuration (FR_ERR_LAUNCH),
    every image is inserted once, and the hook disarms itself."""
    S = 32
    batches = [inputs.make_batch(S, 90, 150 + b) for b in range(2)]
    Vr, Wr, _ = oracle_insert(S, batches)
    ctx = L.fr_create(S)
    try:
        cfg = next(i for i in range(L.fr_num_configs())
                   if L.fr_describe_config(i).startswith(family) and L.fr_config_valid(ctx, i))
        L.fr_set_options(ctx, tuning=0, forced_config=cfg, fault_alloc=1)
        s1 = L.fr_insert(ctx, *[t.cuda() for t in batches[0]])
        s2 = L.fr_insert(ctx, *[t.cuda() for t in batches[1]])
        armed = L.fr_get_options(ctx).fault_alloc
        V, W = _finalize(ctx, S)
    finally:
        L.fr_destroy(ctx)
    assert s1 == L.FR_ERR_LAUNCH and s2 == L.FR_OK and armed == 0
    assert rel_err(V.astype(np.complex128), Vr) <= TOL_F32
    assert rel_err(W.astype(np.float64), Wr) <= TOL_F32


def test_nvtx_ranges_leave_results_unchanged():
    """fr_options.debug bit 2 (an NVTX range per insertion step) changes no result."""
    S = 32
    batches = [inputs.make_batch(S, 70, 160 + b) for b in range(3)]
    Vr, Wr, _ = oracle_insert(S, batches)
    ctx = L.fr_create(S)
    try:
        L.fr_set_options(ctx, debug=4)
        st = [L.fr_insert(ctx, *[t.cuda() for t in b]) for b in batches]
        V, W = _finalize(ctx, S)
    finally:
        L.fr_destroy(ctx)
    assert all(s == L.FR_OK for s in st)
    assert rel_err(V.astype(np.complex128), Vr) <= TOL_F32
    assert rel_err(W.astype(np.float64), Wr) <= TOL_F32


def test_bulk_gemm_wait_timeout_is_reported_and_recovers():
    """fr_gemm_set_wait_limit(0): the bulk-copy kernel's waits give up at once;
    the launch reports FR_ERR_TIMEOUT through the status word, ends (after
    letting its copies in flight land), and the next launch with the default
    limit computes every instance."""
    m, n, k, batch = 8, 8, 8, 200000
    g = torch.Generator(device="cuda").manual_seed(3)
    A = torch.randn(batch, m, k, device="cuda", generator=g)
    B = torch.randn(batch, k, n, device="cuda", generator=g)
    C = torch.empty(batch, m, n, device="cuda")
    cfg = next(i for i in range(L.fr_gemm_num_configs())
               if "bulk" in L.fr_gemm_describe_config(i) and L.fr_gemm_config_valid(i, m, n, k))
    assert L.fr_gemm_device_status() == L.FR_OK
    L.fr_gemm_set_wait_limit(0)
    try:
        L.fr_gemm_run_config(cfg, A, B, C)
        torch.cuda.synchronize()
        status = L.fr_gemm_device_status()
    finally:
        L.fr_gemm_set_wait_limit(1_000_000_000)
    assert status == L.FR_ERR_TIMEOUT
    assert L.fr_gemm_device_status() == L.FR_OK  # read once, cleared
    C.fill_(float("nan"))
    L.fr_gemm_run_config(cfg, A, B, C)
    torch.cuda.synchronize()
    assert L.fr_gemm_device_status() == L.FR_OK
    idx = torch.arange(0, batch, 331)
    As, Bs = A[idx].cpu().numpy(), B[idx].cpu().numpy()
    err = np.abs(C[idx].cpu().numpy().astype(np.float64) - gemm.bgemm(As, Bs))
    assert np.all(err <= gemm.fp32_error_bound(As, Bs) + 1e-30)
