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
    batches = [inputs.make_batch(S, 80, 120 + b) for b in range(14)]
    Vr, Wr, _ = oracle_insert(S, batches)
    bad = 7  # a gather configuration of the exhaustive order
    ctx = L.fr_create(S)
    try:
        L.fr_set_options(ctx, tuning=1, search=L.FR_SEARCH_EXHAUSTIVE, steps_per_insert=4,
                         fault_config=bad + 1)
        statuses = [L.fr_insert(ctx, img.cuda(), rot.cuda()) for img, rot in batches]
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
    S = 48
    batches = [[t.cuda() for t in inputs.make_batch(S, 60, 130 + b)] for b in range(4)]
    full = L.fr_create(S)
    first = L.fr_create(S)
    second = L.fr_create(S)
    try:
        for c in (full, first, second):
            L.fr_set_options(c, tuning=0, forced_config=-1)
        for img, rot in batches:
            L.fr_insert(full, img, rot)
        for img, rot in batches[:2]:
            L.fr_insert(first, img, rot)
        nbytes = L.fr_state_bytes(first)
        assert nbytes == 6 * 4 * (S + 1) ** 2 * (S // 2 + 1 + 1)  # x from -floor(a) = -1 to S/2
        buf = torch.empty(nbytes // 4, dtype=torch.float32, device=where)
        L.fr_state_save(first, buf)
        L.fr_state_load(second, buf)
        for img, rot in batches[2:]:
            L.fr_insert(second, img, rot)
        V1, W1 = _finalize(full, S)
        V2, W2 = _finalize(second, S)
    finally:
        for c in (full, first, second):
            L.fr_destroy(c)
    assert np.array_equal(V1, V2) and np.array_equal(W1, W2)
