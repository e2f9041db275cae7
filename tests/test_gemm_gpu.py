"""Batched small-matrix GEMM on the GPU (the dynamic-tuning workload of
Sec. 5.2): every configuration against the FP64 reference within the FP32
error bound gamma_k sum |a||b|, and the non-blocking tuner under size
changes -- every instance computed once per call whatever the tuning state,
the stop rule (budget, or a configuration reaching a bandwidth target), and
a return to a size reusing its result."""
import numpy as np
import pytest
import torch

from oracle import gemm
from paper_1910_08498_gb300 import _lib as L

pytestmark = pytest.mark.gpu

SIZES = [(2, 2, 2), (3, 5, 7), (16, 16, 16), (32, 32, 32), (32, 2, 17), (5, 31, 3), (9, 12, 32)]


def _data(m, n, k, batch, seed):
    g = torch.Generator().manual_seed(seed)
    A = torch.randn(batch, m, k, generator=g)
    B = torch.randn(batch, k, n, generator=g)
    return A, B


def _check(C, A, B):
    ref = gemm.bgemm(A.numpy(), B.numpy())
    bound = gemm.fp32_error_bound(A.numpy(), B.numpy())
    err = np.abs(C.cpu().numpy().astype(np.float64) - ref)
    assert np.all(err <= bound + 1e-30), float(np.max(err / (bound + 1e-30)))


@pytest.mark.parametrize("m,n,k", SIZES)
def test_every_configuration(m, n, k):
    A, B = _data(m, n, k, 257, m * 100 + n * 10 + k)
    Ad, Bd = A.cuda(), B.cuda()
    ran = 0
    for cfg in range(L.fr_gemm_num_configs()):
        if not L.fr_gemm_config_valid(cfg, m, n, k):
            continue
        C = torch.full((257, m, n), float("nan"), device="cuda")
        L.fr_gemm_run_config(cfg, Ad, Bd, C)
        torch.cuda.synchronize()
        _check(C, A, B)
        ran += 1
    assert ran >= 4


def test_dynamic_tuning_under_size_changes():
    ctx = L.fr_gemm_create()
    try:
        L.fr_gemm_set_tuning(ctx, tuning=1, search=L.FR_SEARCH_RANDOM, budget=6, steps=2)
        plan = [(16, 16, 16)] * 4 + [(5, 31, 3)] * 4 + [(16, 16, 16)] * 2
        for it, (m, n, k) in enumerate(plan):
            A, B = _data(m, n, k, 1000 + it, it)
            C = torch.full((1000 + it, m, n), float("nan"), device="cuda")
            L.fr_gemm_run(ctx, A.cuda(), B.cuda(), C)
            torch.cuda.synchronize()
            _check(C, A, B)  # every instance, whatever configuration computed it
        r1 = L.fr_gemm_report(ctx, 16, 16, 16)
        r2 = L.fr_gemm_report(ctx, 5, 31, 3)
        assert r1["tuned"] == 1 and r1["evaluated"] == 6 and r1["best"] >= 0 and r1["best_gbs"] > 0
        assert r2["tuned"] == 1 and r2["evaluated"] == 6
    finally:
        L.fr_gemm_destroy(ctx)


@pytest.mark.parametrize("search", [L.FR_SEARCH_ANNEALING, L.FR_SEARCH_MCMC, L.FR_SEARCH_EXHAUSTIVE])
def test_stop_rule_bandwidth_target(search):
    ctx = L.fr_gemm_create()
    try:
        # a target every configuration reaches: the search stops after the first call's steps
        L.fr_gemm_set_tuning(ctx, tuning=1, search=search, budget=20, steps=2, bw_gbs=1e-3, bw_frac=0.75)
        A, B = _data(8, 8, 8, 4096, 5)
        C = torch.empty(4096, 8, 8, device="cuda")
        for _ in range(3):
            L.fr_gemm_run(ctx, A.cuda(), B.cuda(), C)
            torch.cuda.synchronize()
        r = L.fr_gemm_report(ctx, 8, 8, 8)
        assert r["tuned"] == 1 and r["evaluated"] == 2
        _check(C, A, B)
    finally:
        L.fr_gemm_destroy(ctx)


def _bulk_configs(m, n, k):
    return [c for c in range(L.fr_gemm_num_configs())
            if "bulk" in L.fr_gemm_describe_config(c) and L.fr_gemm_config_valid(c, m, n, k)]


@pytest.mark.parametrize("m,n,k", [(2, 2, 2), (3, 5, 7), (9, 12, 32), (31, 30, 29)])
@pytest.mark.parametrize("off", [1, 2, 3])
def test_bulk_copies_at_unaligned_offsets(m, n, k, off):
    """Blocks that start at any 4-byte offset: the bulk-copy kernels move the
    16-byte aligned interior and the ragged ends separately; nothing outside
    the caller's C range is written."""
    batch = 389
    A, B = _data(m, n, k, batch + off, 7 * m + n + k + off)
    Ad, Bd = A.cuda(), B.cuda()
    cfgs = _bulk_configs(m, n, k)
    assert cfgs
    for cfg in cfgs:
        Cfull = torch.full((batch + off + 1, m, n), float("nan"), device="cuda")
        L.fr_gemm_run_config(cfg, Ad[off:], Bd[off:], Cfull[off:off + batch])
        torch.cuda.synchronize()
        _check(Cfull[off:off + batch], A[off:], B[off:])
        assert torch.isnan(Cfull[:off]).all() and torch.isnan(Cfull[off + batch:]).all(), \
            L.fr_gemm_describe_config(cfg)
    assert L.fr_gemm_device_status() == L.FR_OK


@pytest.mark.parametrize("batch", [1, 2, 3, 5, 4099])
def test_bulk_copies_ragged_batches(batch):
    """Batches from one instance up to many groups per CTA (the last group partial)."""
    m, n, k = 7, 3, 5
    A, B = _data(m, n, k, batch, batch)
    Ad, Bd = A.cuda(), B.cuda()
    for cfg in _bulk_configs(m, n, k):
        C = torch.full((batch, m, n), float("nan"), device="cuda")
        L.fr_gemm_run_config(cfg, Ad, Bd, C)
        torch.cuda.synchronize()
        _check(C, A, B)
    assert L.fr_gemm_device_status() == L.FR_OK


@pytest.mark.parametrize("m,n,k", [(23, 22, 21), (6, 14, 2)])
def test_full_size_batch_sampled_instances(m, n, k):
    """The batch size the study times (about 512 MB of matrices): every bulk
    configuration, and the tuner, checked on sampled instances."""
    per = 4 * (m * k + k * n + m * n)
    batch = int(512e6 // per)
    g = torch.Generator(device="cuda").manual_seed(m * n * k)
    Ad = torch.randn(batch, m, k, device="cuda", generator=g)
    Bd = torch.randn(batch, k, n, device="cuda", generator=g)
    idx = torch.arange(0, batch, 997)
    idx = torch.cat([idx, torch.tensor([batch - 1])])
    As, Bs = Ad[idx].cpu(), Bd[idx].cpu()
    C = torch.empty(batch, m, n, device="cuda")
    for cfg in _bulk_configs(m, n, k):
        C.fill_(float("nan"))
        L.fr_gemm_run_config(cfg, Ad, Bd, C)
        torch.cuda.synchronize()
        _check(C[idx], As, Bs)
        assert not torch.isnan(C).any(), L.fr_gemm_describe_config(cfg)
    ctx = L.fr_gemm_create()
    try:
        L.fr_gemm_set_tuning(ctx, tuning=1, search=L.FR_SEARCH_RANDOM, budget=20, steps=2)
        for _ in range(12):
            C.fill_(float("nan"))
            L.fr_gemm_run(ctx, Ad, Bd, C)
        torch.cuda.synchronize()
        _check(C[idx], As, Bs)
        assert not torch.isnan(C).any()
        assert L.fr_gemm_report(ctx, m, n, k)["tuned"] == 1
    finally:
        L.fr_gemm_destroy(ctx)
    assert L.fr_gemm_device_status() == L.FR_OK
