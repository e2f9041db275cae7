"""Parity at the benchmark's full size (S = 256, one batch of 5000 FP32
images, the launch configurations bench.py times), on sampled voxels the
oracle computes one by one (brute force over every pixel of every image),
plus properties that hold at any size."""
import numpy as np
import pytest
import torch

import oracle
from paper_1910_08498_gb300 import _lib as L
from paper_1910_08498_gb300 import inputs
from tests.helpers import A32, ALPHA, TOL_F32

pytestmark = pytest.mark.gpu

S, N = 256, 5000


@pytest.fixture(scope="module")
def batch():
    c = inputs.CONFIG_LARGE
    img, rot = inputs.make_batch(S, N, c["seed"] * 1000)
    return img, rot


@pytest.fixture(scope="module")
def samples(batch):
    img, rot = batch
    H = S // 2
    rng = np.random.default_rng(11)
    pts = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, -1), (2, -3, 1), (-2, 5, 7), (H, H, H),
           (H, -H, 0), (0, H, -H), (-1, -H, H), (40, -60, 17), (100, 3, -90)]
    # near the centre (many planes), in the fold columns, and random
    pts += [tuple(int(v) for v in rng.integers(-6, 7, 3)) for _ in range(8)]
    pts += [(int(rng.integers(-2, 2)), int(rng.integers(-H, H + 1)), int(rng.integers(-H, H + 1)))
            for _ in range(6)]
    pts += [(int(rng.integers(-2, H + 1)), int(rng.integers(-H, H + 1)), int(rng.integers(-H, H + 1)))
            for _ in range(14)]
    pts = [p for p in pts if p[0] >= -2]
    Vo, Wo = oracle.voxels(S, img.numpy(), rot.numpy(), pts, a=A32, alpha=ALPHA)
    return np.array(pts), Vo, Wo


def _first_gather2():
    try:
        return next(c for c in range(L.fr_num_configs())
                    if L.fr_describe_config(c).startswith("gather2 "))
    except Exception:
        return 44


@pytest.mark.parametrize("cfg", [13, 4, 43, _first_gather2(), _first_gather2() + 5])
def test_full_size_sampled_voxels(batch, samples, cfg):
    img, rot = batch
    pts, Vo, Wo = samples
    ctx = L.fr_create(S, A32, ALPHA, 0, 10000)
    try:
        if not L.fr_config_valid(ctx, cfg):
            pytest.skip("configuration not valid here")
        L.fr_set_options(ctx, tuning=0, forced_config=cfg)
        L.fr_insert(ctx, img.cuda(), rot.cuda())
        D = S + 1
        V = torch.empty(D ** 3, dtype=torch.complex64, device="cuda")
        W = torch.empty(D ** 3, dtype=torch.float32, device="cuda")
        L.fr_finalize(ctx, V, W)
        torch.cuda.synchronize()
        assert L.fr_last_device_error(ctx) == L.FR_OK
        # properties at full size: voxels x < -floor(a) untouched, W >= 0,
        # total weight positive and finite
        H = S // 2
        Wg = W.view(D, D, D)
        assert torch.count_nonzero(Wg[:, :, : H - 1]).item() == 0
        assert torch.all(Wg >= 0).item() and torch.isfinite(V).all().item()
        scale_v = V.abs().max().item()
        scale_w = W.max().item()
        idx = torch.tensor([((z + H) * D + (y + H)) * D + (x + H) for x, y, z in pts])
        Vg = V[idx.cuda()].cpu().numpy().astype(np.complex128)
        Wg = W[idx.cuda()].cpu().numpy().astype(np.float64)
    finally:
        L.fr_destroy(ctx)
    ev = np.abs(Vg - Vo) / scale_v
    ew = np.abs(Wg - Wo) / scale_w
    assert ev.max() <= TOL_F32, (cfg, ev.max(), pts[int(ev.argmax())])
    assert ew.max() <= TOL_F32, (cfg, ew.max(), pts[int(ew.argmax())])


@pytest.mark.parametrize("cfg", [-1, 41])
def test_largest_image_size_sampled_voxels(cfg):
    """S = 512, the largest size the library accepts (default gather and a
    scatter configuration), on sampled voxels computed one by one."""
    S2, n2 = 512, 120
    img, rot = inputs.make_batch(S2, n2, 512)
    H = S2 // 2
    rng = np.random.default_rng(12)
    pts = [(0, 0, 0), (1, 0, 0), (H, H, H), (-1, -H, H), (200, -100, 50)]
    pts += [tuple(int(v) for v in rng.integers(-4, 5, 3)) for _ in range(6)]
    pts += [(int(rng.integers(-1, H + 1)), int(rng.integers(-H, H + 1)), int(rng.integers(-H, H + 1)))
            for _ in range(9)]
    Vo, Wo = oracle.voxels(S2, img.numpy(), rot.numpy(), pts, a=A32, alpha=ALPHA)
    ctx = L.fr_create(S2, A32, ALPHA, 0, 10000)
    try:
        if cfg >= 0 and not L.fr_config_valid(ctx, cfg):
            pytest.skip("configuration not valid here")
        L.fr_set_options(ctx, tuning=0, forced_config=cfg)
        L.fr_insert(ctx, img.cuda(), rot.cuda())
        D = S2 + 1
        V = torch.empty(D ** 3, dtype=torch.complex64, device="cuda")
        W = torch.empty(D ** 3, dtype=torch.float32, device="cuda")
        L.fr_finalize(ctx, V, W)
        torch.cuda.synchronize()
        assert L.fr_last_device_error(ctx) == L.FR_OK
        scale_v, scale_w = V.abs().max().item(), W.max().item()
        idx = torch.tensor([((z + H) * D + (y + H)) * D + (x + H) for x, y, z in pts]).cuda()
        Vg = V[idx].cpu().numpy().astype(np.complex128)
        Wg = W[idx].cpu().numpy().astype(np.float64)
    finally:
        L.fr_destroy(ctx)
    assert np.max(np.abs(Vg - Vo)) <= TOL_F32 * scale_v
    assert np.max(np.abs(Wg - Wo)) <= TOL_F32 * scale_w


@pytest.mark.parametrize("cfg", [13, -1])
def test_full_size_whole_grid_small_batch(cfg):
    """S = 256 with a small batch (40 images): the whole 257^3 grid against
    the oracle, including the total weight (the sum of the inserted pixels'
    clipped blob masses, which the oracle's W sums to)."""
    n = 40
    img, rot = inputs.make_batch(S, n, 4242)
    Vr, Wr, _ = oracle.insert(S, img.numpy(), rot.numpy(), a=A32, alpha=ALPHA)
    ctx = L.fr_create(S, A32, ALPHA, 0, 10000)
    try:
        if cfg >= 0 and not L.fr_config_valid(ctx, cfg):
            pytest.skip("configuration not valid here")
        L.fr_set_options(ctx, tuning=0, forced_config=cfg)
        L.fr_insert(ctx, img.cuda(), rot.cuda())
        D = S + 1
        V = torch.empty(D ** 3, dtype=torch.complex64, device="cuda")
        W = torch.empty(D ** 3, dtype=torch.float32, device="cuda")
        L.fr_finalize(ctx, V, W)
        torch.cuda.synchronize()
        assert L.fr_last_device_error(ctx) == L.FR_OK
        Vg = V.cpu().numpy().astype(np.complex128)
        Wg = W.cpu().numpy().astype(np.float64)
    finally:
        L.fr_destroy(ctx)
    assert np.max(np.abs(Vg - Vr)) <= TOL_F32 * np.max(np.abs(Vr))
    assert np.max(np.abs(Wg - Wr)) <= TOL_F32 * np.max(np.abs(Wr))
    assert abs(Wg.sum() - Wr.sum()) <= 1e-5 * Wr.sum()


def test_large_reconstruction_scale_sampled_voxels():
    """The large-reconstruction scale: 20 batches of 5000 S = 256 FP32 images
    (100,000 images, about a million terms in a voxel at the centre) into one
    context with the tuned-space default, against the oracle on sampled
    voxels, accumulated batch by batch; the double-float accumulators keep
    the error at the one-batch level."""
    S2, nb, n = 256, 20, 5000
    H = S2 // 2
    c = inputs.CONFIG_LARGE
    rng = np.random.default_rng(13)
    pts = [(0, 0, 0), (1, 0, 0), (0, 1, 1), (-1, 2, -1), (3, -2, 0)]
    pts += [(int(rng.integers(-1, H + 1)), int(rng.integers(-H, H + 1)), int(rng.integers(-H, H + 1)))
            for _ in range(5)]
    Vo = np.zeros(len(pts), dtype=np.complex128)
    Wo = np.zeros(len(pts), dtype=np.float64)
    ctx = L.fr_create(S2, A32, ALPHA, 0, 10000)
    try:
        L.fr_set_options(ctx, tuning=0, forced_config=-1)
        for b in range(nb):
            img, rot = inputs.make_batch(S2, n, c["seed"] * 1000 + 7000 + b, device="cuda")
            L.fr_insert(ctx, img, rot)
            v, w = oracle.voxels(S2, img.cpu().numpy(), rot.cpu().numpy(), pts, a=A32, alpha=ALPHA)
            Vo += v
            Wo += w
            del img, rot
        D = S2 + 1
        V = torch.empty(D ** 3, dtype=torch.complex64, device="cuda")
        W = torch.empty(D ** 3, dtype=torch.float32, device="cuda")
        L.fr_finalize(ctx, V, W)
        torch.cuda.synchronize()
        assert L.fr_last_device_error(ctx) == L.FR_OK
        scale_v, scale_w = V.abs().max().item(), W.max().item()
        idx = torch.tensor([((z + H) * D + (y + H)) * D + (x + H) for x, y, z in pts]).cuda()
        Vg = V[idx].cpu().numpy().astype(np.complex128)
        Wg = W[idx].cpu().numpy().astype(np.float64)
    finally:
        L.fr_destroy(ctx)
    assert Wo[0] > 1e5  # the centre voxel sums about a million blob terms
    assert np.max(np.abs(Vg - Vo)) <= TOL_F32 * scale_v, np.max(np.abs(Vg - Vo)) / scale_v
    assert np.max(np.abs(Wg - Wo)) <= TOL_F32 * scale_w, np.max(np.abs(Wg - Wo)) / scale_w
