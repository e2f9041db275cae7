"""GPU parity of the CUDA insertion path against the FP64 oracle (-m gpu).

Every comparison calls the library through its C ABI (ctypes) on seeded
inputs and checks max|X_gpu - X_ref| / max|X_ref| over the full grid against
2e-5 (FP32 images) or 2e-3 (FP16 images, against the oracle fed the original
FP32 values), for V and W; integer work (fold predicate, update count) is
compared bit-exactly.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1910_08498_gb300 import _lib as L
from paper_1910_08498_gb300 import inputs
from tests.helpers import (A32, ALPHA, TOL_F16, TOL_F32, gpu_insert, oracle_insert, rel_err,
                           sym_np, worst)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib_loaded():
    L.lib()


# ------------------------------------------------------------------ fold predicate

def test_fold_predicate_bit_exact():
    rng = np.random.default_rng(3)
    m = 200_000
    r = rng.standard_normal((m, 2)).astype(np.float32)
    k = np.stack([rng.integers(0, 257, m), rng.integers(-256, 257, m)], 1).astype(np.int32)
    # near-ties: r01 chosen so r00*kx + r01*ky is within a few ulps of zero
    t = 50_000
    kx = rng.integers(1, 257, t)
    ky = rng.integers(1, 257, t) * rng.choice([-1, 1], t)
    r00 = rng.standard_normal(t).astype(np.float32)
    r01 = (-(r00.astype(np.float64) * kx) / ky).astype(np.float32)
    r01 = np.nextafter(r01, np.where(rng.random(t) < 0.5, np.inf, -np.inf).astype(np.float32))
    r[:t, 0], r[:t, 1] = r00, r01
    k[:t, 0], k[:t, 1] = kx, ky
    # exact ties
    r[t:t + 4] = [[0.5, -0.25], [0.0, 1.0], [0.0, 0.0], [-0.75, 0.375]]
    k[t:t + 4] = [[2, 4], [3, 0], [5, 5], [1, 2]]
    out = torch.empty(m, dtype=torch.int32, device="cuda")
    L.fr_debug_fold(torch.from_numpy(r).cuda(), torch.from_numpy(k).cuda(), out)
    got = out.cpu().numpy()
    ref = ((r[:, 0].astype(np.float64) * k[:, 0] + r[:, 1].astype(np.float64) * k[:, 1]) < 0)
    assert np.array_equal(got.astype(bool), ref)
    for i in range(t, t + 4):
        assert bool(got[i]) == oracle.fold(float(r[i, 0]), float(r[i, 1]), int(k[i, 0]), int(k[i, 1]))


# ------------------------------------------------------------------ blob weights

@pytest.mark.parametrize("a,alpha,table", [(A32, ALPHA, 10000), (float(np.float32(2.5)), 15.0, 4096),
                                           (1.5, 10.0, 10000)])
def test_blob_table_and_on_the_fly(a, alpha, table):
    ctx = L.fr_create(32, a, alpha, 0, table)
    try:
        a2 = np.float32(a) * np.float32(a)
        r2 = np.linspace(0, a2, 20001, dtype=np.float32)
        r2_d = torch.from_numpy(r2).cuda()
        ref = np.array([oracle.blob_r2(float(x), a, alpha) for x in r2[::10]])
        for mode, tol in [(0, 3e-7 if table >= 10000 else 2e-6), (1, 1e-6), (2, 1e-6)]:
            out = torch.empty_like(r2_d)
            L.fr_debug_blob(ctx, r2_d, mode, out)
            got = out.cpu().numpy()[::10].astype(np.float64)
            assert np.max(np.abs(got - ref)) < tol, (mode, np.max(np.abs(got - ref)))
    finally:
        L.fr_destroy(ctx)


# ------------------------------------------------------------------ insertion parity

def small_batch():
    c = inputs.CONFIG_SMALL
    return inputs.make_batch(c["S"], c["n"], c["seed"])


@pytest.fixture(scope="module")
def small_ref():
    img, rot = small_batch()
    V, W, cnt = oracle_insert(32, [(img, rot)])
    return img, rot, V, W, cnt


def _num_configs():
    try:
        return L.fr_num_configs()
    except Exception:
        return 44


@pytest.mark.parametrize("cfg", list(range(_num_configs())))
def test_every_configuration_matches_oracle_S32(small_ref, cfg):
    img, rot, Vr, Wr, _ = small_ref
    V, W, _ = gpu_insert(32, [(img, rot)], config=cfg, tuning=False)
    assert rel_err(V, Vr) <= TOL_F32
    assert rel_err(W, Wr) <= TOL_F32
    Vs, Ws = sym_np(V, W, 32)
    Vsr, Wsr = sym_np(Vr, Wr, 32)
    assert rel_err(Vs, Vsr) <= TOL_F32 and rel_err(Ws, Wsr) <= TOL_F32


@pytest.fixture(scope="module")
def small_ref_f16(small_ref):
    img, rot, *_ = small_ref
    V16, W16, _ = oracle_insert(32, [(img, rot)], f16=True)
    return V16, W16


@pytest.mark.parametrize("cfg", list(range(_num_configs())))
def test_every_configuration_fp16_images_S32(small_ref, small_ref_f16, cfg):
    """FP16-stored images through every configuration: within 2e-3 of the
    oracle fed the FP32 values and within 2e-5 of the oracle fed the
    FP16-rounded values."""
    img, rot, Vr, Wr, _ = small_ref
    V16, W16 = small_ref_f16
    V, W, _ = gpu_insert(32, [(img, rot)], config=cfg, tuning=False, f16=True)
    assert rel_err(V, Vr) <= TOL_F16 and rel_err(W, Wr) <= TOL_F16
    assert rel_err(V, V16) <= TOL_F32 and rel_err(W, W16) <= TOL_F32


@pytest.fixture(scope="module")
def mid_ref():
    img, rot = inputs.make_batch(128, 48, 21)
    V, W, _ = oracle_insert(128, [(img, rot)])
    return img, rot, V, W


@pytest.mark.parametrize("cfg", list(range(_num_configs())))
def test_every_configuration_matches_oracle_S128(mid_ref, cfg):
    """Every configuration at S = 128 (bricks of every shape span many tiles
    and a ragged edge of the 129^3 volume), full grid against the oracle."""
    img, rot, Vr, Wr = mid_ref
    V, W, _ = gpu_insert(128, [(img, rot)], config=cfg, tuning=False)
    assert rel_err(V, Vr) <= TOL_F32, (cfg, rel_err(V, Vr), worst(V, Vr, 128))
    assert rel_err(W, Wr) <= TOL_F32, (cfg, rel_err(W, Wr), worst(W, Wr, 128))


def test_gather_is_deterministic(small_ref):
    """With no brick split over several units (fewer than 16 images: a split
    unit takes at least 8), every voxel is summed by one warp in a fixed
    order, with no atomics, so two runs agree bit for bit.  Split units add
    through float atomics, whose order (and last bits) may vary."""
    img, rot, *_ = small_ref
    img, rot = img[:15], rot[:15]
    for cfg in (1, L.fr_num_configs() - 6):  # a per-voxel and a direct-drain gather
        V1, W1, _ = gpu_insert(32, [(img, rot)], config=cfg, tuning=False)
        V2, W2, _ = gpu_insert(32, [(img, rot)], config=cfg, tuning=False)
        assert np.array_equal(V1, V2) and np.array_equal(W1, W2), cfg


@pytest.mark.parametrize("S,n,seed", [(8, 1, 5), (8, 7, 6), (16, 33, 7), (64, 37, 8), (96, 101, 9),
                                      (128, 257, 10)])
def test_ragged_sizes_default_and_scatter(S, n, seed):
    img, rot = inputs.make_batch(S, n, seed)
    Vr, Wr, _ = oracle_insert(S, [(img, rot)])
    for cfg in (-1, 37):  # tuner default path and a scatter configuration
        V, W, _ = gpu_insert(S, [(img, rot)], config=cfg, tuning=False)
        assert rel_err(V, Vr) <= TOL_F32, (cfg, rel_err(V, Vr), worst(V, Vr, S))
        assert rel_err(W, Wr) <= TOL_F32, (cfg, rel_err(W, Wr), worst(W, Wr, S))


def test_empty_batch_is_noop():
    img, rot = inputs.make_batch(16, 3, 1)
    ctx = L.fr_create(16)
    try:
        assert L.fr_insert(ctx, img.cuda(), rot.cuda(), n=0) == L.FR_OK
        D = 17
        V = torch.ones(D ** 3, dtype=torch.complex64, device="cuda")
        W = torch.ones(D ** 3, dtype=torch.float32, device="cuda")
        L.fr_finalize(ctx, V, W)
        assert torch.count_nonzero(W).item() == 0 and torch.count_nonzero(V).item() == 0
    finally:
        L.fr_destroy(ctx)


def test_identity_and_right_angle_rotations():
    S = 32
    img, _ = inputs.make_batch(S, 24, 12)
    P = inputs.proper_signed_permutations()
    Vr, Wr, _ = oracle_insert(S, [(img, P)])
    for cfg in (-1, 9, 39):
        V, W, _ = gpu_insert(S, [(img, P)], config=cfg, tuning=False)
        assert rel_err(V, Vr) <= TOL_F32 and rel_err(W, Wr) <= TOL_F32


@pytest.mark.parametrize("a,alpha", [(1.5, 10.0), (float(np.float32(2.5)), 15.0),
                                     (2.0, 12.0)])
def test_other_blob_radii(a, alpha):
    S = 48
    img, rot = inputs.make_batch(S, 40, 13)
    Vr, Wr, _ = oracle_insert(S, [(img, rot)], a=a, alpha=alpha)
    for cfg in (-1, 4, 20, 40):
        V, W, _ = gpu_insert(S, [(img, rot)], a=a, alpha=alpha, config=cfg, tuning=False)
        assert rel_err(V, Vr) <= TOL_F32, (cfg, rel_err(V, Vr), worst(V, Vr, S), worst(W, Wr, S))
        assert rel_err(W, Wr) <= TOL_F32, (cfg, rel_err(W, Wr), worst(W, Wr, S))


def test_fp16_images():
    S = 64
    img, rot = inputs.make_batch(S, 200, 14)
    Vr32, Wr32, _ = oracle_insert(S, [(img, rot)])
    Vr16, Wr16, _ = oracle_insert(S, [(img, rot)], f16=True)
    for cfg in (-1, 13, 26, 37):
        V, W, _ = gpu_insert(S, [(img, rot)], f16=True, config=cfg, tuning=False)
        assert rel_err(V, Vr32) <= TOL_F16 and rel_err(W, Wr32) <= TOL_F16
        assert rel_err(V, Vr16) <= TOL_F32 and rel_err(W, Wr16) <= TOL_F32


def test_n_copies_accumulation_stress():
    """1000 copies of one image at one rotation: V = 1000 V1; checks the
    compensated accumulation (a plain FP32 running sum drifts past 2e-5)."""
    S = 32
    img, rot = inputs.make_batch(S, 1, 15)
    n = 1000
    imgs = img.repeat(n, 1, 1)
    rots = rot.repeat(n, 1, 1)
    V1, W1, _ = oracle_insert(S, [(img, rot)])
    V, W, _ = gpu_insert(S, [(imgs, rots)], config=-1, tuning=False)
    assert rel_err(V, n * V1) <= TOL_F32 and rel_err(W, n * W1) <= TOL_F32


# ------------------------------------------------------------------ update count

@pytest.mark.parametrize("S,n,a", [(32, 64, A32), (64, 50, A32), (48, 20, 2.0), (40, 30, 1.5)])
def test_update_count_exact(S, n, a):
    _, rot = inputs.make_batch(S, n, 16)
    ctx = L.fr_create(S, a)
    try:
        got = L.fr_count_updates(ctx, rot.cuda())
    finally:
        L.fr_destroy(ctx)
    assert got == oracle.count(S, rot.numpy(), a=a)


# ------------------------------------------------------------------ non-blocking tuning

def test_tuning_steps_keep_every_image_once():
    """Config-2 style cold start: the tuner splits batches into sub-batches run
    with different configurations; the volume is still the oracle's."""
    S = 64
    batches = [inputs.make_batch(S, 120, 100 + b) for b in range(6)]
    Vr, Wr, _ = oracle_insert(S, batches)
    V, W, rep = gpu_insert(S, batches, tuning=True, steps=4)
    assert rel_err(V, Vr) <= TOL_F32 and rel_err(W, Wr) <= TOL_F32
    assert rep["evaluated"] >= 20
    assert rep["images"] == 720


def test_largest_blob_radius():
    """a just below 3 (the largest radius accepted; 6 x 6 candidate boxes with
    no spare cell) on every weight variant of the default shape and a scatter
    configuration."""
    S = 40
    a = float(np.float32(2.99))
    img, rot = inputs.make_batch(S, 50, 17)
    Vr, Wr, _ = oracle_insert(S, [(img, rot)], a=a, alpha=ALPHA)
    for cfg in (-1, 3, 4, 5, 41):
        V, W, _ = gpu_insert(S, [(img, rot)], a=a, alpha=ALPHA, config=cfg, tuning=False)
        assert rel_err(V, Vr) <= TOL_F32, (cfg, rel_err(V, Vr), worst(V, Vr, S))
        assert rel_err(W, Wr) <= TOL_F32, (cfg, rel_err(W, Wr), worst(W, Wr, S))


def test_invalid_arguments_leave_the_volume_untouched():
    S = 16
    img, rot = inputs.make_batch(S, 4, 18)
    ctx = L.fr_create(S)
    try:
        lib = L.lib()
        assert lib.fr_insert(ctx, L._ptr(img.cuda()), 7, L._ptr(rot.cuda()), 4, None) == L.FR_ERR_INVALID_ARG
        assert lib.fr_insert(ctx, None, 0, None, 4, None) == L.FR_ERR_INVALID_ARG
        assert lib.fr_insert(ctx, L._ptr(img.cuda()), 0, L._ptr(rot.cuda()), -1, None) == L.FR_ERR_INVALID_ARG
        D = S + 1
        V = torch.ones(D ** 3, dtype=torch.complex64, device="cuda")
        W = torch.ones(D ** 3, dtype=torch.float32, device="cuda")
        L.fr_finalize(ctx, V, W)
        torch.cuda.synchronize()
        assert torch.count_nonzero(W).item() == 0
    finally:
        L.fr_destroy(ctx)
