"""GPU parity of fr_insert_batched (multi-batch launches over uneven batches).

Every batch's volume is compared with the FP64 oracle (2e-5 FP32, 2e-3 FP16
against the oracle fed the FP32 values), including a context that receives
two batches of one call (its units go through the scratch with atomics) and
an empty batch; graph capture and replay is checked by replaying a captured
call and comparing with twice the oracle; one call mixes every kind of
configuration (direct-drain gather groups of two shapes, the persistent
per-voxel gather with 4- and 6-wide boxes, and the batches run with their own
launches: scatter and tabulated weights); batches run with the configurations
loaded from a tuning cache; at the uneven-batch workload's own size
distribution (reduced in count) the batched path is compared with one
fr_insert per batch.
"""
import numpy as np
import pytest
import torch

from paper_1910_08498_gb300 import _lib as L
from paper_1910_08498_gb300 import inputs
from tests.helpers import A32, ALPHA, TOL_F16, TOL_F32, oracle_insert, rel_err, worst

pytestmark = pytest.mark.gpu


def _finalize(ctx, S):
    D = S + 1
    V = torch.empty(D ** 3, dtype=torch.complex64, device="cuda")
    W = torch.empty(D ** 3, dtype=torch.float32, device="cuda")
    L.fr_finalize(ctx, V, W)
    torch.cuda.synchronize()
    assert L.fr_last_device_error(ctx) == L.FR_OK
    return V.cpu().numpy().astype(np.complex128), W.cpu().numpy().astype(np.float64)


def _ctx(S, config=-1):
    ctx = L.fr_create(S, A32, ALPHA, 0, 10000)
    L.fr_set_options(ctx, tuning=0, forced_config=config)
    return ctx


@pytest.mark.parametrize("f16", [False, True])
@pytest.mark.parametrize("capture", [0, 1])
def test_batched_matches_oracle(f16, capture):
    # (S, n, seed, context slot): slot 2 receives two batches
    spec = [(32, 70, 51, 0), (48, 33, 52, 1), (16, 5, 53, 2), (64, 120, 54, 3), (16, 9, 55, 2),
            (24, 0, 56, 4), (40, 64, 57, 5)]
    S_of = {}
    for S, n, seed, slot in spec:
        S_of[slot] = S
    ctxs = {slot: _ctx(S) for slot, S in S_of.items()}
    try:
        host = [inputs.make_batch(S, n, seed) for S, n, seed, _ in spec]
        imgs = [(inputs.to_half(i) if f16 else i).cuda() for i, _ in host]
        rots = [r.cuda() for _, r in host]
        order = [ctxs[slot] for *_, slot in spec]
        L.fr_insert_batched(order, imgs, rots, capture=capture)
        reps = 1
        if capture:  # replay the captured graph once more
            L.fr_insert_batched(order, imgs, rots, capture=capture)
            reps = 2
        for slot, S in S_of.items():
            mine = [(i, r) for (i, r), (_, _, _, sl) in zip(host, spec) if sl == slot]
            Vr, Wr, _ = oracle_insert(S, mine)
            V, W = _finalize(ctxs[slot], S)
            tol = TOL_F16 if f16 else TOL_F32
            assert rel_err(V, reps * Vr) <= tol, (slot, rel_err(V, reps * Vr), worst(V, reps * Vr, S))
            assert rel_err(W, reps * Wr) <= TOL_F32, (slot, rel_err(W, reps * Wr), worst(W, reps * Wr, S))
    finally:
        for c in ctxs.values():
            L.fr_destroy(c)


def _config(pred):
    for i in range(L.fr_num_configs()):
        if pred(L.fr_describe_config(i)):
            return i
    raise AssertionError("no such configuration")


@pytest.mark.parametrize("f16", [False, True])
def test_batched_mixed_configurations(f16):
    g2a = _config(lambda d: d.startswith("gather2 bx=16 by=8 zc=8") and "warps=24" in d)
    g2b = _config(lambda d: d.startswith("gather2 bx=16 by=8 zc=16 chunk=32"))
    g2c = _config(lambda d: d.startswith("gather2 bx=16 by=16 zc=8") and "warps=16" in d)
    old_poly = _config(lambda d: d == "gather bx=16 by=8 zc=8 chunk=64 w=poly")
    old_lut = _config(lambda d: d == "gather bx=32 by=8 zc=4 chunk=32 w=lut")
    old_otf = _config(lambda d: d == "gather bx=16 by=16 zc=4 chunk=64 w=otf")
    scat = _config(lambda d: d.startswith("scatter threads=256 sub=256 w=poly"))
    # (S, n, seed, a, configuration, context slot); slot 1 receives two batches
    spec = [(32, 90, 61, A32, g2a, 0), (48, 70, 62, A32, g2b, 1), (16, 12, 63, A32, g2c, 2),
            (40, 60, 64, A32, old_poly, 3), (32, 50, 65, 2.5, -1, 4), (24, 40, 66, A32, scat, 5),
            (32, 45, 67, A32, old_lut, 6), (48, 21, 68, A32, g2b, 1), (24, 33, 69, A32, old_otf, 7),
            (64, 80, 70, A32, -1, 8)]
    ctxs = {}
    for S, n, seed, a, cfg, slot in spec:
        if slot not in ctxs:
            c = L.fr_create(S, float(np.float32(a)), ALPHA, 0, 10000)
            assert cfg < 0 or L.fr_config_valid(c, cfg)
            L.fr_set_options(c, tuning=0, forced_config=cfg)
            ctxs[slot] = (c, S, float(np.float32(a)))
    try:
        host = [inputs.make_batch(S, n, seed) for S, n, seed, *_ in spec]
        imgs = [(inputs.to_half(i) if f16 else i).cuda() for i, _ in host]
        rots = [r.cuda() for _, r in host]
        order = [ctxs[slot][0] for *_, slot in spec]
        L.fr_insert_batched(order, imgs, rots, capture=1)
        L.fr_insert_batched(order, imgs, rots, capture=1)  # graph replay
        for slot, (c, S, a) in ctxs.items():
            mine = [(i, r) for (i, r), sp in zip(host, spec) if sp[-1] == slot]
            Vr, Wr, _ = oracle_insert(S, mine, a=a, alpha=ALPHA)
            V, W = _finalize(c, S)
            tol = TOL_F16 if f16 else TOL_F32
            assert rel_err(V, 2 * Vr) <= tol, (slot, rel_err(V, 2 * Vr), worst(V, 2 * Vr, S))
            assert rel_err(W, 2 * Wr) <= TOL_F32, (slot, rel_err(W, 2 * Wr), worst(W, 2 * Wr, S))
    finally:
        for c, *_ in ctxs.values():
            L.fr_destroy(c)


def test_batched_runs_tuned_configurations(tmp_path):
    """A tuning cache measured on one context and loaded into others: the
    batched call runs each batch with the loaded best, and its volumes match
    one fr_insert per batch on contexts with the same cache."""
    S, n = 32, 200
    tun = L.fr_create(S, A32, ALPHA, 0, 10000)
    img, rot = inputs.make_batch(S, n, 71, device="cuda")
    try:
        for _ in range(200):
            L.fr_insert(tun, img, rot)
            if L.fr_tuning_report(tun)["tuned"]:
                break
        rep = L.fr_tuning_report(tun)
        assert rep["tuned"]
        path = str(tmp_path / "tune.json")
        L.fr_tuning_save(tun, path)
    finally:
        L.fr_destroy(tun)
    spec = [(S, n, 72), (S, n - 17, 73), (S, n + 30, 74)]
    bat, per = [], []
    try:
        data = [inputs.make_batch(S_, n_, seed, device="cuda") for S_, n_, seed in spec]
        for _ in spec:
            for lst in (bat, per):
                c = L.fr_create(S, A32, ALPHA, 0, 10000)
                L.fr_set_options(c, tuning=0)
                L.fr_tuning_load(c, path)
                lst.append(c)
        L.fr_insert_batched(bat, [d[0] for d in data], [d[1] for d in data], capture=0)
        for c, (i, r) in zip(per, data):
            L.fr_insert(c, i, r)
            assert L.fr_tuning_report(c)["last_config"] == rep["best_config"]
        for (S_, n_, seed), (i, r), c1, c2 in zip(spec, data, per, bat):
            V1, W1 = _finalize(c1, S)
            V2, W2 = _finalize(c2, S)
            assert rel_err(V2, V1) <= TOL_F32 and rel_err(W2, W1) <= TOL_F32
            Vr, Wr, _ = oracle_insert(S, [(i.cpu(), r.cpu())])
            assert rel_err(V2, Vr) <= TOL_F32 and rel_err(W2, Wr) <= TOL_F32
    finally:
        for c in bat + per:
            L.fr_destroy(c)


def test_batched_equals_per_batch_inserts_on_uneven_sizes():
    spec = inputs.uneven_batches(batches=6)
    # the workload's S choices and n range, fewer batches
    per, bat = [], []
    try:
        data = []
        for S, n, seed in spec:
            img, rot = inputs.make_batch(S, n, seed, device="cuda")
            data.append((S, img, rot))
            per.append(_ctx(S))
            bat.append(_ctx(S))
        for c, (S, img, rot) in zip(per, data):
            L.fr_insert(c, img, rot)
        L.fr_insert_batched(bat, [d[1] for d in data], [d[2] for d in data], capture=1)
        for (S, *_), c1, c2 in zip(data, per, bat):
            V1, W1 = _finalize(c1, S)
            V2, W2 = _finalize(c2, S)
            assert rel_err(V2, V1) <= TOL_F32 and rel_err(W2, W1) <= TOL_F32, (S, rel_err(V2, V1))
        # sampled voxels of the largest batch against the oracle, one by one
        k = max(range(len(data)), key=lambda i: data[i][0] * spec[i][1])
        S, img, rot = data[k]
        V2, W2 = _finalize(bat[k], S)
        rng = np.random.default_rng(7)
        H = S // 2
        coords = np.stack([rng.integers(-2, H + 1, 24), rng.integers(-H, H + 1, 24),
                           rng.integers(-H, H + 1, 24)], 1)
        coords[:4] = [[0, 0, 0], [1, 0, 0], [2, 3, -1], [H, H, H]]
        import oracle
        Vo, Wo = oracle.voxels(S, img.cpu().numpy(), rot.cpu().numpy(), coords, a=A32, alpha=ALPHA)
        D = S + 1
        idx = [((z + H) * D + (y + H)) * D + (x + H) for x, y, z in coords]
        scale_v = np.max(np.abs(V2))
        scale_w = np.max(np.abs(W2))
        assert np.max(np.abs(V2[idx] - Vo)) <= TOL_F32 * scale_v
        assert np.max(np.abs(W2[idx] - Wo)) <= TOL_F32 * scale_w
    finally:
        for c in per + bat:
            L.fr_destroy(c)
