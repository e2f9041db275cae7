"""GPU parity of fr_insert_batched (persistent gather over uneven batches).

Every batch's volume is compared with the FP64 oracle (2e-5 FP32, 2e-3 FP16
against the oracle fed the FP32 values), including a context that receives
two batches of one call (its units go through the scratch with atomics) and
an empty batch; graph capture and replay is checked by replaying a captured
call and comparing with twice the oracle; at the uneven-batch workload's own
size distribution (reduced in count) the persistent path is compared with
one fr_insert per batch.
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
