"""GPU parity of Algorithm 1's last step (fr_reconstruct: symmetrise, weight,
inverse FFT) against the FP64 reference oracle/recon.py.

(1) On the same raw sums: the GPU's own V, W (fr_finalize) fed to the FP64
reference.  Bar: 1e-5 of max|f| -- the inputs agree, the GPU adds hi + lo and
divides in FP32 (relative 1e-7) and runs an FP32 inverse FFT, whose error is
a few times 1e-7 of the RMS per output for these sizes.
(2) End to end from the images: oracle insertion + reference against the
GPU insertion + fr_reconstruct, bar 2e-5 of max|f| (the insertion's own bar).
"""
import numpy as np
import pytest
import torch

from oracle import recon
from paper_1910_08498_gb300 import _lib as L
from paper_1910_08498_gb300 import inputs
from tests.helpers import A32, ALPHA, oracle_insert

pytestmark = pytest.mark.gpu


def _run(S, batches, a, f16=False, w_clip=1.0):
    ctx = L.fr_create(S, a, ALPHA, 0, 10000)
    try:
        L.fr_set_options(ctx, tuning=0, forced_config=-1)
        for img, rot in batches:
            L.fr_insert(ctx, (inputs.to_half(img) if f16 else img).cuda(), rot.cuda())
        D = S + 1
        V = torch.empty(D ** 3, dtype=torch.complex64, device="cuda")
        W = torch.empty(D ** 3, dtype=torch.float32, device="cuda")
        L.fr_finalize(ctx, V, W)
        out = torch.empty(S ** 3, dtype=torch.float32, device="cuda")
        L.fr_reconstruct(ctx, out, w_clip)
        torch.cuda.synchronize()
        return (V.cpu().numpy(), W.cpu().numpy(),
                out.cpu().numpy().astype(np.float64).reshape(S, S, S))
    finally:
        L.fr_destroy(ctx)


@pytest.mark.parametrize("S,n,a,w_clip", [(32, 64, A32, 1.0), (48, 40, 2.5, 1.0), (32, 30, A32, 0.05)])
def test_reconstruct_matches_reference_on_same_sums(S, n, a, w_clip):
    batch = inputs.make_batch(S, n, 90 + S)
    V, W, f = _run(S, [batch], a, w_clip=w_clip)
    ref = recon.reconstruct(S, V.astype(np.complex128), W.astype(np.float64), w_clip)
    err = np.max(np.abs(f - ref)) / np.max(np.abs(ref))
    assert err <= 1e-5, err


@pytest.mark.parametrize("f16", [False, True])
def test_reconstruct_end_to_end(f16):
    S = 32
    batches = [inputs.make_batch(S, 50, 95 + b) for b in range(2)]
    _, _, f = _run(S, batches, A32, f16=f16)
    Vr, Wr, _ = oracle_insert(S, batches, f16=f16)
    ref = recon.reconstruct(S, Vr, Wr, 1.0)
    err = np.max(np.abs(f - ref)) / np.max(np.abs(ref))
    assert err <= 2e-5, err


def test_reconstruct_rejects_bad_clip():
    ctx = L.fr_create(16)
    try:
        out = torch.empty(16 ** 3, dtype=torch.float32, device="cuda")
        assert L.lib().fr_reconstruct(ctx, L._ptr(out), 0.0, None) == L.FR_ERR_INVALID_ARG
    finally:
        L.fr_destroy(ctx)
