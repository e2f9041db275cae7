"""GPU parity of the image-side step (fr_prepare_images: batched 2D R2C
transforms staged into the insertion input) against the FP64 numpy
reference oracle/recon.image_spectra.

Bars: FP32 output within 1e-5 of max|F| (an FP32 FFT of S^2 points errs by a
few times 1e-7 of the RMS); FP16 output within half an FP16 ulp of the FP64
value plus the FP32 FFT error; end to end, images transformed on the GPU and
inserted match the oracle insertion of the FP64 spectra within 2e-5."""
import numpy as np
import pytest
import torch

from oracle import recon
from paper_1910_08498_gb300 import _lib as L
from paper_1910_08498_gb300 import inputs
from tests.helpers import TOL_F32, oracle_insert, rel_err

pytestmark = pytest.mark.gpu


def _real(S, n, seed):
    g = torch.Generator().manual_seed(seed)
    return torch.randn(n, S, S, generator=g, dtype=torch.float32)


@pytest.mark.parametrize("S,n,center", [(32, 300, False), (32, 300, True), (48, 257, True), (64, 5, False),
                                         (30, 301, True), (14, 9, True)])
def test_prepare_fp32(S, n, center):
    real = _real(S, n, S + n)
    ctx = L.fr_create(S)
    try:
        out = torch.empty(n, S, S // 2 + 1, dtype=torch.complex64, device="cuda")
        L.fr_prepare_images(ctx, real.cuda(), out, center=center)
        torch.cuda.synchronize()
    finally:
        L.fr_destroy(ctx)
    ref = recon.image_spectra(real.numpy(), center=center)
    got = out.cpu().numpy().astype(np.complex128)
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(ref))


@pytest.mark.parametrize("S,n", [(32, 70), (30, 33)])
def test_prepare_fp16(S, n):
    real = _real(S, n, 5 + S)
    ctx = L.fr_create(S)
    try:
        out = torch.empty(n, S, S // 2 + 1, 2, dtype=torch.float16, device="cuda")
        L.fr_prepare_images(ctx, real.cuda(), out, center=True)
        torch.cuda.synchronize()
    finally:
        L.fr_destroy(ctx)
    ref = recon.image_spectra(real.numpy(), center=True)
    got = out.cpu().numpy().astype(np.float64)
    ref2 = np.stack([ref.real, ref.imag], -1)
    bound = np.abs(ref2) * 2.0 ** -11 + 1e-5 * np.max(np.abs(ref))
    assert np.all(np.abs(got - ref2) <= bound)


@pytest.mark.parametrize("f16", [False, True])
def test_prepare_across_a_chunk_boundary(f16):
    """S = 256: the transforms run in chunks of about 256 MB of spectra (1016
    images here); images on both sides of the first boundary and the last
    image of the tail chunk match the reference."""
    S, n = 256, 1100
    real = _real(S, n, 77)
    ctx = L.fr_create(S)
    try:
        if f16:
            out = torch.empty(n, S, S // 2 + 1, 2, dtype=torch.float16, device="cuda")
        else:
            out = torch.empty(n, S, S // 2 + 1, dtype=torch.complex64, device="cuda")
        L.fr_prepare_images(ctx, real.cuda(), out, center=True)
        torch.cuda.synchronize()
    finally:
        L.fr_destroy(ctx)
    pick = [0, 1015, 1016, 1099]
    ref = recon.image_spectra(real[pick].numpy(), center=True)
    got = out[pick].cpu()
    if f16:
        got = got.float().numpy().astype(np.float64)
        ref2 = np.stack([ref.real, ref.imag], -1)
        assert np.all(np.abs(got - ref2) <= np.abs(ref2) * 2.0 ** -11 + 1e-5 * np.max(np.abs(ref)))
    else:
        got = got.numpy().astype(np.complex128)
        assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(ref))


def test_prepared_images_insert_like_the_oracle():
    S, n = 32, 64
    real = _real(S, n, 9)
    _, rot = inputs.make_batch(S, n, 10)
    ctx = L.fr_create(S)
    try:
        spec = torch.empty(n, S, S // 2 + 1, dtype=torch.complex64, device="cuda")
        L.fr_prepare_images(ctx, real.cuda(), spec, center=True)
        L.fr_set_options(ctx, tuning=0, forced_config=-1)
        L.fr_insert(ctx, spec, rot.cuda())
        D = S + 1
        V = torch.empty(D ** 3, dtype=torch.complex64, device="cuda")
        W = torch.empty(D ** 3, dtype=torch.float32, device="cuda")
        L.fr_finalize(ctx, V, W)
        torch.cuda.synchronize()
    finally:
        L.fr_destroy(ctx)
    F = recon.image_spectra(real.numpy(), center=True)
    Vr, Wr, _ = oracle_insert(S, [(torch.from_numpy(F.astype(np.complex64)), rot)])
    V = V.cpu().numpy().astype(np.complex128)
    W = W.cpu().numpy().astype(np.float64)
    assert rel_err(V, Vr) <= TOL_F32 and rel_err(W, Wr) <= TOL_F32
