"""fr_insert_noalloc: the insertion entry point that allocates no device memory.

The file name sorts last so that, in a full run, these tests also execute
after every other test has used the library on the same device.

* GPU: two calls in a row into zeroed caller-owned V, W give, within the
  FP32 tolerance, what the FP64 oracle gives for the two seeded batches (and
  what the context entry point gives), at the largest size the fixed scratch
  holds and with the largest blob radius (the scratch filled to its last
  cell); FP16 images within the FP16 bound; a call after the one-time setup
  changes the device's free memory by nothing.
* CPU: sizes above the fixed scratch are rejected with FR_ERR_NOALLOC_LIMIT
  before any CUDA call.
"""
import numpy as np
import pytest
import torch

from paper_1910_08498_gb300 import _lib as L
from paper_1910_08498_gb300 import inputs
from tests.helpers import A32, ALPHA, TOL_F16, TOL_F32, gpu_insert, oracle_insert, rel_err, worst


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib = L.lib()
    S = L.FR_NOALLOC_MAX_S + 2
    rc = lib.fr_insert_noalloc(S, 1.9, 15.0, None, L.FR_F32, None, 10, None, None, None)
    assert rc == L.FR_ERR_NOALLOC_LIMIT
    assert b"fr_insert_noalloc" in lib.fr_error_string(rc)
    # odd and tiny sizes keep their usual statuses
    assert lib.fr_insert_noalloc(63, 1.9, 15.0, None, L.FR_F32, None, 10, None, None, None) == \
        L.FR_ERR_UNSUPPORTED
    assert lib.fr_insert_noalloc(6, 1.9, 15.0, None, L.FR_F32, None, 10, None, None, None) == \
        L.FR_ERR_INVALID_ARG


@pytest.mark.gpu
@pytest.mark.parametrize("a", [A32, 2.5, 2.9])
def test_noalloc_two_calls_match_oracle(a):
    a = float(np.float32(a))
    S = L.FR_NOALLOC_MAX_S
    b1 = inputs.make_batch(S, 300, 41)
    b2 = inputs.make_batch(S, 257, 42)
    Vr, Wr, _ = oracle_insert(S, [b1, b2], a=a, alpha=ALPHA)
    Vc, Wc, _ = gpu_insert(S, [b1, b2], a=a, alpha=ALPHA, tuning=False)

    D3 = (S + 1) ** 3
    V = torch.zeros(D3, dtype=torch.complex64, device="cuda")
    W = torch.zeros(D3, dtype=torch.float32, device="cuda")
    for img, rot in (b1, b2):
        rc = L.fr_insert_noalloc(S, img.cuda(), rot.cuda(), V, W, a=a, alpha=ALPHA)
        assert rc == L.FR_OK
    torch.cuda.synchronize()
    Vn = V.cpu().numpy().astype(np.complex128)
    Wn = W.cpu().numpy().astype(np.float64)
    assert rel_err(Vn, Vr) <= TOL_F32, (rel_err(Vn, Vr), worst(Vn, Vr, S))
    assert rel_err(Wn, Wr) <= TOL_F32, (rel_err(Wn, Wr), worst(Wn, Wr, S))
    # and the context entry point on the same batches
    assert rel_err(Vn, Vc) <= TOL_F32 and rel_err(Wn, Wc) <= TOL_F32
    # voxels the fold never reaches stay exactly zero
    H = S // 2
    xa0 = -int(np.floor(np.float32(a)))
    Wg = Wn.reshape(S + 1, S + 1, S + 1)
    assert not Wg[:, :, : xa0 + H].any()


@pytest.mark.gpu
def test_noalloc_call_after_setup_allocates_nothing():
    S = 32
    img, rot = inputs.make_batch(S, 64, 43)
    img, rot = img.cuda(), rot.cuda()
    D3 = (S + 1) ** 3
    V = torch.zeros(D3, dtype=torch.complex64, device="cuda")
    W = torch.zeros(D3, dtype=torch.float32, device="cuda")
    L.fr_insert_noalloc(S, img, rot, V, W)  # first call on the device: one-time setup
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    L.fr_insert_noalloc(S, img, rot, V, W)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    # two identical calls: W is twice one call's W
    W1 = torch.zeros_like(W)
    V1 = torch.zeros_like(V)
    L.fr_insert_noalloc(S, img, rot, V1, W1)
    torch.cuda.synchronize()
    assert rel_err(W.cpu().numpy(), 2 * W1.cpu().numpy().astype(np.float64)) <= TOL_F32


@pytest.mark.gpu
def test_noalloc_fp16_images():
    """FP16-stored images through the no-allocation entry point: within the
    FP16 bound of the oracle fed the FP32 values, within the FP32 bound of
    the oracle fed the FP16-rounded values."""
    S = L.FR_NOALLOC_MAX_S
    img, rot = inputs.make_batch(S, 200, 44)
    Vr, Wr, _ = oracle_insert(S, [(img, rot)])
    V16, W16, _ = oracle_insert(S, [(img, rot)], f16=True)
    D3 = (S + 1) ** 3
    V = torch.zeros(D3, dtype=torch.complex64, device="cuda")
    W = torch.zeros(D3, dtype=torch.float32, device="cuda")
    assert L.fr_insert_noalloc(S, inputs.to_half(img).cuda(), rot.cuda(), V, W, a=A32,
                               alpha=ALPHA) == L.FR_OK
    torch.cuda.synchronize()
    Vn = V.cpu().numpy().astype(np.complex128)
    Wn = W.cpu().numpy().astype(np.float64)
    assert rel_err(Vn, Vr) <= TOL_F16 and rel_err(Wn, Wr) <= TOL_F16
    assert rel_err(Vn, V16) <= TOL_F32 and rel_err(Wn, W16) <= TOL_F32
