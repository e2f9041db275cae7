"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and compare with the FP64 oracle on the same seeded inputs."""
from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_1910_08498_gb300 import _lib as L
from paper_1910_08498_gb300 import inputs

A32 = float(np.float32(1.9))   # the FP32 blob radius the library receives, fed to the oracle too
ALPHA = 15.0
TOL_F32 = 2e-5
TOL_F16 = 2e-3


def rel_err(x_gpu, x_ref):
    """max |x_gpu - x_ref| / max |x_ref| over the whole grid (complex modulus for V)."""
    x_gpu = np.asarray(x_gpu).ravel()
    x_ref = np.asarray(x_ref).ravel()
    den = np.max(np.abs(x_ref))
    return float(np.max(np.abs(x_gpu - x_ref)) / den) if den > 0 else float(np.max(np.abs(x_gpu)))


def worst(x_gpu, x_ref, S):
    """Description of the worst voxel (coordinates, values) for failure messages."""
    x_gpu = np.asarray(x_gpu).ravel()
    x_ref = np.asarray(x_ref).ravel()
    i = int(np.argmax(np.abs(x_gpu - x_ref)))
    D, H = S + 1, S // 2
    z, r = divmod(i, D * D)
    y, x = divmod(r, D)
    return f"worst voxel (x,y,z)=({x - H},{y - H},{z - H}) gpu={x_gpu[i]} ref={x_ref[i]}"


def sym_np(V, W, S):
    D = S + 1
    V = V.reshape(D, D, D)
    W = W.reshape(D, D, D)
    return V + np.conj(V[::-1, ::-1, ::-1]), W + W[::-1, ::-1, ::-1]


def gpu_insert(S, batches, a=A32, alpha=ALPHA, config=-1, tuning=True, table=10000, f16=False,
               steps=4, search=L.FR_SEARCH_EXHAUSTIVE, budget=0):
    """Insert a list of (images complex64 CPU, rotations float32 CPU) batches
    on the GPU; returns (V complex128 flat, W float64 flat, report)."""
    ctx = L.fr_create(S, a, alpha, 0, table)
    try:
        if config >= 0 and not L.fr_config_valid(ctx, config):
            import pytest
            pytest.skip(f"configuration {config} cannot run for this context")
        L.fr_set_options(ctx, forced_config=config, tuning=int(tuning), steps_per_insert=steps,
                         search=search, budget=budget)
        for img, rot in batches:
            rot_d = rot.contiguous().cuda()
            if f16:
                img_d = inputs.to_half(img).cuda()
            else:
                img_d = img.contiguous().cuda()
            L.fr_insert(ctx, img_d, rot_d)
        D = S + 1
        V = torch.empty(D ** 3, dtype=torch.complex64, device="cuda")
        W = torch.empty(D ** 3, dtype=torch.float32, device="cuda")
        L.fr_finalize(ctx, V, W)
        torch.cuda.synchronize()
        rep = L.fr_tuning_report(ctx)
        assert L.fr_last_device_error(ctx) == L.FR_OK
        return V.cpu().numpy().astype(np.complex128), W.cpu().numpy().astype(np.float64), rep
    finally:
        L.fr_destroy(ctx)


def oracle_insert(S, batches, a=A32, alpha=ALPHA, f16=False):
    V = W = None
    cnt = 0
    for img, rot in batches:
        vals = inputs.half_values(inputs.to_half(img)) if f16 else img
        V, W, c = oracle.insert(S, vals.numpy(), rot.numpy(), a=a, alpha=alpha, V=V, W=W)
        cnt += c
    return V, W, cnt
