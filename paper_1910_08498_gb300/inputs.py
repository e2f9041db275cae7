"""Seeded synthetic inputs for 3D Fourier insertion.

This module holds no insertion arithmetic: it only draws the images and
rotations that both the CUDA library and the FP64 oracle consume.  It does
not load the CUDA library.

Recipe (stand-in for the cryo-EM particle stacks of Sec. 5.3.2, whose dataset
is not available here):

* images: ``[n][S][S/2+1]`` complex Hermitian half planes in ``torch.fft.rfft2``
  order (row ``j`` <-> ``ky = j`` for ``j < S/2`` else ``j - S``; column
  ``kx = 0..S/2``).  Real and imaginary parts are iid N(0, 1), each divided by
  ``1 + |k|`` with ``|k| = sqrt(kx^2 + ky^2)`` in pixel units, so that low
  frequencies dominate as in real projection spectra.
* rotations: uniform on SO(3): a unit quaternion from a normalised 4-D standard
  normal draw, turned into a matrix in FP64 and rounded to FP32.  Row-major
  ``[n][3][3]``; ``q = R (kx, ky, 0)^T`` maps image to volume coordinates.
* FP16 copies are the FP32 values rounded to half precision.

Seeds go through ``torch.Generator(device).manual_seed(seed)``.  The CPU and
CUDA generators give different streams; a comparison always feeds both sides
the same tensors.
"""
from __future__ import annotations

import torch


def freq_radius(S: int, device="cpu") -> torch.Tensor:
    """|k| for every stored pixel of an S x (S/2+1) half plane, [S, S/2+1]."""
    j = torch.arange(S, device=device, dtype=torch.float64)
    ky = torch.where(j < S // 2, j, j - S)
    kx = torch.arange(S // 2 + 1, device=device, dtype=torch.float64)
    return torch.sqrt(ky[:, None] ** 2 + kx[None, :] ** 2)


def random_images(S: int, n: int, gen: torch.Generator, device="cpu") -> torch.Tensor:
    """complex64 [n, S, S/2+1]: iid complex Gaussian scaled by 1/(1+|k|)."""
    if S % 2:
        raise ValueError("S must be even")
    scale = (1.0 / (1.0 + freq_radius(S, device))).to(torch.float32)
    re_im = torch.randn((n, S, S // 2 + 1, 2), generator=gen, device=device, dtype=torch.float32)
    re_im *= scale[None, :, :, None]
    return torch.view_as_complex(re_im)


def quat_to_matrix(q: torch.Tensor) -> torch.Tensor:
    """Unit quaternions (w, x, y, z) [n, 4] FP64 -> rotation matrices [n, 3, 3] FP64."""
    w, x, y, z = q.unbind(-1)
    return torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1),
    ], -2)


def random_rotations(n: int, gen: torch.Generator, device="cpu") -> torch.Tensor:
    """float32 [n, 3, 3], uniform on SO(3) (normalised Gaussian quaternions)."""
    q = torch.randn((n, 4), generator=gen, device=device, dtype=torch.float64)
    q = q / q.norm(dim=-1, keepdim=True)
    return quat_to_matrix(q).to(torch.float32)


def make_batch(S: int, n: int, seed: int, device="cpu"):
    """(images complex64 [n,S,S/2+1], rotations float32 [n,3,3]) from one seed."""
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    rot = random_rotations(n, gen, device)
    img = random_images(S, n, gen, device)
    return img, rot


def to_half(images: torch.Tensor) -> torch.Tensor:
    """FP16 storage copy: [n, S, S/2+1, 2] float16 (interleaved re, im)."""
    return torch.view_as_real(images).to(torch.float16).contiguous()


def half_values(images_f16: torch.Tensor) -> torch.Tensor:
    """The exact complex64 values of an FP16 copy (half -> float is exact)."""
    return torch.view_as_complex(images_f16.to(torch.float32).contiguous())


def proper_signed_permutations() -> torch.Tensor:
    """The 24 rotation matrices with entries in {-1, 0, 1} (det = +1), [24,3,3]."""
    import itertools
    out = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1.0, -1.0), repeat=3):
            m = torch.zeros(3, 3, dtype=torch.float32)
            for r, c in enumerate(perm):
                m[r, c] = signs[r]
            if torch.det(m.double()) > 0:
                out.append(m)
    return torch.stack(out)


# Workload configurations (Sec. 5.3.2 stand-ins); sizes only, no arithmetic.
CONFIG_SMALL = dict(S=32, n=64, seed=1, a=1.9, alpha=15.0, table=10000)
CONFIG_TUNING = dict(S=128, batches=10, n=1000, seed=2, a=1.9, alpha=15.0)
CONFIG_UNEVEN = dict(batches=40, S_choices=(64, 96, 128, 192, 256), n_range=(500, 5000), seed=3)
CONFIG_LARGE = dict(S=256, n_total=100_000, n=5000, seed=5, a=1.9, alpha=15.0, S_switch=192)


def uneven_batches(cfg=CONFIG_UNEVEN, batches=None):
    """(S, n, seed) of each batch of the uneven-batch workload: S uniform over
    cfg["S_choices"], n uniform over cfg["n_range"] (inclusive), drawn from a
    CPU torch generator seeded with cfg["seed"]; batch b's images use seed
    cfg["seed"] * 1000 + b."""
    gen = torch.Generator()
    gen.manual_seed(int(cfg["seed"]))
    nb = cfg["batches"] if batches is None else batches
    choices = cfg["S_choices"]
    lo, hi = cfg["n_range"]
    out = []
    for b in range(nb):
        S = int(choices[int(torch.randint(len(choices), (1,), generator=gen))])
        n = int(torch.randint(lo, hi + 1, (1,), generator=gen))
        out.append((S, n, int(cfg["seed"]) * 1000 + b))
    return out

