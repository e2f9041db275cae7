"""FP64 references of the FFT steps of Algorithm 1 (Sec. 5.3.1) around the
insertion: the images' forward transforms (image_spectra) and the last step,
applying the weights W to G and transforming back (reconstruct) -- TEST
INFRASTRUCTURE ONLY (tests, smoke and the benchmark's CPU legs may import
it; the product never does).

Readings (the paper does not spell the step out): the half-space fold is
undone by Hermitian symmetrisation, Vs(v) = V(v) + conj(V(-v)) and
Ws(v) = W(v) + W(-v); the weighting divides by the weight clipped from below,
F = Vs / max(Ws, w_clip); the spectrum is taken on k in [-S/2, S/2)^3 with
the Nyquist planes (k_x = S/2, k_y = -S/2, k_z = -S/2) set to zero, so that
it is exactly Hermitian; the volume is its real inverse DFT normalised by
1/S^3 (numpy's irfftn), origin at index 0.
"""
from __future__ import annotations

import numpy as np


def symmetrise(S, V, W):
    D = S + 1
    V = np.asarray(V, dtype=np.complex128).reshape(D, D, D)
    W = np.asarray(W, dtype=np.float64).reshape(D, D, D)
    return V + np.conj(V[::-1, ::-1, ::-1]), W + W[::-1, ::-1, ::-1]


def half_spectrum(S, F):
    """Centred (S+1)^3 spectrum -> [kz][ky][kx] with kz, ky in FFT order and
    kx = 0..S/2, Nyquist planes zeroed."""
    H = S // 2
    fft_order = np.r_[0:H, -H:0] + H  # FFT index j -> centred index of frequency j or j - S
    Fh = F[np.ix_(fft_order, fft_order, np.arange(H, S + 1))].copy()
    Fh[:, :, H] = 0  # k_x = S/2
    Fh[H, :, :] = 0  # k_z = -S/2 (FFT index S/2)
    Fh[:, H, :] = 0  # k_y = -S/2
    return Fh


def reconstruct(S, V, W, w_clip=1.0):
    """Real volume [z][y][x] (S^3, float64) from the raw sums V, W ((S+1)^3)."""
    Vs, Ws = symmetrise(S, V, W)
    F = Vs / np.maximum(Ws, w_clip)
    return np.fft.irfftn(half_spectrum(S, F), s=(S, S, S), axes=(0, 1, 2))


def image_spectra(real, center=False):
    """FP64 2D transforms of real images [n][S][S] in the insertion's layout
    [n][S][S/2+1] (numpy's rfft2); with center, the image origin is taken at
    pixel (S/2, S/2) (equivalently, the spectrum times (-1)^(kx + j))."""
    real = np.asarray(real, dtype=np.float64)
    if center:
        real = np.fft.ifftshift(real, axes=(-2, -1))
    return np.fft.rfft2(real, axes=(-2, -1))
