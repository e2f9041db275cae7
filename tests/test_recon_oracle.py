"""Pins of the FP64 reference of Algorithm 1's last step (oracle/recon.py)
against what the mathematics fixes, independently of its own code path:

* round trip: a band-limited real volume f0, its spectrum written into the
  centred raw-sum layout as the insertion would leave it (half of the k_x = 0
  plane's value, the other half coming back through symmetrisation) with
  W = 1/2 everywhere, reconstructs to f0;
* the weighting divides by the symmetrised weight and clips it from below;
* a single frequency k0 (k_x > 0) of value c gives the closed form
  (2/S^3) Re(c exp(2 pi i k0.r / S)), written out with cos and sin;
* a volume whose only content is on the Nyquist planes reconstructs to 0.
"""
import numpy as np
import pytest

from oracle import recon


def _raw_from_spectrum(S, F0):
    H, D = S // 2, S + 1
    V = np.zeros((D, D, D), complex)
    for jz in range(S):
        kz = jz if jz < H else jz - S
        for jy in range(S):
            ky = jy if jy < H else jy - S
            for kx in range(H + 1):
                v = F0[jz, jy, kx]
                V[kz + H, ky + H, kx + H] = v / 2 if kx == 0 else v
    return V


def _bandlimited(S, seed):
    H = S // 2
    f0 = np.random.default_rng(seed).standard_normal((S, S, S))
    F0 = np.fft.rfftn(f0)
    F0[:, :, H] = 0
    F0[H, :, :] = 0
    F0[:, H, :] = 0
    return np.fft.irfftn(F0, s=(S, S, S), axes=(0, 1, 2)), F0


@pytest.mark.parametrize("S", [8, 16])
def test_round_trip(S):
    f0, F0 = _bandlimited(S, S)
    D = S + 1
    V = _raw_from_spectrum(S, F0)
    f = recon.reconstruct(S, V, np.full((D, D, D), 0.5), 1.0)
    assert np.max(np.abs(f - f0)) < 1e-12 * np.max(np.abs(f0)) * S ** 3


def test_weighting_divides_and_clips():
    S = 8
    f0, F0 = _bandlimited(S, 3)
    D = S + 1
    V = _raw_from_spectrum(S, F0)
    f = recon.reconstruct(S, V, np.full((D, D, D), 5.0), 1.0)       # Ws = 10
    assert np.allclose(f, f0 / 10, atol=1e-12)
    f = recon.reconstruct(S, V, np.full((D, D, D), 0.05), 1.0)      # Ws = 0.1 -> clipped to 1
    assert np.allclose(f, f0, atol=1e-12)
    f = recon.reconstruct(S, V, np.full((D, D, D), 0.05), 0.01)     # no clip: divide by 0.1
    assert np.allclose(f, 10 * f0, atol=1e-11)


def test_single_frequency_closed_form():
    S, H, D = 16, 8, 17
    k0 = (3, -2, 5)  # (kx, ky, kz), kx > 0
    c = 0.7 - 1.3j
    V = np.zeros((D, D, D), complex)
    V[k0[2] + H, k0[1] + H, k0[0] + H] = c
    f = recon.reconstruct(S, V, np.full((D, D, D), 0.5), 1.0)
    z, y, x = np.meshgrid(np.arange(S), np.arange(S), np.arange(S), indexing="ij")
    ph = 2 * np.pi * (k0[0] * x + k0[1] * y + k0[2] * z) / S
    ref = 2.0 / S ** 3 * (c.real * np.cos(ph) - c.imag * np.sin(ph))
    assert np.max(np.abs(f - ref)) < 1e-15


def test_nyquist_planes_are_dropped():
    S, H, D = 8, 4, 9
    V = np.zeros((D, D, D), complex)
    V[:, :, S] = 1.0      # k_x = +S/2
    V[0, :, H:] = 2.0     # k_z = -S/2
    V[:, 0, H:] = 3.0     # k_y = -S/2
    f = recon.reconstruct(S, V, np.ones((D, D, D)), 1.0)
    # what survives is only the symmetrised image of those planes at k = +S/2 in y, z,
    # which lies outside [-S/2, S/2)^3
    assert np.max(np.abs(f)) == 0.0


def test_image_spectra_closed_forms():
    S = 8
    # a unit impulse at the origin: flat spectrum; at the centre with
    # center=True: flat as well (the origin is moved there)
    d = np.zeros((1, S, S))
    d[0, 0, 0] = 1.0
    assert np.allclose(recon.image_spectra(d), 1.0)
    c = np.zeros((1, S, S))
    c[0, S // 2, S // 2] = 1.0
    assert np.allclose(recon.image_spectra(c, center=True), 1.0)
    # without centring, the centre impulse gives (-1)^(kx + ky), written out
    F = recon.image_spectra(c)[0]
    j = np.arange(S)[:, None]
    kx = np.arange(S // 2 + 1)[None, :]
    assert np.allclose(F, (-1.0) ** (kx + j))
    # a single cosine along x of frequency 2: two bins of value S^2 / 2 at kx = 2, ky = 0
    y, x = np.meshgrid(np.arange(S), np.arange(S), indexing="ij")
    F = recon.image_spectra(np.cos(2 * np.pi * 2 * x / S)[None])[0]
    ref = np.zeros_like(F)
    ref[0, 2] = S * S / 2
    assert np.allclose(F, ref, atol=1e-12)
