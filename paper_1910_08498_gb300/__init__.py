"""GB300-native 3D Fourier insertion with non-blocking dynamic autotuning.

The work is done by libfr.so (hand-written sm_103a CUDA kernels behind the C
ABI in include/fr.h); ``_lib`` is its ctypes binding with the same function
names, and :class:`FourierInserter` is a small convenience wrapper around it.
Importing this package does not load the library; the first call does, and
fails loudly if it is not built.
"""
from __future__ import annotations

__all__ = ["FourierInserter", "build", "inputs"]


def build(verbose: bool = False) -> str:
    from .build import build as _b
    return _b(verbose=verbose)


class FourierInserter:
    """One reconstruction volume of side S+1 (a context of libfr).

    >>> fi = FourierInserter(128)              # a = 1.9, alpha = 15, 10000-entry table
    >>> fi.insert(images, rotations)           # CUDA tensors, any number of times
    >>> V, W = fi.finalize()                   # complex64 / float32 [(S+1)^3] tensors
    """

    def __init__(self, S: int, a: float = 1.9, alpha: float = 15.0, table_size: int = 10000):
        from . import _lib
        self._L = _lib
        self.S = S
        self.ctx = _lib.fr_create(S, a, alpha, 0, table_size)

    def insert(self, images, rotations, stream=None):
        return self._L.fr_insert(self.ctx, images, rotations, stream=stream)

    def finalize(self, stream=None):
        import torch
        D = self.S + 1
        V = torch.empty((D, D, D), dtype=torch.complex64, device="cuda")
        W = torch.empty((D, D, D), dtype=torch.float32, device="cuda")
        self._L.fr_finalize(self.ctx, V, W, stream=stream)
        return V, W

    def reset(self, stream=None):
        self._L.fr_reset(self.ctx, stream)

    def retune(self, all: bool = False):
        self._L.fr_retune(self.ctx, all)

    def set_options(self, **kw):
        self._L.fr_set_options(self.ctx, **kw)

    def report(self) -> dict:
        return self._L.fr_tuning_report(self.ctx)

    def count_updates(self, rotations) -> int:
        return self._L.fr_count_updates(self.ctx, rotations)

    def close(self):
        if self.ctx is not None:
            self._L.fr_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
