"""FP64 CPU oracle for 3D Fourier insertion -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline /
reference leg may import this package.  The product library never loads it,
and it loads nothing from the product library.

``fr_oracle.c`` (plain C, FP64) holds the definition; ``mlp.py`` holds the
FP64 reference of the cost-model network.  This module compiles the C file
with gcc on first use (or via :func:`build`) and wraps it with ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fr_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile fr_oracle.c into liboracle.so (gcc -O2 -fopenmp)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB)
        d, i, ll = ctypes.c_double, ctypes.c_int, ctypes.c_longlong
        vp = ctypes.c_void_p
        lib.fro_i0.restype = d
        lib.fro_i0.argtypes = [d]
        lib.fro_blob.restype = d
        lib.fro_blob.argtypes = [d, d, d]
        lib.fro_blob_r2.restype = d
        lib.fro_blob_r2.argtypes = [d, d, d]
        lib.fro_fold.restype = i
        lib.fro_fold.argtypes = [ctypes.c_float, ctypes.c_float, i, i]
        lib.fro_insert.restype = ll
        lib.fro_insert.argtypes = [i, vp, vp, i, d, d, vp, vp, i]
        lib.fro_voxels.restype = i
        lib.fro_voxels.argtypes = [i, vp, vp, i, d, d, vp, i, vp, vp, i]
        lib.fro_count.restype = ll
        lib.fro_count.argtypes = [i, vp, i, d, i]
        lib.fro_max_threads.restype = i
        lib.fro_max_threads.argtypes = []
        _lib = lib
        return lib


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _images_f32(images):
    """Accept complex64/complex128 [n,S,S/2+1] or float [n,S,S/2+1,2] arrays;
    FP16 values are promoted exactly."""
    a = np.asarray(images)
    if np.iscomplexobj(a):
        a = np.stack([a.real, a.imag], axis=-1)
    return _f32(a)


def i0(x: float) -> float:
    return _load().fro_i0(float(x))


def blob(r: float, a: float = 1.9, alpha: float = 15.0) -> float:
    return _load().fro_blob(float(r), float(a), float(alpha))


def blob_r2(r2: float, a: float = 1.9, alpha: float = 15.0) -> float:
    return _load().fro_blob_r2(float(r2), float(a), float(alpha))


def fold(r00: float, r01: float, kx: int, ky: int) -> bool:
    return bool(_load().fro_fold(float(r00), float(r01), int(kx), int(ky)))


def max_threads() -> int:
    return _load().fro_max_threads()


def insert(S, images, rotations, a=1.9, alpha=15.0, V=None, W=None, nthreads=0):
    """Scatter images [n,S,S/2+1] (complex) with rotations [n,3,3] into V, W.

    Returns (V complex128 [(S+1)^3] flat, W float64 [(S+1)^3] flat, updates).
    V, W (if given) are accumulated into, in place."""
    img = _images_f32(images)
    rot = _f32(rotations).reshape(-1, 9)
    n = rot.shape[0]
    assert img.shape == (n, S, S // 2 + 1, 2), img.shape
    D3 = (S + 1) ** 3
    if V is None:
        V = np.zeros(D3, dtype=np.complex128)
    if W is None:
        W = np.zeros(D3, dtype=np.float64)
    assert V.dtype == np.complex128 and V.flags.c_contiguous and V.size == D3
    assert W.dtype == np.float64 and W.flags.c_contiguous and W.size == D3
    cnt = _load().fro_insert(S, img.ctypes.data, rot.ctypes.data, n, float(a), float(alpha),
                             V.ctypes.data, W.ctypes.data, int(nthreads))
    if cnt < 0:
        raise ValueError("oracle rejected arguments")
    return V, W, int(cnt)


def voxels(S, images, rotations, coords, a=1.9, alpha=15.0, nthreads=0):
    """V, W at the given voxel coordinates [(x,y,z), ...] (brute force)."""
    img = _images_f32(images)
    rot = _f32(rotations).reshape(-1, 9)
    n = rot.shape[0]
    c = np.ascontiguousarray(np.asarray(coords, dtype=np.int32).reshape(-1, 3))
    nv = c.shape[0]
    Vo = np.zeros(2 * nv, dtype=np.float64)
    Wo = np.zeros(nv, dtype=np.float64)
    rc = _load().fro_voxels(S, img.ctypes.data, rot.ctypes.data, n, float(a), float(alpha),
                            c.ctypes.data, nv, Vo.ctypes.data, Wo.ctypes.data, int(nthreads))
    if rc != 0:
        raise ValueError("oracle rejected arguments")
    return Vo[0::2] + 1j * Vo[1::2], Wo


def count(S, rotations, a=1.9, nthreads=0) -> int:
    rot = _f32(rotations).reshape(-1, 9)
    return int(_load().fro_count(S, rot.ctypes.data, rot.shape[0], float(a), int(nthreads)))


def volume_shape(S):
    return (S + 1, S + 1, S + 1)
