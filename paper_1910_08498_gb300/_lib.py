"""ctypes binding of libfr.so (include/fr.h) -- argument marshalling only.

Each ``fr_*`` function here has the name and argument order of the C entry
point; torch tensors are passed by ``data_ptr()`` and the stream defaults to
``torch.cuda.current_stream()``.  Every step of the insertion runs in the
library's CUDA kernels; there is no Python or CPU fallback: if libfr.so is not
built, loading fails loudly.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfr.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "fr.h")

FR_OK, FR_ERR_INVALID_ARG, FR_ERR_UNSUPPORTED, FR_ERR_OOM, FR_ERR_CUDA = 0, 1, 2, 3, 4
FR_ERR_LAUNCH, FR_ERR_DEVICE_ASSERT, FR_ERR_TIMEOUT, FR_ERR_IO, FR_ERR_STATE = 5, 6, 7, 8, 9
FR_ERR_NOALLOC_LIMIT = 10
FR_NOALLOC_MAX_S = 64
FR_F32, FR_F16 = 0, 1
FR_SEARCH_EXHAUSTIVE, FR_SEARCH_RANDOM, FR_SEARCH_LEARNED, FR_SEARCH_ANNEALING, FR_SEARCH_MCMC = 0, 1, 2, 3, 4
MLP_NPARAM = 5313


class FrError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = _lib().fr_error_string(status).decode() if _LIB is not None else str(status)
        if status in (FR_ERR_CUDA, FR_ERR_OOM) and _LIB is not None:
            msg += f" [cudaError {_LIB.fr_last_cuda_error()}]"
        super().__init__(f"{where}: {msg} (status {status})")
        self.status = status


class fr_blob(ctypes.Structure):
    _fields_ = [("a", ctypes.c_float), ("alpha", ctypes.c_float), ("order", ctypes.c_int),
                ("table_size", ctypes.c_int)]


class fr_options(ctypes.Structure):
    _fields_ = [("tuning", ctypes.c_int), ("search", ctypes.c_int), ("budget", ctypes.c_int),
                ("steps_per_insert", ctypes.c_int), ("forced_config", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("debug", ctypes.c_int), ("fault_config", ctypes.c_int),
                ("fault_alloc", ctypes.c_int), ("reserved", ctypes.c_int * 6)]


class fr_report(ctypes.Structure):
    _fields_ = [("S", ctypes.c_int), ("n_bucket", ctypes.c_int), ("space_size", ctypes.c_int),
                ("evaluated", ctypes.c_int), ("tuned", ctypes.c_int),
                ("best_config", ctypes.c_int), ("last_config", ctypes.c_int),
                ("launches", ctypes.c_int), ("best_ns_per_image", ctypes.c_double),
                ("mean_ns_per_image", ctypes.c_double), ("tuning_overhead_pct", ctypes.c_double),
                ("images", ctypes.c_ulonglong), ("retunes", ctypes.c_int),
                ("reserved", ctypes.c_int * 7)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"} | {
            "predicted_best": self.reserved[0]}


_LIB = None
_LOCK = threading.Lock()


def declared_symbols(header: str | None = None) -> list[str]:
    """Names of the functions one header (default: every include/*.h) declares."""
    import glob
    paths = [header] if header else sorted(glob.glob(os.path.join(os.path.dirname(HEADER), "*.h")))
    names = set()
    for path in paths:
        txt = re.sub(r"/\*.*?\*/", "", open(path).read(), flags=re.S)
        names.update(re.findall(r"\b(fr_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built: call paper_1910_08498_gb300.build.build() "
                               "(or __graft_entry__.build()) first; there is no fallback path")
        L = ctypes.CDLL(LIB_PATH)
        i, d, vp, f = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_float
        P = ctypes.POINTER
        sig = {
            "fr_create": (i, [i, P(fr_blob), P(vp)]),
            "fr_destroy": (i, [vp]),
            "fr_reset": (i, [vp, vp]),
            "fr_insert": (i, [vp, vp, i, vp, i, vp]),
            "fr_insert_batched": (i, [P(vp), P(vp), P(i), P(vp), P(i), i, i, vp]),
            "fr_finalize": (i, [vp, vp, vp, vp]),
            "fr_retune": (i, [vp, i]),
            "fr_set_options": (i, [vp, P(fr_options)]),
            "fr_get_options": (i, [vp, P(fr_options)]),
            "fr_tuning_report": (i, [vp, P(fr_report)]),
            "fr_tuning_measurements": (i, [vp, P(i), P(d), P(d), i]),
            "fr_tuning_save": (i, [vp, ctypes.c_char_p]),
            "fr_tuning_load": (i, [vp, ctypes.c_char_p]),
            "fr_num_configs": (i, []),
            "fr_describe_config": (i, [i, ctypes.c_char_p, i]),
            "fr_config_valid": (i, [vp, i]),
            "fr_insert_launches": (i, [vp, i, i, P(i)]),
            "fr_config_features": (i, [i, i, i, f, P(f)]),
            "fr_count_updates": (i, [vp, vp, i, vp, P(ctypes.c_ulonglong)]),
            "fr_relative_performance": (d, [d, d, d, d]),
            "fr_invocations_to_amortize": (d, [d, d, d, d]),
            "fr_random_search_steps": (d, [d, d]),
            "fr_error_string": (ctypes.c_char_p, [i]),
            "fr_last_device_error": (i, [vp]),
            "fr_last_cuda_error": (i, []),
            "fr_debug_fold": (i, [vp, vp, i, vp, vp]),
            "fr_debug_blob": (i, [vp, vp, i, i, vp, vp]),
            "fr_debug_phase_counters": (i, [vp, P(ctypes.c_ulonglong), i]),
            "fr_mlp_num_params": (i, []),
            "fr_mlp_forward": (i, [vp, vp, i, vp, vp]),
            "fr_mlp_backward": (i, [vp, vp, vp, i, vp, vp, vp]),
            "fr_mlp_adam": (i, [vp, vp, vp, vp, i, f, f, f, f, vp]),
            "fr_mlp_train": (i, [vp, P(f), P(f), i, i, f, ctypes.c_uint64, P(f)]),
            "fr_mlp_get": (i, [vp, P(f)]),
            "fr_mlp_set": (i, [vp, P(f)]),
            "fr_insert_noalloc": (i, [i, f, f, vp, i, vp, i, vp, vp, vp]),
            "fr_reconstruct": (i, [vp, vp, f, vp]),
            "fr_state_bytes": (ctypes.c_size_t, [vp]),
            "fr_state_save": (i, [vp, vp]),
            "fr_state_load": (i, [vp, vp]),
            "fr_prepare_images": (i, [vp, vp, i, i, vp, i, vp]),
            "fr_search_simulate": (i, [i, P(d), i, i, ctypes.c_uint64, i, P(i)]),
            "fr_probe_fp32_peak": (i, [i, i, P(d), P(d), vp]),
            "fr_gemm_create": (i, [P(vp)]),
            "fr_gemm_destroy": (i, [vp]),
            "fr_gemm_set_tuning": (i, [vp, i, i, i, i, d, d, ctypes.c_uint64]),
            "fr_gemm_run": (i, [vp, i, i, i, vp, vp, vp, i, vp]),
            "fr_gemm_run_config": (i, [i, i, i, i, vp, vp, vp, i, vp]),
            "fr_gemm_num_configs": (i, []),
            "fr_gemm_device_status": (i, []),
            "fr_gemm_set_wait_limit": (i, [ctypes.c_longlong]),
            "fr_gemm_describe_config": (i, [i, ctypes.c_char_p, i]),
            "fr_gemm_config_valid": (i, [i, i, i, i]),
            "fr_gemm_report": (i, [vp, i, i, i, P(i), P(i), P(i), P(d), P(d)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
        return L


def lib():
    """The loaded ctypes library (raises if it is not built)."""
    return _lib()


def _check(rc: int, where: str, ok=(FR_OK,)):
    if rc not in ok:
        raise FrError(rc, where)
    return rc


def _stream(stream):
    import torch
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _dtype_of(images):
    import torch
    if images.dtype in (torch.complex64, torch.float32):
        return FR_F32
    if images.dtype == torch.float16:
        return FR_F16
    raise TypeError(f"images must be complex64/float32 or float16 (got {images.dtype})")


# ------------------------------------------------------------------ C entry points

def fr_create(S: int, a: float = 1.9, alpha: float = 15.0, order: int = 0, table_size: int = 10000):
    h = ctypes.c_void_p()
    b = fr_blob(a, alpha, order, table_size)
    _check(_lib().fr_create(S, ctypes.byref(b), ctypes.byref(h)), "fr_create")
    return h


def fr_destroy(ctx):
    return _check(_lib().fr_destroy(ctx), "fr_destroy")


def fr_reset(ctx, stream=None):
    return _check(_lib().fr_reset(ctx, _stream(stream)), "fr_reset")


def fr_insert(ctx, images, rotations, n: int | None = None, stream=None, allow_fallback=True):
    """images: CUDA tensor [n,S,S/2+1] complex64 (or [...,2] float32, or [...,2]
    float16); rotations: CUDA float32 [n,3,3].  Returns the status (FR_OK or
    FR_ERR_LAUNCH when a configuration was replaced by the fallback)."""
    if n is None:
        n = rotations.shape[0]
    assert images.is_cuda and rotations.is_cuda and images.is_contiguous() and rotations.is_contiguous()
    ok = (FR_OK, FR_ERR_LAUNCH) if allow_fallback else (FR_OK,)
    return _check(_lib().fr_insert(ctx, _ptr(images), _dtype_of(images), _ptr(rotations), int(n),
                                   _stream(stream)), "fr_insert", ok)


def fr_insert_noalloc(S, images, rotations, V, W, a=1.9, alpha=15.0, n=None, stream=None):
    """Insertion with no device allocation (S <= FR_NOALLOC_MAX_S): adds the
    batch to caller-owned V (complex64, (S+1)^3) and W (float32, (S+1)^3)."""
    if n is None:
        n = rotations.shape[0]
    for t in (images, rotations, V, W):
        assert t.is_cuda and t.is_contiguous()
    return _check(_lib().fr_insert_noalloc(int(S), float(a), float(alpha), _ptr(images),
                                           _dtype_of(images), _ptr(rotations), int(n), _ptr(V),
                                           _ptr(W), _stream(stream)), "fr_insert_noalloc")


def fr_probe_fp32_peak(packed=False, repeats=5, stream=None) -> tuple[float, float]:
    """Measured FP32 FMA peak: (TFLOP/s, ms) of the fastest of `repeats`
    launches of the FMA-chain kernel (packed: two-lane f32x2 FMAs)."""
    tf = ctypes.c_double()
    ms = ctypes.c_double()
    _check(_lib().fr_probe_fp32_peak(int(bool(packed)), int(repeats), ctypes.byref(tf),
                                     ctypes.byref(ms), _stream(stream)), "fr_probe_fp32_peak")
    return tf.value, ms.value


def fr_search_simulate(search, ns_per_image, budget, seed=1, start=-1) -> list[int]:
    """Configurations a searcher would measure, in order, on a table of known
    times (host only; <= 0 marks an invalid configuration)."""
    t = (ctypes.c_double * len(ns_per_image))(*[float(x) for x in ns_per_image])
    out = (ctypes.c_int * max(1, budget))()
    m = _lib().fr_search_simulate(int(search), t, len(ns_per_image), int(budget), int(seed),
                                  int(start), out)
    if m < 0:
        raise FrError(-m, "fr_search_simulate")
    return [out[k] for k in range(m)]


def fr_prepare_images(ctx, real, out, center=False, n=None, stream=None):
    """2D FFTs of real images [n,S,S] (CUDA float32) into out: complex64
    [n,S,S/2+1] (or float32 [...,2]) for FP32, float16 [n,S,S/2+1,2] for FP16."""
    if n is None:
        n = real.shape[0]
    assert real.is_cuda and out.is_cuda and real.is_contiguous() and out.is_contiguous()
    return _check(_lib().fr_prepare_images(ctx, _ptr(real), int(n), int(bool(center)), _ptr(out),
                                           _dtype_of(out), _stream(stream)), "fr_prepare_images")


def fr_state_bytes(ctx) -> int:
    return int(_lib().fr_state_bytes(ctx))


def fr_state_save(ctx, dst):
    """Copy the accumulator planes into dst (a torch tensor on the host or the
    device with at least fr_state_bytes bytes)."""
    assert dst.is_contiguous() and dst.numel() * dst.element_size() >= fr_state_bytes(ctx)
    return _check(_lib().fr_state_save(ctx, _ptr(dst)), "fr_state_save")


def fr_state_load(ctx, src):
    assert src.is_contiguous() and src.numel() * src.element_size() >= fr_state_bytes(ctx)
    return _check(_lib().fr_state_load(ctx, _ptr(src)), "fr_state_load")


def fr_reconstruct(ctx, out, w_clip=1.0, stream=None):
    """Weighted inverse transform of the context's volume into out (CUDA
    float32, S^3, [z][y][x])."""
    assert out.is_cuda and out.is_contiguous() and out.dtype.is_floating_point
    return _check(_lib().fr_reconstruct(ctx, _ptr(out), float(w_clip), _stream(stream)),
                  "fr_reconstruct")


def fr_insert_batched(ctxs, images, rotations, ns=None, capture=0, stream=None):
    nb = len(ctxs)
    if ns is None:
        ns = [r.shape[0] for r in rotations]
    C = (ctypes.c_void_p * nb)(*[c.value if isinstance(c, ctypes.c_void_p) else c for c in ctxs])
    I = (ctypes.c_void_p * nb)(*[t.data_ptr() for t in images])
    R = (ctypes.c_void_p * nb)(*[t.data_ptr() for t in rotations])
    D = (ctypes.c_int * nb)(*[_dtype_of(t) for t in images])
    N = (ctypes.c_int * nb)(*[int(x) for x in ns])
    return _check(_lib().fr_insert_batched(C, I, D, R, N, nb, int(capture), _stream(stream)),
                  "fr_insert_batched")


def fr_finalize(ctx, V, W, stream=None):
    return _check(_lib().fr_finalize(ctx, _ptr(V), _ptr(W), _stream(stream)), "fr_finalize")


def fr_retune(ctx, all: bool = False):
    return _check(_lib().fr_retune(ctx, int(bool(all))), "fr_retune")


def fr_get_options(ctx) -> fr_options:
    o = fr_options()
    _check(_lib().fr_get_options(ctx, ctypes.byref(o)), "fr_get_options")
    return o


def fr_set_options(ctx, opt: fr_options | None = None, **kw):
    o = opt if opt is not None else fr_get_options(ctx)
    for k, v in kw.items():
        setattr(o, k, v)
    return _check(_lib().fr_set_options(ctx, ctypes.byref(o)), "fr_set_options")


def fr_tuning_report(ctx) -> dict:
    r = fr_report()
    _check(_lib().fr_tuning_report(ctx, ctypes.byref(r)), "fr_tuning_report")
    return r.as_dict()


def fr_tuning_measurements(ctx) -> list[tuple[int, float, float]]:
    """[(config id, ns per image, images timed)] of the current key."""
    n = _lib().fr_tuning_measurements(ctx, None, None, None, 0)
    if n < 0:
        raise FrError(-n, "fr_tuning_measurements")
    c = (ctypes.c_int * max(n, 1))()
    t = (ctypes.c_double * max(n, 1))()
    im = (ctypes.c_double * max(n, 1))()
    n = _lib().fr_tuning_measurements(ctx, c, t, im, n)
    return [(c[k], t[k], im[k]) for k in range(n)]


def fr_tuning_save(ctx, path: str):
    return _check(_lib().fr_tuning_save(ctx, path.encode()), "fr_tuning_save")


def fr_tuning_load(ctx, path: str):
    return _check(_lib().fr_tuning_load(ctx, path.encode()), "fr_tuning_load")


def fr_num_configs() -> int:
    return _lib().fr_num_configs()


def fr_describe_config(i: int) -> str:
    buf = ctypes.create_string_buffer(160)
    rc = _lib().fr_describe_config(i, buf, 160)
    if rc < 0:
        raise FrError(-rc, "fr_describe_config")
    return buf.value.decode()


def fr_config_valid(ctx, i: int) -> bool:
    return bool(_lib().fr_config_valid(ctx, i))


def fr_insert_launches(ctx, i: int, n: int) -> int:
    """Kernel launches of one insertion step of n images with configuration i."""
    out = ctypes.c_int(0)
    _check(_lib().fr_insert_launches(ctx, int(i), int(n), ctypes.byref(out)), "fr_insert_launches")
    return out.value


def fr_config_features(i: int, S: int, n: int, a: float):
    out = (ctypes.c_float * 16)()
    _check(_lib().fr_config_features(i, S, n, a, out), "fr_config_features")
    return list(out)


def fr_count_updates(ctx, rotations, n=None, stream=None) -> int:
    if n is None:
        n = rotations.shape[0]
    out = ctypes.c_ulonglong(0)
    _check(_lib().fr_count_updates(ctx, _ptr(rotations), int(n), _stream(stream), ctypes.byref(out)),
           "fr_count_updates")
    return int(out.value)


def fr_relative_performance(s, t_avg, t_well, n) -> float:
    return _lib().fr_relative_performance(s, t_avg, t_well, n)


def fr_invocations_to_amortize(rp, s, t_avg, t_well) -> float:
    return _lib().fr_invocations_to_amortize(rp, s, t_avg, t_well)


def fr_random_search_steps(r, p) -> float:
    return _lib().fr_random_search_steps(r, p)


def fr_error_string(status: int) -> str:
    return _lib().fr_error_string(status).decode()


def fr_last_device_error(ctx) -> int:
    return _lib().fr_last_device_error(ctx)


def fr_last_cuda_error() -> int:
    return _lib().fr_last_cuda_error()


def fr_debug_fold(r, k, out, stream=None):
    return _check(_lib().fr_debug_fold(_ptr(r), _ptr(k), out.numel(), _ptr(out), _stream(stream)),
                  "fr_debug_fold")


def fr_debug_blob(ctx, r2, mode, out, stream=None):
    return _check(_lib().fr_debug_blob(ctx, _ptr(r2), r2.numel(), int(mode), _ptr(out),
                                       _stream(stream)), "fr_debug_blob")


PHASES = ["cull", "queue", "drain_fast", "drain_edge", "drain_careful", "flush", "items_fast",
          "items_edge", "items_careful", "list_images", "warp_cycles", "rounds_fast", "drain_fold",
          "items_fold"]


def fr_debug_phase_counters(ctx) -> dict:
    out = (ctypes.c_ulonglong * 16)()
    _check(_lib().fr_debug_phase_counters(ctx, out, 16), "fr_debug_phase_counters")
    return {name: int(out[k]) for k, name in enumerate(PHASES)}


def fr_mlp_num_params() -> int:
    return _lib().fr_mlp_num_params()


def fr_mlp_forward(params, x, y, stream=None):
    return _check(_lib().fr_mlp_forward(_ptr(params), _ptr(x), x.shape[0], _ptr(y), _stream(stream)),
                  "fr_mlp_forward")


def fr_mlp_backward(params, x, target, grad, loss, stream=None):
    return _check(_lib().fr_mlp_backward(_ptr(params), _ptr(x), _ptr(target), x.shape[0],
                                         _ptr(grad), _ptr(loss), _stream(stream)), "fr_mlp_backward")


def fr_mlp_adam(params, grad, m1, m2, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    return _check(_lib().fr_mlp_adam(_ptr(params), _ptr(grad), _ptr(m1), _ptr(m2), int(t), lr,
                                     beta1, beta2, eps, _stream(stream)), "fr_mlp_adam")


def fr_mlp_train(ctx, feat, logt, epochs=2000, lr=3e-3, seed=1) -> float:
    import numpy as np
    f = np.ascontiguousarray(np.asarray(feat, dtype=np.float32))
    t = np.ascontiguousarray(np.asarray(logt, dtype=np.float32))
    m = t.shape[0]
    assert f.shape == (m, 16)
    loss = ctypes.c_float(0)
    FP = ctypes.POINTER(ctypes.c_float)
    _check(_lib().fr_mlp_train(ctx, f.ctypes.data_as(FP), t.ctypes.data_as(FP), m, int(epochs),
                               float(lr), int(seed), ctypes.byref(loss)), "fr_mlp_train")
    return float(loss.value)


def fr_mlp_get(ctx):
    import numpy as np
    out = np.zeros(MLP_NPARAM, np.float32)
    _check(_lib().fr_mlp_get(ctx, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))), "fr_mlp_get")
    return out


def fr_mlp_set(ctx, params):
    import numpy as np
    p = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
    assert p.size == MLP_NPARAM
    return _check(_lib().fr_mlp_set(ctx, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
                  "fr_mlp_set")


# ---------------------------------------------------------------- batched GEMM (fr_gemm.h)

def fr_gemm_create():
    h = ctypes.c_void_p()
    _check(_lib().fr_gemm_create(ctypes.byref(h)), "fr_gemm_create")
    return h


def fr_gemm_destroy(ctx):
    return _check(_lib().fr_gemm_destroy(ctx), "fr_gemm_destroy")


def fr_gemm_set_tuning(ctx, tuning=1, search=FR_SEARCH_RANDOM, budget=20, steps=2, bw_gbs=0.0,
                       bw_frac=0.75, seed=1):
    return _check(_lib().fr_gemm_set_tuning(ctx, int(tuning), int(search), int(budget), int(steps),
                                            float(bw_gbs), float(bw_frac), int(seed)),
                  "fr_gemm_set_tuning")


def _gemm_args(A, B, C):
    batch, m, k = A.shape
    assert B.shape[0] == batch and B.shape[1] == k and C.shape == (batch, m, B.shape[2])
    for t in (A, B, C):
        assert t.is_cuda and t.is_contiguous()
    return m, B.shape[2], k, batch


def fr_gemm_run(ctx, A, B, C, stream=None):
    """C[b] = A[b] B[b] (CUDA float32 [batch, m, k] x [batch, k, n]), tuned dynamically."""
    m, n, k, batch = _gemm_args(A, B, C)
    return _check(_lib().fr_gemm_run(ctx, m, n, k, _ptr(A), _ptr(B), _ptr(C), batch, _stream(stream)),
                  "fr_gemm_run")


def fr_gemm_run_config(config, A, B, C, stream=None):
    m, n, k, batch = _gemm_args(A, B, C)
    return _check(_lib().fr_gemm_run_config(int(config), m, n, k, _ptr(A), _ptr(B), _ptr(C), batch,
                                            _stream(stream)), "fr_gemm_run_config")


def fr_gemm_device_status() -> int:
    """FR_OK, or FR_ERR_TIMEOUT if a bulk-copy launch's bounded wait gave up
    since the last call (clears it)."""
    return _lib().fr_gemm_device_status()


def fr_gemm_set_wait_limit(ns: int):
    """Test hook: limit (ns) of the bulk-copy kernels' waits for their copies."""
    return _check(_lib().fr_gemm_set_wait_limit(int(ns)), "fr_gemm_set_wait_limit")


def fr_gemm_num_configs() -> int:
    return _lib().fr_gemm_num_configs()


def fr_gemm_describe_config(i: int) -> str:
    buf = ctypes.create_string_buffer(64)
    _check(_lib().fr_gemm_describe_config(i, buf, 64), "fr_gemm_describe_config")
    return buf.value.decode()


def fr_gemm_config_valid(i, m, n, k) -> bool:
    return bool(_lib().fr_gemm_config_valid(int(i), int(m), int(n), int(k)))


def fr_gemm_report(ctx, m, n, k) -> dict:
    t, e, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    g, o = ctypes.c_double(), ctypes.c_double()
    _check(_lib().fr_gemm_report(ctx, m, n, k, ctypes.byref(t), ctypes.byref(e), ctypes.byref(b),
                                 ctypes.byref(g), ctypes.byref(o)), "fr_gemm_report")
    return {"tuned": t.value, "evaluated": e.value, "best": b.value, "best_gbs": g.value,
            "overhead_pct": o.value}

