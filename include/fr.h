/*
 * fr.h -- C ABI of the GB300 3D Fourier insertion library (libfr.so).
 *
 * The library performs the insertion step of cryo-EM 3D Fourier
 * reconstruction (the step of Algorithm 1, Sec. 5.3.1, that adds the Fourier
 * transforms of a buffer of projection images into the volumes G and W) on
 * one GPU, with the non-blocking dynamic autotuning of Sec. 3.2 / Sec. 5.3.
 *
 *   for each image i, each stored pixel k = (kx, ky) of its half plane:
 *       q = R_i (kx, ky, 0)^T ;  p = image_i[k]
 *       if R_i[0][0]*kx + R_i[0][1]*ky < 0 (exact sign): q = -q, p = conj(p)
 *       for every voxel v with |v - q| <= a inside [-S/2, S/2]^3:
 *           w = b(|v - q|);  V[v] += w p;  W[v] += w
 *   b(r) = I0(alpha sqrt(1 - (r/a)^2)) / I0(alpha)   (Kaiser-Bessel, order 0)
 *
 * Conventions shared by every entry point
 *   - Pointers named "device" are CUDA device (or managed) pointers owned by
 *     the caller and borrowed until the work enqueued on `stream` completes.
 *   - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Every call that takes a stream only enqueues work on it and
 *     returns without waiting, unless its comment says otherwise.
 *   - Every call returns an fr_status.  FR_OK is 0.  Errors raised by device
 *     work already enqueued surface on a later call (fr_finalize,
 *     fr_last_device_error).
 *   - A context is not thread-safe: calls on one context must be serialised
 *     by the caller.  Different contexts are independent.
 *   - Layouts:
 *       images    [n][S][S/2+1] complex, interleaved (re, im); row j holds
 *                 ky = j for j < S/2 and ky = j - S otherwise, column kx =
 *                 0..S/2 (the torch.fft.rfft2 order).  FR_F32: 8 bytes per
 *                 pixel; FR_F16: two IEEE halves, 4 bytes per pixel.  The
 *                 base address must be 16-byte aligned.
 *       rotations [n][3][3] float32, row-major, mapping image coordinates to
 *                 volume coordinates (q = R k).  Only orthonormal inputs
 *                 (rounded to FP32) are meaningful; they are not checked.
 *       V, W      [z][y][x] with x fastest, (S+1)^3 elements, index i <->
 *                 coordinate i - S/2.  V is complex64 (interleaved float
 *                 re, im), W is float32.
 */
#ifndef FR_H
#define FR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FR_ABI_VERSION 1

typedef enum fr_status {
    FR_OK = 0,
    FR_ERR_INVALID_ARG = 1,   /* a null pointer, a size out of range, a bad enum */
    FR_ERR_UNSUPPORTED = 2,   /* valid but not supported (odd S, order != 0, a >= 3) */
    FR_ERR_OOM = 3,           /* a device or host allocation failed */
    FR_ERR_CUDA = 4,          /* a CUDA runtime call failed (see fr_last_cuda_error) */
    FR_ERR_LAUNCH = 5,        /* a configuration could not launch; the work was re-run
                                 with the fallback configuration, so results are valid */
    FR_ERR_DEVICE_ASSERT = 6, /* a device-side range check fired (results invalid) */
    FR_ERR_TIMEOUT = 7,       /* a bounded device wait gave up (results invalid) */
    FR_ERR_IO = 8,            /* a tuning file could not be read or written */
    FR_ERR_STATE = 9,         /* the call is not valid in the context's current state */
    FR_ERR_NOALLOC_LIMIT = 10 /* the size exceeds the fixed scratch of fr_insert_noalloc */
} fr_status;

typedef enum fr_dtype { FR_F32 = 0, FR_F16 = 1 } fr_dtype;

/* Interpolation kernel: generalised Kaiser-Bessel blob (Lewitt 1990).
 *   a          radius in voxels, 0 < a < 3
 *   alpha      taper parameter, 0 <= alpha <= 40
 *   order      must be 0 (FR_ERR_UNSUPPORTED otherwise)
 *   table_size entries of the tabulated blob, 2..16384; the table samples
 *              b at r^2 = i a^2 / (table_size - 1) and is read with linear
 *              interpolation in r^2 (the "precomputed weights" of
 *              Sec. 4.2.10).  The on-the-fly variant ignores it. */
typedef struct fr_blob {
    float a;
    float alpha;
    int order;
    int table_size;
} fr_blob;

typedef struct fr_ctx fr_ctx;

/* Search strategies of the dynamic tuner (Sec. 3 lists random search among
 * KTT's searchers; exhaustive is the "oraculum" protocol of Sec. 5.3.2). */
typedef enum fr_search {
    FR_SEARCH_EXHAUSTIVE = 0, /* every valid configuration once, in a seeded order */
    FR_SEARCH_RANDOM = 1,     /* `budget` configurations drawn without replacement */
    FR_SEARCH_LEARNED = 2,    /* the cost model ranks the space; its top `budget` are measured */
    FR_SEARCH_ANNEALING = 3,  /* simulated annealing over neighbouring configurations */
    FR_SEARCH_MCMC = 4        /* Metropolis walk (constant temperature) over neighbours */
} fr_search;

typedef struct fr_options {
    int tuning;          /* 1: tune dynamically (default); 0: use the cached best or the default */
    int search;          /* fr_search, default FR_SEARCH_EXHAUSTIVE */
    int budget;          /* configurations to measure per key; 0 = the whole space */
    int steps_per_insert;/* tuning steps (sub-batches) one fr_insert may take: >= 1 that many
                            (at most the configurations left and n); 0 (default): automatic, as
                            many as keep every step at >= 2e7 estimated voxel updates (about
                            0.1 ms, so its event timing is accurate), at most 32 */
    int forced_config;   /* >= 0: always use this configuration id; -1 (default): tuner decides */
    uint64_t seed;       /* seed of the search order (default 1) */
    int debug;           /* bit 0: synchronise after every launch and check the device error
                            word; bit 1: collect gather phase counters; bit 2: an NVTX range
                            around every insertion step (named by configuration and images) */
    int fault_config;    /* test hook (host-side fault injection): > 0 makes every launch of
                            configuration fault_config - 1 report a launch failure without
                            enqueuing work, so the fallback path runs; 0 (default): none */
    int fault_alloc;     /* test hook (host-side fault injection): k > 0 makes the k-th device
                            allocation the insertion path attempts after this call (work-unit
                            lists, scratch) fail as out of memory; the step then falls back as
                            for a failed launch.  One shot: reads back as 0 once it has fired.
                            0 (default): none */
    int reserved[6];
} fr_options;

/* What the tuner has done for the context's current key. */
typedef struct fr_report {
    int S;                  /* image size of the current key */
    int n_bucket;           /* batch-size bucket of the current key (log2 of n, rounded down) */
    int space_size;         /* valid configurations for this key */
    int evaluated;          /* configurations measured so far */
    int tuned;              /* 1 once the search has finished */
    int best_config;        /* best configuration id so far (-1 if none) */
    int last_config;        /* configuration used by the last launch */
    int launches;           /* insertion launches on this context */
    double best_ns_per_image;    /* measured time of the best configuration */
    double mean_ns_per_image;    /* mean over the measured configurations (t_avg) */
    double tuning_overhead_pct;  /* 100 (rp - 1), rp of Eq. (performance) over this key's launches */
    unsigned long long images;   /* images inserted since create / reset */
    int retunes;            /* times the tuner started over (fr_retune or a key change) */
    int reserved[7];
} fr_report;

/* ---------------------------------------------------------------- lifecycle */

/* Create a context for images of size S (even, 8 <= S <= 512) and the given
 * blob.  Allocates the context's accumulators on the current CUDA device
 * (about 24 (S+1)^2 (S/2+2) bytes) and its blob table; they are zeroed.
 * Synchronous.  On error *out is set to NULL. */
int fr_create(int S, const fr_blob *blob, fr_ctx **out);

/* Free the context and everything it owns.  Waits for the context's work.
 * NULL is accepted. */
int fr_destroy(fr_ctx *ctx);

/* Zero the accumulators (V = W = 0) on `stream`.  Tuning state is kept. */
int fr_reset(fr_ctx *ctx, void *stream);

/* ---------------------------------------------------------------- insertion */

/* Add the contribution of n images to the context's volume (the insertion
 * step of Algorithm 1).  images: device, [n][S][S/2+1] complex of `dtype`.  rotations:
 * device, [n][9] float32.  0 <= n <= 2^24; n = 0 is a no-op.  Every image is
 * inserted exactly once whatever the tuning state: while tuning, the batch may
 * be split into sub-batches, each run with a different configuration and
 * timed with CUDA events (non-blocking dynamic tuning, Sec. 3.2).  When the
 * search ran in such sub-batch steps, the fastest configuration of each kernel
 * family (direct-drain gather, per-voxel gather, scatter) then runs one whole
 * insert each, and the key's best is the fastest of those whole-insert
 * timings (a gather launch has a fixed cost that a small step does not
 * amortise).  The S of the images is the context's S; a new batch-size bucket
 * starts a new tuning key (cached keys are reused).  images must be 16-byte
 * aligned. */
int fr_insert(fr_ctx *ctx, const void *images, fr_dtype dtype, const float *rotations,
              int n, void *stream);

/* Insert nb batches, batch b into context ctxs[b] (contexts may differ in S
 * and blob and may repeat): several samples in one launch, which the atomic
 * accumulation makes possible (Sec. 5.3.2).  All arrays are host arrays of nb
 * entries; images[b] (16-byte aligned) and rotations[b] are device pointers.
 * Each batch runs the configuration its context's tuner picked for its key
 * (else the context's forced configuration or the default).  Batches whose
 * configurations share a kernel instantiation run in ONE launch over the
 * pooled work units (a brick and a share of a batch's images) of all of them,
 * heaviest units first, so uneven S and n share the GPU without a tail per
 * batch: the direct-drain gather as one CTA per unit (its fold columns in a
 * second launch on a high-priority side stream), the per-voxel gather as a
 * persistent kernel whose CTAs take units from a device counter.  Batches
 * whose configuration has no multi-batch kernel (scatter, tabulated weights)
 * run their own launches after those.  A context that appears more than once
 * receives its sums through its scratch volume with atomics.  The first call
 * with a given (contexts, pointers, sizes, dtypes, configurations) builds a
 * plan and uploads it (synchronously); later calls reuse it.  With capture =
 * 1 the plan's launch sequence is captured, on a stream the library owns,
 * into a CUDA graph at the first call; that call and later ones launch the
 * graph on `stream`.  Same semantics per batch as fr_insert (every image
 * exactly once); no tuning steps are taken here.  Returns FR_ERR_INVALID_ARG
 * for a null context, a misaligned or null pointer with n > 0, n out of
 * range, a bad dtype or contexts on different devices. */
int fr_insert_batched(fr_ctx *const *ctxs, const void *const *images, const fr_dtype *dtypes,
                      const float *const *rotations, const int *n, int nb, int capture,
                      void *stream);

/* Checkpoint of the accumulated volume: the context's six accumulator planes
 * (hi and lo of V.re, V.im, W; fr_state_bytes bytes).  fr_state_save copies
 * them to dst, fr_state_load replaces them with src (host or device memory,
 * any alignment), so that a context of the same S and blob resumes where the
 * saved one stopped: later inserts add to the loaded sums exactly as they
 * would have to the original ones.  Both wait for the context's queued work.
 * Tuning state is saved separately (fr_tuning_save). */
size_t fr_state_bytes(const fr_ctx *ctx);
int fr_state_save(fr_ctx *ctx, void *dst);
int fr_state_load(fr_ctx *ctx, const void *src);

/* Write the accumulated volume: V (device, complex64 (S+1)^3) and W (device,
 * float32 (S+1)^3), [z][y][x].  Raw sums: no normalisation and no Hermitian
 * symmetrisation.  Does not reset.  Checks the device error word first
 * (synchronising the stream). */
int fr_finalize(fr_ctx *ctx, void *V, float *W, void *stream);

/* The image-side step of Algorithm 1 (Sec. 5.3.1; the paper runs it on the
 * CPU and uploads the result): the 2D Fourier transforms of n real images,
 * written in the insertion's input layout and dtype, ready for fr_insert.
 *   real   device float32 [n][S][S] (x fastest), 16-byte aligned; S is the
 *          context's.
 *   out    device [n][S][S/2+1] complex of `dtype` (fr_insert's layout), 16-byte
 *          aligned: out[i][j][kx] = sum_{y,x} real[i][y][x] exp(-2 pi i (kx x +
 *          ky y) / S), ky = j for j < S/2 and j - S otherwise (numpy's rfft2),
 *          times (-1)^(kx + j) when center != 0 (the image origin taken at
 *          pixel (S/2, S/2) instead of (0, 0)); FR_F16 rounds to nearest half.
 *   n      0 <= n <= 2^24 (0: nothing).
 * The transforms are the CUDA toolkit's cuFFT (batched R2C, loaded at run
 * time; FR_ERR_UNSUPPORTED if it cannot be loaded), in chunks of about 256 MB
 * of spectra (at least 256 images); the sign and the FP16 conversion are a
 * kernel of this library.  Allocates on first use the plans and, for FR_F16,
 * a staging buffer of one chunk.
 * Work is enqueued on `stream`. */
int fr_prepare_images(fr_ctx *ctx, const float *real, int n, int center, void *out,
                      fr_dtype dtype, void *stream);

/* The last step of Algorithm 1 (Sec. 5.3.1): apply the weights W to G and
 * transform back, from the context's accumulated sums.  With V, W the raw
 * sums of fr_finalize:
 *     Vs(v) = V(v) + conj(V(-v)),  Ws(v) = W(v) + W(-v)  (undo the fold)
 *     F(k)  = Vs(k) / max(Ws(k), w_clip) / S^3,  k in [-S/2, S/2)^3,
 *             F = 0 on the Nyquist planes kx = S/2, ky = -S/2, kz = -S/2
 *     out   = the real inverse DFT of F: out[z][y][x] (float32, S^3, device,
 *             x fastest, origin at index 0) = sum_k F(k) exp(2 pi i k.r / S)
 * The paper does not spell the weighting out; the clip w_clip > 0 (1 is a
 * good value: a voxel met by about one blob of weight keeps its sum) keeps
 * the division away from zero.  Allocates, on first use, a half-spectrum
 * buffer (8 S^2 (S/2+1) bytes) and an inverse-FFT plan; the inverse FFT is
 * the CUDA toolkit's cuFFT, loaded at run time (FR_ERR_UNSUPPORTED if it
 * cannot be loaded).  Work is enqueued on `stream`.  Returns FR_OK,
 * FR_ERR_INVALID_ARG (null pointer, w_clip <= 0), FR_ERR_OOM, FR_ERR_CUDA. */
int fr_reconstruct(fr_ctx *ctx, float *out, float w_clip, void *stream);

/* ---------------------------------------------------------------- tuning */

/* Forget the tuning results of the current key (or of every key if all != 0);
 * the next inserts tune again. */
int fr_retune(fr_ctx *ctx, int all);

int fr_set_options(fr_ctx *ctx, const fr_options *opt);
int fr_get_options(const fr_ctx *ctx, fr_options *opt);
/* Fill *rep for the context's current key.  Harvests finished timings; does
 * not block. */
int fr_tuning_report(fr_ctx *ctx, fr_report *rep);

/* Per-configuration timings of the current key: up to cap entries of
 * (configuration id, mean ns per image, images timed) into cfg / ns / images
 * (host arrays).  Returns the number of measured configurations (which may
 * exceed cap), or a negative fr_status.  Harvests finished timings first. */
int fr_tuning_measurements(fr_ctx *ctx, int *cfg, double *ns_per_image, double *images, int cap);

/* Persist / restore the tuning cache as JSON keyed by device name, SM count,
 * S, n bucket, a, dtype and the hash of the configuration space. */
int fr_tuning_save(const fr_ctx *ctx, const char *path);
int fr_tuning_load(fr_ctx *ctx, const char *path);

/* Size of the configuration space and a text description of configuration
 * `id` ("gather bx=16 by=16 zc=8 t=2 w=lut" ...).  Returns the number of
 * configurations, or a negative fr_status. */
int fr_num_configs(void);
int fr_describe_config(int id, char *buf, int len);
/* 1 if configuration id can run for this context (resources, blob radius). */
int fr_config_valid(const fr_ctx *ctx, int id);

/* Feature vector (16 floats, normalised) the cost model sees for (config,
 * S, n, a).  Host function. */
int fr_config_features(int id, int S, int n, float a, float *out16);

/* Number of kernel launches one insertion step of n images with
 * configuration id enqueues (*out): the insertion kernels plus the scratch
 * merges.  Builds the configuration's work units if needed (host work and a
 * small device upload, as the first insert with it would); enqueues no
 * kernel.  FR_ERR_INVALID_ARG for a bad id, n < 1 or a null out. */
int fr_insert_launches(fr_ctx *ctx, int id, int n, int *out);

/* ---------------------------------------------------------------- measurement */

/* Exact number of (pixel, voxel) updates that inserting images with these
 * rotations performs (independent of pixel values): pairs with |v - q| <= a
 * inside the volume.  rotations: device [n][9].  Synchronous on `stream`. */
int fr_count_updates(fr_ctx *ctx, const float *rotations, int n, void *stream,
                     unsigned long long *out);

/* Amortisation arithmetic of Sec. 5.4.
 * Eq. (performance): rp = (s t_avg + (n - s) t_well) / (n t_well).
 * Eq. (invocations): n = rp s (t_avg / t_well - 1) / (1 - rp).
 * Eq. (samples):     s = log(1 - p) / log(1 - r)  (random-search steps). */
double fr_relative_performance(double s, double t_avg, double t_well, double n);
double fr_invocations_to_amortize(double rp, double s, double t_avg, double t_well);
double fr_random_search_steps(double r, double p);

/* ---------------------------------------------------------------- diagnostics */

const char *fr_error_string(int status);
/* Reads (synchronising `ctx`'s last stream) and clears the device error word:
 * FR_OK, FR_ERR_DEVICE_ASSERT or FR_ERR_TIMEOUT. */
int fr_last_device_error(fr_ctx *ctx);
/* The last cudaError_t seen by the library (0 if none). */
int fr_last_cuda_error(void);

/* Evaluate the device's exact Hermitian-fold predicate (R00 kx + R01 ky < 0)
 * for m cases: r (device float[2m] pairs R00, R01), k (device int[2m] pairs
 * kx, ky, |k| <= 4096), out (device int[m], 1 = folded).  Test hook for the
 * predicate the insertion kernels use. */
int fr_debug_fold(const float *r, const int *k, int m, int *out, void *stream);

/* Diagnostics of the gather kernel, collected while fr_options.debug has bit
 * 1 set (16 counters): 0 cull, 1 queue, 2-4 drain of fast, edge and kx = 0
 * crossing items, 5 flush (SM clock cycles summed over warps); 6-8 item counts
 * of those three kinds; 9 list images; 10 warp cycles in total; 11 rounds of
 * fast items; 12 drain of fold-column items (cycles); 13 fold-column items.
 * Copies up to cap counters to out (host) and clears them.  Synchronises the
 * device. */
int fr_debug_phase_counters(fr_ctx *ctx, unsigned long long *out, int cap);

/* Evaluate the device blob weight for m squared distances r2 (device float[m])
 * into out (device float[m]): mode 0 the table, mode 1 the Abramowitz & Stegun
 * Bessel approximations, mode 2 the register polynomial.  Test hook. */
int fr_debug_blob(const fr_ctx *ctx, const float *r2, int m, int mode, float *out, void *stream);

/* Host-only simulation of a search order over a table of known times, to
 * compare searchers at equal budgets on measured sweeps.  ns_per_image:
 * host double[nconfig] (nconfig must equal fr_num_configs(); a value <= 0
 * marks an invalid configuration); budget >= 1 distinct configurations;
 * start: the configuration an adaptive walk starts from (any invalid value:
 * a random valid one); order: host int[budget] receives the configurations
 * in the order the searcher measures them (adaptive searchers see each
 * time as soon as they propose it).  search: FR_SEARCH_EXHAUSTIVE, _RANDOM,
 * _ANNEALING or _MCMC (the learned order needs the model: see
 * fr_mlp_forward).  Returns the number of configurations written, or a
 * negative fr_status.  Touches no device. */
int fr_search_simulate(int search, const double *ns_per_image, int nconfig, int budget,
                       uint64_t seed, int start, int *order);

/* ---------------------------------------------------------------- learned tuner */

/* The cost model is a 16-64-64-1 ReLU MLP in FP32 (weights owned by the
 * context's tuner) predicting log(ns per image) of a configuration.  These
 * entry points expose its hand-written CUDA kernels. */

/* Number of parameters (16*64+64 + 64*64+64 + 64+1 = 5313). */
int fr_mlp_num_params(void);
/* params: device float[5313] in the order W1[64][16], b1[64], W2[64][64],
 * b2[64], W3[64], b3 (W[out][in]).  x: device float[m][16]; y: device
 * float[m].  m >= 0. */
int fr_mlp_forward(const float *params, const float *x, int m, float *y, void *stream);
/* Mean-squared-error loss L = (1/m) sum (y - target)^2 over m >= 1 rows and
 * its gradient grad (device float[5313], overwritten); loss (device
 * float[1]).  Deterministic (fixed reduction order). */
int fr_mlp_backward(const float *params, const float *x, const float *target, int m,
                    float *grad, float *loss, void *stream);
/* One Adam step (Kingma & Ba 2015) on params with moments m1, m2 (device
 * float[5313] each), step t >= 1, bias-corrected. */
int fr_mlp_adam(float *params, const float *grad, float *m1, float *m2, int t, float lr,
                float beta1, float beta2, float eps, void *stream);
/* Train the context's model on rows (host arrays: feat[m][16], log time[m])
 * for `epochs` full-batch Adam steps on the GPU (parameters initialised
 * from `seed`, He-uniform); *final_loss receives the last loss.  Synchronous.
 * After training, FR_SEARCH_LEARNED ranks configurations with this model. */
int fr_mlp_train(fr_ctx *ctx, const float *feat, const float *logt, int m, int epochs,
                 float lr, uint64_t seed, float *final_loss);
/* Copy the context's model parameters to / from a host float[5313]. */
int fr_mlp_get(const fr_ctx *ctx, float *params_host);
int fr_mlp_set(fr_ctx *ctx, const float *params_host);

#ifdef __cplusplus
}
#endif

#endif /* FR_H */
