/*
 * fr_oracle.c -- plain FP64 CPU oracle for 3D Fourier insertion.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file: only the tests, the smoke check and the benchmark's
 * cpu_baseline / reference leg use it.  It shares no code, header, table or
 * constant with the CUDA library.
 *
 * What it computes (Algorithm 1, the insertion step of Sec. 5.3.1, with the
 * Fourier-reconstruction tuning space of Sec. 4.2.10 naming the interpolation
 * weights; the paper defers the formula itself to its Xmipp citation, so the
 * following readings are taken: Kaiser-Bessel blob of order 0 normalised to
 * b(0) = 1 with r <= a inclusive; fold iff R00*kx + R01*ky < 0 exactly, zero
 * not folded; every stored pixel of the half plane inserted once, no
 * resolution cut-off; voxels outside the volume dropped; q = R k with R
 * row-major, mapping image to volume coordinates):
 *
 *   for each image i (in order), each stored pixel (row j, column kx):
 *       ky = j < S/2 ? j : j - S                (rfft2 row order)
 *       p  = image[i][j][kx]                    (complex, promoted exactly)
 *       q  = R_i * (kx, ky, 0)^T                (FP64 from the FP32 entries)
 *       if R_i[0][0]*kx + R_i[0][1]*ky < 0:     (Hermitian half-space fold)
 *           q = -q ; p = conj(p)
 *       for every lattice voxel v, |v - q|^2 <= a^2, v in [-S/2, S/2]^3:
 *           w = b(|v - q|) ;  V[v] += w * p ;  W[v] += w
 *
 *   b(r) = I0(alpha * sqrt(1 - (r/a)^2)) / I0(alpha)   (Kaiser-Bessel blob,
 *          order 0, Lewitt 1990), r <= a inclusive, 0 beyond.
 *   I0(x) = sum_k ((x/2)^k / k!)^2                      (textbook series).
 *
 * The scatter is written exactly as above.  The only liberty taken is that
 * several threads may run at once, each owning a contiguous range of z
 * planes of the output and skipping the voxels outside its range; every
 * voxel still receives its contributions in (image, row, column) order, so
 * the result is bit-identical to a single-threaded run.
 *
 * Volume layout: index ((z * (S+1)) + y) * (S+1) + x, coordinate = index - S/2.
 * V is interleaved (re, im) doubles; W is doubles.
 *
 * Parity of every function here is pinned by tests/test_oracle_pins.py
 * (brute force, closed forms, symmetries); none is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Modified Bessel function of the first kind, order 0, by its power series
 * sum_k ((x/2)^k / k!)^2, summed until a term falls below 1e-18 of the sum. */
double fro_i0(double x)
{
    double q = 0.25 * x * x;   /* (x/2)^2 */
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 500; ++k) {
        term *= q / ((double)k * (double)k);
        sum += term;
        if (term < 1e-18 * sum) break;
    }
    return sum;
}

/* Kaiser-Bessel blob of order 0 at distance r (given as r^2). */
double fro_blob_r2(double r2, double a, double alpha)
{
    if (r2 > a * a) return 0.0;
    double s = 1.0 - r2 / (a * a);
    if (s < 0.0) s = 0.0;
    return fro_i0(alpha * sqrt(s)) / fro_i0(alpha);
}

double fro_blob(double r, double a, double alpha)
{
    return fro_blob_r2(r * r, a, alpha);
}

/* Hermitian fold predicate: R00*kx + R01*ky < 0, evaluated so that the sign
 * is exact: each product of an FP32 entry (24-bit significand) and an integer
 * |k| <= 2^9 is exact in FP64, and a correctly rounded sum keeps the sign of
 * the exact sum. */
int fro_fold(float r00, float r01, int kx, int ky)
{
    double x = (double)r00 * (double)kx + (double)r01 * (double)ky;
    return x < 0.0;
}

/* Windowed FP64 scatter of n images into V, W (which are ADDED to, not
 * cleared).  Returns the number of (pixel, voxel) updates performed, or -1 on
 * bad arguments.  nthreads <= 0 uses the OpenMP default. */
long long fro_insert(int S, const float *images, const float *rot, int n,
                     double a, double alpha, double *V, double *W, int nthreads)
{
    if (S < 2 || (S & 1) || n < 0 || a <= 0.0) return -1;
    if (n == 0) return 0;
    const int H = S / 2, NX = S / 2 + 1, D = S + 1;
    const double i0a = fro_i0(alpha);
    const double a2 = a * a;
    long long total = 0;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#else
    nthreads = 1;
#endif
    if (nthreads > D) nthreads = D;

#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads) reduction(+ : total)
#endif
    {
#ifdef _OPENMP
        int t = omp_get_thread_num(), nt = omp_get_num_threads();
#else
        int t = 0, nt = 1;
#endif
        /* this thread owns z indices [z0, z1) */
        int z0 = (int)((long long)D * t / nt), z1 = (int)((long long)D * (t + 1) / nt);
        long long cnt = 0;
        for (int i = 0; i < n; ++i) {
            const float *R = rot + 9 * (size_t)i;
            const float *img = images + (size_t)i * S * NX * 2;
            for (int j = 0; j < S; ++j) {
                int ky = j < H ? j : j - S;
                for (int kx = 0; kx < NX; ++kx) {
                    double pr = img[((size_t)j * NX + kx) * 2 + 0];
                    double pi = img[((size_t)j * NX + kx) * 2 + 1];
                    double qx = (double)R[0] * kx + (double)R[1] * ky;
                    double qy = (double)R[3] * kx + (double)R[4] * ky;
                    double qz = (double)R[6] * kx + (double)R[7] * ky;
                    if (fro_fold(R[0], R[1], kx, ky)) {
                        qx = -qx; qy = -qy; qz = -qz; pi = -pi;
                    }
                    /* lattice box [ceil(q-a), floor(q+a)] clipped to the volume */
                    int xlo = (int)ceil(qx - a), xhi = (int)floor(qx + a);
                    int ylo = (int)ceil(qy - a), yhi = (int)floor(qy + a);
                    int zlo = (int)ceil(qz - a), zhi = (int)floor(qz + a);
                    if (xlo < -H) xlo = -H;
                    if (xhi > H) xhi = H;
                    if (ylo < -H) ylo = -H;
                    if (yhi > H) yhi = H;
                    if (zlo < z0 - H) zlo = z0 - H;
                    if (zhi > z1 - 1 - H) zhi = z1 - 1 - H;
                    for (int z = zlo; z <= zhi; ++z) {
                        double dz = z - qz;
                        for (int y = ylo; y <= yhi; ++y) {
                            double dy = y - qy;
                            for (int x = xlo; x <= xhi; ++x) {
                                double dx = x - qx;
                                double r2 = dx * dx + dy * dy + dz * dz;
                                if (r2 > a2) continue;
                                double s = 1.0 - r2 / a2;
                                if (s < 0.0) s = 0.0;
                                double w = fro_i0(alpha * sqrt(s)) / i0a;
                                size_t v = ((size_t)(z + H) * D + (size_t)(y + H)) * D + (size_t)(x + H);
                                V[2 * v + 0] += w * pr;
                                V[2 * v + 1] += w * pi;
                                W[v] += w;
                                ++cnt;
                            }
                        }
                    }
                }
            }
        }
        total += cnt;
    }
    return total;
}

/* The same definition evaluated at single voxels, by brute force over every
 * pixel of every image: used to check full-size GPU results at sampled
 * voxels.  vox holds nv (x, y, z) coordinates in [-S/2, S/2].  Outputs
 * Vout[2*nv] (re, im) and Wout[nv] (overwritten). */
int fro_voxels(int S, const float *images, const float *rot, int n, double a,
               double alpha, const int *vox, int nv, double *Vout, double *Wout,
               int nthreads)
{
    if (S < 2 || (S & 1) || n < 0 || nv < 0) return -1;
    const int H = S / 2, NX = S / 2 + 1;
    const double i0a = fro_i0(alpha), a2 = a * a;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 1)
#endif
    for (int s = 0; s < nv; ++s) {
        double vx = vox[3 * s], vy = vox[3 * s + 1], vz = vox[3 * s + 2];
        double sr = 0, si = 0, sw = 0;
        for (int i = 0; i < n; ++i) {
            const float *R = rot + 9 * (size_t)i;
            const float *img = images + (size_t)i * S * NX * 2;
            for (int j = 0; j < S; ++j) {
                int ky = j < H ? j : j - S;
                for (int kx = 0; kx < NX; ++kx) {
                    double qx = (double)R[0] * kx + (double)R[1] * ky;
                    double qy = (double)R[3] * kx + (double)R[4] * ky;
                    double qz = (double)R[6] * kx + (double)R[7] * ky;
                    double sg = 1.0;
                    if (fro_fold(R[0], R[1], kx, ky)) { qx = -qx; qy = -qy; qz = -qz; sg = -1.0; }
                    double dx = vx - qx, dy = vy - qy, dz = vz - qz;
                    double r2 = dx * dx + dy * dy + dz * dz;
                    if (r2 > a2) continue;
                    double t = 1.0 - r2 / a2;
                    if (t < 0.0) t = 0.0;
                    double w = fro_i0(alpha * sqrt(t)) / i0a;
                    sr += w * img[((size_t)j * NX + kx) * 2 + 0];
                    si += w * sg * img[((size_t)j * NX + kx) * 2 + 1];
                    sw += w;
                }
            }
        }
        Vout[2 * s] = sr; Vout[2 * s + 1] = si; Wout[s] = sw;
    }
    return 0;
}

/* Number of (pixel, voxel) updates the definition performs for these
 * rotations (independent of the pixel values). */
long long fro_count(int S, const float *rot, int n, double a, int nthreads)
{
    if (S < 2 || (S & 1) || n < 0) return -1;
    const int H = S / 2, NX = S / 2 + 1;
    const double a2 = a * a;
    long long total = 0;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for num_threads(nthreads) reduction(+ : total) schedule(dynamic, 1)
#endif
    for (int i = 0; i < n; ++i) {
        const float *R = rot + 9 * (size_t)i;
        long long cnt = 0;
        for (int j = 0; j < S; ++j) {
            int ky = j < H ? j : j - S;
            for (int kx = 0; kx < NX; ++kx) {
                double qx = (double)R[0] * kx + (double)R[1] * ky;
                double qy = (double)R[3] * kx + (double)R[4] * ky;
                double qz = (double)R[6] * kx + (double)R[7] * ky;
                if (fro_fold(R[0], R[1], kx, ky)) { qx = -qx; qy = -qy; qz = -qz; }
                int xlo = (int)ceil(qx - a), xhi = (int)floor(qx + a);
                int ylo = (int)ceil(qy - a), yhi = (int)floor(qy + a);
                int zlo = (int)ceil(qz - a), zhi = (int)floor(qz + a);
                if (xlo < -H) xlo = -H;
                if (xhi > H) xhi = H;
                if (ylo < -H) ylo = -H;
                if (yhi > H) yhi = H;
                if (zlo < -H) zlo = -H;
                if (zhi > H) zhi = H;
                for (int z = zlo; z <= zhi; ++z)
                    for (int y = ylo; y <= yhi; ++y)
                        for (int x = xlo; x <= xhi; ++x) {
                            double dx = x - qx, dy = y - qy, dz = z - qz;
                            if (dx * dx + dy * dy + dz * dz <= a2) ++cnt;
                        }
            }
        }
        total += cnt;
    }
    return total;
}

int fro_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
