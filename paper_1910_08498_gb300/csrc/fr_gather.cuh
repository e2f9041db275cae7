// fr_gather.cuh -- the per-voxel gather insertion kernel (primary variant).
//
// The volume half x >= -floor(a) that folding can reach is cut into warp
// footprints of 8 x 4 voxel columns, ZC voxels deep; a CTA groups BX/8 x BY/4
// footprints (and shares the blob table in shared memory).  Each warp is the
// only writer of its footprint's voxels for the whole launch, so V and W in
// HBM need no atomics, and warps never wait for one another.
//
// Per warp and launch:
//  1. cull (A2): one image per lane; an image is kept if its central plane
//     passes within a + (footprint radius) of the footprint centre and its
//     extended plane reaches the footprint.  Kept images go, in order, to a
//     warp-private shared-memory list (one 64-byte record per image, read as
//     four 16-byte groups) holding the plane basis and the footprint centre's
//     projection R^T c, formed with error-free
//     products and split into an integer part and a small remainder so that
//     in-plane positions keep ~1e-7 absolute accuracy at any |k|;
//  2. queue: for each list image the warp marks the voxels within a of the
//     plane (|u_z| <= a, u = R^T v) whose projection lies within the extended
//     plane [-S/2-a, S/2+a]^2, and appends them, as (image, voxel) items, to a
//     warp-private queue (warp prefix sums, image-major order);
//  3. accumulate (A4): all 32 lanes drain the queue, one item per lane, so no
//     lane idles on a voxel that is far from the plane.  An item visits the
//     KB x KB pixel box around (u_x, u_y) of the Hermitian-extended, folded
//     image plane and forms sum b(r) p and sum b(r) over the pixels with
//     r^2 = (u_x-kx)^2 + (u_y-ky)^2 + u_z^2 <= a^2 (weights from the blob
//     table in shared memory, or on the fly: a register-held polynomial in
//     r^2 or the Abramowitz & Stegun Bessel approximations).
//     Pixels are read through L1; consecutive items are neighbouring voxels of
//     one image, so their boxes share sectors.  A box wholly in the stored half
//     plane (kx >= 1) or wholly in its mirror (kx <= -1), inside the image, for
//     a voxel away from the fold plane (x > floor(a)), needs no fold or range
//     test (the mirror half is read point-reflected and conjugated); every
//     other box takes a careful path with the exact fold predicate and range
//     tests per pixel.  The item's three sums are added to the warp's
//     shared-memory accumulators;
//  4. write back (A5): every FLUSH list images and at the end, the warp folds
//     its shared-memory partial sums into the HBM double-float accumulators
//     (error-free TwoSum), so no FP32 partial sum runs over more than FLUSH
//     images.  A launch may split the images of a batch across nsplit CTAs
//     per brick (the bricks at the centre meet every plane and would otherwise
//     run alone at the end); then each CTA adds its partial sums to a float4
//     scratch volume with atomics, folded into the accumulators after the
//     launch.
//  Fast and careful items are queued apart, so a careful item never holds a
//  whole round of fast ones; for polynomial weights the fast box is branch
//  free (packed FP32x2 FMAs, weights masked to 0 outside the blob).
#pragma once

#include "fr_device.cuh"

namespace fr {

// number of 4-byte fields per kept image in the shared-memory list: one
// 64-byte record per image, the fields grouped by use so that each group is
// one 16-byte load (plane normal and distance; first in-plane axis and the
// fractional x; second axis and fractional y; integer centre and the
// image's address)
constexpr int LIST_FIELDS = 16;
enum ListField {
  LF_MX, LF_MY, LF_MZ, LF_UZ, LF_E1X, LF_E1Y, LF_E1Z, LF_FX,
  LF_E2X, LF_E2Y, LF_E2Z, LF_FY, LF_CIX, LF_CIY, LF_ADLO, LF_ADHI
};

// the image address held by a list entry
__device__ __forceinline__ const unsigned char *list_image(const float *L) {
  const unsigned long long lo = __float_as_uint(L[LF_ADLO]), hi = __float_as_uint(L[LF_ADHI]);
  return reinterpret_cast<const unsigned char *>(lo | (hi << 32));
}

// e . c with compensated products and sums (Ogita-Rump-Oishi Dot2), returned
// as an unevaluated pair hi + lo; accurate to ~2^-48 relative.
__device__ __forceinline__ void dot3_dd(float e0, float e1, float e2, float c0, float c1,
                                        float c2, float &hi, float &lo) {
  float p0 = e0 * c0, q0 = fmaf(e0, c0, -p0);
  float p1 = e1 * c1, q1 = fmaf(e1, c1, -p1);
  float p2 = e2 * c2, q2 = fmaf(e2, c2, -p2);
  float s, t1, t2;
  two_sum(p0, p1, s, t1);
  two_sum(s, p2, hi, t2);
  lo = (q0 + q1 + q2) + (t1 + t2);
}

// true if any column of a warp footprint whose lowest column is (fx0, fy0) is inside the volume
__device__ __forceinline__ bool col_in_any(const Geom &g, int fx0, int fy0) {
  return fx0 <= g.H && fy0 <= g.H;
}

constexpr int GATHER_FLUSH = 256;  // list images between flushes of the shared partial sums

template <int F16>
__device__ __forceinline__ float2 ld_px(const unsigned char *p) {
  if (F16) return __half22float2(__ldg(reinterpret_cast<const __half2 *>(p)));
  return __ldg(reinterpret_cast<const float2 *>(p));
}

// Fast path: every pixel of the box is stored (sgn = +1: pixels (kx0+j,
// ky0+l)) or point-reflected (sgn = -1: pixels (-kx0-j, -ky0-l), conjugated
// by the caller); no fold, range or multiplicity test.  One copy of the body
// serves both (runtime sign), rows are not unrolled, and a row whose distance
// to the voxel already exceeds a is skipped.
template <int WMODE, int KB, int F16>
__device__ __forceinline__ void box_fast(const InsertArgs &args, const float2 *lut,
                                         const unsigned char *ibase, int sgn, int kx0, int ky0,
                                         float fx, float fy, float uz2, float inv_a2, float &sr,
                                         float &si, float &sw) {
  const Geom &g = args.g;
  constexpr int ESZ = F16 ? 4 : 8;
  const int row_bytes = g.NX * ESZ;
  const int step = sgn * ESZ;
#pragma unroll 1
  for (int l = 0; l < KB; ++l) {
    const float dy = fy - (float)l;
    const float ry = fmaf(dy, dy, uz2);
    if (ry > g.a2) continue;
    int ky = sgn * (ky0 + l);
    ky += ky < 0 ? g.S : 0;
    const unsigned char *row = ibase + (ky * row_bytes + sgn * kx0 * ESZ);
#pragma unroll
    for (int j = 0; j < KB; ++j) {
      const float dx = fx - (float)j;
      const float r2 = fmaf(dx, dx, ry);
      if (r2 <= g.a2) {
        const float w = blob_w<WMODE>(lut, r2, args, inv_a2);
        const float2 p = ld_px<F16>(row + j * step);
        sr = fmaf(w, p.x, sr);
        si = fmaf(w, p.y, si);
        sw += w;
      }
    }
  }
}

// Branch-free fast boxes for the polynomial weights.  The polynomial is split
// into even and odd parts, E(x^2) + x O(x^2), evaluated together with packed
// FP32x2 FMAs (c holds (c_0, c_1), (c_2, c_3), ... pairs).
__device__ __forceinline__ float poly_eo(const float2 *c, float x) {
  constexpr int NP = POLY_N / 2;
  const float x2 = x * x;
  float2 eo = c[NP - 1];
#pragma unroll
  for (int k = NP - 2; k >= 0; --k) eo = __ffma2_rn(eo, make_float2(x2, x2), c[k]);
  return fmaf(eo.y, x, eo.x);
}

// Interior box: every pixel of the KB x KB box exists, so all candidates are
// evaluated with no branch at all; weights outside r <= a are masked to 0.
template <int KB, int F16>
__device__ __forceinline__ void box_poly_interior(const InsertArgs &args, const float2 *c,
                                                  const unsigned char *ibase, int sgn, int kx0,
                                                  int ky0, float fx, float fy, float uz2,
                                                  float two_inv_a2, float &sr, float &si,
                                                  float &sw) {
  const Geom &g = args.g;
  constexpr int ESZ = F16 ? 4 : 8;
  const int row_bytes = g.NX * ESZ;
  // columns in memory order: the box's columns kx0 .. kx0 + KB - 1 when
  // direct, the mirrored -(kx0 + KB - 1) .. -kx0 when mirrored; memory column
  // m is box column j = m (direct) or KB - 1 - m (mirrored), so
  // dx = fx - j = dx0 + dxs m, and the loads take constant offsets
  const int cfirst = sgn > 0 ? kx0 : -(kx0 + KB - 1);
  const float dx0 = sgn > 0 ? fx : fx - (float)(KB - 1);
  const float dxs = sgn > 0 ? -1.0f : 1.0f;
  // all pixel loads first (they do not depend on the weights), then the math
  float2 px[KB * KB];
#pragma unroll
  for (int l = 0; l < KB; ++l) {
    int ky = sgn * (ky0 + l);
    ky += ky < 0 ? g.S : 0;
    const unsigned char *row = ibase + (ky * row_bytes + cfirst * ESZ);
#pragma unroll
    for (int m = 0; m < KB; ++m) px[l * KB + m] = ld_px<F16>(row + m * ESZ);
  }
  float ar = sr, ai = si, aw = sw;
#pragma unroll
  for (int l = 0; l < KB; ++l) {
    const float dy = fy - (float)l;
    const float ry = fmaf(dy, dy, uz2);
#pragma unroll
    for (int j = 0; j < KB; ++j) {
      const float dx = fmaf(dxs, (float)j, dx0);
      const float r2 = fmaf(dx, dx, ry);
      const float pv = poly_eo(c, fmaf(r2, two_inv_a2, -1.0f));
      const float w = r2 <= g.a2 ? pv : 0.0f;
      const float2 p = px[l * KB + j];
      ar = fmaf(w, p.x, ar);
      ai = fmaf(w, p.y, ai);
      aw += w;
    }
  }
  sr = ar;
  si = ai;
  sw = aw;
}

// Edge box: the box crosses the image border; rows and columns outside the
// stored (or mirrored) pixels get weight 0 and read a valid pixel instead.
template <int KB, int F16>
__device__ __forceinline__ void box_poly_edge(const InsertArgs &args, const float2 *c,
                                              const unsigned char *ibase, int sgn, int kx0,
                                              int ky0, float fx, float fy, float uz2,
                                              float two_inv_a2, float &sr, float &si,
                                              float &sw) {
  const Geom &g = args.g;
  constexpr int ESZ = F16 ? 4 : 8;
  const int row_bytes = g.NX * ESZ;
  const int step = sgn * ESZ;
  unsigned colok = 0;  // valid pixel columns pc = sgn (kx0 + j) in [1, H]
#pragma unroll
  for (int j = 0; j < KB; ++j) {
    const int pc = sgn * (kx0 + j);
    colok |= (pc >= 1 && pc <= g.H ? 1u : 0u) << j;
  }
  if (!colok) return;
  const int jsafe = __ffs(colok) - 1;
  float ar = sr, ai = si, aw = sw;
#pragma unroll 1
  for (int l = 0; l < KB; ++l) {
    int ky = sgn * (ky0 + l);
    if (ky < -g.H || ky >= g.H) continue;
    ky += ky < 0 ? g.S : 0;
    const float dy = fy - (float)l;
    const float ry = fmaf(dy, dy, uz2);
    const unsigned char *row = ibase + (ky * row_bytes + sgn * kx0 * ESZ);
#pragma unroll
    for (int j = 0; j < KB; ++j) {
      const float dx = fx - (float)j;
      const float r2 = fmaf(dx, dx, ry);
      const bool ok = ((colok >> j) & 1u) != 0;
      const float pv = poly_eo(c, fmaf(r2, two_inv_a2, -1.0f));
      const float w = (r2 <= g.a2 && ok) ? pv : 0.0f;
      const float2 p = ld_px<F16>(row + (ok ? j : jsafe) * step);
      ar = fmaf(w, p.x, ar);
      ai = fmaf(w, p.y, ai);
      aw += w;
    }
  }
  sr = ar;
  si = ai;
  sw = aw;
}

// Box crossing the column kx = 0, for a voxel with x > floor(a).  Every point
// R c of the extended plane within a of such a voxel has (R c)_x > 0, so no
// fold test is needed: a column c_x > 0 reads the stored pixel c, a column
// c_x < 0 reads the stored -c conjugated, and the column c_x = 0 reads both
// (0, c_y) and, conjugated, (0, -c_y) -- the rfft column kx = 0 holds both
// halves, and the stored one of each pair that lands at -R c is folded onto
// R c.  Branch free: pixels outside the image get weight 0 and read pixel 0.
template <int KB, int F16>
__device__ __forceinline__ void box_poly_straddle(const InsertArgs &args, const float2 *c,
                                                  const unsigned char *ibase, int kx0, int ky0,
                                                  float fx, float fy, float uz2,
                                                  float two_inv_a2, float &sr, float &si,
                                                  float &sw) {
  const Geom &g = args.g;
  constexpr int ESZ = F16 ? 4 : 8;
  const int row_bytes = g.NX * ESZ;
  const int j0 = -kx0;  // box column of kx = 0, in [0, KB)
  const float dx0 = fx - (float)j0;
  float ar = 0.f, ai = 0.f, aw = 0.f;
#pragma unroll 1
  for (int l = 0; l < KB; ++l) {
    const int cy = ky0 + l;
    const bool dok = cy >= -g.H && cy < g.H;  // row of the direct pixel (., cy) is stored
    const bool mok = cy > -g.H && cy <= g.H;  // row of the mirrored pixel (., -cy) is stored
    const int drow = dok ? (cy < 0 ? cy + g.S : cy) : 0;
    const int mrow = mok ? (cy > 0 ? g.S - cy : -cy) : 0;
    const float dy = fy - (float)l;
    const float ry = fmaf(dy, dy, uz2);
#pragma unroll
    for (int j = 0; j < KB; ++j) {
      const int cx = kx0 + j;
      const bool neg = cx < 0;
      const int pc = neg ? -cx : cx;
      const bool ok = pc <= g.H && (neg ? mok : dok);
      const float dx = fx - (float)j;
      const float r2 = fmaf(dx, dx, ry);
      const float pv = poly_eo(c, fmaf(r2, two_inv_a2, -1.0f));
      const float w = (r2 <= g.a2 && ok) ? pv : 0.0f;
      const int off = ok ? ((neg ? mrow : drow) * row_bytes + pc * ESZ) : 0;
      const float2 p = ld_px<F16>(ibase + off);
      ar = fmaf(w, p.x, ar);
      ai = fmaf(neg ? -w : w, p.y, ai);
      aw += w;
    }
    // column kx = 0, second half: stored (0, -cy), conjugated
    const float r2 = fmaf(dx0, dx0, ry);
    const float pv = poly_eo(c, fmaf(r2, two_inv_a2, -1.0f));
    const float w = (r2 <= g.a2 && mok) ? pv : 0.0f;
    const float2 p = ld_px<F16>(ibase + mrow * row_bytes);
    ar = fmaf(w, p.x, ar);
    ai = fmaf(-w, p.y, ai);
    aw += w;
  }
  sr = ar;
  si = ai;
  sw = aw;
}

// Box of a voxel in a fold column (x <= floor(a)): the point R c of the
// extended plane receives the stored pixel c when it is not folded (c_x >= 0,
// R00 c_x + R01 c_y >= 0) and, conjugated, the stored pixel -c when that one is
// folded (-c_x >= 0, R00 c_x + R01 c_y > 0) -- both for c_x = 0.  The signs are
// exact (fold_pred).  Candidates whose FP32 r^2 is within rounding of a^2 are
// left out of the branch-free pass and re-decided exactly afterwards (rare);
// the DC pixel takes the exact |v|^2.
template <int KB, int F16>
__device__ __forceinline__ void box_poly_fold(const InsertArgs &args, const float2 *c,
                                              const unsigned char *ibase, const float *e,
                                              int kx0, int ky0, float fx, float fy, float uz2,
                                              int vx, int vy, int vz, float two_inv_a2,
                                              float &sr, float &si, float &sw) {
  const Geom &g = args.g;
  constexpr int ESZ = F16 ? 4 : 8;
  const int row_bytes = g.NX * ESZ;
  const float r00 = e[0], r01 = e[3];  // e = (e1x, e1y, e1z, e2x, e2y, e2z)
  const float vr2 = (float)(vx * vx + vy * vy + vz * vz);
  const float a2 = g.a2, tie_band = 1e-5f * g.a2;
  const int j0 = -kx0;  // box column of kx = 0 (may lie outside [0, KB))
  const bool has0 = j0 >= 0 && j0 < KB;
  const float dx0 = fx - (float)j0;
  unsigned long long ties = 0;
  float ar = 0.f, ai = 0.f, aw = 0.f;
  // contributions of box pixel (j, l) with weight w: the main pixel (c itself
  // for c_x >= 0, -c for c_x < 0) and, in column kx = 0, the mirrored one
  auto pixel = [&](int j, int l, float w) {
    const int cx = kx0 + j, cy = ky0 + l;
    const bool neg = cx < 0;
    const int pc = neg ? -cx : cx, pr = neg ? -cy : cy;
    const bool st = pc <= g.H && pr >= -g.H && pr < g.H;
    const bool fo = st && fold_pred(r00, r01, pc, pr);
    const bool ok = st && (neg ? fo : !fo);
    const float wm = ok ? w : 0.f;
    const float2 p = ld_px<F16>(ibase + (ok ? (pr < 0 ? pr + g.S : pr) * row_bytes + pc * ESZ : 0));
    ar = fmaf(wm, p.x, ar);
    ai = fmaf(neg ? -wm : wm, p.y, ai);
    aw += wm;
  };
  auto column0 = [&](int l, float w) {
    const int my = -(ky0 + l);
    const bool st = my >= -g.H && my < g.H;
    const bool ok = st && fold_pred(r00, r01, 0, my);
    const float wm = ok ? w : 0.f;
    const float2 p = ld_px<F16>(ibase + (ok ? (my < 0 ? my + g.S : my) * row_bytes : 0));
    ar = fmaf(wm, p.x, ar);
    ai = fmaf(-wm, p.y, ai);
    aw += wm;
  };
#pragma unroll 1
  for (int l = 0; l < KB; ++l) {
    const int cy = ky0 + l;
    const float dy = fy - (float)l;
    const float ry = fmaf(dy, dy, uz2);
#pragma unroll
    for (int j = 0; j < KB; ++j) {
      const int cx = kx0 + j;
      const bool dc = cx == 0 && cy == 0;
      const float dx = fx - (float)j;
      const float r2 = dc ? vr2 : fmaf(dx, dx, ry);
      const bool tie = !dc && fabsf(r2 - a2) <= tie_band;
      ties |= (tie ? 1ull : 0ull) << (l * KB + j);
      const float pv = poly_eo(c, fmaf(r2, two_inv_a2, -1.0f));
      pixel(j, l, (r2 <= a2 && !tie) ? pv : 0.f);
    }
    // the kx = 0 column's second pixel (0, -cy), when the box holds that column
    if (has0) {
      const bool dc0 = cy == 0;
      const float r2 = dc0 ? vr2 : fmaf(dx0, dx0, ry);
      const bool tie0 = !dc0 && fabsf(r2 - a2) <= tie_band;
      const float pv = poly_eo(c, fmaf(r2, two_inv_a2, -1.0f));
      column0(l, (r2 <= a2 && !tie0) ? pv : 0.f);
    }
  }
  // candidates within rounding of the blob edge: decide as the real numbers do
  while (ties) {
    const int b = __ffsll((long long)ties) - 1;
    ties &= ties - 1;
    const int l = b / KB, j = b - l * KB;
    const int cx = kx0 + j, cy = ky0 + l;
    if (!exact_r2_le_a2(vx, vy, vz, e[0], e[1], e[2], e[3], e[4], e[5], cx, cy, g.a)) continue;
    const float dx = fx - (float)j, dy = fy - (float)l;
    const float r2 = fminf(fmaf(dx, dx, fmaf(dy, dy, uz2)), a2);
    const float w = poly_eo(c, fmaf(r2, two_inv_a2, -1.0f));
    pixel(j, l, w);
    if (cx == 0) column0(l, w);
  }
  sr = ar;
  si = ai;
  sw = aw;
}

// Careful path: any box, exact fold predicate (when near the fold plane) and
// range tests per pixel; the W weight counts each contribution.
template <int WMODE, int KB, int F16>
__device__ __noinline__ void box_careful(const InsertArgs &args, const float2 *lut,
                                         const unsigned char *ibase, const float *e,
                                         int kx0, int ky0, float fx, float fy, float uz2,
                                         bool fold_check, int vx, int vy, int vz, float inv_a2,
                                         float &sr, float &si, float &sw) {
  const float r00 = e[0], r01 = e[3];  // e = (e1x, e1y, e1z, e2x, e2y, e2z)
  const float vr2 = (float)(vx * vx + vy * vy + vz * vz);
  const Geom &g = args.g;
  constexpr int ESZ = F16 ? 4 : 8;
  for (int l = 0; l < KB; ++l) {
    const float dy = fy - (float)l;
    const float ry = fmaf(dy, dy, uz2);
    const int cy = ky0 + l;
    for (int j = 0; j < KB; ++j) {
      const int cx = kx0 + j;
      const float dx = fx - (float)j;
      // the DC pixel sits at q = 0 exactly for every rotation: use the exact
      // |v|^2 so that a lattice voxel at distance exactly a is decided as the
      // definition decides it
      const float r2 = (cx == 0 && cy == 0) ? vr2 : fmaf(dx, dx, ry);
      // within rounding of the blob edge: decide as the real numbers do
      if (fabsf(r2 - g.a2) <= 1e-5f * g.a2 && !(cx == 0 && cy == 0)) {
        if (!exact_r2_le_a2(vx, vy, vz, e[0], e[1], e[2], e[3], e[4], e[5], cx, cy, g.a)) continue;
      } else if (!(r2 <= g.a2)) {
        continue;
      }
      const float w = blob_w<WMODE>(lut, r2, args, inv_a2);
      // stored pixel c, not folded
      if (cx >= 0 && cx <= g.H && cy >= -g.H && cy < g.H &&
          (!fold_check || !fold_pred(r00, r01, cx, cy))) {
        const int row = cy < 0 ? cy + g.S : cy;
        float2 p = ld_px<F16>(ibase + ((size_t)row * g.NX + cx) * ESZ);
        sr = fmaf(w, p.x, sr);
        si = fmaf(w, p.y, si);
        sw += w;
      }
      // stored pixel -c, folded, enters conjugated
      const int mx = -cx, my = -cy;
      if (mx >= 0 && mx <= g.H && my >= -g.H && my < g.H &&
          (!fold_check || fold_pred(r00, r01, mx, my))) {
        const int row = my < 0 ? my + g.S : my;
        float2 p = ld_px<F16>(ibase + ((size_t)row * g.NX + mx) * ESZ);
        sr = fmaf(w, p.x, sr);
        si = fmaf(-w, p.y, si);
        sw += w;
      }
    }
  }
}

// Cull one step of 32 images [cs, cs + 32) ∩ [cs, img1) for a warp footprint
// centred at (cx, cy, cz) with half extents (hx, hy, hz): one image per lane;
// an image is kept if its plane passes within a of the footprint box and its
// extended plane [-H - a, H + a]^2 can reach the footprint (|R^T c| <= ext in
// plane).  Kept images are appended in order to the warp's list s_list
// (LIST_FIELDS floats per entry) starting at entry nl, with the centre's
// projection R^T c formed with compensated products (Dot2) and split into an
// integer part and a small remainder, and the address of the image (imgs +
// i img_stride, as two 32-bit halves).  Returns the new list length.
__device__ __forceinline__ int cull_step(const InsertArgs &args, const unsigned char *imgs,
                                         size_t img_stride, float *s_list, int nl, int cs,
                                         int img1, float cx, float cy, float cz, float hx,
                                         float hy, float hz, float ext, bool any_col) {
  const int lane = threadIdx.x & 31;
  const int i = cs + lane;
  bool keep = false;
  float e1x = 0, e1y = 0, e1z = 0, e2x = 0, e2y = 0, e2z = 0, mx = 0, my = 0, mz = 0;
  if (i < img1) {
    const float *R = args.rot + 9 * (size_t)i;
    e1x = __ldg(R + 0); e1y = __ldg(R + 3); e1z = __ldg(R + 6);
    e2x = __ldg(R + 1); e2y = __ldg(R + 4); e2z = __ldg(R + 7);
    mx = __ldg(R + 2);  my = __ldg(R + 5);  mz = __ldg(R + 8);
    const float d = mx * cx + my * cy + mz * cz;
    const float ux = e1x * cx + e1y * cy + e1z * cz;
    const float uy = e2x * cx + e2y * cy + e2z * cz;
    // the plane's distance to the footprint box is |d| minus its support
    const float supp = fabsf(mx) * hx + fabsf(my) * hy + fabsf(mz) * hz;
    keep = any_col && fabsf(d) <= args.g.a + supp + 1e-3f && fabsf(ux) <= ext && fabsf(uy) <= ext;
  }
  const unsigned bal = __ballot_sync(0xffffffffu, keep);
  if (keep) {
    const int o = nl + __popc(bal & ((1u << lane) - 1u));
    float *L = s_list + (size_t)o * LIST_FIELDS;
    float hxx, lx, hyy, ly, hzz, lz;
    dot3_dd(e1x, e1y, e1z, cx, cy, cz, hxx, lx);
    dot3_dd(e2x, e2y, e2z, cx, cy, cz, hyy, ly);
    dot3_dd(mx, my, mz, cx, cy, cz, hzz, lz);
    const float rx = rintf(hxx), ry = rintf(hyy);
    L[LF_E1X] = e1x; L[LF_E1Y] = e1y; L[LF_E1Z] = e1z;
    L[LF_E2X] = e2x; L[LF_E2Y] = e2y; L[LF_E2Z] = e2z;
    L[LF_MX] = mx;   L[LF_MY] = my;   L[LF_MZ] = mz;
    L[LF_FX] = (hxx - rx) + lx;  // hxx - rx is exact
    L[LF_FY] = (hyy - ry) + ly;
    L[LF_UZ] = hzz + lz;
    L[LF_CIX] = __int_as_float((int)rx);
    L[LF_CIY] = __int_as_float((int)ry);
    const unsigned long long ad = reinterpret_cast<unsigned long long>(imgs + (size_t)i * img_stride);
    L[LF_ADLO] = __uint_as_float((unsigned)ad);
    L[LF_ADHI] = __uint_as_float((unsigned)(ad >> 32));
  }
  return nl + __popc(bal);
}

// Fold a warp's shared partial sums (s_acc: [3][32 ZC], slot lane * ZC + t for
// the voxel (fx0 + lane % FW, fy0 + lane / FW, z0 + t); FW = 8 for the 8 x 4
// footprint, 4 for the 4 x 8 one) into HBM and clear them:
// straight into the double-float accumulators (error-free TwoSum) when the
// warp is the only writer of its voxels, else into the float4 scratch with
// atomics (merged after the launch).
template <int ZC, int FW = 8>
__device__ __forceinline__ void flush_partials(const InsertArgs &args, float *s_acc, int fx0,
                                               int fy0, int z0, bool to_scratch) {
  constexpr int WV = 32 * ZC;
  const Geom &g = args.g;
  const int lane = threadIdx.x & 31;
  const int vx = fx0 + lane % FW, vy = fy0 + lane / FW;
  __syncwarp();
  if (vx <= g.H && vy <= g.H) {
#pragma unroll
    for (int t = 0; t < ZC; ++t) {
      const int vz = z0 + t;
      if (vz > g.H) break;
      const size_t v =
          ((size_t)(vz + g.H) * g.D + (size_t)(vy + g.H)) * g.NXa + (size_t)(vx - g.xa0);
      const float ar = s_acc[lane * ZC + t], ai = s_acc[WV + lane * ZC + t],
                  aw = s_acc[2 * WV + lane * ZC + t];
      if (aw != 0.f || ar != 0.f || ai != 0.f) {
        if (!to_scratch) {
          const float add[3] = {ar, ai, aw};
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            float h = args.acc[c * args.plane + v], l = args.acc[(3 + c) * args.plane + v];
            dd_add(h, l, add[c]);
            args.acc[c * args.plane + v] = h;
            args.acc[(3 + c) * args.plane + v] = l;
          }
        } else {
          atomicAdd(args.scratch + v, make_float4(ar, ai, aw, 0.f));
        }
      }
    }
  }
#pragma unroll
  for (int t = 0; t < ZC; ++t)
#pragma unroll
    for (int c = 0; c < 3; ++c) s_acc[c * WV + lane * ZC + t] = 0.f;
  __syncwarp();
}

// Per-warp shared memory of the gather: image list, partial sums, item queues.
__host__ __device__ constexpr size_t gather_warp_smem(int zc, int chunk) {
  return (size_t)LIST_FIELDS * chunk * 4 + (size_t)3 * (32 * zc) * 4 + (size_t)4 * (32 * zc + 32) * 2;
}

// Bytes of the InsertArgs copy at the head of each warp's shared memory in
// the persistent gather.
constexpr size_t GATHER_ARGS_BYTES = (sizeof(InsertArgs) + 15) & ~(size_t)15;

// One warp's share of one work unit: the 8 x 4 x ZC footprint `warp` of the
// brick (unit.x, unit.y, unit.z), over the images of the unit's split.
// unit.w = split | nsplit << 16 | scratch << 30; partial sums go to the
// double-float accumulators when the unit is the only writer of its brick
// (nsplit == 1, no scratch flag), else to the float4 scratch with atomics.
// wsmem is the warp's gather_warp_smem(args.chunk) bytes; lut the shared blob
// table (W_LUT only).  No CTA-wide barrier is taken.
template <int BX, int BY, int ZC, int WMODE, int KB, int F16>
__device__ __forceinline__ void gather_warp(const InsertArgs &args, const InsertArgs &cst,
                                            const void *images, const float2 *lut,
                                            unsigned char *wsmem, const int4 unit,
                                            const int warp) {
  constexpr int WV = 32 * ZC;                   // voxels per warp footprint
  constexpr int QCAP = WV + 32;                 // entries per queue
  constexpr int ESZ = F16 ? 4 : 8;
  static_assert(BX % 8 == 0 && BY % 4 == 0 && (BX * BY) % 32 == 0,
                "warp footprint is 8 x 4 columns");
  static_assert(ZC <= 8, "item encoding holds 3 bits of z");
  const Geom &g = cst.g;
  const int lane = threadIdx.x & 31;
  const int lcap = cst.chunk;  // list capacity per warp (<= 128: 7 bits of the item tags)
  if (lcap > 128) {
    if ((threadIdx.x & 31) == 0) set_err(args.err, DERR_RANGE);
    return;
  }

  float *s_list = reinterpret_cast<float *>(__builtin_assume_aligned(wsmem, 16));  // [lcap][LIST_FIELDS]
  float *s_acc = s_list + (size_t)LIST_FIELDS * lcap;   // [3][WV]
  // item queues of 16-bit tags li << 9 | mirrored << 8 | column << 3 | z level
  // (list capacity <= 128): the less shared memory the warps take, the more
  // of the SM's L1 is left for the pixel reads
  using qtag = unsigned short;
  qtag *s_qf = reinterpret_cast<qtag *>(s_acc + 3 * WV);  // fast items
  qtag *s_qe = s_qf + QCAP;                              // fast items at the image edge
  qtag *s_qc = s_qe + QCAP;                              // boxes crossing kx = 0
  qtag *s_qd = s_qc + QCAP;                              // voxels in fold columns
  auto LF = [&](int f, int i) -> float & { return s_list[i * LIST_FIELDS + f]; };
  auto LI = [&](int f, int i) -> int { return __float_as_int(s_list[i * LIST_FIELDS + f]); };

  const int split = unit.w & 0xffff, nsplit = (unit.w >> 16) & 0x3fff;
  const bool to_scratch = nsplit > 1 || ((unit.w >> 30) & 1);
  const int img0 = (int)((long long)args.n * split / nsplit);
  const int img1 = (int)((long long)args.n * (split + 1) / nsplit);
  const int wx = warp % (BX / 8), wy = warp / (BX / 8);
  const int fx0 = g.xa0 + unit.x * BX + wx * 8;
  const int fy0 = -g.H + unit.y * BY + wy * 4;
  const int z0 = -g.H + unit.z * ZC;
  const float cx = fx0 + 3.5f, cy = fy0 + 1.5f, cz = z0 + 0.5f * (ZC - 1);  // footprint centre
  const float hz = 0.5f * (ZC - 1);
  const float rw = sqrtf(3.5f * 3.5f + 1.5f * 1.5f + hz * hz);
  const float a = g.a;
  const float inv_a2 = 1.0f / g.a2;
  // The box starts at ceil(u - a_box).  When the box has a spare cell
  // (KB > floor(2a) + 1) it is shifted down by a small margin, so a pixel at
  // distance exactly a (possible for the DC pixel, which sits at q = 0) is
  // never lost to rounding of u; the r^2 <= a^2 test decides it.
  const float a_box = KB > (int)floorf(2.0f * a) + 1 ? a + 1e-4f : a;
  const float a_plane = a + 1e-4f;  // conservative |u_z| <= a test for queueing
  const float reach = (float)g.H + a;  // the extended plane spans [-H, H]^2
  const float ext = reach + rw + 1.0f;
  const int vx = fx0 + (lane & 7), vy = fy0 + (lane >> 3);
  const float dvx = (float)vx - cx, dvy = (float)vy - cy;
  const bool fold_col = vx <= -g.xa0;  // x <= floor(a): pixels from both sides of the fold
  const bool col_in = vx <= g.H && vy <= g.H;
  const unsigned char *imgs = reinterpret_cast<const unsigned char *>(images);
  const size_t img_stride = (size_t)g.S * g.NX * ESZ;
  float2 cpair[POLY_N / 2];
#pragma unroll
  for (int k = 0; k < POLY_N / 2; ++k) cpair[k] = make_float2(cst.poly[2 * k], cst.poly[2 * k + 1]);

  for (int i = lane; i < 3 * WV; i += 32) s_acc[i] = 0.f;
  __syncwarp();
  // optional phase counters (warp-uniform control, lane 0 keeps the clocks)
  const bool prof = args.phase != nullptr;
  unsigned long long ph[PH_COUNT];
#pragma unroll
  for (int k = 0; k < PH_COUNT; ++k) ph[k] = 0;
  const long long t_start = prof ? clock64() : 0;
  auto tick = [&]() -> long long { return prof ? clock64() : 0; };

  // fold the warp's shared partial sums into HBM (lane owns its column's voxels):
  // straight into the double-float accumulators when this CTA is the only one
  // writing its brick, else into the float4 scratch (merged after the launch)
  auto flush = [&]() {
    const long long tf = tick();
    flush_partials<ZC>(args, s_acc, fx0, fy0, z0, to_scratch);
    if (prof) ph[PH_FLUSH] += (unsigned long long)(clock64() - tf);
  };

  // one queued (image, voxel) item: form the box sums and add them to the
  // warp's partial sums
  // kinds: 0 fast, 1 fast at the image edge, 2 box crossing kx = 0, 3 fold column
  auto process = [&](unsigned it, int kind) {
    const int li = (int)(it >> 9), src = (int)((it >> 3) & 31), t = (int)(it & 7);
    const int sgn = (it >> 8) & 1 ? -1 : 1;
    const int sx = fx0 + (src & 7), sy = fy0 + (src >> 3), sz = z0 + t;
    const float sdx = (float)sx - cx, sdy = (float)sy - cy, sdz = (float)sz - cz;
    const float uz = fmaf(LF(LF_MZ, li), sdz, fmaf(LF(LF_MY, li), sdy, fmaf(LF(LF_MX, li), sdx, LF(LF_UZ, li))));
    const float uxr = fmaf(LF(LF_E1Z, li), sdz, fmaf(LF(LF_E1Y, li), sdy, fmaf(LF(LF_E1X, li), sdx, LF(LF_FX, li))));
    const float uyr = fmaf(LF(LF_E2Z, li), sdz, fmaf(LF(LF_E2Y, li), sdy, fmaf(LF(LF_E2X, li), sdx, LF(LF_FY, li))));
    const float ixf = ceilf(uxr - a_box), iyf = ceilf(uyr - a_box);
    const float fx = uxr - ixf, fy = uyr - iyf;
    const int kx0 = LI(LF_CIX, li) + (int)ixf, ky0 = LI(LF_CIY, li) + (int)iyf;
    const float uz2 = uz * uz;
    const unsigned char *ibase = list_image(s_list + (size_t)li * LIST_FIELDS);
    float sr = 0.f, si = 0.f, sw = 0.f;
    if (kind == 0 || (kind == 1 && WMODE == W_POLY)) {
      if (WMODE == W_POLY) {
        if (kind == 0)
          box_poly_interior<KB, F16>(cst, cpair, ibase, sgn, kx0, ky0, fx, fy, uz2,
                                     2.0f * inv_a2, sr, si, sw);
        else
          box_poly_edge<KB, F16>(cst, cpair, ibase, sgn, kx0, ky0, fx, fy, uz2, 2.0f * inv_a2,
                                 sr, si, sw);
      } else {
        box_fast<WMODE, KB, F16>(cst, lut, ibase, sgn, kx0, ky0, fx, fy, uz2, inv_a2, sr, si, sw);
      }
      si *= (float)sgn;
    } else if (kind == 2 && WMODE == W_POLY) {
      // a box crossing kx = 0 for a voxel away from the fold plane
      box_poly_straddle<KB, F16>(cst, cpair, ibase, kx0, ky0, fx, fy, uz2, 2.0f * inv_a2, sr,
                                 si, sw);
    } else {
      const float e[6] = {LF(LF_E1X, li), LF(LF_E1Y, li), LF(LF_E1Z, li),
                          LF(LF_E2X, li), LF(LF_E2Y, li), LF(LF_E2Z, li)};
      if (kind == 3 && WMODE == W_POLY)
        box_poly_fold<KB, F16>(cst, cpair, ibase, e, kx0, ky0, fx, fy, uz2, sx, sy, sz,
                               2.0f * inv_a2, sr, si, sw);
      else
        box_careful<WMODE, KB, F16>(cst, lut, ibase, e, kx0, ky0, fx, fy, uz2, kind == 3, sx,
                                    sy, sz, inv_a2, sr, si, sw);
    }
    const int slot = src * ZC + t;
    atomicAdd(&s_acc[slot], sr);
    atomicAdd(&s_acc[WV + slot], si);
    atomicAdd(&s_acc[2 * WV + slot], sw);
  };

  // drain full rounds of 32 items (all of them if `all`); the remainder moves
  // to the front of the queue
  auto drain = [&](qtag *q, int &qlen, int kind, bool all) {
    __syncwarp();
    const long long t0 = tick();
    const int nfull = all ? qlen : (qlen & ~31);
    for (int k = lane; k < nfull; k += 32) process(q[k], kind);
    if (prof) {
      __syncwarp();
      ph[kind < 3 ? PH_DRAIN_FAST + kind : PH_DRAIN_FOLD] += (unsigned long long)(clock64() - t0);
      ph[kind < 3 ? PH_ITEMS_FAST + kind : PH_ITEMS_FOLD] += (unsigned long long)nfull;
      if (kind == 0) ph[PH_ROUNDS] += (unsigned long long)((nfull + 31) / 32);
    }
    __syncwarp();
    const int rest = qlen - nfull;
    if (rest) {
      const qtag v = lane < rest ? q[nfull + lane] : (qtag)0;
      __syncwarp();
      if (lane < rest) q[lane] = v;
    }
    qlen = rest;
    __syncwarp();
  };

  // queue the footprint's voxels near the plane of list entry li that the
  // extended plane reaches: fast, fast at the image edge, and careful apart
  int qf = 0, qe = 0, qc = 0, qd = 0;
  auto enqueue = [&](int li) {
    const float mx = LF(LF_MX, li), my = LF(LF_MY, li), mz = LF(LF_MZ, li);
    const float bz = fmaf(my, dvy, fmaf(mx, dvx, LF(LF_UZ, li)));
    const float bx = fmaf(LF(LF_E1Y, li), dvy, fmaf(LF(LF_E1X, li), dvx, LF(LF_FX, li)));
    const float by = fmaf(LF(LF_E2Y, li), dvy, fmaf(LF(LF_E2X, li), dvx, LF(LF_FY, li)));
    const int cix = LI(LF_CIX, li), ciy = LI(LF_CIY, li);
    const float e1z = LF(LF_E1Z, li), e2z = LF(LF_E2Z, li);
    // phase 1: voxels of this column within a of the plane (cheap, all lanes)
    unsigned near = 0;
#pragma unroll
    for (int t = 0; t < ZC; ++t) {
      const float uz = fmaf(mz, (float)(z0 + t) - cz, bz);
      near |= (fabsf(uz) <= a_plane ? 1u : 0u) << t;
    }
    if (!col_in) near = 0;
    if (!__any_sync(0xffffffffu, near != 0)) return;
    // Shortcut: every voxel of the footprint projects within rw of the
    // centre's projection uc, so its box starts at kx0 in [uc_x - rw - a_box,
    // uc_x + rw - a_box + 1).  If all boxes lie inside the stored half (or all
    // inside the mirrored half) of the image, with a margin against rounding,
    // and no column is a fold column, every near voxel is a fast item and the
    // per-voxel classification is skipped.
    unsigned mf = 0, me = 0, mc = 0, md = 0, mneg = 0;
    const float ucx = (float)cix + LF(LF_FX, li), ucy = (float)ciy + LF(LF_FY, li);
    const float xlo = ucx - rw - a_box - 0.01f, xhi = ucx + rw - a_box + (float)KB + 0.01f;
    const float ylo = ucy - rw - a_box - 0.01f, yhi = ucy + rw - a_box + (float)KB + 0.01f;
    const float Hf = (float)g.H;
    const bool direct_all = xlo >= 1.f && xhi <= Hf && ylo >= -Hf && yhi <= Hf - 1.f;
    const bool mirror_all = xhi <= -1.f && xlo >= -Hf && ylo > -Hf && yhi <= Hf;
    if (fx0 > -g.xa0 && (direct_all || mirror_all)) {
      // every near voxel is a fast item.  A column's near voxels are one run
      // of z levels [t0, t0 + c), so the lane-major positions come from a
      // prefix sum over lanes done with one ballot per bit of c (c <= 8), and
      // the stores are predicated, without a loop
      const int c = __popc(near);
      const int t0 = near ? __ffs(near) - 1 : 0;
      const unsigned lt = (1u << lane) - 1u;
      int excl = 0, tot = 0;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const unsigned bal = __ballot_sync(0xffffffffu, (c >> b) & 1);
        excl += __popc(bal & lt) << b;
        tot += __popc(bal) << b;
      }
      const unsigned base = ((unsigned)li << 9) | (mirror_all ? 1u << 8 : 0u) | ((unsigned)lane << 3);
      const int p0 = qf + excl - t0;
#pragma unroll
      for (int t = 0; t < ZC; ++t)
        if ((near >> t) & 1u) s_qf[p0 + t] = (qtag)(base | (unsigned)t);
      qf += tot;
      return;
    } else {
      // phase 2: classify the near voxels one by one
      for (unsigned m = near; m; m &= m - 1) {
        const int t = __ffs(m) - 1;
        const float dz = (float)(z0 + t) - cz;
        const float uxr = fmaf(e1z, dz, bx), uyr = fmaf(e2z, dz, by);
        const float ux = (float)cix + uxr, uy = (float)ciy + uyr;
        if (fabsf(ux) <= reach && fabsf(uy) <= reach) {
          const int kx0 = cix + (int)ceilf(uxr - a_box), ky0 = ciy + (int)ceilf(uyr - a_box);
          const bool direct = kx0 >= 1, mirror = kx0 + KB - 1 <= -1;
          if (!fold_col && (direct || mirror)) {
            const bool interior = direct
                ? (kx0 + KB - 1 <= g.H && ky0 >= -g.H && ky0 + KB - 1 < g.H)
                : (kx0 >= -g.H && ky0 > -g.H && ky0 + KB - 1 <= g.H);
            if (interior) mf |= 1u << t; else me |= 1u << t;
            if (mirror) mneg |= 1u << t;
          } else if (fold_col) {
            md |= 1u << t;
          } else {
            mc |= 1u << t;
          }
        }
      }
    }
    // warp prefix sums of the three counts (packed 10 bits each)
    const int cnt = __popc(mf) | (__popc(me) << 10) | (__popc(mc) << 20);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    const int excl = incl - cnt;
    int pf = qf + (excl & 1023), pe = qe + ((excl >> 10) & 1023), pc = qc + (excl >> 20);
    const unsigned base = ((unsigned)li << 9) | ((unsigned)lane << 3);
    while (mf) {
      const int t = __ffs(mf) - 1;
      mf &= mf - 1;
      s_qf[pf++] = (qtag)(base | (((mneg >> t) & 1u) << 8) | (unsigned)t);
    }
    while (me) {
      const int t = __ffs(me) - 1;
      me &= me - 1;
      s_qe[pe++] = (qtag)(base | (((mneg >> t) & 1u) << 8) | (unsigned)t);
    }
    while (mc) {
      const int t = __ffs(mc) - 1;
      mc &= mc - 1;
      s_qc[pc++] = (qtag)(base | (unsigned)t);
    }
    qf += total & 1023;
    qe += (total >> 10) & 1023;
    qc += total >> 20;
    // voxels of fold columns (rare: only footprints at x <= floor(a))
    if (__any_sync(0xffffffffu, md != 0)) {
      const int cd = __popc(md);
      int incd = cd;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incd, o);
        if (lane >= o) incd += v;
      }
      int pd = qd + incd - cd;
      while (md) {
        const int t = __ffs(md) - 1;
        md &= md - 1;
        s_qd[pd++] = (qtag)(base | (unsigned)t);
      }
      qd += __shfl_sync(0xffffffffu, incd, 31);
    }
  };

  // drain the queues that hold a full round (every queue entirely if `all`);
  // the only place the boxes are evaluated, so each box's code exists once
  auto service = [&](bool all) {
    if (qf >= 32 || (all && qf > 0)) drain(s_qf, qf, 0, all);
    if (qe >= 32 || (all && qe > 0)) drain(s_qe, qe, 1, all);
    if (qc >= 32 || (all && qc > 0)) drain(s_qc, qc, 2, all);
    if (qd >= 32 || (all && qd > 0)) drain(s_qd, qd, 3, all);
  };

  int nl = 0;           // entries in the warp's list
  int since_flush = 0;  // list entries queued since the last flush
  // Cull 32 images per step into the list; when the list is nearly full, or
  // after the last image, queue and drain it.  Written as one loop with one
  // site of each step so the code of every step exists once.
  for (int cs = img0;; cs += 32) {
    const bool last = cs >= img1;
    if (!last) {
      // ---- cull: one image per lane; kept images go to the warp's list in order
      const long long tc = tick();
      nl = cull_step(args, imgs, img_stride, s_list, nl, cs, img1, cx, cy, cz, 3.5f, 1.5f, hz, ext,
                     col_in_any(g, fx0, fy0));
      __syncwarp();
      if (prof) ph[PH_CULL] += (unsigned long long)(clock64() - tc);
    }
    if (last || nl > lcap - 32) {
      // ---- queue and accumulate the list's images; every GATHER_FLUSH
      // images, drain everything and fold the partial sums into HBM
      if (prof) ph[PH_LIST_IMAGES] += (unsigned long long)nl;
      for (int li = 0; li <= nl; ++li) {
        const bool end = li == nl;
        bool all = end;  // the list is rebuilt next: nothing may refer to it afterwards
        if (!end) {
          enqueue(li);
          if (++since_flush >= GATHER_FLUSH) all = true;
        }
        service(all);
        if (all && since_flush >= GATHER_FLUSH) {
          flush();
          since_flush = 0;
        }
      }
      nl = 0;
    }
    if (last) break;
  }
  flush();
  if (prof && lane == 0) {
    ph[PH_WARP_CYCLES] = (unsigned long long)(clock64() - t_start);
    // queueing time = total minus the other phases
    unsigned long long other = ph[PH_CULL] + ph[PH_DRAIN_FAST] + ph[PH_DRAIN_EDGE] +
                               ph[PH_DRAIN_CAREFUL] + ph[PH_DRAIN_FOLD] + ph[PH_FLUSH];
    ph[PH_QUEUE] = ph[PH_WARP_CYCLES] > other ? ph[PH_WARP_CYCLES] - other : 0;
#pragma unroll
    for (int k = 0; k < PH_COUNT; ++k)
      if (ph[k]) atomicAdd(args.phase + k, ph[k]);
  }
}

// One CTA per work unit (args.units[blockIdx.x]); the CTA shares the blob
// table, its warps then run independently.
template <int BX, int BY, int ZC, int WMODE, int KB, int F16>
__global__ void __launch_bounds__(BX * BY, 512 / (BX * BY))
gather_kernel(const InsertArgs args) {
  constexpr int NT = BX * BY;
  const int tid = threadIdx.x, warp = tid >> 5;
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char *sp = smem;
  float2 *s_lut = reinterpret_cast<float2 *>(sp);
  if (WMODE == W_LUT) {
    sp += ((size_t)args.lut_n * sizeof(float2) + 15) & ~(size_t)15;
    for (int i = tid; i < args.lut_n; i += NT) s_lut[i] = args.lut[i];
    __syncthreads();  // the only CTA-wide barrier: warps run independently from here
  }
  gather_warp<BX, BY, ZC, WMODE, KB, F16>(args, args, args.images, s_lut,
                                          sp + (size_t)warp * gather_warp_smem(ZC, args.chunk),
                                          args.units[blockIdx.x], warp);
}

// Persistent gather over the work units of several batches (A8): each CTA
// takes units from a device counter until none are left, so batches of
// different S and n share one launch; the CTA's warps work on the footprints
// of one unit at a time (neighbouring columns, the same images: pixels shared
// in L1).  items[i] = {bx | by << 10 | bz << 20, split word, batch, 0}.  The
// batch's arguments are copied to shared memory when the batch changes.
// Weights on the fly (polynomial or Bessel).  The counter is only
// incremented, never waited on; the CTA barriers are between units.
template <int BX, int BY, int ZC, int WMODE, int KB, int F16>
__global__ void __launch_bounds__(BX * BY, 512 / (BX * BY))
gather_persistent_kernel(const InsertArgs *__restrict__ descs, const int4 *__restrict__ items,
                         int nitems, int chunk, unsigned *counter) {
  static_assert(WMODE != W_LUT, "the persistent gather evaluates weights on the fly");
  constexpr int NT = BX * BY;
  const int tid = threadIdx.x, warp = tid >> 5;
  extern __shared__ __align__(16) unsigned char smem[];
  InsertArgs *s_args = reinterpret_cast<InsertArgs *>(smem);
  __shared__ int4 s_item;
  unsigned char *wsmem = smem + GATHER_ARGS_BYTES + (size_t)warp * gather_warp_smem(ZC, chunk);
  int cur = -1;
  for (;;) {
    if (tid == 0) {
      const unsigned k = atomicAdd(counter, 1u);
      s_item = k < (unsigned)nitems ? items[k] : make_int4(0, 0, -1, 0);
    }
    __syncthreads();
    const int4 it = s_item;
    if (it.z < 0) break;
    if (it.z != cur) {
      const int *src = reinterpret_cast<const int *>(descs + it.z);
      int *dst = reinterpret_cast<int *>(s_args);
      for (int i = tid; i < (int)(sizeof(InsertArgs) / 4); i += NT) dst[i] = src[i];
      cur = it.z;
    }
    __syncthreads();
    const int4 unit = make_int4(it.x & 1023, (it.x >> 10) & 1023, (it.x >> 20) & 1023, it.y);
    gather_warp<BX, BY, ZC, WMODE, KB, F16>(*s_args, *s_args, s_args->images, nullptr, wsmem,
                                            unit, warp);
    __syncthreads();  // s_item and s_args are rewritten next
  }
}

// Several batches in one launch, one CTA per work item: CTA b takes
// p.items[b] (encoded as for the persistent gather) and copies its batch's
// arguments p.descs[batch] to shared memory; geometry, weights and list
// capacity, common to the launch's batches, are read from p.base (kernel
// parameters).  Weights on the fly.
template <int BX, int BY, int ZC, int WMODE, int KB, int F16>
__global__ void __launch_bounds__(BX * BY, 512 / (BX * BY))
gather_multi_kernel(const MultiLaunch p) {
  static_assert(WMODE != W_LUT, "the multi-batch gather evaluates weights on the fly");
  constexpr int NT = BX * BY;
  const int tid = threadIdx.x, warp = tid >> 5;
  extern __shared__ __align__(16) unsigned char smem[];
  InsertArgs *s_args = reinterpret_cast<InsertArgs *>(smem);
  const int4 it = p.items[blockIdx.x];
  const int *src = reinterpret_cast<const int *>(p.descs + it.z);
  int *dst = reinterpret_cast<int *>(s_args);
  for (int i = tid; i < (int)(sizeof(InsertArgs) / 4); i += NT) dst[i] = src[i];
  __syncthreads();
  const int4 unit = make_int4(it.x & 1023, (it.x >> 10) & 1023, (it.x >> 20) & 1023, it.y);
  gather_warp<BX, BY, ZC, WMODE, KB, F16>(
      *s_args, p.base, p.images[it.w], nullptr,
      smem + GATHER_ARGS_BYTES + (size_t)warp * gather_warp_smem(ZC, p.base.chunk), unit, warp);
}

}  // namespace fr
