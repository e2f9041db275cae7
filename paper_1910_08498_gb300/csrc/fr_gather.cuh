// fr_gather.cuh -- the per-voxel gather insertion kernel (primary variant).
//
// One CTA owns a brick of BX x BY voxel columns, ZC voxels deep along z, in
// the half volume x >= -floor(a) that folding can reach; each warp owns an
// 8 x 4-column footprint of it (32 * ZC voxels) and is the only writer of
// those voxels for the whole launch, so V and W in HBM need no atomics.
//
// Per launch, for each chunk of images:
//  1. cull (A2): the CTA keeps, in image order, the images whose central
//     plane passes within a + (brick radius) of the brick centre, compacted
//     with warp ballots into a shared-memory list (structure of arrays) that
//     holds each kept image's plane basis and the brick centre's projection
//     R^T c, formed with error-free products and split into an integer part
//     and a small remainder so in-plane positions keep ~1e-7 absolute accuracy
//     at any |k|;
//  2. queue: each warp walks the list; for an image whose plane passes near
//     its footprint it marks the voxels within a of the plane (|u_z| <= a,
//     u = R^T v) and appends them, as (image, voxel) items, to a warp-private
//     shared-memory queue (warp prefix sums, image-major order);
//  3. accumulate (A4): all 32 lanes drain the queue, one item per lane, so no
//     lane idles on a voxel that is far from the plane.  An item visits the
//     KB x KB pixel box around (u_x, u_y) of the Hermitian-extended, folded
//     image plane and forms sum b(r) p and sum b(r) over the pixels with
//     r^2 = (u_x-kx)^2 + (u_y-ky)^2 + u_z^2 <= a^2 (weights from the blob
//     table in shared memory, the same table through L1, or on the fly).
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
//     images.
#pragma once

#include "fr_device.cuh"

namespace fr {

// number of 4-byte fields per kept image in the shared-memory list
constexpr int LIST_FIELDS = 15;
enum ListField {
  LF_E1X, LF_E1Y, LF_E1Z, LF_E2X, LF_E2Y, LF_E2Z, LF_MX, LF_MY, LF_MZ,
  LF_FX, LF_FY, LF_UZ, LF_CIX, LF_CIY, LF_IMG
};

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

constexpr int GATHER_FLUSH = 256;  // list images between flushes of the shared partial sums
constexpr int GATHER_QUEUE = 512;  // queue entries per warp

template <int F16>
__device__ __forceinline__ float2 ld_px(const unsigned char *p) {
  if (F16) return __half22float2(__ldg(reinterpret_cast<const __half2 *>(p)));
  return __ldg(reinterpret_cast<const float2 *>(p));
}

// Fast path: every pixel of the box is stored (SGN = +1: pixels (kx0+j,
// ky0+l)) or point-reflected (SGN = -1: pixels (-kx0-j, -ky0-l), conjugated
// by the caller); no fold, range or multiplicity test.
template <int WMODE, int KB, int F16, int SGN>
__device__ __forceinline__ void box_fast(const InsertArgs &args, const float2 *lut,
                                         const unsigned char *ibase, int kx0, int ky0, float fx,
                                         float fy, float uz2, float inv_a2, float &sr, float &si,
                                         float &sw) {
  const Geom &g = args.g;
  constexpr int ESZ = F16 ? 4 : 8;
  const size_t row_bytes = (size_t)g.NX * ESZ;
#pragma unroll
  for (int l = 0; l < KB; ++l) {
    int ky = SGN * (ky0 + l);
    ky += ky < 0 ? g.S : 0;
    const unsigned char *row = ibase + (size_t)ky * row_bytes + (size_t)(SGN * kx0) * ESZ;
    const float dy = fy - (float)l;
    const float ry = fmaf(dy, dy, uz2);
#pragma unroll
    for (int j = 0; j < KB; ++j) {
      const float dx = fx - (float)j;
      const float r2 = fmaf(dx, dx, ry);
      if (r2 <= g.a2) {
        const float w = blob_w<WMODE>(lut, r2, args, inv_a2);
        const float2 p = ld_px<F16>(row + SGN * j * ESZ);
        sr = fmaf(w, p.x, sr);
        si = fmaf(w, p.y, si);
        sw += w;
      }
    }
  }
}

// Careful path: any box, exact fold predicate (when near the fold plane) and
// range tests per pixel; the W weight counts each contribution.
template <int WMODE, int KB, int F16>
__device__ __noinline__ void box_careful(const InsertArgs &args, const float2 *lut,
                                         const unsigned char *ibase, float r00, float r01,
                                         int kx0, int ky0, float fx, float fy, float uz2,
                                         bool fold_check, float inv_a2, float &sr, float &si,
                                         float &sw) {
  const Geom &g = args.g;
  constexpr int ESZ = F16 ? 4 : 8;
  for (int l = 0; l < KB; ++l) {
    const float dy = fy - (float)l;
    const float ry = fmaf(dy, dy, uz2);
    const int cy = ky0 + l;
    for (int j = 0; j < KB; ++j) {
      const float dx = fx - (float)j;
      const float r2 = fmaf(dx, dx, ry);
      if (!(r2 <= g.a2)) continue;
      const int cx = kx0 + j;
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

template <int BX, int BY, int ZC, int WMODE, int KB, int F16>
__global__ void __launch_bounds__(BX * BY)
gather_kernel(const InsertArgs args) {
  constexpr int NT = BX * BY;
  constexpr int NW = NT / 32;
  constexpr int WV = 32 * ZC;  // voxels per warp footprint
  constexpr int ESZ = F16 ? 4 : 8;
  static_assert(BX % 8 == 0 && BY % 4 == 0 && NT % 32 == 0, "warp footprint is 8 x 4 columns");
  static_assert(ZC <= 8, "item encoding holds 3 bits of z");
  const Geom &g = args.g;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int chunk = args.chunk;

  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char *sp = smem;
  float2 *s_lut = reinterpret_cast<float2 *>(sp);
  if (WMODE == W_LUT) sp += ((size_t)args.lut_n * sizeof(float2) + 15) & ~(size_t)15;
  float *s_list = reinterpret_cast<float *>(sp);  // [LIST_FIELDS][chunk]
  sp += (size_t)LIST_FIELDS * chunk * 4;
  float *s_acc = reinterpret_cast<float *>(sp) + (size_t)warp * 3 * WV;  // [3][WV] per warp
  sp += (size_t)NW * 3 * WV * 4;
  unsigned *s_q = reinterpret_cast<unsigned *>(sp) + (size_t)warp * GATHER_QUEUE;
  __shared__ int s_wcount[NW];
  __shared__ int s_nlist;
  const float2 *lut = WMODE == W_LUT ? s_lut : args.lut;
  auto LF = [&](int f, int i) -> float & { return s_list[f * chunk + i]; };
  auto LI = [&](int f, int i) -> int { return __float_as_int(s_list[f * chunk + i]); };

  // brick and warp footprint
  const int wx = warp % (BX / 8), wy = warp / (BX / 8);
  const int x0 = g.xa0 + blockIdx.x * BX, y0 = -g.H + blockIdx.y * BY, z0 = -g.H + blockIdx.z * ZC;
  const float cxb = x0 + 0.5f * (BX - 1), cyb = y0 + 0.5f * (BY - 1), czb = z0 + 0.5f * (ZC - 1);
  const float hxb = 0.5f * (BX - 1), hyb = 0.5f * (BY - 1), hzb = 0.5f * (ZC - 1);
  const float rb = sqrtf(hxb * hxb + hyb * hyb + hzb * hzb);
  const float a = g.a;
  const float inv_a2 = 1.0f / g.a2;
  const float cull = a + rb + 1e-3f;
  const float ext = (float)g.H + rb + a + 1.0f;  // the extended plane spans [-H, H]^2
  // this lane's column and the warp footprint centre, relative to the brick centre
  const int tx = wx * 8 + (lane & 7), ty = wy * 4 + (lane >> 3);
  const int vx = x0 + tx, vy = y0 + ty;
  const float dvx = (float)vx - cxb, dvy = (float)vy - cyb;
  const float wcx = (float)(wx * 8) + 3.5f - hxb, wcy = (float)(wy * 4) + 1.5f - hyb;
  const float wrad = sqrtf(3.5f * 3.5f + 1.5f * 1.5f + hzb * hzb) + a + 1e-3f;
  const bool col_in = vx <= g.H && vy <= g.H;
  const unsigned char *imgs = reinterpret_cast<const unsigned char *>(args.images);
  const size_t img_stride = (size_t)g.S * g.NX * ESZ;

  if (WMODE == W_LUT) {
    for (int i = tid; i < args.lut_n; i += NT) s_lut[i] = args.lut[i];
  }
  for (int i = lane; i < 3 * WV; i += 32) s_acc[i] = 0.f;

  // fold the warp's shared partial sums into HBM (lane owns its column's voxels)
  auto flush = [&]() {
    __syncwarp();
    if (col_in) {
#pragma unroll
      for (int t = 0; t < ZC; ++t) {
        const int vz = z0 + t;
        if (vz > g.H) break;
        const size_t v =
            ((size_t)(vz + g.H) * g.D + (size_t)(vy + g.H)) * g.NXa + (size_t)(vx - g.xa0);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float add = s_acc[c * WV + lane * ZC + t];
          if (add != 0.f) {
            float h = args.acc[c * args.plane + v], l = args.acc[(3 + c) * args.plane + v];
            dd_add(h, l, add);
            args.acc[c * args.plane + v] = h;
            args.acc[(3 + c) * args.plane + v] = l;
          }
        }
      }
    }
#pragma unroll
    for (int t = 0; t < ZC; ++t)
#pragma unroll
      for (int c = 0; c < 3; ++c) s_acc[c * WV + lane * ZC + t] = 0.f;
    __syncwarp();
  };

  // process every queued item; one item per lane per round
  auto drain = [&](int qlen) {
    __syncwarp();
    for (int k = lane; k < qlen; k += 32) {
      const unsigned it = s_q[k];
      const int li = (int)(it >> 8), src = (int)((it >> 3) & 31), t = (int)(it & 7);
      const int stx = wx * 8 + (src & 7), sty = wy * 4 + (src >> 3);
      const float sdx = (float)(x0 + stx) - cxb, sdy = (float)(y0 + sty) - cyb;
      const float dvz = (float)(z0 + t) - czb;
      const float uz = fmaf(LF(LF_MZ, li), dvz, fmaf(LF(LF_MY, li), sdy, fmaf(LF(LF_MX, li), sdx, LF(LF_UZ, li))));
      const float uxr = fmaf(LF(LF_E1Z, li), dvz, fmaf(LF(LF_E1Y, li), sdy, fmaf(LF(LF_E1X, li), sdx, LF(LF_FX, li))));
      const float uyr = fmaf(LF(LF_E2Z, li), dvz, fmaf(LF(LF_E2Y, li), sdy, fmaf(LF(LF_E2X, li), sdx, LF(LF_FY, li))));
      const float ixf = ceilf(uxr - a), iyf = ceilf(uyr - a);
      const float fx = uxr - ixf, fy = uyr - iyf;
      const int kx0 = LI(LF_CIX, li) + (int)ixf, ky0 = LI(LF_CIY, li) + (int)iyf;
      const float uz2 = uz * uz;
      const unsigned char *ibase = imgs + (size_t)LI(LF_IMG, li) * img_stride;
      const bool fold_vox = (x0 + stx) <= -g.xa0;
      float sr = 0.f, si = 0.f, sw = 0.f;
      if (!fold_vox && kx0 >= 1 && kx0 + KB - 1 <= g.H && ky0 >= -g.H && ky0 + KB - 1 < g.H) {
        box_fast<WMODE, KB, F16, 1>(args, lut, ibase, kx0, ky0, fx, fy, uz2, inv_a2, sr, si, sw);
      } else if (!fold_vox && kx0 + KB - 1 <= -1 && kx0 >= -g.H && ky0 > -g.H &&
                 ky0 + KB - 1 <= g.H) {
        box_fast<WMODE, KB, F16, -1>(args, lut, ibase, kx0, ky0, fx, fy, uz2, inv_a2, sr, si, sw);
        si = -si;
      } else {
        box_careful<WMODE, KB, F16>(args, lut, ibase, LF(LF_E1X, li), LF(LF_E2X, li), kx0, ky0,
                                    fx, fy, uz2, fold_vox, inv_a2, sr, si, sw);
      }
      const int slot = src * ZC + t;
      atomicAdd(&s_acc[slot], sr);
      atomicAdd(&s_acc[WV + slot], si);
      atomicAdd(&s_acc[2 * WV + slot], sw);
    }
    __syncwarp();
  };

  const float *rot = args.rot;
  int since_flush = 0;
  for (int cs = 0; cs < args.n; cs += chunk) {
    const int ce = min(args.n, cs + chunk);
    // ---- 1. cull this chunk into an ordered list
    if (tid == 0) s_nlist = 0;
    __syncthreads();
    for (int base = cs; base < ce; base += NT) {
      const int i = base + tid;
      bool keep = false;
      float e1x = 0, e1y = 0, e1z = 0, e2x = 0, e2y = 0, e2z = 0, mx = 0, my = 0, mz = 0;
      if (i < ce) {
        const float *R = rot + 9 * (size_t)i;
        e1x = __ldg(R + 0); e1y = __ldg(R + 3); e1z = __ldg(R + 6);
        e2x = __ldg(R + 1); e2y = __ldg(R + 4); e2z = __ldg(R + 7);
        mx = __ldg(R + 2);  my = __ldg(R + 5);  mz = __ldg(R + 8);
        const float d = mx * cxb + my * cyb + mz * czb;
        const float ux = e1x * cxb + e1y * cyb + e1z * czb;
        const float uy = e2x * cxb + e2y * cyb + e2z * czb;
        keep = fabsf(d) <= cull && fabsf(ux) <= ext && fabsf(uy) <= ext;
      }
      const unsigned bal = __ballot_sync(0xffffffffu, keep);
      if (lane == 0) s_wcount[warp] = __popc(bal);
      __syncthreads();
      int off = s_nlist;
      for (int w = 0; w < warp; ++w) off += s_wcount[w];
      if (keep) {
        const int o = off + __popc(bal & ((1u << lane) - 1u));
        float hx, lx, hy, ly, hz, lz;
        dot3_dd(e1x, e1y, e1z, cxb, cyb, czb, hx, lx);
        dot3_dd(e2x, e2y, e2z, cxb, cyb, czb, hy, ly);
        dot3_dd(mx, my, mz, cxb, cyb, czb, hz, lz);
        const float rx = rintf(hx), ry = rintf(hy);
        LF(LF_E1X, o) = e1x; LF(LF_E1Y, o) = e1y; LF(LF_E1Z, o) = e1z;
        LF(LF_E2X, o) = e2x; LF(LF_E2Y, o) = e2y; LF(LF_E2Z, o) = e2z;
        LF(LF_MX, o) = mx;   LF(LF_MY, o) = my;   LF(LF_MZ, o) = mz;
        LF(LF_FX, o) = (hx - rx) + lx;  // hx - rx is exact
        LF(LF_FY, o) = (hy - ry) + ly;
        LF(LF_UZ, o) = hz + lz;
        LF(LF_CIX, o) = __int_as_float((int)rx);
        LF(LF_CIY, o) = __int_as_float((int)ry);
        LF(LF_IMG, o) = __int_as_float(i);
      }
      __syncthreads();
      if (tid == 0) {
        int tot = 0;
        for (int w = 0; w < NW; ++w) tot += s_wcount[w];
        s_nlist += tot;
      }
      __syncthreads();
    }
    const int nlist = s_nlist;

    // ---- 2./3. queue the warp's near-plane voxels and drain
    int qlen = 0;
    for (int li = 0; li < nlist; ++li) {
      const float mx = LF(LF_MX, li), my = LF(LF_MY, li), mz = LF(LF_MZ, li);
      // the plane must pass near this warp's footprint
      const float dw = fmaf(my, wcy, fmaf(mx, wcx, LF(LF_UZ, li)));
      if (fabsf(dw) <= wrad) {
        const float bz = fmaf(my, dvy, fmaf(mx, dvx, LF(LF_UZ, li)));
        unsigned mask = 0;
#pragma unroll
        for (int t = 0; t < ZC; ++t) {
          const float uz = fmaf(mz, (float)(z0 + t) - czb, bz);
          mask |= (fabsf(uz) <= a ? 1u : 0u) << t;
        }
        if (!col_in) mask = 0;
        // warp prefix sum of the item counts
        const int cnt = __popc(mask);
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int v = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += v;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        int pos = qlen + incl - cnt;
        while (mask) {
          const int t = __ffs(mask) - 1;
          mask &= mask - 1;
          s_q[pos++] = ((unsigned)li << 8) | ((unsigned)lane << 3) | (unsigned)t;
        }
        qlen += total;
        if (qlen > GATHER_QUEUE - WV) {
          drain(qlen);
          qlen = 0;
        }
      }
      if (++since_flush >= GATHER_FLUSH) {
        if (qlen) { drain(qlen); qlen = 0; }
        flush();
        since_flush = 0;
      }
    }
    if (qlen) drain(qlen);
    __syncthreads();  // the list is rebuilt for the next chunk
  }
  // ---- 4. final write back
  flush();
}

}  // namespace fr
