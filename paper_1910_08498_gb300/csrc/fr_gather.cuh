// fr_gather.cuh -- the per-voxel gather insertion kernel (primary variant).
//
// One CTA owns a brick of BX x BY voxel columns, ZC voxels deep along z, in
// the half volume x >= -floor(a) that folding can reach.  Each thread owns
// one column and keeps its voxels' sums in registers for the whole launch, so
// V and W are read and written once per launch (A5), never per image.
//
// Per launch:
//  1. cull: the CTA keeps, in image order, the images whose central plane
//     passes within a + (brick radius) of the brick centre (a test of the
//     plane normal against the brick's bounding sphere), compacted with warp
//     ballots into a shared-memory list;
//  2. stage: for TD images at a time it builds, in shared memory, the patch of
//     the Hermitian-extended, folded image plane that the brick projects onto
//     (A3): cell c holds the sum of p(c) if pixel c is stored and not folded
//     and conj(p(-c)) if pixel -c is stored and folded, plus the count of
//     those contributions (the W weight), so the inner loop needs no fold,
//     mirror or range logic;
//  3. accumulate (A4): for each of its voxels with |u_z| <= a (u = R^T v),
//     the thread visits the KB x KB pixel box around (u_x, u_y) and adds
//     b(r) p and b(r) for the pixels with r^2 = (u_x-kx)^2 + (u_y-ky)^2 + u_z^2
//     <= a^2, b from the shared-memory table or on the fly;
//  4. write back (A5): register sums are folded into double-float running
//     sums every FLUSH images and into the HBM accumulators at the end, with
//     error-free TwoSum, so a voxel's error stays at FP32 rounding of a short
//     partial sum whatever the number of images.
#pragma once

#include "fr_device.cuh"

namespace fr {

struct SlotParam {
  float e1x, e1y, e1z;  // R column 0: image x axis in the volume
  float e2x, e2y, e2z;  // R column 1: image y axis
  float mx, my, mz;     // R column 2: plane normal
  float ucx, ucy, ucz;  // R^T c - (cx0, cy0, 0) for the brick centre c, to ~1e-7 absolute
  float r00, r01;       // fold predicate coefficients
  int img;              // image index in the launch
  int cx0, cy0;         // patch origin (plane cell coordinates)
  int pw, ph;           // patch extent (cells)
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

// Cell extent bound of a patch for this brick shape: projection half width of
// the brick onto a unit vector is at most the half diagonal h, plus the blob
// radius, the candidate box and one cell of margin on either side.
__host__ __device__ inline int gather_pw_bound(int bx, int by, int zc, float a, int KB) {
  float hx = 0.5f * (bx - 1), hy = 0.5f * (by - 1), hz = 0.5f * (zc - 1);
  float h = sqrtf(hx * hx + hy * hy + hz * hz);
  return (int)ceilf(2.0f * h) + KB + 4;
}

constexpr int GATHER_FLUSH = 32;  // images between register-to-double-float flushes

template <int BX, int BY, int ZC, int WMODE, int KB>
__global__ void __launch_bounds__(BX * BY)
gather_kernel(const InsertArgs args) {
  constexpr int NT = BX * BY;
  constexpr int NW = NT / 32;
  static_assert(BX % 8 == 0 && BY % 4 == 0 && NT % 32 == 0, "warp footprint is 8 x 4 columns");
  const Geom &g = args.g;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;

  extern __shared__ __align__(16) unsigned char smem[];
  // layout: [lut float2 x lut_n (LUT mode)] [list int x chunk] [slots] [patch val] [patch mult]
  unsigned char *sp = smem;
  float2 *s_lut = reinterpret_cast<float2 *>(sp);
  if (WMODE == W_LUT) sp += ((size_t)args.lut_n * sizeof(float2) + 15) & ~(size_t)15;
  int *s_list = reinterpret_cast<int *>(sp);
  sp += ((size_t)args.chunk * sizeof(int) + 15) & ~(size_t)15;
  SlotParam *s_slot = reinterpret_cast<SlotParam *>(sp);
  sp += ((size_t)args.tdepth * sizeof(SlotParam) + 15) & ~(size_t)15;
  const int pcells = args.pw_max * args.pw_max;
  float2 *s_pval = reinterpret_cast<float2 *>(sp);
  sp += (size_t)args.tdepth * pcells * sizeof(float2);
  float *s_pmul = reinterpret_cast<float *>(sp);
  __shared__ int s_wcount[NW];
  __shared__ int s_nlist;
  __shared__ int s_off[9];

  // brick and column of this thread (warps cover 8 x 4 column footprints)
  const int bxi = blockIdx.x, byi = blockIdx.y, bzi = blockIdx.z;
  const int wx = warp % (BX / 8), wy = warp / (BX / 8);
  const int tx = wx * 8 + (lane & 7), ty = wy * 4 + (lane >> 3);
  const int x0 = g.xa0 + bxi * BX, y0 = -g.H + byi * BY, z0 = -g.H + bzi * ZC;
  const int vx = x0 + tx, vy = y0 + ty;
  const float cxb = x0 + 0.5f * (BX - 1), cyb = y0 + 0.5f * (BY - 1), czb = z0 + 0.5f * (ZC - 1);
  const float hxb = 0.5f * (BX - 1), hyb = 0.5f * (BY - 1), hzb = 0.5f * (ZC - 1);
  const float rb = sqrtf(hxb * hxb + hyb * hyb + hzb * hzb);
  const float a = g.a, a2 = g.a2;
  const float inv_a2 = 1.0f / a2;
  const float cull = a + rb + 1e-3f;
  const float ext = (float)g.H + rb + a + 1.0f;  // the extended plane spans [-H, H]^2

  if (WMODE == W_LUT) {
    for (int i = tid; i < args.lut_n; i += NT) s_lut[i] = args.lut[i];
  }

  float part[ZC][3], hi[ZC][3], lo[ZC][3];
#pragma unroll
  for (int t = 0; t < ZC; ++t)
#pragma unroll
    for (int c = 0; c < 3; ++c) { part[t][c] = 0.f; hi[t][c] = 0.f; lo[t][c] = 0.f; }
  int since_flush = 0;

  const float *rot = args.rot;
  for (int cs = 0; cs < args.n; cs += args.chunk) {
    const int ce = min(args.n, cs + args.chunk);
    // ---- 1. cull this chunk into an ordered list
    if (tid == 0) s_nlist = 0;
    __syncthreads();
    for (int base = cs; base < ce; base += NT) {
      int i = base + tid;
      bool keep = false;
      if (i < ce) {
        const float *R = rot + 9 * (size_t)i;
        float mx = __ldg(R + 2), my = __ldg(R + 5), mz = __ldg(R + 8);
        float d = mx * cxb + my * cyb + mz * czb;
        float ux = __ldg(R + 0) * cxb + __ldg(R + 3) * cyb + __ldg(R + 6) * czb;
        float uy = __ldg(R + 1) * cxb + __ldg(R + 4) * cyb + __ldg(R + 7) * czb;
        keep = fabsf(d) <= cull && fabsf(ux) <= ext && fabsf(uy) <= ext;
      }
      unsigned bal = __ballot_sync(0xffffffffu, keep);
      if (lane == 0) s_wcount[warp] = __popc(bal);
      __syncthreads();
      int off = s_nlist;
      for (int w = 0; w < warp; ++w) off += s_wcount[w];
      if (keep) s_list[off + __popc(bal & ((1u << lane) - 1u))] = i;
      __syncthreads();
      if (tid == 0) {
        int tot = 0;
        for (int w = 0; w < NW; ++w) tot += s_wcount[w];
        s_nlist += tot;
      }
      __syncthreads();
    }
    const int nlist = s_nlist;

    // ---- 2./3. stage TD images, then accumulate them
    for (int g0 = 0; g0 < nlist; g0 += args.tdepth) {
      const int ns = min(args.tdepth, nlist - g0);
      if (tid < ns) {
        SlotParam P;
        int i = s_list[g0 + tid];
        const float *R = rot + 9 * (size_t)i;
        P.e1x = __ldg(R + 0); P.e1y = __ldg(R + 3); P.e1z = __ldg(R + 6);
        P.e2x = __ldg(R + 1); P.e2y = __ldg(R + 4); P.e2z = __ldg(R + 7);
        P.mx = __ldg(R + 2);  P.my = __ldg(R + 5);  P.mz = __ldg(R + 8);
        P.r00 = P.e1x; P.r01 = P.e2x;
        P.img = i;
        float ucx, ucx_lo, ucy, ucy_lo, ucz, ucz_lo;
        dot3_dd(P.e1x, P.e1y, P.e1z, cxb, cyb, czb, ucx, ucx_lo);
        dot3_dd(P.e2x, P.e2y, P.e2z, cxb, cyb, czb, ucy, ucy_lo);
        dot3_dd(P.mx, P.my, P.mz, cxb, cyb, czb, ucz, ucz_lo);
        float h1 = fabsf(P.e1x) * hxb + fabsf(P.e1y) * hyb + fabsf(P.e1z) * hzb;
        float h2 = fabsf(P.e2x) * hxb + fabsf(P.e2y) * hyb + fabsf(P.e2z) * hzb;
        int cx0 = (int)floorf(ucx - h1 - a) - 1;
        int cy0 = (int)floorf(ucy - h2 - a) - 1;
        int cx1 = (int)floorf(ucx + h1 - a) + KB + 2;  // exclusive
        int cy1 = (int)floorf(ucy + h2 - a) + KB + 2;
        P.cx0 = cx0; P.cy0 = cy0;
        // patch-relative centre: hi - cx0 is exact (|hi| < 2^9, cx0 integer)
        P.ucx = (ucx - (float)cx0) + ucx_lo;
        P.ucy = (ucy - (float)cy0) + ucy_lo;
        P.ucz = ucz + ucz_lo;
        P.pw = min(cx1 - cx0, args.pw_max);
        P.ph = min(cy1 - cy0, args.pw_max);
        if (cx1 - cx0 > args.pw_max || cy1 - cy0 > args.pw_max) set_err(args.err, DERR_RANGE);
        s_slot[tid] = P;
      }
      __syncthreads();
      if (tid == 0) {
        int o = 0;
        for (int s = 0; s < ns; ++s) { s_off[s] = o; o += s_slot[s].pw * s_slot[s].ph; }
        s_off[ns] = o;
      }
      __syncthreads();
      // build the folded, Hermitian-extended patches
      const int total = s_off[ns];
      for (int idx = tid; idx < total; idx += NT) {
        int s = 0;
        while (idx >= s_off[s + 1]) ++s;
        const SlotParam &P = s_slot[s];
        int local = idx - s_off[s];
        int ly = local / P.pw, lx = local - ly * P.pw;
        int cx = P.cx0 + lx, cy = P.cy0 + ly;
        float vr = 0.f, vi = 0.f, mu = 0.f;
        const size_t ibase = (size_t)P.img * g.S * g.NX;
        // direct: stored pixel (cx, cy), not folded
        if (cx >= 0 && cx <= g.H && cy >= -g.H && cy < g.H) {
          if (!fold_pred(P.r00, P.r01, cx, cy)) {
            int row = cy < 0 ? cy + g.S : cy;
            float2 p = load_pixel(args.images, args.f16, ibase + (size_t)row * g.NX + cx);
            vr += p.x; vi += p.y; mu += 1.f;
          }
        }
        // mirrored: stored pixel (-cx, -cy), folded, enters conjugated
        int mx_ = -cx, my_ = -cy;
        if (mx_ >= 0 && mx_ <= g.H && my_ >= -g.H && my_ < g.H) {
          if (fold_pred(P.r00, P.r01, mx_, my_)) {
            int row = my_ < 0 ? my_ + g.S : my_;
            float2 p = load_pixel(args.images, args.f16, ibase + (size_t)row * g.NX + mx_);
            vr += p.x; vi -= p.y; mu += 1.f;
          }
        }
        s_pval[(size_t)s * pcells + local] = make_float2(vr, vi);
        s_pmul[(size_t)s * pcells + local] = mu;
      }
      __syncthreads();

      // accumulate: u' = R^T (v - c) + (R^T c - patch origin), small magnitudes
      const float dvx = (float)vx - cxb, dvy = (float)vy - cyb;
      for (int s = 0; s < ns; ++s) {
        const SlotParam P = s_slot[s];
        const float2 *pv = s_pval + (size_t)s * pcells;
        const float *pm = s_pmul + (size_t)s * pcells;
        const float bx = fmaf(P.e1y, dvy, fmaf(P.e1x, dvx, P.ucx));
        const float by = fmaf(P.e2y, dvy, fmaf(P.e2x, dvx, P.ucy));
        const float bz = fmaf(P.my, dvy, fmaf(P.mx, dvx, P.ucz));
#pragma unroll
        for (int t = 0; t < ZC; ++t) {
          const float dvz = (float)(z0 + t) - czb;
          const float uz = fmaf(P.mz, dvz, bz);
          if (fabsf(uz) <= a) {
            const float ux = fmaf(P.e1z, dvz, bx), uy = fmaf(P.e2z, dvz, by);
            int ix = (int)ceilf(ux - a), iy = (int)ceilf(uy - a);
            const float fx = ux - (float)ix, fy = uy - (float)iy;
            if (ix < 0 || iy < 0 || ix > P.pw - KB || iy > P.ph - KB) {
              set_err(args.err, DERR_RANGE);
              ix = min(max(ix, 0), P.pw - KB);
              iy = min(max(iy, 0), P.ph - KB);
            }
            const float uz2 = uz * uz;
            const float2 *rv = pv + iy * P.pw + ix;
            const float *rm = pm + iy * P.pw + ix;
            float sr = 0.f, si = 0.f, sw = 0.f;
#pragma unroll
            for (int l = 0; l < KB; ++l) {
              const float dy = fy - (float)l;
              const float ry = fmaf(dy, dy, uz2);
#pragma unroll
              for (int j = 0; j < KB; ++j) {
                const float dx = fx - (float)j;
                const float r2 = fmaf(dx, dx, ry);
                if (r2 <= a2) {
                  const float w = blob_w<WMODE>(s_lut, r2, args, inv_a2);
                  const float2 v = rv[l * P.pw + j];
                  sr = fmaf(w, v.x, sr);
                  si = fmaf(w, v.y, si);
                  sw = fmaf(w, rm[l * P.pw + j], sw);
                }
              }
            }
            part[t][0] += sr; part[t][1] += si; part[t][2] += sw;
          }
        }
      }
      since_flush += ns;
      if (since_flush >= GATHER_FLUSH) {
        since_flush = 0;
#pragma unroll
        for (int t = 0; t < ZC; ++t)
#pragma unroll
          for (int c = 0; c < 3; ++c) { dd_add(hi[t][c], lo[t][c], part[t][c]); part[t][c] = 0.f; }
      }
      __syncthreads();  // patches are rebuilt next
    }
  }

  // ---- 4. fold into the HBM double-float accumulators
  if (vx > g.H || vy > g.H) return;
  const size_t plane = args.plane;
#pragma unroll
  for (int t = 0; t < ZC; ++t) {
    const int vz = z0 + t;
    if (vz > g.H) break;
    const size_t v = ((size_t)(vz + g.H) * g.D + (size_t)(vy + g.H)) * g.NXa + (size_t)(vx - g.xa0);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      dd_add(hi[t][c], lo[t][c], part[t][c]);
      float gh = args.acc[c * plane + v];
      float gl = args.acc[(3 + c) * plane + v];
      dd_add2(gh, gl, hi[t][c], lo[t][c]);
      args.acc[c * plane + v] = gh;
      args.acc[(3 + c) * plane + v] = gl;
    }
  }
}

}  // namespace fr
