// fr_gather2.cuh -- the direct-drain gather insertion kernel.
//
// Same decomposition as the per-voxel gather of fr_gather.cuh (a warp owns an
// 8 x 4 x ZC footprint of voxel columns, culls the images of its work unit
// into a shared-memory list, and accumulates (image, voxel) items into
// shared-memory partial sums that are folded into HBM with TwoSum), with far
// fewer instructions spent per item:
//
//  * item generation: for each list image every lane marks the run of z
//    levels of its column that lie within a of the plane (u_z is linear in z,
//    so the run is contiguous) and appends one 16-bit tag per item (list entry,
//    column, z level) to the warp's tag queue, at lane-major positions found
//    with one ballot per bit of the run length (8- or 16-deep columns);
//  * evaluation: each full round of 32 tags (one item per lane) forms
//    u = R^T v from the footprint centre's compensated projection, reflects
//    u through the origin when it lies in the mirrored half plane (the pixel is
//    then read at -c and conjugated: Hermitian symmetry), puts the 4 x 4
//    candidate box at ceil(u - a) clamped into the stored half plane
//    kx in [0, H], ky in [-H, H - 1] (box rows and columns moved in by the
//    clamp lie outside the blob and are masked), reads each box row as two
//    two-pixel loads, evaluates the Chebyshev weight polynomial in
//    x = 2 r^2 / a^2 - 1 for two candidates at a time with packed FP32x2
//    FMAs (masked to 0 outside r <= a) and adds the complex and weight sums to
//    the voxel's partial sums with shared-memory atomics.
//
// An item whose box crosses the column kx = 0 is evaluated twice: the box
// clamped to kx >= 0 read directly, and the point-reflected box clamped to
// kx >= 0 read conjugated (its tag is queued again with the half forced).  Away
// from the fold columns every point of the extended plane within a of the
// voxel has (R c)_x > 0, so a column c_x > 0 receives the stored pixel c, a
// column c_x < 0 the stored -c conjugated, and the column c_x = 0 both (0, c_y)
// and, conjugated, (0, -c_y): exactly what the two boxes read.  The bricks of
// this kernel's main launch tile x >= floor(a) + 1.  The fold columns |x| <=
// floor(a), where the fold predicate itself has to be evaluated per pixel,
// are computed by a second instantiation over those columns only (FOLD), in
// footprints 4 columns wide so that three of four lanes hold fold columns:
// there a stored pixel k counts in the directly read box when it is not
// folded and in the reflected box when it is (exact sign of R00 k_x + R01
// k_y).  Polynomial weights only, 4 x 4 boxes only (a < 2).
#pragma once

#include "fr_gather.cuh"

namespace fr {

constexpr int G2_T2CAP = 64;  // forced second halves: < 32 carried over + <= 32 per round

// tags of one list image (<= 32 columns x ZC levels) + < 32 carried over
template <int ZC>
__host__ __device__ constexpr int g2_tcap() {
  return 32 * ZC + 32;
}

// Per-warp shared memory: image list, partial sums, tag queues, phase counters.
template <int ZC>
__host__ __device__ constexpr size_t gather2_warp_smem(int chunk) {
  return ((size_t)LIST_FIELDS * chunk * 4 + (size_t)3 * (32 * ZC) * 4 + (size_t)G2_T2CAP * 4 +
          (size_t)g2_tcap<ZC>() * 2 + (size_t)PH_COUNT * 8 + 15) &
         ~(size_t)15;
}

// The 4 pixels of a box row starting at `row`, read as two two-pixel loads
// from the aligned unit at or before `row` (the images are 16-byte aligned,
// so every image's storage row 0 starts aligned and the unit before an
// unaligned row start lies in the image's previous storage row), plus one
// single-pixel load when `row` is not aligned: no load leaves the images.
template <int F16>
__device__ __forceinline__ void load_row4(const unsigned char *row, float2 &p0, float2 &p1,
                                          float2 &p2, float2 &p3) {
  const uintptr_t u = reinterpret_cast<uintptr_t>(row);
  if (!F16) {
    const bool odd = (u & 8) != 0;
    const float4 *al = reinterpret_cast<const float4 *>(u & ~(uintptr_t)15);
    const float4 A = __ldg(al), B = __ldg(al + 1);
    float2 C = make_float2(0.f, 0.f);
    if (odd) C = __ldg(reinterpret_cast<const float2 *>(al + 2));
    p0 = odd ? make_float2(A.z, A.w) : make_float2(A.x, A.y);
    p1 = odd ? make_float2(B.x, B.y) : make_float2(A.z, A.w);
    p2 = odd ? make_float2(B.z, B.w) : make_float2(B.x, B.y);
    p3 = odd ? C : make_float2(B.z, B.w);
  } else {
    const bool odd = (u & 4) != 0;
    const uint2 *al = reinterpret_cast<const uint2 *>(u & ~(uintptr_t)7);
    const uint2 A = __ldg(al), B = __ldg(al + 1);
    unsigned C = 0u;
    if (odd) C = __ldg(reinterpret_cast<const unsigned *>(al + 2));
    const unsigned h0 = odd ? A.y : A.x, h1 = odd ? B.x : A.y, h2 = odd ? B.y : B.x,
                   h3 = odd ? C : B.y;
    p0 = __half22float2(*reinterpret_cast<const __half2 *>(&h0));
    p1 = __half22float2(*reinterpret_cast<const __half2 *>(&h1));
    p2 = __half22float2(*reinterpret_cast<const __half2 *>(&h2));
    p3 = __half22float2(*reinterpret_cast<const __half2 *>(&h3));
  }
}

// The 4 x 4 box of an item: candidates (kx0 + j, ky0 + l) of the stored half
// plane (ibase points at pixel kx0 of the image), u at (kx0 + fx, ky0 + fy),
// u_z^2 = uz2; returns the sums of w p (complex) and of w over the candidates
// with r <= a.  FOLD: a stored pixel k is inserted at R k when it is not
// folded and at -R k (conjugated) when it is, folded meaning R00 k_x + R01 k_y
// < 0 (exact sign; r00, r01 = R00, R01): the box read directly (refl = 0)
// keeps the candidates that are not folded, the point-reflected box (refl =
// 1) those that are.  Away from the fold columns that test always passes.
template <int F16, int FOLD = 0>
__device__ __forceinline__ void g2_box(const InsertArgs &args, const float2 *cp,
                                       const unsigned char *ibase, int kx0, int ky0, float fx,
                                       float fy, float uz2, float cs, float sq, float2 &acc,
                                       float &aw, float r00 = 0.f, float r01 = 0.f,
                                       bool refl = false) {
  constexpr int NP = POLY_N;
  constexpr int ESZ = F16 ? 4 : 8;
  const Geom &g = args.g;
  // cp: coefficient pairs (c_k, c_k), kernel-parameter constants
  const int row_bytes = g.NX * ESZ;
  // scaled column offsets sq (fx - j): x = (sq dx)^2 + cs (dy^2 + u_z^2) - 1
  const float2 d01 = make_float2(sq * fx, sq * (fx - 1.0f));
  const float2 d23 = make_float2(sq * (fx - 2.0f), sq * (fx - 3.0f));
  const float U = fmaf(cs, uz2, -1.0f);
  float2 a2 = make_float2(0.f, 0.f), w2 = make_float2(0.f, 0.f);
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    int ky = ky0 + r;
    ky += ky < 0 ? g.S : 0;
    float2 p0, p1, p2, p3;
    load_row4<F16>(ibase + ky * row_bytes, p0, p1, p2, p3);
    const float dy = fy - (float)r;
    const float Y = fmaf(cs * dy, dy, U);
    const float2 YY = make_float2(Y, Y);
    const float2 xa = __ffma2_rn(d01, d01, YY), xb = __ffma2_rn(d23, d23, YY);
    float2 ha = cp[NP - 1], hb = cp[NP - 1];
#pragma unroll
    for (int k = NP - 2; k >= 0; --k) {
      ha = __ffma2_rn(ha, xa, cp[k]);
      hb = __ffma2_rn(hb, xb, cp[k]);
    }
    float w0 = xa.x <= 1.0f ? ha.x : 0.0f, w1 = xa.y <= 1.0f ? ha.y : 0.0f;
    float w2_ = xb.x <= 1.0f ? hb.x : 0.0f, w3 = xb.y <= 1.0f ? hb.y : 0.0f;
    if (FOLD) {
      const int kyr = ky0 + r;
      if (fold_pred(r00, r01, kx0, kyr) != refl) w0 = 0.f;
      if (fold_pred(r00, r01, kx0 + 1, kyr) != refl) w1 = 0.f;
      if (fold_pred(r00, r01, kx0 + 2, kyr) != refl) w2_ = 0.f;
      if (fold_pred(r00, r01, kx0 + 3, kyr) != refl) w3 = 0.f;
    }
    a2 = __ffma2_rn(make_float2(w0, w0), p0, a2);
    a2 = __ffma2_rn(make_float2(w1, w1), p1, a2);
    a2 = __ffma2_rn(make_float2(w2_, w2_), p2, a2);
    a2 = __ffma2_rn(make_float2(w3, w3), p3, a2);
    w2 = __fadd2_rn(w2, make_float2(w0 + w2_, w1 + w3));
  }
  acc = a2;
  aw = w2.x + w2.y;
}

// One warp's share of one work unit (see gather_warp for the unit word).
// args: the batch's arguments; cst: the arguments its launch shares (geometry,
// weight polynomial, list capacity) and images the batch's images, both read
// in the inner loops.  The warp footprint is FW x (32 / FW) columns (8 x 4,
// or 4 x 8 for the fold columns).  FOLD = 0: the bricks tile x >= floor(a) +
// 1; FOLD = 1: they tile x >= -floor(a) and only the fold columns |x| <=
// floor(a) are computed, with the fold predicate tested per candidate.
template <int BX, int BY, int ZC, int F16, int FW = 8, int FOLD = 0>
__device__ __forceinline__ void gather2_warp(const InsertArgs &args, const InsertArgs &cst,
                                             const void *images, unsigned char *wsmem,
                                             const int4 unit, const int warp) {
  constexpr int FH = 32 / FW;  // footprint height in y
  static_assert((FW == 8 || FW == 4) && BX % FW == 0 && BY % FH == 0 && (BX * BY) % 32 == 0,
                "warp footprint is 8 x 4 or 4 x 8 columns");
  static_assert(ZC == 8 || ZC == 16, "tags hold 4 bits of z");
  constexpr int WV = 32 * ZC;
  constexpr int ESZ = F16 ? 4 : 8;
  constexpr float HX = 0.5f * (FW - 1), HY = 0.5f * (FH - 1);  // footprint half extents
  const Geom &g = cst.g;
  const int lane = threadIdx.x & 31;
  const int wx = warp % (BX / FW), wy = warp / (BX / FW);
  const int fx0 = (FOLD ? g.xa0 : 1 - g.xa0) + unit.x * BX + wx * FW;
  const int fy0 = -g.H + unit.y * BY + wy * FH;
  const int z0 = -g.H + unit.z * ZC;
  const int lcap = cst.chunk;
  if (lcap > 64) {  // list entries are 6 bits of the tags
    if (lane == 0) set_err(args.err, DERR_RANGE);
    return;
  }
  float *s_list = reinterpret_cast<float *>(__builtin_assume_aligned(wsmem, 16));
  float *s_acc = s_list + (size_t)LIST_FIELDS * lcap;                               // [3][WV]
  unsigned *s_tag2 = reinterpret_cast<unsigned *>(s_acc + 3 * WV);                  // [G2_T2CAP]
  unsigned long long *s_ph = reinterpret_cast<unsigned long long *>(s_tag2 + G2_T2CAP);  // [PH_COUNT]
  unsigned short *s_tag = reinterpret_cast<unsigned short *>(s_ph + PH_COUNT);      // [g2_tcap]

  const int split = unit.w & 0xffff, nsplit = (unit.w >> 16) & 0x3fff;
  const bool to_scratch = nsplit > 1 || ((unit.w >> 30) & 1);
  const int img0 = (int)((long long)args.n * split / nsplit);
  const int img1 = (int)((long long)args.n * (split + 1) / nsplit);
  const float cx = fx0 + HX, cy = fy0 + HY, cz = z0 + 0.5f * (ZC - 1);  // footprint centre
  const float hz = 0.5f * (ZC - 1);
  const float rw = sqrtf(HX * HX + HY * HY + hz * hz);
  const float a = g.a;
  // box origin ceil(u - a_box): a spare box cell (KB > floor(2a) + 1) is
  // shifted down by a margin so a pixel at distance exactly a is never lost
  // to the rounding of u (the r^2 <= a^2 mask decides it)
  const float a_box = 4 > (int)floorf(2.0f * a) + 1 ? a + 1e-4f : a;
  const float a_plane = a + 1e-4f;      // conservative |u_z| <= a test
  const float reach = (float)g.H + a;   // the extended plane spans [-H, H]^2
  const float ext = reach + rw + 1.0f;
  const int vx = fx0 + lane % FW, vy = fy0 + lane / FW;
  const bool col_in = vx <= g.H && vy <= g.H && (!FOLD || vx <= -g.xa0);
  const float dvx = (float)(lane % FW) - HX, dvy = (float)(lane / FW) - HY;
  const float cs = 2.0f / g.a2, sq = sqrtf(cs);  // the weight polynomial's argument scales
  const unsigned char *imgs = reinterpret_cast<const unsigned char *>(images);
  const size_t img_stride = (size_t)g.S * g.NX * ESZ;
  const unsigned lt = (1u << lane) - 1u;

  for (int i = lane; i < 3 * WV; i += 32) s_acc[i] = 0.f;
  __syncwarp();
  // optional phase counters (fr_options.debug bit 1): cycles of cull, item
  // generation (PH_QUEUE), evaluation rounds (PH_DRAIN_FAST) and flushes, item
  // and round counts; kept in shared memory (lane 0 counts) so that they hold
  // no registers
  const bool prof = args.phase != nullptr;
  unsigned long long *ph = s_ph;
  if (prof && lane == 0)
    for (int k = 0; k < PH_COUNT; ++k) ph[k] = 0;
  const long long t_start = prof ? clock64() : 0;
  auto tick = [&]() -> long long { return prof ? clock64() : 0; };

  int qt = 0, qt2 = 0;  // queued tags, queued forced second halves

  // One round: lane k evaluates tag q[k] (if k < cnt): li << 9 | column << 4 |
  // z level, plus bit 16 (half forced) and bit 17 (the reflected half) for
  // the second halves; an item whose box crosses kx = 0 queues its other half
  // in s_tag2.
  auto round = [&](unsigned tag, bool alive) {
    const int li = (int)((tag >> 9) & 63), src = (int)((tag >> 4) & 31), t = (int)(tag & 15);
    const bool forced = ((tag >> 16) & 1u) != 0, fneg = ((tag >> 17) & 1u) != 0;
    const float *L = s_list + li * LIST_FIELDS;
    const float4 q0 = *reinterpret_cast<const float4 *>(L + LF_MX);   // m, u_z of the centre
    const float4 q1 = *reinterpret_cast<const float4 *>(L + LF_E1X);  // e1, fractional u_x
    const float4 q2 = *reinterpret_cast<const float4 *>(L + LF_E2X);  // e2, fractional u_y
    const int4 q3 = *reinterpret_cast<const int4 *>(L + LF_CIX);      // integer centre, image address
    const float sdx = (float)(src % FW) - HX, sdy = (float)(src / FW) - HY,
                sdz = (float)t - hz;
    const float uz = fmaf(q0.z, sdz, fmaf(q0.y, sdy, fmaf(q0.x, sdx, q0.w)));
    const float uxr = fmaf(q1.z, sdz, fmaf(q1.y, sdy, fmaf(q1.x, sdx, q1.w)));
    const float uyr = fmaf(q2.z, sdz, fmaf(q2.y, sdy, fmaf(q2.x, sdx, q2.w)));
    const float ux = (float)q3.x + uxr, uy = (float)q3.y + uyr;
    const bool valid = alive && fabsf(ux) <= reach && fabsf(uy) <= reach;
    // the half plane read: the one u lies in, or the forced one
    const bool neg = forced ? fneg : ux < 0.f;
    const float sg = neg ? -1.f : 1.f;
    const int isg = neg ? -1 : 1;
    const float vxr = sg * uxr, vyr = sg * uyr;
    const float ixf = ceilf(vxr - a_box), iyf = ceilf(vyr - a_box);
    const int kx0 = isg * q3.x + (int)ixf, ky0 = isg * q3.y + (int)iyf;
    // the box reaches column kx <= 0: the other half as well
    const bool second = valid && !forced && kx0 < 1;
    const unsigned m2 = __ballot_sync(0xffffffffu, second);
    if (second) s_tag2[qt2 + __popc(m2 & lt)] = (tag & 0xffffu) | (1u << 16) | (neg ? 0u : 1u << 17);
    qt2 += __popc(m2);
    // clamp the box into the stored half plane [0, H] x [-H, H - 1]
    const int kxc = min(max(kx0, 0), g.H - 3);
    const int kyc = min(max(ky0, -g.H), g.H - 4);
    // an item outside the extended plane (or a dead lane) keeps a box far from u
    const float fx = valid ? vxr - ixf + (float)(kx0 - kxc) : 64.f;
    const float fy = vyr - iyf + (float)(ky0 - kyc);
    float2 acc;
    float aw;
    const unsigned char *ibase = reinterpret_cast<const unsigned char *>(
        (unsigned long long)(unsigned)q3.z | ((unsigned long long)(unsigned)q3.w << 32));
    g2_box<F16, FOLD>(cst, cst.poly2, ibase + (size_t)kxc * ESZ, kxc,
                      kyc, fx, fy, uz * uz, cs, sq, acc, aw, q1.x, q2.x, neg);
    if (valid) {
      const int slot = src * ZC + t;
      atomicAdd(&s_acc[slot], acc.x);
      atomicAdd(&s_acc[WV + slot], neg ? -acc.y : acc.y);
      atomicAdd(&s_acc[2 * WV + slot], aw);
    }
    __syncwarp();
  };

  // evaluate full rounds of both queues (every tag if `all`); the remainders
  // move to the fronts
  auto drain = [&](bool all) {
    const long long t0 = tick();
    int nr = 0;
    int head = 0;
    for (; qt - head >= 32 || (all && qt > head); head += 32) {
      const bool alive = lane < qt - head;
      round(alive ? (unsigned)s_tag[head + lane] : 0u, alive);
      ++nr;
      if (qt2 >= 32) {
        const unsigned t2 = s_tag2[lane];
        __syncwarp();
        round(t2, true);
        ++nr;
        qt2 -= 32;
        const unsigned v = lane < qt2 ? s_tag2[32 + lane] : 0u;
        __syncwarp();
        if (lane < qt2) s_tag2[lane] = v;
        __syncwarp();
      }
    }
    if (all && qt2 > 0) {
      const bool alive = lane < qt2;
      const unsigned t2 = alive ? s_tag2[lane] : 0u;
      __syncwarp();
      qt2 = 0;
      round(t2, alive);
      ++nr;
    }
    const int rest = qt - head < 0 ? 0 : qt - head;
    if (head > 0 && rest) {
      const unsigned short v = lane < rest ? s_tag[head + lane] : (unsigned short)0;
      __syncwarp();
      if (lane < rest) s_tag[lane] = v;
      __syncwarp();
    }
    qt = rest;
    if (prof && lane == 0) {
      ph[PH_DRAIN_FAST] += (unsigned long long)(clock64() - t0);
      ph[PH_ROUNDS] += (unsigned long long)nr;
    }
  };

  // generate the items of list entry li (tags at the queue's tail): the run
  // of z levels t with |u_z(t)| <= a of the lane's column, from u_z linear in t
  auto generate = [&](int li) {
    const long long tq = tick();
    const float *L = s_list + li * LIST_FIELDS;
    const float4 q0 = *reinterpret_cast<const float4 *>(L + LF_MX);
    const float bz = fmaf(q0.z, -hz, fmaf(q0.y, dvy, fmaf(q0.x, dvx, q0.w)));
    unsigned near = 0;
#pragma unroll
    for (int t = 0; t < ZC; ++t)
      near |= (fabsf(fmaf(q0.z, (float)t, bz)) <= a_plane ? 1u : 0u) << t;
    if (!col_in) near = 0;
    const int c = __popc(near);
    const int t0 = near ? __ffs(near) - 1 : 0;
    const unsigned lt_ = lt;
    int excl = 0, ntag = 0;
#pragma unroll
    for (int b = 0; b < 5; ++b) {
      if (b == 4 && ZC < 16) break;
      const unsigned bal = __ballot_sync(0xffffffffu, (c >> b) & 1);
      excl += __popc(bal & lt_) << b;
      ntag += __popc(bal) << b;
    }
    const unsigned base = ((unsigned)li << 9) | ((unsigned)lane << 4);
    const int p0 = qt + excl;
#pragma unroll
    for (int t = 0; t < ZC; ++t)
      if ((near >> t) & 1u) s_tag[p0 + (t - t0)] = (unsigned short)(base | (unsigned)t);
    qt += ntag;
    __syncwarp();
    if (prof && lane == 0) {
      ph[PH_QUEUE] += (unsigned long long)(clock64() - tq);
      ph[PH_ITEMS_FAST] += (unsigned long long)ntag;
    }
  };

  int nl = 0;           // entries in the warp's list
  int since_flush = 0;  // list entries processed since the last flush
  for (int cs0 = img0;; cs0 += 32) {
    const bool last = cs0 >= img1;
    if (!last) {
      const long long tc = tick();
      nl = cull_step(args, imgs, img_stride, s_list, nl, cs0, img1, cx, cy, cz, HX, HY, hz, ext,
                     col_in_any(g, fx0, fy0));
      __syncwarp();
      if (prof && lane == 0) ph[PH_CULL] += (unsigned long long)(clock64() - tc);
    }
    if (last || nl > lcap - 32) {
      if (prof && lane == 0) ph[PH_LIST_IMAGES] += (unsigned long long)nl;
      for (int li = 0; li < nl; ++li) {
        generate(li);
        drain(false);
        if (++since_flush >= GATHER_FLUSH) {
          drain(true);
          const long long tf = tick();
          flush_partials<ZC, FW>(args, s_acc, fx0, fy0, z0, to_scratch);
          if (prof && lane == 0) ph[PH_FLUSH] += (unsigned long long)(clock64() - tf);
          since_flush = 0;
        }
      }
      // the list is rebuilt next: nothing may refer to its entries afterwards
      drain(true);
      nl = 0;
    }
    if (last) break;
  }
  const long long tf = tick();
  flush_partials<ZC, FW>(args, s_acc, fx0, fy0, z0, to_scratch);
  if (prof && lane == 0) {
    ph[PH_FLUSH] += (unsigned long long)(clock64() - tf);
    ph[PH_WARP_CYCLES] = (unsigned long long)(clock64() - t_start);
    for (int k = 0; k < PH_COUNT; ++k)
      if (ph[k]) atomicAdd(args.phase + k, ph[k]);
  }
}

// One CTA per work unit (args.units[blockIdx.x]); warps run independently.
// MINW: resident warps per SM the register allocation must allow (16, 20 or
// 24: at most 128, 102 or 85 registers per thread).  FW, FOLD: see
// gather2_warp.
template <int BX, int BY, int ZC, int F16, int MINW, int FW = 8, int FOLD = 0>
__global__ void __launch_bounds__(BX * BY, MINW * 32 / (BX * BY))
gather2_kernel(const InsertArgs args) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5;
  gather2_warp<BX, BY, ZC, F16, FW, FOLD>(args, args, args.images,
                                smem + (size_t)warp * gather2_warp_smem<ZC>(args.chunk),
                                args.units[blockIdx.x], warp);
}

// Several batches in one launch: CTA b takes work item p.items[b] =
// {bx | by << 10 | bz << 20, split word, batch, slot} and copies its batch's
// arguments p.descs[batch] to shared memory; geometry, weight polynomial and
// list capacity, common to the launch's batches, are read from p.base (kernel
// parameters: constant operands in the inner loops).
template <int BX, int BY, int ZC, int F16, int MINW, int FW = 8, int FOLD = 0>
__global__ void __launch_bounds__(BX * BY, MINW * 32 / (BX * BY))
gather2_multi_kernel(const MultiLaunch p) {
  constexpr int NT = BX * BY;
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5;
  InsertArgs *s_args = reinterpret_cast<InsertArgs *>(smem);
  const int4 it = p.items[blockIdx.x];
  const int *src = reinterpret_cast<const int *>(p.descs + it.z);
  int *dst = reinterpret_cast<int *>(s_args);
  for (int i = tid; i < (int)(sizeof(InsertArgs) / 4); i += NT) dst[i] = src[i];
  __syncthreads();
  const int4 unit = make_int4(it.x & 1023, (it.x >> 10) & 1023, (it.x >> 20) & 1023, it.y);
  gather2_warp<BX, BY, ZC, F16, FW, FOLD>(
      *s_args, p.base, p.images[it.w],
      smem + GATHER_ARGS_BYTES + (size_t)warp * gather2_warp_smem<ZC>(p.base.chunk), unit, warp);
}

}  // namespace fr
