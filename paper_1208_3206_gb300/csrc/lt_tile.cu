// lt_tile.cu -- the persistent tile raster of Eq. 6 (and the fragment
// counter built on the same walk).
//
// One CTA takes (frame, tile) work items from an atomic counter. For its
// tile, each warp repeatedly takes a batch of kCB cubes of the tile's cube
// list:
//   0. two lanes per cube project its anchor and its eight corners (four
//      each) into the warp's corner table in shared memory, so every corner
//      is projected once per tile whatever the number of tetrahedra sharing
//      it; then, 32 tetrahedra (one per lane) at a time:
//   1. every lane reads its tetrahedron's four corners from the table and
//      builds its raster form (the per-tetrahedron setup of lt_common.cuh)
//      in tile pixel coordinates; the records of the drawable ones are
//      compacted into a per-warp table in shared memory;
//   2. a warp scan flattens the (tetrahedron, row) jobs of their bounding
//      boxes; 32 jobs at a time, each lane finds the pixel span of its row
//      where every edge function is >= 0;
//   3. a second scan flattens the spans' pixels; 32 pixels at a time, each
//      lane evaluates rho * dl and adds it to the pixel's 64-bit fixed-point
//      accumulator in shared memory with one integer atomic (the owner of a
//      job or pixel is found from the popcount of the step's start mask,
//      without shared memory);
//   4. fragments whose FP32 value may be off by more than the tolerance are
//      queued and evaluated exactly in FP64 after the walk.
// Control flow stays uniform across the warp, so lanes are busy in every
// phase whatever the sizes of the tetrahedra. Integer accumulation makes
// the result independent of the order of the adds. After the walk every
// pixel of the tile is converted and stored once.
#include "lt_internal.h"

namespace lt {

constexpr int kRec = 36;  // words per tetrahedron record (stride 4 mod 32: float4 access is conflict-free)
constexpr int kCB = 16;          // cubes per warp batch (two lanes each in step 0)
constexpr int kTB = 6 * kCB;     // their tetrahedra: kTB / 32 rounds of steps 1-3
constexpr int kCorStride = 9;    // float4 per cube in the corner table (eight corners and a pad)

// Per-warp shared memory.
struct WarpSmem {
  float4 cor[kCB * kCorStride];  // corner (x, y, 1/Z - 1/Z_anchor, Z) relative to the cube's anchor
  float4 anc[kCB];               // anchor pixel coordinate as hi + lo: axh, axl, ayh, ayl
  float4 cinfo[kCB];             // 1/Z_anchor, perspective uncertainty factor, flags, -
  float recs[32 * kRec];         // records of the drawable tetrahedra of the current 32
  int4 jobs[32];                 // (tetrahedron, row) jobs of the current step
};
constexpr unsigned kCubeValid = 0x100u;  // cinfo flags: bits 0..5 zero-volume mask, this bit: drawable
// Ill-conditioned fragments are queued per CTA in global memory (a.xq_cap
// entries per CTA) and evaluated exactly after the tile's walk.

// Record layout, in float4 groups so the walk reads it with a few 128-bit
// loads: [0] qx0, qy0, qx1 | flag << 16 (bounding box in tile pixels),
// first row job; [1] a[4]; [2] b[4]; [3] c[4] (edge functions); [4] 1/a[4]
// (row spans); [5] pa0, pb0, pc0, pa1; [6] pb1, pc1, g (perspective depth
// planes), exact-check flag; [7] edge steepness st[4]; [8] periodic copy
// (sx, sy), tetrahedron index within the tile's list (6 x list position
// + s), vertex uncertainty.

__device__ __forceinline__ unsigned long long pack_frag(unsigned tau, int sx, int sy, int X, int Y) {
  return (unsigned long long)tau | ((unsigned long long)(unsigned)(sx + 64) << 32) |
         ((unsigned long long)(unsigned)(sy + 64) << 39) | ((unsigned long long)(unsigned)X << 46) |
         ((unsigned long long)(unsigned)Y << 52);
}

// 1 / a, or 0 for a == 0 (an edge function constant along the row).
// (Correctly rounded over the whole range: a steep sliver's |a| can pass
// 2^126, where the approximate reciprocal returns 0.)
__device__ __forceinline__ float inv_or_zero(float a) { return a != 0.0f ? __frcp_rn(a) : 0.0f; }

// Narrow [lo, hi] to the X where a X + rr >= 0 (rr the row term b Y + c).
// An edge constant along the row (a == 0) empties the row when rr < 0; the
// unused slot (rr = +inf) never constrains.
__device__ __forceinline__ void span_edge(float a, float rr, float ia, float& lo, float& hi) {
  const float xe = -rr * ia;
  if (a > 0.0f) lo = fmaxf(lo, xe);
  if (a < 0.0f) hi = fminf(hi, xe);
  if (a == 0.0f && rr < 0.0f) hi = __int_as_float(0xff800000);
}

// Exclusive warp scan of n; total receives the warp's sum.
__device__ __forceinline__ int warp_excl_scan(int n, int& total) {
  const int lane = threadIdx.x & 31;
  int incl = n;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  total = __shfl_sync(0xffffffffu, incl, 31);
  return incl - n;
}

#ifndef LT_TILE_MIN_CTAS
#define LT_TILE_MIN_CTAS 2  // resident 256-thread CTAs per SM the register budget is cut for
#endif

template <bool ANY_PERSP, bool COUNT>
__global__ void __launch_bounds__(256, LT_TILE_MIN_CTAS) k_tile(RasterArgs a, unsigned long long* __restrict__ counts) {
  extern __shared__ __align__(16) float4 smem4[];
  const int T = a.tile;
  const int AS = T + 5;  // accumulator row stride: consecutive rows start on different banks
  const int nw = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  WarpSmem& S = reinterpret_cast<WarpSmem*>(smem4)[warp];
  unsigned long long* acc = reinterpret_cast<unsigned long long*>(reinterpret_cast<WarpSmem*>(smem4) + nw);
  float* recs = S.recs;
  int4* jobs = S.jobs;
  __shared__ unsigned long long item_s;
  __shared__ double mass_w[32];
  __shared__ unsigned qn;
  unsigned long long* xq = a.xq + (size_t)blockIdx.x * a.xq_cap;
  const unsigned FULL = 0xffffffffu;
  unsigned long long nfrag = 0;

  for (;;) {
    if (threadIdx.x == 0) {
      item_s = atomicAdd(&a.ctr->work_next, 1ull);
      qn = 0u;
    }
    if (!COUNT)
      for (int q = threadIdx.x; q < T * AS; q += blockDim.x) acc[q] = 0ull;
    __syncthreads();
    const unsigned long long item = item_s;
    if (item >= (unsigned long long)a.n_items) break;
    const long long tg = (long long)a.work[item];
    const long long tpf = (long long)a.frames[0].tiles_x * a.frames[0].tiles_y;
    const int f = (int)(tg / tpf);
    const FrameDev& F = a.frames[f];
    const bool persp = ANY_PERSP && F.persp;
    const long long tl = tg - (long long)f * tpf;
    const int tyi = (int)(tl / F.tiles_x), txi = (int)(tl - (long long)tyi * F.tiles_x);
    const int tx0 = txi * T, ty0 = tyi * T;
    const int tw = min(T, F.W - tx0), th = min(T, F.H - ty0);
    // a graph replayed after the positions changed can need more list entries
    // than it was sized for: the scatter dropped the excess (and latched the
    // error), and the walk reads only what the lists hold
    unsigned long long e0 = a.off[tg], e1 = a.off[tg + 1];
    if (e1 > a.list_cap) {
      if (threadIdx.x == 0) atomicOr(&a.ctr->errors, kErrCapacity);
      e0 = min(e0, a.list_cap);
      e1 = a.list_cap;
    }
    const long long ncl = (long long)(e1 - e0);
    const bool wrap = (!persp) && F.wrap;
    const float Kn0 = 6.0f * F.K;
    const float sig = F.sigma_units;
    const long long snap_off = (long long)F.snapshot * a.L.n_particles;

    for (long long cb = (long long)warp * kCB; cb < ncl; cb += (long long)nw * kCB) {
      // ---- 0. lanes c and c + 16 project cube c: its anchor and corners 0-3 / 4-7
      {
        const int c = lane & (kCB - 1), hh = lane >> 4;
        const long long cidx = cb + c;
        bool ok = true, front = true;
        unsigned zmask = 0;
        float axh = 0.f, axl = 0.f, ayh = 0.f, ayl = 0.f, w0 = 0.f;
        if (cidx < ncl) {
          const unsigned long long li = e0 + (unsigned long long)cidx;
          const long long cube = LT_IN_BOUNDS(li < e1, &a.ctr->errors) ? (long long)a.list[li] : 0;
          zmask = a.L.degen ? (unsigned)__ldg(a.L.degen + snap_off + cube) & 63u : 0u;
          if (cube_far(a.L, F, cube)) ok = false;  // hybrid rendering: drawn as splats
          int i, j, k;
          cube_ijk(a.L, cube, i, j, k);
          float X0 = 0.f, Y0 = 0.f, Z0 = 1.f;
          if (!persp) {
            anchor_affine(F, 0, i, j, k, axh, axl);
            anchor_affine(F, 1, i, j, k, ayh, ayl);
          } else {
            float Xh, Xl, Yh, Yl, Zh, Zl;
            anchor_affine(F, 0, i, j, k, Xh, Xl);
            anchor_affine(F, 1, i, j, k, Yh, Yl);
            anchor_affine(F, 2, i, j, k, Zh, Zl);
            X0 = Xh + Xl; Y0 = Yh + Yl; Z0 = Zh + Zl;
            front = Z0 > F.near_z;
            const float rz = fast_rcp(Zh);
            ff_project(Xh, Xl, Zh, Zl, rz, F.kxh, F.kxl, F.cx, axh, axl);
            ff_project(Yh, Yl, Zh, Zl, rz, F.kyh, F.kyl, F.cy, ayh, ayl);
            w0 = fast_rcp(Z0);
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int n = 4 * hh + q;
            const float3 l = load_corner(a.L, snap_off, i, j, k, n, ok);
            float4 cv;
            if (!persp) {
              cv.x = (F.r[0] * l.x + F.r[1] * l.y + F.r[2] * l.z) * F.sx;
              cv.y = (F.u[0] * l.x + F.u[1] * l.y + F.u[2] * l.z) * F.sy;
              cv.z = 0.f;
              cv.w = 1.f;
            } else {
              const float dX = F.r[0] * l.x + F.r[1] * l.y + F.r[2] * l.z;
              const float dY = F.u[0] * l.x + F.u[1] * l.y + F.u[2] * l.z;
              const float dZ = F.f[0] * l.x + F.f[1] * l.y + F.f[2] * l.z;
              const float Zn = Z0 + dZ;
              front = front && (Zn > F.near_z);
              const float inv = fast_rcp(Zn * Z0);
              // X_n/Z_n - X0/Z0 = (dX Z0 - X0 dZ) / (Z_n Z0), free of cancellation
              cv.x = (dX * Z0 - X0 * dZ) * inv * F.kx;
              cv.y = (dY * Z0 - Y0 * dZ) * inv * F.ky;
              cv.z = -dZ * inv;
              cv.w = Zn;
            }
            S.cor[c * kCorStride + n] = cv;
          }
        }
        // both halves of a cube must be finite and in front of the eye
        const bool good = __shfl_xor_sync(FULL, (int)(ok && front), 16) && ok && front;
        if (hh == 0) {
          // perspective: the anchor's offset from the view axis times the
          // depth offsets enters the vertex uncertainty (per corner |dw| / w0)
          const float offw = persp ? __fdividef(fmaxf(fabsf(axh - F.cx), fabsf(ayh - F.cy)), w0) : 0.f;
          const unsigned flags = zmask | ((cidx < ncl && good) ? kCubeValid : 0u);
          S.anc[c] = make_float4(axh, axl, ayh, ayl);
          S.cinfo[c] = make_float4(w0, offw, __int_as_float((int)flags), 0.f);
        }
      }
      __syncwarp();
#pragma unroll 1
      for (int qr = 0; qr < kTB / 32; ++qr) {
        // ---- 1. one tetrahedron per lane
        const int ts = qr * 32 + lane;  // tetrahedron slot of the batch
        const int c = ts / 6, s = ts - 6 * c;
        const unsigned tau = (unsigned)((cb + c) * 6 + s);  // index within the tile's tetrahedra
        const float4 ci = S.cinfo[c];
        const unsigned cfl = (unsigned)__float_as_int(ci.z);
        const bool ok = (cfl & kCubeValid) && !((cfl >> s) & 1u);  // zero volume: contributes nothing
        float px[4], py[4], pdw[4], pz[4];
        float4 an = make_float4(0.f, 0.f, 0.f, 0.f);
        if (ok) {
          an = S.anc[c];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const float4 v = S.cor[c * kCorStride + tet_corner_dyn(s, k)];
            px[k] = v.x; py[k] = v.y; pdw[k] = v.z; pz[k] = v.w;
          }
        } else {
#pragma unroll
          for (int k = 0; k < 4; ++k) { px[k] = 0.f; py[k] = 0.f; pdw[k] = 0.f; pz[k] = 1.f; }
        }
        float bx0 = 0.f, bx1 = -1.f, by0 = 0.f, by1 = -1.f;
        int sx0 = 0, sx1 = -1, sy0 = 0, sy1 = -1;
        if (ok) {
          bx0 = fminf(fminf(px[0], px[1]), fminf(px[2], px[3]));
          bx1 = fmaxf(fmaxf(px[0], px[1]), fmaxf(px[2], px[3]));
          by0 = fminf(fminf(py[0], py[1]), fminf(py[2], py[3]));
          by1 = fmaxf(fmaxf(py[0], py[1]), fmaxf(py[2], py[3]));
          const float axa = an.x + an.y, aya = an.z + an.w;
          shift_range(axa + bx0, axa + bx1, (float)tx0 - 0.5f, (float)(tx0 + tw) - 0.5f, (float)F.W, wrap, sx0, sx1);
          shift_range(aya + by0, aya + by1, (float)ty0 - 0.5f, (float)(ty0 + th) - 0.5f, (float)F.H, wrap, sy0, sy1);
          sx1 = min(sx1, sx0 + 63);
          sy1 = min(sy1, sy0 + 63);
        }
        const int ncx = max(0, sx1 - sx0 + 1), ncp = ncx * max(0, sy1 - sy0 + 1);
        float delta = 0.f;
        if (ok) {
          const float Rx = fmaxf(fmaxf(fabsf(px[0]), fabsf(px[1])), fmaxf(fabsf(px[2]), fabsf(px[3])));
          const float Ry = fmaxf(fmaxf(fabsf(py[0]), fabsf(py[1])), fmaxf(fabsf(py[2]), fabsf(py[3])));
          float Rv = fmaxf(Rx, Ry);
          if (persp) Rv += ci.y * fmaxf(fmaxf(fabsf(pdw[0]), fabsf(pdw[1])), fmaxf(fabsf(pdw[2]), fabsf(pdw[3])));
          delta = vertex_uncertainty(Rv, persp);
        }
        const float margin = 1e-3f + delta;
        const int rounds = __reduce_max_sync(FULL, ncp);
        float Kn = Kn0, invKn = 0.f;
        if (persp && ok) {
          Kn = __fdividef(Kn0, pz[0] * pz[1] * pz[2] * pz[3]);
          invKn = fast_rcp(Kn);
        }
        for (int r = 0; r < rounds; ++r) {
          int nrows = 0, qx0 = 0, qx1 = 0, qy0 = 0, sx = 0, sy = 0;
          TetRaster t;
          if (r < ncp) {
            sx = sx0 + r % ncx;
            sy = sy0 + r / ncx;
            // vertex coordinates relative to the tile origin: anchor + shift - tile corner
            const float ox = ((float)(tx0 - sx * F.W) - an.x) - an.y;
            const float oy = ((float)(ty0 - sy * F.H) - an.z) - an.w;
            const float x0 = px[0] - ox, x1 = px[1] - ox, x2 = px[2] - ox, x3 = px[3] - ox;
            const float y0 = py[0] - oy, y1 = py[1] - oy, y2 = py[2] - oy, y3 = py[3] - oy;
            qx0 = max(0, (int)ceilf(bx0 - ox - margin));
            qx1 = min(tw - 1, (int)floorf(bx1 - ox + margin));
            qy0 = max(0, (int)ceilf(by0 - oy - margin));
            const int qy1 = min(th - 1, (int)floorf(by1 - oy + margin));
            if (qx0 <= qx1 && qy0 <= qy1) {
              // the raster form relative to the bounding box's first pixel:
              // small coordinates keep the round-off of evaluating a x + b y + c
              // (and with it the exact path's share) small
              const float lx = (float)qx0, ly = (float)qy0;
              const bool set =
                  persp ? tet_setup<true>(x0 - lx, y0 - ly, x1 - lx, y1 - ly, x2 - lx, y2 - ly, x3 - lx, y3 - ly,
                                          pdw[0], pdw[1], pdw[2], pdw[3], Kn, ci.x, invKn, t)
                        : tet_setup<false>(x0 - lx, y0 - ly, x1 - lx, y1 - ly, x2 - lx, y2 - ly, x3 - lx, y3 - ly,
                                           0.f, 0.f, 0.f, 0.f, Kn, 0.f, 0.f, t);
              if (set) nrows = qy1 - qy0 + 1;
            }
          }
          // ---- 2. records of the drawable tetrahedra, compacted, and the
          // flattened (tetrahedron, row) jobs
          const unsigned lt_mask = (1u << lane) - 1u, le_mask = (2u << lane) - 1u;
          const int slot = __popc(__ballot_sync(FULL, nrows > 0) & lt_mask);
          int rtotal;
          const int roff = warp_excl_scan(nrows, rtotal);
          if (nrows > 0 && LT_IN_BOUNDS(slot < 32, &a.ctr->errors)) {
            float4* R = reinterpret_cast<float4*>(recs + slot * kRec);
            const bool flagged = may_need_exact(t, sig, delta);
            const bool whole_rows = may_miss_fragments(t, sig, delta);
            R[0] = make_float4(__int_as_float(qx0), __int_as_float(qy0), __int_as_float(qx1 | (whole_rows ? 0x10000 : 0)),
                               __int_as_float(roff));
            R[1] = make_float4(t.a[0], t.a[1], t.a[2], t.a[3]);
            R[2] = make_float4(t.b[0], t.b[1], t.b[2], t.b[3]);
            R[3] = make_float4(t.c[0], t.c[1], t.c[2], t.c[3]);
            R[4] = make_float4(inv_or_zero(t.a[0]), inv_or_zero(t.a[1]), inv_or_zero(t.a[2]), inv_or_zero(t.a[3]));
            const float flag = flagged ? 1.0f : 0.0f;
            if (persp) {
              R[5] = make_float4(t.pa[0], t.pb[0], t.pc[0], t.pa[1]);
              R[6] = make_float4(t.pb[1], t.pc[1], t.g, flag);
            } else {
              R[6] = make_float4(0.f, 0.f, 0.f, flag);
            }
            R[7] = make_float4(t.st[0], t.st[1], t.st[2], t.st[3]);
            R[8] = make_float4(__int_as_float(sx), __int_as_float(sy), __int_as_float((int)tau), delta);
          }
          __syncwarp();
          // The owner of a position in a 32-wide step is the last run starting
          // at or before it: with runs compacted, its index is the number of
          // runs started before the step plus those started in the step up to
          // the position, minus one.
          int rprev = 0;
          for (int rb = 0; rb < rtotal; rb += 32) {
            const int rrel = roff - rb;
            const unsigned rmask = __reduce_or_sync(FULL, (nrows > 0 && rrel >= 0 && rrel < 32) ? (1u << rrel) : 0u);
            const int o = rprev + __popc(rmask & le_mask) - 1;
            rprev += __popc(rmask);
            // ---- 3. pixel span of each job's row: every edge function >= 0
            // (coordinates relative to the record's bounding-box corner)
            int len = 0, xl = 0, yl = 0, abase = 0;
            if (rb + lane < rtotal) {
              const float4* R = reinterpret_cast<const float4*>(recs + o * kRec);
              const float4 r0 = R[0];
              yl = rb + lane - __float_as_int(r0.w);
              const float fy = (float)yl;
              const float4 ra = R[1], rbv = R[2], rc = R[3], ri = R[4];
              float lo = __int_as_float(0xff800000), hi = __int_as_float(0x7f800000);
              span_edge(ra.x, fmaf(rbv.x, fy, rc.x), ri.x, lo, hi);
              span_edge(ra.y, fmaf(rbv.y, fy, rc.y), ri.y, lo, hi);
              span_edge(ra.z, fmaf(rbv.z, fy, rc.z), ri.z, lo, hi);
              span_edge(ra.w, fmaf(rbv.w, fy, rc.w), ri.w, lo, hi);
              const int qx0 = __float_as_int(r0.x), qy0 = __float_as_int(r0.y), qx1w = __float_as_int(r0.z);
              const float wf = (float)((qx1w & 0xffff) - qx0);  // last pixel of the box, local
              if (qx1w >> 16) {
                // a steep sliver: the whole bounding-box row, so that pixels the
                // vertex uncertainty could move inside are checked too
                lo = 0.0f;
                hi = wf;
              }
              lo = fmaxf(lo - 1e-3f, 0.0f);
              hi = fminf(hi + 1e-3f, wf);
              if (lo <= hi) {
                xl = (int)ceilf(lo);
                len = max(0, (int)floorf(hi) - xl + 1);
              }
              abase = (qy0 + yl) * AS + qx0 + xl;  // accumulator index of the span's first pixel
            }
            int ptotal;
            const int poff = warp_excl_scan(len, ptotal);
            const int jslot = __popc(__ballot_sync(FULL, len > 0) & lt_mask);
            if (len > 0 && LT_IN_BOUNDS(jslot < 32 && o < 32, &a.ctr->errors))
              jobs[jslot] = make_int4(xl | (yl << 16), abase, o, poff);
            __syncwarp();
            // ---- 4. walk the pixels of the jobs, 32 per step
            int pprev = 0;
            for (int pb = 0; pb < ptotal; pb += 32) {
              const int prel = poff - pb;
              const unsigned pmask = __reduce_or_sync(FULL, (len > 0 && prel >= 0 && prel < 32) ? (1u << prel) : 0u);
              const int j = pprev + __popc(pmask & le_mask) - 1;
              pprev += __popc(pmask);
              bool exact = false;
              unsigned long long qent = 0;
              float vq = 0.f;
              int aq = 0;
              if (pb + lane < ptotal) {
                const int4 J = jobs[j];
                const int kx = pb + lane - J.w;  // position within the job's span
                const int ai = J.y + kx;         // accumulator index
                const float4* R = reinterpret_cast<const float4*>(recs + J.z * kRec);
                const float fx = (float)((J.x & 0xffff) + kx), fy = (float)(J.x >> 16);
                const float4 ra = R[1], rbv = R[2], rc = R[3];
                const float f0 = fmaf(ra.x, fx, fmaf(rbv.x, fy, rc.x));
                const float f1 = fmaf(ra.y, fx, fmaf(rbv.y, fy, rc.y));
                const float f2 = fmaf(ra.z, fx, fmaf(rbv.z, fy, rc.z));
                const float f3 = fmaf(ra.w, fx, fmaf(rbv.w, fy, rc.w));
                const float Tv = fmaxf(fminf(fminf(f0, f1), fminf(f2, f3)), 0.0f);
                float v = Tv;
                float4 r6 = make_float4(0.f, 0.f, 0.f, 0.f);
                float M = 1.0f, den = 1.0f;
                if (persp) {
                  const float4 r5 = R[5];
                  r6 = R[6];
                  M = fmaxf(fmaf(r5.x, fx, fmaf(r5.y, fy, r5.z)), fmaf(r5.w, fx, fmaf(r6.x, fy, r6.y)));
                  den = M * fmaf(r6.z, Tv, M);
                  v = __fdividef(Tv, den);
                } else if (!COUNT) {
                  r6 = R[6];
                }
                if (COUNT) {
                  if (v > 0.0f) ++nfrag;
                } else if (v > 0.0f || r6.w != 0.0f) {
                  // flagged tetrahedra: fragments whose error bound is too large,
                  // and pixels the vertex uncertainty could move inside, go to
                  // the exact evaluation
                  if (r6.w != 0.0f) {
                    const float q = persp ? __fdividef(M, den) : 1.0f;  // d value / d T = (M / den)^2
                    exact = fragment_needs_exact(f0, f1, f2, f3, ra, rbv, rc, R[7], fx, fy, R[8].w, q * q, v, sig);
                  }
                  if (!exact) {
                    if (v > 0.0f && LT_IN_BOUNDS(ai >= 0 && ai % AS < tw && ai / AS < th, &a.ctr->errors))
                      accum_fixed(&acc[ai], v, a.ctr);
                  } else {
                    const float4 r8 = R[8];
                    const int Y = ai / AS, X = ai - Y * AS;  // tile pixel of the queued fragment
                    qent = pack_frag((unsigned)__float_as_int(r8.z), __float_as_int(r8.x), __float_as_int(r8.y),
                                     X, Y);
                    vq = v;
                    aq = ai;
                  }
                }
              }
              if (!COUNT) {
                const unsigned em = __ballot_sync(FULL, exact);
                if (em) {
                  const int leader = __ffs(em) - 1;
                  unsigned base = 0;
                  if (lane == leader) base = atomicAdd(&qn, (unsigned)__popc(em));
                  base = __shfl_sync(FULL, base, leader);
                  if (exact) {
                    const unsigned slot = base + __popc(em & lt_mask);
                    if (slot < a.xq_cap) {
                      xq[slot] = qent;
                    } else if (vq > 0.0f) {
                      // queue full: keep the FP32 value (counted in the statistics)
                      accum_fixed(&acc[aq], vq, a.ctr);
                    }
                  }
                }
              }
              __syncwarp();
            }
          }
        }
      }
      __syncwarp();
    }
    if (COUNT) {
      unsigned long long c = nfrag;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(FULL, c, o);
      if (lane == 0 && c) atomicAdd(&counts[f], c);
      nfrag = 0;
      __syncthreads();
      continue;
    }
    __syncthreads();
    // ---- ill-conditioned fragments: exact FP64 evaluation, all lanes busy
    const unsigned nq = min(qn, a.xq_cap);
    if (threadIdx.x == 0 && qn) {
      atomicAdd(&a.ctr->exact_fragments, (unsigned long long)nq);
      atomicMax(&a.ctr->exact_tile_max, (unsigned long long)qn);
      if (qn > a.xq_cap) atomicAdd(&a.ctr->queue_overflow, (unsigned long long)(qn - a.xq_cap));
    }
    for (unsigned qi = threadIdx.x; qi < nq; qi += blockDim.x) {
      const unsigned long long q = xq[qi];
      const unsigned tau_o = (unsigned)(q & 0xffffffffull);
      const int sxo = (int)((q >> 32) & 127u) - 64, syo = (int)((q >> 39) & 127u) - 64;
      const int X = (int)((q >> 46) & 63u), Y = (int)((q >> 52) & 63u);
      const unsigned long long li = e0 + (unsigned long long)(tau_o / 6);
      if (!LT_IN_BOUNDS(li < e1 && X < tw && Y < th, &a.ctr->errors)) continue;
      const long long cube = (long long)a.list[li];
      const double val = exact_fragment(a.L, F, cube, (int)(tau_o % 6), sxo, syo, tx0 + X, ty0 + Y, F.m_tet);
      if (val > 0.0) accum_fixed(&acc[Y * AS + X], (float)(val / F.unit), a.ctr);
    }
    __syncthreads();
    // ---- one store per pixel, and the tile's share of the frame mass
    double msum = 0.0;
    float* img = a.image + (long long)f * a.image_stride;
    for (int li = threadIdx.x; li < tw * th; li += blockDim.x) {
      const int ly = li / tw, lx = li - ly * tw;
      double v = (double)acc[ly * AS + lx] * F.unit;
      if (persp) {
        const float xt = F.tan_x * (2.0f * ((float)(tx0 + lx) + 0.5f) / (float)F.W - 1.0f);
        const float yt = F.tan_y * (2.0f * ((float)(ty0 + ly) + 0.5f) / (float)F.H - 1.0f);
        v *= (double)sqrtf(1.0f + xt * xt + yt * yt);
      }
      const float vf = (float)v;
      img[(long long)(ty0 + ly) * F.W + (tx0 + lx)] = vf;
      msum += (double)vf;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) msum += __shfl_down_sync(FULL, msum, o);
    if (lane == 0) mass_w[warp] = msum;
    __syncthreads();
    if (threadIdx.x < 32) {
      double w = threadIdx.x < (unsigned)nw ? mass_w[threadIdx.x] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(FULL, w, o);
      if (threadIdx.x == 0) a.mass_tile[tg] = w * F.pix_area;
    }
    __syncthreads();
  }
}

static size_t tile_smem(int threads, int tile) {
  const int nw = threads / 32;
  return sizeof(WarpSmem) * nw + sizeof(unsigned long long) * tile * (tile + 5);
}

int raster_max_ctas_per_sm(int threads, int tile, int any_persp) {
  if (threads > 256 || threads % 32) return 0;  // the kernel is compiled for at most 256 threads
  int n = 0;
  const size_t smem = tile_smem(threads, tile);
  cudaError_t e;
  if (any_persp) {
    cudaFuncSetAttribute(k_tile<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_tile<true, false>, threads, smem);
  } else {
    cudaFuncSetAttribute(k_tile<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_tile<false, false>, threads, smem);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

cudaError_t launch_count_fragments(const RasterArgs& a, unsigned long long* d_counts, int n_frames, int ctas,
                                   int threads, cudaStream_t s) {
  (void)n_frames;
  const size_t smem = tile_smem(threads, a.tile);
  cudaFuncSetAttribute(k_tile<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_tile<true, true><<<ctas, threads, smem, s>>>(a, d_counts);
  return cudaGetLastError();
}

cudaError_t launch_raster(const RasterArgs& a, int ctas, int threads, int any_persp, cudaStream_t s) {
  const size_t smem = tile_smem(threads, a.tile);
  if (any_persp) {
    cudaFuncSetAttribute(k_tile<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_tile<true, false><<<ctas, threads, smem, s>>>(a, nullptr);
  } else {
    cudaFuncSetAttribute(k_tile<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_tile<false, false><<<ctas, threads, smem, s>>>(a, nullptr);
  }
  return cudaGetLastError();
}

}  // namespace lt
