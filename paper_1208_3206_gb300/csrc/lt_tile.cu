// lt_tile.cu -- the persistent tile raster of Eq. 6 (and the fragment
// counter built on the same walk).
//
// One CTA takes (frame, tile) work items from an atomic counter. For its
// tile, each warp repeatedly takes 32 tetrahedra (one per lane) of the tile's
// cube list:
//   1. every lane projects its tetrahedron and builds its raster form (the
//      per-tetrahedron setup of lt_common.cuh) in tile pixel coordinates,
//      keeps it in a per-warp shared-memory record, and counts the pixel
//      centres of its bounding box inside the tile;
//   2. a warp scan turns the counts into one flat list of (tetrahedron,
//      pixel) candidates;
//   3. all 32 lanes walk that list together, 32 candidates per step (the
//      owning tetrahedron of a candidate is found from a bit mask of the
//      tetrahedra starting in the step), evaluate rho * dl at the pixel and
//      add it to the tile's fixed-point accumulators in shared memory.
// Control flow stays uniform across the warp, so lanes are busy in every
// phase whatever the sizes of the tetrahedra. Integer accumulation makes
// the result independent of the order of the adds. After the list is done
// every pixel of the tile is converted and stored once.
#include "lt_internal.h"

namespace lt {

constexpr int kRec = 36;  // words per tetrahedron record (stride 4 mod 32: float4 access is conflict-free)
constexpr int kQueue = 2048;  // ill-conditioned fragments queued per tile

// Record layout, in float4 groups so the walk reads it with a few 128-bit
// loads: [0] qx0, qy0, box width, 1/width; [1] a[4]; [2] b[4]; [3] c[4] (edge
// functions); [4] pa0, pb0, pc0, pa1; [5] pb1, pc1, g, exact-check flag
// (perspective depth planes); [6] edge steepness st[4]; [7] periodic copy
// (sx, sy). Words 30-35 pad the stride.

constexpr float kErr = kFragErr;
constexpr float kTol = kFragTol;

__device__ __forceinline__ unsigned long long pack_frag(unsigned tau, int sx, int sy, int X, int Y) {
  return (unsigned long long)tau | ((unsigned long long)(unsigned)(sx + 64) << 32) |
         ((unsigned long long)(unsigned)(sy + 64) << 39) | ((unsigned long long)(unsigned)X << 46) |
         ((unsigned long long)(unsigned)Y << 52);
}

template <bool ANY_PERSP, bool COUNT>
__global__ void __launch_bounds__(256, 2) k_tile(RasterArgs a, unsigned long long* __restrict__ counts) {
  extern __shared__ __align__(16) float smem_f[];
  const int T = a.tile;
  const int nw = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned* acc_lo = reinterpret_cast<unsigned*>(smem_f);
  unsigned* acc_hi = acc_lo + T * T;
  float* recs = reinterpret_cast<float*>(acc_hi + T * T) + warp * 32 * kRec;
  int* starts = reinterpret_cast<int*>(reinterpret_cast<float*>(acc_hi + T * T) + nw * 32 * kRec) + warp * 32;
  __shared__ unsigned long long item_s;
  __shared__ double mass_w[32];
  __shared__ unsigned long long queue[kQueue];
  __shared__ unsigned qn;
  const unsigned FULL = 0xffffffffu;
  unsigned long long nfrag = 0;

  for (;;) {
    if (threadIdx.x == 0) {
      item_s = atomicAdd(&a.ctr->work_next, 1ull);
      qn = 0u;
    }
    if (!COUNT)
      for (int q = threadIdx.x; q < 2 * T * T; q += blockDim.x) acc_lo[q] = 0u;
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
    const unsigned long long e0 = a.off[tg];
    const long long ntet = 6LL * (long long)(a.off[tg + 1] - e0);
    const bool wrap = (!persp) && F.wrap;
    const float Kn0 = 6.0f * F.K;
    const float sig = F.sigma_units;

    // tb / 6 and tb % 6 carried along the loop (tb advances by nw * 32)
    const unsigned step_q = (unsigned)(nw * 32) / 6u, step_r = (unsigned)(nw * 32) % 6u;
    unsigned long long cq = (unsigned long long)warp * 32u / 6u;
    unsigned cr = (unsigned)(warp * 32) % 6u;
    for (long long tb = (long long)warp * 32; tb < ntet; tb += (long long)nw * 32) {
      // ---- 1. one tetrahedron per lane
      const long long tau = tb + lane;
      TetProj P;
      bool ok = false;
      if (tau < ntet) {
        const unsigned rel = cr + (unsigned)lane;  // < 38
        const long long cube = (long long)a.list[e0 + cq + rel / 6u];
        const int s = (int)(rel % 6u);
        ok = persp ? project_tet<true>(a.L, F, cube, s, P) : project_tet<false>(a.L, F, cube, s, P);
      }
      float bx0 = 0.f, bx1 = -1.f, by0 = 0.f, by1 = -1.f;
      int sx0 = 0, sx1 = -1, sy0 = 0, sy1 = -1;
      if (ok) {
        bx0 = fminf(fminf(P.x[0], P.x[1]), fminf(P.x[2], P.x[3]));
        bx1 = fmaxf(fmaxf(P.x[0], P.x[1]), fmaxf(P.x[2], P.x[3]));
        by0 = fminf(fminf(P.y[0], P.y[1]), fminf(P.y[2], P.y[3]));
        by1 = fmaxf(fmaxf(P.y[0], P.y[1]), fmaxf(P.y[2], P.y[3]));
        const float axa = P.axh + P.axl, aya = P.ayh + P.ayl;
        shift_range(axa + bx0, axa + bx1, (float)tx0 - 0.5f, (float)(tx0 + tw) - 0.5f, (float)F.W, wrap, sx0, sx1);
        shift_range(aya + by0, aya + by1, (float)ty0 - 0.5f, (float)(ty0 + th) - 0.5f, (float)F.H, wrap, sy0, sy1);
        sx1 = min(sx1, sx0 + 63);
        sy1 = min(sy1, sy0 + 63);
      }
      const int ncx = max(0, sx1 - sx0 + 1), ncp = ncx * max(0, sy1 - sy0 + 1);
      const int rounds = __reduce_max_sync(FULL, ncp);
      float Kn = Kn0, invKn = 0.f;
      if (persp && ok) {
        Kn = Kn0 / (P.z[0] * P.z[1] * P.z[2] * P.z[3]);
        invKn = 1.0f / Kn;
      }
      for (int r = 0; r < rounds; ++r) {
        int n = 0;
        if (r < ncp) {
          const int sx = sx0 + r % ncx, sy = sy0 + r / ncx;
          // vertex coordinates relative to the tile origin: anchor + shift - tile corner
          const float ox = ((float)(tx0 - sx * F.W) - P.axh) - P.axl;
          const float oy = ((float)(ty0 - sy * F.H) - P.ayh) - P.ayl;
          const float x0 = P.x[0] - ox, x1 = P.x[1] - ox, x2 = P.x[2] - ox, x3 = P.x[3] - ox;
          const float y0 = P.y[0] - oy, y1 = P.y[1] - oy, y2 = P.y[2] - oy, y3 = P.y[3] - oy;
          const int qx0 = max(0, (int)ceilf(bx0 - ox - 1e-3f));
          const int qx1 = min(tw - 1, (int)floorf(bx1 - ox + 1e-3f));
          const int qy0 = max(0, (int)ceilf(by0 - oy - 1e-3f));
          const int qy1 = min(th - 1, (int)floorf(by1 - oy + 1e-3f));
          if (qx0 <= qx1 && qy0 <= qy1) {
            TetRaster t;
            bool set = persp ? tet_setup<true>(x0, y0, x1, y1, x2, y2, x3, y3, P.dw[0], P.dw[1], P.dw[2], P.dw[3],
                                               Kn, P.w0, invKn, t)
                             : tet_setup<false>(x0, y0, x1, y1, x2, y2, x3, y3, 0.f, 0.f, 0.f, 0.f, Kn, 0.f, 0.f, t);
            if (set) {
              float4* R = reinterpret_cast<float4*>(recs + lane * kRec);
              const int qw = qx1 - qx0 + 1;
              R[0] = make_float4(__int_as_float(qx0), __int_as_float(qy0), __int_as_float(qw), 1.0f / (float)qw);
              R[1] = make_float4(t.a[0], t.a[1], t.a[2], t.a[3]);
              R[2] = make_float4(t.b[0], t.b[1], t.b[2], t.b[3]);
              R[3] = make_float4(t.c[0], t.c[1], t.c[2], t.c[3]);
              const float flag = may_need_exact(t, sig) ? 1.0f : 0.0f;
              if (persp) {
                R[4] = make_float4(t.pa[0], t.pb[0], t.pc[0], t.pa[1]);
                R[5] = make_float4(t.pb[1], t.pc[1], t.g, flag);
              } else {
                R[5] = make_float4(0.f, 0.f, 0.f, flag);
              }
              R[6] = make_float4(t.st[0], t.st[1], t.st[2], t.st[3]);
              R[7] = make_float4(__int_as_float(sx), __int_as_float(sy), 0.f, 0.f);
              n = qw * (qy1 - qy0 + 1);
            }
          }
        }
        // ---- 2. flatten the candidates of the 32 tetrahedra
        int incl = n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(FULL, incl, o);
          if (lane >= o) incl += y;
        }
        const int off = incl - n;
        const int total = __shfl_sync(FULL, incl, 31);
        __syncwarp();
        // ---- 3. walk the candidates, 32 per step
        int carry = 0;
        for (int base = 0; base < total; base += 32) {
          const int bp = off - base;
          const bool in = n > 0 && bp >= 0 && bp < 32;
          const unsigned mask = __reduce_or_sync(FULL, in ? (1u << bp) : 0u);
          if (in) starts[bp] = lane;
          __syncwarp();
          const unsigned m = mask & (FULL >> (31 - lane));
          const int owner = m ? starts[31 - __clz(m)] : carry;
          const int own_off = __shfl_sync(FULL, off, owner);
          const int pos = base + lane;
          if (pos < total) {
            const float4* R = reinterpret_cast<const float4*>(recs + owner * kRec);
            const int kk = pos - own_off;
            const float4 r0 = R[0];
            const int w = __float_as_int(r0.z);
            const int dy = (int)(((float)kk + 0.5f) * r0.w);
            const int dx = kk - dy * w;
            const int X = __float_as_int(r0.x) + dx, Y = __float_as_int(r0.y) + dy;
            const float fx = (float)X, fy = (float)Y;
            const float4 ra = R[1], rb = R[2], rc = R[3];
            const float f0 = fmaf(ra.x, fx, fmaf(rb.x, fy, rc.x));
            const float f1 = fmaf(ra.y, fx, fmaf(rb.y, fy, rc.y));
            const float f2 = fmaf(ra.z, fx, fmaf(rb.z, fy, rc.z));
            const float f3 = fmaf(ra.w, fx, fmaf(rb.w, fy, rc.w));
            const float Tv = fmaxf(fminf(fminf(f0, f1), fminf(f2, f3)), 0.0f);
            float v = Tv;
            float4 r5;
            if (persp) {
              const float4 r4 = R[4];
              r5 = R[5];
              const float M = fmaxf(fmaf(r4.x, fx, fmaf(r4.y, fy, r4.z)), fmaf(r4.w, fx, fmaf(r5.x, fy, r5.y)));
              v = __fdividef(Tv, M * fmaf(r5.z, Tv, M));
            } else if (!COUNT) {
              r5 = R[5];
            }
            if (v > 0.0f) {
              bool risky = false;
              if (!COUNT && r5.w != 0.0f) {
                // steepness of the edge that bounds the value here
                const float4 r6 = R[6];
                float sa = r6.x, mn = f0;
                if (f1 < mn) { mn = f1; sa = r6.y; }
                if (f2 < mn) { mn = f2; sa = r6.z; }
                if (f3 < mn) { sa = r6.w; }
                risky = sa * kErr * v > kTol * fmaxf(v, sig);
              }
              if (COUNT) {
                ++nfrag;
              } else if (!risky) {
                accum_fixed(&acc_lo[Y * T + X], &acc_hi[Y * T + X], v, &a.ctr->errors);
              } else {
                const float4 r7 = R[7];
                const int sxo = __float_as_int(r7.x), syo = __float_as_int(r7.y);
                const unsigned slot = atomicAdd(&qn, 1u);
                if (slot < (unsigned)kQueue) {
                  queue[slot] = pack_frag((unsigned)(tb + owner), sxo, syo, X, Y);
                } else {
                  // queue full: keep the FP32 value (counted in the statistics)
                  accum_fixed(&acc_lo[Y * T + X], &acc_hi[Y * T + X], v, &a.ctr->errors);
                }
              }
            }
          }
          carry = mask ? starts[31 - __clz(mask)] : carry;
          __syncwarp();
        }
      }
      cr += step_r;
      cq += step_q + (cr >= 6u ? 1u : 0u);
      cr = cr >= 6u ? cr - 6u : cr;
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
    const unsigned nq = min(qn, (unsigned)kQueue);
    if (threadIdx.x == 0 && qn) {
      atomicAdd(&a.ctr->exact_fragments, (unsigned long long)nq);
      if (qn > (unsigned)kQueue) atomicAdd(&a.ctr->queue_overflow, (unsigned long long)(qn - kQueue));
    }
    for (unsigned qi = threadIdx.x; qi < nq; qi += blockDim.x) {
      const unsigned long long q = queue[qi];
      const unsigned tau_o = (unsigned)(q & 0xffffffffull);
      const int sxo = (int)((q >> 32) & 127u) - 64, syo = (int)((q >> 39) & 127u) - 64;
      const int X = (int)((q >> 46) & 63u), Y = (int)((q >> 52) & 63u);
      const long long cube = (long long)a.list[e0 + (unsigned long long)(tau_o / 6)];
      const double val = exact_fragment(a.L, F, cube, (int)(tau_o % 6), sxo, syo, tx0 + X, ty0 + Y, F.m_tet);
      if (val > 0.0) accum_fixed(&acc_lo[Y * T + X], &acc_hi[Y * T + X], (float)(val / F.unit), &a.ctr->errors);
    }
    __syncthreads();
    // ---- one store per pixel, and the tile's share of the frame mass
    double msum = 0.0;
    float* img = a.image + (long long)f * a.image_stride;
    for (int li = threadIdx.x; li < tw * th; li += blockDim.x) {
      const int ly = li / tw, lx = li - ly * tw;
      const int si = ly * T + lx;
      const unsigned long long q = ((unsigned long long)acc_hi[si] << 16) + (unsigned long long)acc_lo[si];
      double v = (double)q * F.unit;
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
  return sizeof(unsigned) * 2 * tile * tile + sizeof(float) * nw * 32 * kRec + sizeof(int) * nw * 32;
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
