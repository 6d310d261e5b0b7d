// lt_raster.cu -- the plain one-cube-per-thread atomic form of Eq. 6 and the
// per-frame mass reduction (the tiled raster is in lt_tile.cu).
#include "lt_internal.h"

namespace lt {

// Visit every (tetrahedron, pixel) fragment candidate of one cube inside the
// pixel rectangle [px0, px1] x [py0, py1] (absolute, inclusive), for every
// periodic copy of the cube that reaches it. fn(px, py, value) is called for
// candidates with value > 0 (value in accumulator units, before the
// perspective ray-length factor).
template <bool PERSP, bool EXACT, typename Fn>
__device__ __forceinline__ void cube_fragments(const CubeProj& P, const FrameDev& F, int px0, int px1, int py0,
                                               int py1, const Lattice& Lat, long long cube, Fn&& fn) {
  int sx0, sx1, sy0, sy1;
  const bool wrap = (!PERSP) && F.wrap;
  const float axa = P.axh + P.axl, aya = P.ayh + P.ayl;  // approximate anchor, for ranges only
  shift_range(axa + P.xmin, axa + P.xmax, (float)px0 - 0.5f, (float)px1 + 0.5f, (float)F.W, wrap, sx0, sx1);
  shift_range(aya + P.ymin, aya + P.ymax, (float)py0 - 0.5f, (float)py1 + 0.5f, (float)F.H, wrap, sy0, sy1);
  // a cube cannot span more than a few periods of a periodic window when its
  // particles moved less than half a box; cap the copies of invalid input
  sx1 = min(sx1, sx0 + 63);
  sy1 = min(sy1, sy0 + 63);
  for (int sy = sy0; sy <= sy1; ++sy) {
    for (int sx = sx0; sx <= sx1; ++sx) {
      const int shx = sx * F.W, shy = sy * F.H;
      const float ax = axa + (float)shx, ay = aya + (float)shy;
#pragma unroll
      for (int s = 0; s < 6; ++s) {
        if (tet_degenerate(Lat, F.snapshot, cube, s)) continue;  // zero volume: contributes nothing
        const int c0 = tet_corner(s, 0), c1 = tet_corner(s, 1), c2 = tet_corner(s, 2), c3 = tet_corner(s, 3);
        const float txmin = fminf(fminf(P.x[c0], P.x[c1]), fminf(P.x[c2], P.x[c3]));
        const float txmax = fmaxf(fmaxf(P.x[c0], P.x[c1]), fmaxf(P.x[c2], P.x[c3]));
        const float tymin = fminf(fminf(P.y[c0], P.y[c1]), fminf(P.y[c2], P.y[c3]));
        const float tymax = fmaxf(fmaxf(P.y[c0], P.y[c1]), fmaxf(P.y[c2], P.y[c3]));
        float Rv = fmaxf(fmaxf(fabsf(txmin), fabsf(txmax)), fmaxf(fabsf(tymin), fabsf(tymax)));
        if (PERSP) {
          const float dwm = fmaxf(fmaxf(fabsf(P.dw[c0]), fabsf(P.dw[c1])), fmaxf(fabsf(P.dw[c2]), fabsf(P.dw[c3])));
          Rv += fmaxf(fabsf(P.axh - F.cx), fabsf(P.ayh - F.cy)) * __fdividef(dwm, P.w0);
        }
        const float delta = vertex_uncertainty(Rv, PERSP);
        const float mg = 1e-3f + delta;
        const int qx0 = max(px0, (int)ceilf(ax + txmin - mg)), qx1 = min(px1, (int)floorf(ax + txmax + mg));
        const int qy0 = max(py0, (int)ceilf(ay + tymin - mg)), qy1 = min(py1, (int)floorf(ay + tymax + mg));
        if (qx0 > qx1 || qy0 > qy1) continue;
        float Kn = 6.0f * F.K, invKn = 0.0f;
        if (PERSP) {
          const float zz = P.z[c0] * P.z[c1] * P.z[c2] * P.z[c3];
          Kn = __fdividef(Kn, zz);
          invKn = fast_rcp(Kn);
        }
        TetRaster t;
        if (!tet_setup<PERSP>(P.x[c0], P.y[c0], P.x[c1], P.y[c1], P.x[c2], P.y[c2], P.x[c3], P.y[c3],
                              PERSP ? P.dw[c0] : 0.f, PERSP ? P.dw[c1] : 0.f, PERSP ? P.dw[c2] : 0.f,
                              PERSP ? P.dw[c3] : 0.f, Kn, P.w0, invKn, t))
          continue;
        for (int py = qy0; py <= qy1; ++py) {
          const float Y = rel_coord(py, shy, P.ayh, P.ayl);
          float erow[4], prow[2];
#pragma unroll
          for (int e = 0; e < 4; ++e) erow[e] = fmaf(t.b[e], Y, t.c[e]);
          if (PERSP) {
            prow[0] = fmaf(t.pb[0], Y, t.pc[0]);
            prow[1] = fmaf(t.pb[1], Y, t.pc[1]);
          }
          float lo, hi;
          row_span(t, erow, lo, hi);
          const bool check = EXACT && may_need_exact(t, F.sigma_units, delta);
          // a steep sliver visits its whole bounding-box row: pixels the
          // vertex uncertainty could move inside are checked too
          const bool whole = EXACT && may_miss_fragments(t, F.sigma_units, delta);
          const int xa = whole ? qx0 : max(qx0, (int)ceilf(fmaxf(lo + ax, -1.0e9f)));
          const int xb = whole ? qx1 : min(qx1, (int)floorf(fminf(hi + ax, 1.0e9f)));
          for (int px = xa; px <= xb; ++px) {
            const float X = rel_coord(px, shx, P.axh, P.axl);
            const float f0 = fmaf(t.a[0], X, erow[0]), f1 = fmaf(t.a[1], X, erow[1]);
            const float f2 = fmaf(t.a[2], X, erow[2]), f3 = fmaf(t.a[3], X, erow[3]);
            const float T = fmaxf(fminf(fminf(f0, f1), fminf(f2, f3)), 0.0f);
            float v = T, dvdT = 1.0f;
            if (PERSP) {
              const float M = fmaxf(fmaf(t.pa[0], X, prow[0]), fmaf(t.pa[1], X, prow[1]));
              const float den = M * fmaf(t.g, T, M);
              v = __fdividef(T, den);
              const float q = __fdividef(M, den);
              dvdT = q * q;
            }
            if (check && fragment_needs_exact(f0, f1, f2, f3, make_float4(t.a[0], t.a[1], t.a[2], t.a[3]),
                                              make_float4(t.b[0], t.b[1], t.b[2], t.b[3]),
                                              make_float4(t.c[0], t.c[1], t.c[2], t.c[3]),
                                              make_float4(t.st[0], t.st[1], t.st[2], t.st[3]), X, Y, delta, dvdT,
                                              v, F.sigma_units)) {
              const double ex = exact_fragment(Lat, F, cube, s, sx, sy, px, py, F.m_tet);
              if (ex > 0.0) fn(px, py, (float)(ex / F.unit));
              continue;
            }
            if (v > 0.0f) fn(px, py, v);
          }
        }
      }
    }
  }
}

// Perspective ray-direction length |d| = sqrt(1 + x^2 + y^2) of pixel (px, py).
__device__ __forceinline__ float ray_len(const FrameDev& F, int px, int py) {
  const float xt = F.tan_x * (2.0f * ((float)px + 0.5f) / (float)F.W - 1.0f);
  const float yt = F.tan_y * (2.0f * ((float)py + 0.5f) / (float)F.H - 1.0f);
  return sqrtf(1.0f + xt * xt + yt * yt);
}

// Per-frame mass: fixed-order sum of the frame's tile partials.
__global__ void k_mass_reduce(const double* __restrict__ mass_tile, long long tpf, double* __restrict__ d_mass) {
  __shared__ double ws[32];
  const int f = blockIdx.x;
  double s = 0.0;
  for (long long t = threadIdx.x; t < tpf; t += blockDim.x) s += mass_tile[(long long)f * tpf + t];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double w = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
    if (threadIdx.x == 0) d_mass[f] = w;
  }
}

cudaError_t launch_mass_reduce(const double* mass_tile, long long tpf, int n_frames, double* d_mass,
                               cudaStream_t s) {
  k_mass_reduce<<<n_frames, 256, 0, s>>>(mass_tile, tpf, d_mass);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Plain form: one thread per (frame, cube), float atomics into the image.

template <bool PERSP>
__device__ __forceinline__ void atomic_cube(const Lattice& L, const FrameDev& F, long long cube, float* img,
                                            DevCounters* ctr) {
  CubeProj P;
  bool ok = true;
  if (!project_cube<PERSP>(L, F, cube, P, ok)) return;
  const double unit = F.unit;
  cube_fragments<PERSP, true>(P, F, 0, F.W - 1, 0, F.H - 1, L, cube, [&](int px, int py, float v) {
    float val = (float)((double)v * unit);
    if (PERSP) val *= ray_len(F, px, py);
    atomicAdd(&img[(long long)py * F.W + px], val);
  });
}

__global__ void __launch_bounds__(256) k_atomic(Lattice L, const FrameDev* __restrict__ frames, long long stride,
                                                float* __restrict__ image, DevCounters* ctr) {
  const FrameDev& F = frames[blockIdx.y];
  float* img = image + (long long)blockIdx.y * stride;
  for (long long cube = (long long)blockIdx.x * blockDim.x + threadIdx.x; cube < L.n_particles;
       cube += (long long)gridDim.x * blockDim.x) {
    if (F.persp) atomic_cube<true>(L, F, cube, img, ctr);
    else atomic_cube<false>(L, F, cube, img, ctr);
  }
}

cudaError_t launch_atomic(const Lattice& L, const FrameDev* d_frames, long long stride, int n_frames, float* image,
                          DevCounters* ctr, cudaStream_t s) {
  long long b = (L.n_particles + 255) / 256;
  if (b > 4096) b = 4096;
  dim3 grid((unsigned)(b < 1 ? 1 : b), n_frames);
  k_atomic<<<grid, 256, 0, s>>>(L, d_frames, stride, image, ctr);
  return cudaGetLastError();
}

}  // namespace lt
