// lt_backward.cu -- adjoint of the orthographic projection: dL/d(position)
// from dL/dI, differentiating the per-tetrahedron pyramid form of
// rho_t * dl_t (Eq. 6, 3, 9) with respect to the projected vertices.
//
// Inside the region where hull edge e = (j, k) is the lowest of the pyramid
// faces, the value is f_e(x) = Kn * sigma * N(x) / (o1 o2) with
// N(x) = orient(v_j, v_k, x) and o1, o2 = orient(v_j, v_k, v_l1 / v_l2).
// Its derivative with respect to any vertex is affine in x, so the sums over
// a tetrahedron's fragments only need the moments sum g, sum g X, sum g Y
// of dL/dI per active edge. One thread per cube walks its fragments as a
// gather from dL/dI (no atomics), keeps the 8 corner gradients in registers
// over all frames, and a second kernel gathers them per particle in a fixed
// order.
#include "lt_internal.h"

namespace lt {

struct Moments {
  float g0[4], gx[4], gy[4];
};

// Gradient of the projected canonical vertices (pixel units) from the moments.
__device__ __forceinline__ void edge_grad(const TetCanon& K, int e, float Kn, float tiny, const Moments& m,
                                          float* gxv, float* gyv) {
  const EdgeRef r = edge_ref(K, e);
  const float prod = r.o1 * r.o2;
  if (!(fabsf(prod) > tiny) || m.g0[e] == 0.0f) return;
  if (!K.caseB && e == 3) return;
  const float sg = (r.o1 + r.o2) < 0.0f ? -1.0f : 1.0f;
  const float A = Kn * sg / prod;
  const float xj = sel4(K.x, r.j), yj = sel4(K.y, r.j);
  const float xl1 = sel4(K.x, r.l1), yl1 = sel4(K.y, r.l1);
  const float xl2 = sel4(K.x, r.l2), yl2 = sel4(K.y, r.l2);
  const float SGy = m.gy[e] - yj * m.g0[e];  // sum g (Y - y_j)
  const float SGx = m.gx[e] - xj * m.g0[e];  // sum g (X - x_j)
  const float SN = r.ex * SGy - r.ey * SGx;  // sum g N
  const float R1 = SN / r.o1, R2 = SN / r.o2;
  const float s1x = xl1 - xj, s1y = yl1 - yj, s2x = xl2 - xj, s2y = yl2 - yj;
  // vertex k
  const float gkx = A * (SGy - R1 * s1y - R2 * s2y);
  const float gky = A * (-SGx + R1 * s1x + R2 * s2x);
  // vertex j
  const float gjx = A * ((-SGy + r.ey * m.g0[e]) - R1 * (-s1y + r.ey) - R2 * (-s2y + r.ey));
  const float gjy = A * ((SGx - r.ex * m.g0[e]) - R1 * (s1x - r.ex) - R2 * (s2x - r.ex));
  // the two others
  const float gl1x = A * R1 * r.ey, gl1y = -A * R1 * r.ex;
  const float gl2x = A * R2 * r.ey, gl2y = -A * R2 * r.ex;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    gxv[v] += (v == r.k ? gkx : 0.f) + (v == r.j ? gjx : 0.f) + (v == r.l1 ? gl1x : 0.f) + (v == r.l2 ? gl2x : 0.f);
    gyv[v] += (v == r.k ? gky : 0.f) + (v == r.j ? gjy : 0.f) + (v == r.l1 ? gl1y : 0.f) + (v == r.l2 ? gl2y : 0.f);
  }
}

__global__ void __launch_bounds__(128) k_backward(Lattice L, const FrameDev* __restrict__ frames, int n_frames,
                                                  long long stride, const float* __restrict__ dLdI,
                                                  float* __restrict__ corner_grad) {
  const long long ncube = L.n_particles;
  const int snap = blockIdx.y;
  for (long long cube = (long long)blockIdx.x * blockDim.x + threadIdx.x; cube < ncube;
       cube += (long long)gridDim.x * blockDim.x) {
    float G[8][3];
#pragma unroll
    for (int n = 0; n < 8; ++n) G[n][0] = G[n][1] = G[n][2] = 0.f;
    for (int f = 0; f < n_frames; ++f) {
      const FrameDev& F = frames[f];
      if (F.snapshot != snap || F.persp) continue;
      CubeProj P;
      bool ok = true;
      if (!project_cube<false>(L, F, cube, P, ok)) continue;
      const float* gimg = dLdI + (long long)f * stride;
      float gpx[8], gpy[8];
#pragma unroll
      for (int n = 0; n < 8; ++n) gpx[n] = gpy[n] = 0.f;
      int sx0, sx1, sy0, sy1;
      const float axa = P.axh + P.axl, aya = P.ayh + P.ayl;
      shift_range(axa + P.xmin, axa + P.xmax, -0.5f, (float)F.W - 0.5f, (float)F.W, F.wrap != 0, sx0, sx1);
      shift_range(aya + P.ymin, aya + P.ymax, -0.5f, (float)F.H - 0.5f, (float)F.H, F.wrap != 0, sy0, sy1);
      const float Kn = 6.0f * F.K;
      sx1 = min(sx1, sx0 + 63);
      sy1 = min(sy1, sy0 + 63);
      for (int sy = sy0; sy <= sy1; ++sy)
        for (int sx = sx0; sx <= sx1; ++sx) {
          const int shx = sx * F.W, shy = sy * F.H;
          const float ax = axa + (float)shx, ay = aya + (float)shy;
#pragma unroll
          for (int s = 0; s < 6; ++s) {
            if (tet_degenerate(L, snap, cube, s)) continue;  // zero volume: contributes nothing
            const int c0 = tet_corner(s, 0), c1 = tet_corner(s, 1), c2 = tet_corner(s, 2), c3 = tet_corner(s, 3);
            TetRaster t;
            if (!tet_setup<false>(P.x[c0], P.y[c0], P.x[c1], P.y[c1], P.x[c2], P.y[c2], P.x[c3], P.y[c3], 0.f, 0.f,
                                  0.f, 0.f, Kn, 0.f, 0.f, t))
              continue;
            const int qx0 = max(0, (int)ceilf(ax + t.xmin - 1e-3f)), qx1 = min(F.W - 1, (int)floorf(ax + t.xmax + 1e-3f));
            const int qy0 = max(0, (int)ceilf(ay + t.ymin - 1e-3f)), qy1 = min(F.H - 1, (int)floorf(ay + t.ymax + 1e-3f));
            if (qx0 > qx1 || qy0 > qy1) continue;
            Moments m;
#pragma unroll
            for (int e = 0; e < 4; ++e) m.g0[e] = m.gx[e] = m.gy[e] = 0.f;
            for (int py = qy0; py <= qy1; ++py) {
              const float Y = rel_coord(py, shy, P.ayh, P.ayl);
              float erow[4];
#pragma unroll
              for (int e = 0; e < 4; ++e) erow[e] = fmaf(t.b[e], Y, t.c[e]);
              float lo, hi;
              row_span(t, erow, lo, hi);
              const int xa = max(qx0, (int)ceilf(fmaxf(lo + ax, -1.0e9f)));
              const int xb = min(qx1, (int)floorf(fminf(hi + ax, 1.0e9f)));
              for (int px = xa; px <= xb; ++px) {
                const float X = rel_coord(px, shx, P.axh, P.axl);
                float v[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) v[e] = fmaf(t.a[e], X, erow[e]);
                int am = 0;
                float mn = v[0];
#pragma unroll
                for (int e = 1; e < 4; ++e)
                  if (v[e] < mn) { mn = v[e]; am = e; }
                if (!(mn > 0.0f)) continue;
                const float g = __ldg(gimg + (long long)py * F.W + px);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                  const float w = (am == e) ? g : 0.f;
                  m.g0[e] += w;
                  m.gx[e] = fmaf(w, X, m.gx[e]);
                  m.gy[e] = fmaf(w, Y, m.gy[e]);
                }
              }
            }
            TetCanon K;
            if (!tet_canon(P.x[c0], P.y[c0], P.x[c1], P.y[c1], P.x[c2], P.y[c2], P.x[c3], P.y[c3], 0.f, 0.f, 0.f,
                           0.f, K))
              continue;
            const float tiny = K.S * K.S * 1e-12f;
            float gx[4] = {0.f, 0.f, 0.f, 0.f}, gy[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int e = 0; e < 4; ++e) edge_grad(K, e, Kn, tiny, m, gx, gy);
            // canonical position -> table slot -> cube corner
            const int cs[4] = {c0, c1, c2, c3};
#pragma unroll
            for (int v = 0; v < 4; ++v) {
              const int slot = K.perm[v];
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                if (slot == q) {
#pragma unroll
                  for (int n = 0; n < 8; ++n)
                    if (n == cs[q]) { gpx[n] += gx[v]; gpy[n] += gy[v]; }
                }
              }
            }
          }
        }
      // pixel -> world: x_pix = (r . P) sx + const, y_pix = (u . P) sy + const; the
      // edge functions are in fixed-point accumulator units, converted by F.unit
      const float unit = (float)F.unit;
#pragma unroll
      for (int n = 0; n < 8; ++n)
#pragma unroll
        for (int q = 0; q < 3; ++q) G[n][q] += (gpx[n] * F.sx * F.r[q] + gpy[n] * F.sy * F.u[q]) * unit;
    }
    float* out = corner_grad + ((long long)snap * ncube + cube) * 24;
#pragma unroll
    for (int n = 0; n < 8; ++n)
#pragma unroll
      for (int q = 0; q < 3; ++q) out[n * 3 + q] = G[n][q];
  }
}

// dL/d(particle) = sum over the 8 cubes sharing the particle as corner n.
__global__ void k_gather(Lattice L, const float* __restrict__ corner_grad, float* __restrict__ dLdpos) {
  const long long np = L.n_particles;
  const int snap = blockIdx.y;
  const int N = L.N;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(p % N), j = (int)((p / N) % N), k = (int)(p / ((long long)N * N));
    float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      const int a = n & 1, b = (n >> 1) & 1, c = (n >> 2) & 1;
      const int ci = (i - a + N) % N, cj = (j - b + N) % N, ck = (k - c + N) % N;
      const long long cube = particle_id(ci, cj, ck, N);
      const float* g = corner_grad + ((long long)snap * np + cube) * 24 + n * 3;
      gx += g[0];
      gy += g[1];
      gz += g[2];
    }
    float* o = dLdpos + ((long long)snap * np + p) * 3;
    o[0] = gx;
    o[1] = gy;
    o[2] = gz;
  }
}

cudaError_t launch_backward(const Lattice& L, const FrameDev* d_frames, long long stride, int n_frames, int n_snap,
                            const float* dLdI, float* corner_grad, cudaStream_t s) {
  long long b = (L.n_particles + 127) / 128;
  if (b > 8192) b = 8192;
  dim3 grid((unsigned)(b < 1 ? 1 : b), n_snap);
  k_backward<<<grid, 128, 0, s>>>(L, d_frames, n_frames, stride, dLdI, corner_grad);
  return cudaGetLastError();
}

cudaError_t launch_gather_grad(const Lattice& L, int n_snap, const float* corner_grad, float* dLdpos,
                               cudaStream_t s) {
  long long b = (L.n_particles + 255) / 256;
  if (b > 8192) b = 8192;
  dim3 grid((unsigned)(b < 1 ? 1 : b), n_snap);
  k_gather<<<grid, 256, 0, s>>>(L, corner_grad, dLdpos);
  return cudaGetLastError();
}

}  // namespace lt
