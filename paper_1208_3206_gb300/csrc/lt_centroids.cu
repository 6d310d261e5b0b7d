// lt_centroids.cu -- the centroid rendering of Sec. 4.2: every tetrahedron
// drawn as a 2D kernel in the image plane at its centroid (its centre of
// mass), scaled with (m / rho)^(1/3) = |V|^(1/3), carrying its mass.
//
// The paper names a cubic-spline kernel and leaves its form and the scale
// factor open. This takes the 2D M4 cubic spline with unit integral and
// smoothing length h = |V|^(1/3):
//   W(r, h) = 10 / (7 pi h^2) w(r / h),
//   w(q) = 1 - 3/2 q^2 + 3/4 q^3 (q < 1), (2 - q)^3 / 4 (1 <= q < 2), 0 else,
// so a pixel holds an estimate of the column density. The billboards face
// the view direction: a perspective ray picks one up over the cosine of its
// angle to that direction. A periodic orthographic window draws every
// periodic copy. With the frame's near radius set (hybrid rendering) only
// the far cubes are drawn.
//
// Each warp takes 32 tetrahedra (one per lane): in FP64, the lane forms the
// vertices (relative to the cube's Lagrangian corner), the volume, the
// centroid projected to pixel coordinates and the splat's pixel rectangle.
// Then, tetrahedron by tetrahedron, the warp's lanes walk the rectangle 32
// pixels at a time and evaluate the spline in FP32 relative to the centroid's
// fractional pixel position, adding m W as a 64-bit fixed-point integer with
// a global atomic (order-independent sums: the image is bitwise
// reproducible). A second kernel converts the sums to float.
#include "lt_internal.h"

namespace lt {

struct CentroidArgs {
  Lattice L;
  const FrameDev* frame;
  double m_tet, inv_unit;
  unsigned long long* acc;  // [H][W]
  DevCounters* ctr;
};

__global__ void __launch_bounds__(128) k_centroids(CentroidArgs a) {
  const FrameDev& F = *a.frame;
  const int N = a.L.N, W = F.W, H = F.H;
  const double h_lat = (double)a.L.box / N;
  const long long soff = (long long)F.snapshot * a.L.n_particles;
  const long long ntet = 6LL * a.L.n_particles;
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  const long long wid = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const bool wrap = F.wrap != 0;
  for (long long base = wid * 32; base < ntet; base += warps * 32) {
    // ---- one tetrahedron per lane: its splat in pixel units
    const long long tau = base + lane;
    bool live = false;
    double cx = 0.0, cy = 0.0;   // centroid in pixel coordinates (pixel p has its centre at p)
    float sxh = 0.f, syh = 0.f;  // pixel width and height over h
    float norm = 0.f;            // m W(0) / w(0), accumulator units
    int x0 = 0, x1 = -1, y0 = 0, y1 = -1;
    if (tau < ntet) {
      const long long cube = tau / 6;
      const int s = (int)(tau - 6 * cube);
      // hybrid rendering: the near cubes are drawn by the exact projection
      const bool skip = F.near_r2 > 0.0 && !cube_far(a.L, F, cube);
      if (!skip && !tet_degenerate(a.L, F.snapshot, cube, s)) {
        int i, j, k;
        cube_ijk(a.L, cube, i, j, k);
        bool ok = true;
        TetF64 t;
        tet_f64(a.L, soff, i, j, k, s, ok, t);
        if (ok && t.V != 0.0) {
          double c[3];
#pragma unroll
          for (int q = 0; q < 3; ++q) c[q] = 0.25 * (t.v[0][q] + t.v[1][q] + t.v[2][q] + t.v[3][q]);
          c[0] += i * h_lat;
          c[1] += j * h_lat;
          c[2] += k * h_lat;
          const double h = cbrt(fabs(t.V));
          // pixel sizes (at the billboard) in the units of h
          double pw, ph;
          bool front = true;
          if (!F.persp) {
            const double wa = F.rd[0] * c[0] + F.rd[1] * c[1] + F.rd[2] * c[2];
            const double wb = F.ud[0] * c[0] + F.ud[1] * c[1] + F.ud[2] * c[2];
            cx = (wa - F.lod[0]) / F.pxd[0] - 0.5;
            cy = (wb - F.lod[1]) / F.pxd[1] - 0.5;
            pw = F.pxd[0];
            ph = F.pxd[1];
          } else {
            // camera coordinates of the centroid; the ray of the pixel at
            // tan (xt, yt) meets the billboard at Z (xt, yt) - (X, Y)
            const double e[3] = {c[0] - F.eyed[0], c[1] - F.eyed[1], c[2] - F.eyed[2]};
            const double Z = F.fd[0] * e[0] + F.fd[1] * e[1] + F.fd[2] * e[2];
            const double X = F.rd[0] * e[0] + F.rd[1] * e[1] + F.rd[2] * e[2];
            const double Y = F.ud[0] * e[0] + F.ud[1] * e[1] + F.ud[2] * e[2];
            front = Z > 0.0;
            const double ptx = 2.0 * F.tand[0] / W, pty = 2.0 * F.tand[1] / H;  // pixel size in tan units
            cx = front ? (X / Z / F.tand[0] + 1.0) * 0.5 * W - 0.5 : 0.0;
            cy = front ? (Y / Z / F.tand[1] + 1.0) * 0.5 * H - 0.5 : 0.0;
            pw = Z * ptx;
            ph = Z * pty;
          }
          const double rx = 2.0 * h / pw, ry = 2.0 * h / ph;  // support radius in pixels
          x0 = (int)fmax(ceil(cx - rx), -2.0e9);
          x1 = (int)fmin(floor(cx + rx), 2.0e9);
          y0 = (int)fmax(ceil(cy - ry), -2.0e9);
          y1 = (int)fmin(floor(cy + ry), 2.0e9);
          if (!wrap) {
            x0 = max(x0, 0); x1 = min(x1, W - 1);
            y0 = max(y0, 0); y1 = min(y1, H - 1);
          } else {
            // at most one period of pixels per axis (a splat wider than the
            // window covers each pixel once per copy it reaches)
            x1 = min(x1, x0 + 4 * W);
            y1 = min(y1, y0 + 4 * H);
          }
          sxh = (float)(pw / h);
          syh = (float)(ph / h);
          norm = (float)(a.m_tet * 10.0 / (7.0 * M_PI * h * h) * a.inv_unit);
          live = front && x0 <= x1 && y0 <= y1;
          if (live && (long long)(x1 - x0 + 1) * (y1 - y0 + 1) > 0x7fffffffLL) {
            // more than 2^31 pixels (a window zoomed far into one splat): the
            // walk's 32-bit pixel index cannot hold it
            atomicOr(&a.ctr->errors, kErrRange);
            live = false;
          }
        }
      }
    }
    // ---- tetrahedron by tetrahedron, the warp walks the splat's rectangle
    unsigned todo = __ballot_sync(0xffffffffu, live);
    while (todo) {
      const int src = __ffs(todo) - 1;
      todo &= todo - 1u;
      const double tcx = __shfl_sync(0xffffffffu, cx, src), tcy = __shfl_sync(0xffffffffu, cy, src);
      const float tsx = __shfl_sync(0xffffffffu, sxh, src), tsy = __shfl_sync(0xffffffffu, syh, src);
      const float tn = __shfl_sync(0xffffffffu, norm, src);
      const int tx0 = __shfl_sync(0xffffffffu, x0, src), tx1 = __shfl_sync(0xffffffffu, x1, src);
      const int ty0 = __shfl_sync(0xffffffffu, y0, src), ty1 = __shfl_sync(0xffffffffu, y1, src);
      // the centroid as an integer pixel plus a fraction, so that offsets are exact
      const double bx = floor(tcx), by = floor(tcy);
      const float fx = (float)(tcx - bx), fy = (float)(tcy - by);
      const int ibx = (int)bx, iby = (int)by;
      const int wx = tx1 - tx0 + 1;
      const int np = wx * (ty1 - ty0 + 1);
      for (int p = lane; p < np; p += 32) {
        const int ry = p / wx;
        const int px = tx0 + (p - ry * wx), py = ty0 + ry;
        const float dx = ((float)(px - ibx) - fx) * tsx, dy = ((float)(py - iby) - fy) * tsy;
        const float q = sqrtf(dx * dx + dy * dy);
        if (!(q < 2.0f)) continue;
        const float w = q < 1.0f ? fmaf(q * q, fmaf(0.75f, q, -1.5f), 1.0f) : 0.25f * (2.0f - q) * (2.0f - q) * (2.0f - q);
        float v = tn * w;
        if (F.persp) {
          // the ray crosses the billboard at an angle: over the cosine, |(xt, yt, 1)|
          const float xt = F.tan_x * (2.0f * ((float)px + 0.5f) / (float)W - 1.0f);
          const float yt = F.tan_y * (2.0f * ((float)py + 0.5f) / (float)H - 1.0f);
          v *= sqrtf(1.0f + xt * xt + yt * yt);
        }
        const int pxw = wrap ? ((px % W) + W) % W : px, pyw = wrap ? ((py % H) + H) % H : py;
        if (!LT_IN_BOUNDS(pxw >= 0 && pxw < W && pyw >= 0 && pyw < H, &a.ctr->errors)) continue;
        unsigned long long* cell = a.acc + ((long long)pyw * W + pxw);
        if (v < 4294967040.0f) {
          const unsigned long long add = (unsigned long long)__float2uint_rn(v);
          if (add) {
            const unsigned long long old = atomicAdd(cell, add);
            if (old > ~0ull - add) {
              atomicOr(&a.ctr->errors, kErrRange);
              atomicAdd(&a.ctr->range_overflow, 1ull);
            }
          }
        } else if (v < 9223372036854775808.0f) {
          const unsigned long long add = __float2ull_rn(v);
          const unsigned long long old = atomicAdd(cell, add);
          if (old > ~0ull - add) {
            atomicOr(&a.ctr->errors, kErrRange);
            atomicAdd(&a.ctr->range_overflow, 1ull);
          }
        } else {
          atomicOr(&a.ctr->errors, kErrRange);
          atomicAdd(&a.ctr->range_overflow, 1ull);
        }
      }
    }
  }
}

__global__ void k_centroids_finalize(const unsigned long long* __restrict__ acc, long long np, double unit, bool add,
                                     float* __restrict__ out) {
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (long long)gridDim.x * blockDim.x) {
    const float v = (float)((double)acc[p] * unit);
    out[p] = add ? out[p] + v : v;
  }
}

cudaError_t launch_centroids(const Lattice& L, const FrameDev* d_frame, int W, int H, double m_tet, double unit,
                             unsigned long long* d_acc, float* d_out, bool add, DevCounters* ctr, cudaStream_t s) {
  const long long np = (long long)W * H;
  cudaError_t e = cudaMemsetAsync(d_acc, 0, sizeof(unsigned long long) * np, s);
  if (e != cudaSuccess) return e;
  CentroidArgs a;
  a.L = L;
  a.frame = d_frame;
  a.m_tet = m_tet;
  a.inv_unit = 1.0 / unit;
  a.acc = d_acc;
  a.ctr = ctr;
  long long blocks = (6LL * L.n_particles + 127) / 128;
  if (blocks > 152LL * 32) blocks = 152LL * 32;
  k_centroids<<<(unsigned)(blocks < 1 ? 1 : blocks), 128, 0, s>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_fixed_finalize(d_acc, np, unit, add, d_out, s);
}

cudaError_t launch_fixed_finalize(const unsigned long long* d_acc, long long np, double unit, bool add, float* d_out,
                                  cudaStream_t s) {
  long long fb = (np + 255) / 256;
  if (fb > 152LL * 32) fb = 152LL * 32;
  k_centroids_finalize<<<(unsigned)(fb < 1 ? 1 : fb), 256, 0, s>>>(d_acc, np, unit, add, d_out);
  return cudaGetLastError();
}

}  // namespace lt
