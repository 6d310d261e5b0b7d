// lt_area.cu -- area-averaged pixels of an orthographic view: each pixel holds
// the mean of the column density of Eq. 6 over its square, instead of the
// value at its centre.
//
// In an orthographic view the chord of one tetrahedron is a continuous,
// piecewise-linear function of the image point: zero on the boundary of the
// projected hull and linear on each triangle that joins the apex to a hull
// edge. The apex is the projected vertex lying inside the triangle of the
// other three, or for a four-vertex hull the crossing of its diagonals. The
// pyramid the chord forms over the hull holds the tetrahedron's volume, so
// rho times the chord at the apex is 3 m / A, with A the hull's area. On the
// triangle of hull edge e the column density is k_e d_e(p), where d_e is that
// edge's line function. Its integral over a pixel is then
// k_e (a_e Mx + b_e My + c_e |P|), where |P|, Mx and My are the area and
// first moments of the triangle clipped to the pixel's square.
//
// Each warp takes 32 tetrahedra (one per lane). In FP64 a lane projects the
// vertices to pixel units, finds the apex and the hull, and forms the lines of
// the hull edges and of the rays from the apex through the hull vertices. The
// lines are relative to the apex's pixel, normalised to |a| + |b| = 1, and
// kept as float-float pairs. Then the warp walks the bounding rectangles one
// tetrahedron at a time, 32 pixels per pass. Each lane evaluates the lines at
// its pixel's corner in float-float arithmetic (error-free products and sums;
// GB300's FP64 pipe is narrow), so a line's offset there carries only its own
// rounding, however far the pixel lies from the apex. The lane clips the
// square against each triangle and sums the integrals. That step runs in FP32,
// or in FP64 for hulls thinner than kThinHull pixels and for apexes within
// kThinSector pixels of a hull edge: there FP32 rounding of the clip would
// show next to the pixel's own small value. The sums are 64-bit
// fixed-point integers added by global atomics, so the image is bitwise
// reproducible. A second kernel converts them to float.
#include "lt_internal.h"

namespace lt {

namespace {

constexpr double kThinHull = 0.05;     // pixels: hull width below which the clip runs in FP64
constexpr double kThinSector = 1e-3;  // pixels: apex distance to a hull edge below which it does too
constexpr int kAreaThreads = 128;

struct AreaArgs {
  Lattice L;
  const FrameDev* frame;
  double m_tet, inv_unit;
  unsigned long long* acc;  // [H][W]
  DevCounters* ctr;
};

// One tetrahedron's pyramid, lines relative to the anchor pixel (ax, ay).
struct AreaTet {
  float2 hull[4][3];  // hull edge e (from vertex e to e + 1): a x + b y + c >= 0 inside; (hi, lo) pairs
  float2 ray[4][3];   // ray from the apex through hull vertex e: >= 0 on the side of edge e
  float k[4];         // column density per unit of hull line e, in accumulator units
  int n, ax, ay, thin;
  int x0, x1, y0, y1;
};

__device__ __forceinline__ double orient(double ax, double ay, double bx, double by, double cx, double cy) {
  return (bx - ax) * (cy - ay) - (by - ay) * (cx - ax);
}

__device__ __forceinline__ float2 split_ff(double x) {
  const float hi = (float)x;
  return make_float2(hi, (float)(x - (double)hi));
}

__device__ __forceinline__ double join_ff(float2 v) { return (double)v.x + (double)v.y; }

// Line through (px, py) with direction (dx, dy), positive on its left.
__device__ __forceinline__ void make_line(double px, double py, double dx, double dy, float2* l) {
  const double a = -dy, b = dx, s = fabs(a) + fabs(b);
  const double inv = s > 0.0 ? 1.0 / s : 0.0;
  l[0] = split_ff(a * inv);
  l[1] = split_ff(b * inv);
  l[2] = split_ff((dy * px - dx * py) * inv);
}

// a ox + b oy + c for float-float a, b, c and integer ox, oy (exact in FP32):
// error-free products and two-sums, then the small terms (Dekker, Knuth).
__device__ __forceinline__ float line_ff(const float2* l, float ox, float oy) {
  const float p1 = l[0].x * ox, e1 = fmaf(l[0].y, ox, fmaf(l[0].x, ox, -p1));
  const float p2 = l[1].x * oy, e2 = fmaf(l[1].y, oy, fmaf(l[1].x, oy, -p2));
  const float s = p1 + p2, sb = s - p1, es = (p1 - (s - sb)) + (p2 - sb);
  const float t = l[2].x + s, tb = t - l[2].x, et = (l[2].x - (t - tb)) + (s - tb);
  return t + (((et + es) + (e1 + e2)) + l[2].y);
}

__device__ __forceinline__ double line_f64(const float2* l, double ox, double oy) {
  return fma(join_ff(l[1]), oy, fma(join_ff(l[0]), ox, join_ff(l[2])));
}

// A thread's polygon buffer in shared memory: slot i of thread t at
// p[i * kAreaThreads + t], so that the threads of a warp fall on distinct
// banks whatever slots they touch.
struct SmemPoly {
  float* p;
  __device__ __forceinline__ float& operator[](int i) const { return p[i * kAreaThreads]; }
};

// Clip the convex polygon (xi, yi)[n] to a x + b y + c >= 0 (Sutherland-Hodgman).
template <typename T, typename Buf>
__device__ __forceinline__ int clip_poly(Buf xi, Buf yi, int n, T a, T b, T c, Buf xo, Buf yo) {
  int m = 0;
  T dp = c + a * xi[n - 1] + b * yi[n - 1];
  int j = n - 1;
  for (int i = 0; i < n; ++i) {
    const T d = c + a * xi[i] + b * yi[i];
    if ((d >= T(0)) != (dp >= T(0))) {
      const T t = dp / (dp - d);
      xo[m] = xi[j] + t * (xi[i] - xi[j]);
      yo[m] = yi[j] + t * (yi[i] - yi[j]);
      ++m;
    }
    if (d >= T(0)) {
      xo[m] = xi[i];
      yo[m] = yi[i];
      ++m;
    }
    dp = d;
    j = i;
  }
  return m;
}

// Integral over the unit square of the hull line function l0 = (a0, b0, c0),
// restricted to l0 >= 0, l1 >= 0 and l2 >= 0; xa, ya, xb, yb hold 8 vertices each.
template <typename T, typename Buf>
__device__ T sector_integral(T a0, T b0, T c0, T a1, T b1, T c1, T a2, T b2, T c2, Buf xa, Buf ya, Buf xb, Buf yb) {
  const T la[3] = {a0, a1, a2}, lb[3] = {b0, b1, b2}, lc[3] = {c0, c1, c2};
  bool inside[3];
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    // largest and smallest value over the square's corners
    const T hi = lc[l] + (la[l] > T(0) ? la[l] : T(0)) + (lb[l] > T(0) ? lb[l] : T(0));
    const T lo = lc[l] + (la[l] < T(0) ? la[l] : T(0)) + (lb[l] < T(0) ? lb[l] : T(0));
    if (hi <= T(0)) return T(0);
    inside[l] = lo >= T(0);
  }
  if (inside[0] && inside[1] && inside[2]) return T(0.5) * (a0 + b0) + c0;
  xa[0] = T(0); xa[1] = T(1); xa[2] = T(1); xa[3] = T(0);
  ya[0] = T(0); ya[1] = T(0); ya[2] = T(1); ya[3] = T(1);
  int n = 4;
  bool in_a = true;
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    if (inside[l]) continue;
    if (in_a) n = clip_poly(xa, ya, n, la[l], lb[l], lc[l], xb, yb);
    else n = clip_poly(xb, yb, n, la[l], lb[l], lc[l], xa, ya);
    in_a = !in_a;
    if (n < 3) return T(0);
  }
  const Buf x = in_a ? xa : xb;
  const Buf y = in_a ? ya : yb;
  // twice the area and six times the first moments, relative to vertex 0 (a
  // fan of triangles), so that a thin piece keeps its relative accuracy (the
  // square is counter-clockwise; clipping keeps it)
  T A = T(0), Mx = T(0), My = T(0);
  for (int i = 1; i + 1 < n; ++i) {
    const T ux = x[i] - x[0], uy = y[i] - y[0], vx = x[i + 1] - x[0], vy = y[i + 1] - y[0];
    const T cr = ux * vy - vx * uy;
    A += cr;
    Mx += (ux + vx) * cr;
    My += (uy + vy) * cr;
  }
  // the line's integral: its value at vertex 0 times the area plus the moments
  const T d0 = c0 + a0 * x[0] + b0 * y[0];
  const T v = d0 * (A / T(2)) + a0 * (Mx / T(6)) + b0 * (My / T(6));
  return v > T(0) ? v : T(0);
}

// Mean column density over pixel (ox, oy) (offsets from the anchor) of one
// tetrahedron, in accumulator units: the lines at the pixel's corner to about
// 2^-44 relative, the clip in T.
template <typename T, typename Buf>
__device__ __forceinline__ float pixel_mean(const AreaTet& t, int ox, int oy, Buf xa, Buf ya, Buf xb, Buf yb) {
  T ha[4], hb[4], hc[4], ra[4], rb[4], rc[4];
  // the hull lines first: a square outside one of them gets nothing
  bool outside = false;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    if (sizeof(T) == 4) {
      ha[e] = (T)t.hull[e][0].x;
      hb[e] = (T)t.hull[e][1].x;
      hc[e] = (T)line_ff(t.hull[e], (float)ox, (float)oy);
    } else {
      ha[e] = (T)join_ff(t.hull[e][0]);
      hb[e] = (T)join_ff(t.hull[e][1]);
      hc[e] = (T)line_f64(t.hull[e], (double)ox, (double)oy);
    }
    const T hi = hc[e] + (ha[e] > T(0) ? ha[e] : T(0)) + (hb[e] > T(0) ? hb[e] : T(0));
    outside = outside || (e < t.n && hi <= T(0));
  }
  if (outside) return 0.0;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    if (sizeof(T) == 4) {
      ra[e] = (T)t.ray[e][0].x;
      rb[e] = (T)t.ray[e][1].x;
      rc[e] = (T)line_ff(t.ray[e], (float)ox, (float)oy);
    } else {
      ra[e] = (T)join_ff(t.ray[e][0]);
      rb[e] = (T)join_ff(t.ray[e][1]);
      rc[e] = (T)line_f64(t.ray[e], (double)ox, (double)oy);
    }
  }
  T v = T(0);
  for (int e = 0; e < t.n; ++e) {
    const int f = e + 1 == t.n ? 0 : e + 1;
    const T s = sector_integral<T, Buf>(ha[e], hb[e], hc[e], ra[e], rb[e], rc[e], -ra[f], -rb[f], -rc[f], xa, ya, xb, yb);
    v += (T)t.k[e] * s;
  }
  return (float)v;
}

// The FP64 clip of thin hulls, out of line (rare: it keeps the hot loop small).
__device__ __noinline__ float pixel_mean_f64(const AreaTet& t, int ox, int oy) {
  double xa[8], ya[8], xb[8], yb[8];
  return pixel_mean<double, double*>(t, ox, oy, xa, ya, xb, yb);
}

// FP64 setup of the lane's tetrahedron; false when it covers no area.
__device__ bool setup_tet(const AreaArgs& a, const FrameDev& F, long long tau, AreaTet& t) {
  const long long cube = tau / 6;
  const int s = (int)(tau - 6 * cube);
  if (tet_degenerate(a.L, F.snapshot, cube, s)) return false;
  int i, j, k;
  cube_ijk(a.L, cube, i, j, k);
  bool ok = true;
  TetF64 tf;
  tet_f64(a.L, (long long)F.snapshot * a.L.n_particles, i, j, k, s, ok, tf);
  if (!ok || tf.V == 0.0) return false;
  const double hl = (double)a.L.box / a.L.N;
  const double base[3] = {i * hl, j * hl, k * hl};
  double P[4][2];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    double w[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) w[q] = base[q] + tf.v[c][q];
    P[c][0] = (F.rd[0] * w[0] + F.rd[1] * w[1] + F.rd[2] * w[2] - F.lod[0]) / F.pxd[0];
    P[c][1] = (F.ud[0] * w[0] + F.ud[1] * w[1] + F.ud[2] * w[2] - F.lod[1]) / F.pxd[1];
  }
  // the apex and the hull, counter-clockwise: a vertex inside the triangle of
  // the other three is the apex
  double Ax = 0.0, Ay = 0.0, Hx[4], Hy[4];
  int n = 0;
  int inner = -1;
  for (int c = 0; c < 4 && inner < 0; ++c) {
    const int p = (c + 1) & 3, q = (c + 2) & 3, r = (c + 3) & 3;
    const double o = orient(P[p][0], P[p][1], P[q][0], P[q][1], P[r][0], P[r][1]);
    if (o == 0.0) continue;
    const double s1 = orient(P[p][0], P[p][1], P[q][0], P[q][1], P[c][0], P[c][1]) * o;
    const double s2 = orient(P[q][0], P[q][1], P[r][0], P[r][1], P[c][0], P[c][1]) * o;
    const double s3 = orient(P[r][0], P[r][1], P[p][0], P[p][1], P[c][0], P[c][1]) * o;
    // on the boundary counts too: coincident projections (the undeformed
    // lattice seen along an axis) put the apex on a hull vertex or edge,
    // where the triangles beside it have no area
    if (s1 >= 0.0 && s2 >= 0.0 && s3 >= 0.0) {
      inner = c;
      Ax = P[c][0];
      Ay = P[c][1];
      const bool ccw = o > 0.0;
      const int ord[3] = {p, ccw ? q : r, ccw ? r : q};
      for (int e = 0; e < 3; ++e) {
        Hx[e] = P[ord[e]][0];
        Hy[e] = P[ord[e]][1];
      }
      n = 3;
    }
  }
  if (inner < 0) {
    // four vertices in convex position: vertex 0's diagonal partner d is the
    // one whose segment from vertex 0 separates the other two
    int d = -1, u = -1, w = -1;
    for (int c = 1; c < 4 && d < 0; ++c) {
      const int p = c == 1 ? 2 : 1, q = 6 - c - p;
      const double sp = orient(P[0][0], P[0][1], P[c][0], P[c][1], P[p][0], P[p][1]);
      const double sq = orient(P[0][0], P[0][1], P[c][0], P[c][1], P[q][0], P[q][1]);
      if ((sp > 0.0 && sq < 0.0) || (sp < 0.0 && sq > 0.0)) {
        d = c;
        // counter-clockwise: 0, u, d, w with u on the right of 0 -> d
        u = sp < 0.0 ? p : q;
        w = sp < 0.0 ? q : p;
      }
    }
    if (d < 0) return false;
    const double o0 = orient(P[u][0], P[u][1], P[w][0], P[w][1], P[0][0], P[0][1]);
    const double od = orient(P[u][0], P[u][1], P[w][0], P[w][1], P[d][0], P[d][1]);
    if (!((o0 > 0.0 && od < 0.0) || (o0 < 0.0 && od > 0.0))) return false;  // not a crossing
    const double tt = o0 / (o0 - od);
    Ax = P[0][0] + tt * (P[d][0] - P[0][0]);
    Ay = P[0][1] + tt * (P[d][1] - P[0][1]);
    const int ord[4] = {0, u, d, w};
    for (int e = 0; e < 4; ++e) {
      Hx[e] = P[ord[e]][0];
      Hy[e] = P[ord[e]][1];
    }
    n = 4;
  }
  double area2 = 0.0, emax = 0.0;
  for (int e = 0; e < n; ++e) {
    const int f = e + 1 == n ? 0 : e + 1;
    area2 += Hx[e] * Hy[f] - Hx[f] * Hy[e];
    emax = fmax(emax, hypot(Hx[f] - Hx[e], Hy[f] - Hy[e]));
  }
  if (!(area2 > 0.0)) return false;
  // column density at the apex: 3 m / (hull area in world units)
  const double h = 3.0 * a.m_tet / (0.5 * area2 * F.pxd[0] * F.pxd[1]);
  t.ax = (int)fmin(fmax(floor(Ax), -1.0e9), 1.0e9);
  t.ay = (int)fmin(fmax(floor(Ay), -1.0e9), 1.0e9);
  const double qx = Ax - t.ax, qy = Ay - t.ay;
  double xmn = Hx[0], xmx = Hx[0], ymn = Hy[0], ymx = Hy[0];
  bool thin_sector = false;
  for (int e = 0; e < n; ++e) {
    const int f = e + 1 == n ? 0 : e + 1;
    make_line(Hx[e] - t.ax, Hy[e] - t.ay, Hx[f] - Hx[e], Hy[f] - Hy[e], t.hull[e]);
    make_line(qx, qy, Hx[e] - Ax, Hy[e] - Ay, t.ray[e]);
    const double dA = join_ff(t.hull[e][0]) * qx + join_ff(t.hull[e][1]) * qy + join_ff(t.hull[e][2]);
    t.k[e] = dA > 0.0 ? (float)(h / dA * a.inv_unit) : 0.0f;
    // an apex next to a hull edge: a long thin face whose FP32 clip would lose
    // its relative accuracy while k_e grows as 1 / dA
    thin_sector = thin_sector || (dA > 0.0 && dA < kThinSector);
    xmn = fmin(xmn, Hx[e]); xmx = fmax(xmx, Hx[e]);
    ymn = fmin(ymn, Hy[e]); ymx = fmax(ymx, Hy[e]);
  }
  for (int e = n; e < 4; ++e) {
    for (int q = 0; q < 3; ++q) t.hull[e][q] = t.ray[e][q] = make_float2(0.f, 0.f);
    t.k[e] = 0.0f;
  }
  t.n = n;
  t.thin = 0.5 * area2 < kThinHull * emax || thin_sector;
  int x0 = (int)fmax(floor(xmn), -2.0e9), x1 = (int)fmin(floor(xmx), 2.0e9);
  int y0 = (int)fmax(floor(ymn), -2.0e9), y1 = (int)fmin(floor(ymx), 2.0e9);
  if (!F.wrap) {
    x0 = max(x0, 0); x1 = min(x1, F.W - 1);
    y0 = max(y0, 0); y1 = min(y1, F.H - 1);
  } else {
    // at most a few periods per axis (a tetrahedron spans less than one)
    x1 = min(x1, x0 + 4 * F.W);
    y1 = min(y1, y0 + 4 * F.H);
  }
  t.x0 = x0; t.x1 = x1; t.y0 = y0; t.y1 = y1;
  if (x0 > x1 || y0 > y1) return false;
  if ((long long)(x1 - x0 + 1) * (y1 - y0 + 1) > 0x7fffffffLL) {
    // more than 2^31 pixels (a window zoomed far into one tetrahedron): the
    // walk's 32-bit pixel index cannot hold it
    atomicOr(&a.ctr->errors, kErrRange);
    return false;
  }
  return true;
}

__global__ void __launch_bounds__(kAreaThreads) k_area(AreaArgs a) {
  __shared__ AreaTet tets[kAreaThreads];
  __shared__ float poly[4 * 8 * kAreaThreads];  // the FP32 clip's vertex buffers
  const SmemPoly pxa{poly + threadIdx.x}, pya{poly + 8 * kAreaThreads + threadIdx.x};
  const SmemPoly pxb{poly + 16 * kAreaThreads + threadIdx.x}, pyb{poly + 24 * kAreaThreads + threadIdx.x};
  const FrameDev& F = *a.frame;
  const int W = F.W, H = F.H;
  const long long ntet = 6LL * a.L.n_particles;
  const int lane = threadIdx.x & 31;
  AreaTet* wt = tets + (threadIdx.x & ~31);
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  const long long wid = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  for (long long base = wid * 32; base < ntet; base += warps * 32) {
    const long long tau = base + lane;
    const bool live = tau < ntet && setup_tet(a, F, tau, wt[lane]);
    unsigned todo = __ballot_sync(0xffffffffu, live);
    __syncwarp();
    while (todo) {
      const int src = __ffs(todo) - 1;
      todo &= todo - 1u;
      const AreaTet& t = wt[src];
      const int wx = t.x1 - t.x0 + 1;
      const int np = wx * (t.y1 - t.y0 + 1);
      if (lane == 0) {
        atomicAdd(&a.ctr->area_pairs, (unsigned long long)np);
        if (t.thin) atomicAdd(&a.ctr->area_fp64_pairs, (unsigned long long)np);
      }
      for (int p = lane; p < np; p += 32) {
        const int ry = p / wx;
        const int px = t.x0 + (p - ry * wx), py = t.y0 + ry;
        const int ox = px - t.ax, oy = py - t.ay;
        const float v = t.thin ? pixel_mean_f64(t, ox, oy) : pixel_mean<float, SmemPoly>(t, ox, oy, pxa, pya, pxb, pyb);
        const int pxw = F.wrap ? ((px % W) + W) % W : px, pyw = F.wrap ? ((py % H) + H) % H : py;
        if (!LT_IN_BOUNDS(pxw >= 0 && pxw < W && pyw >= 0 && pyw < H, &a.ctr->errors)) continue;
        accum_fixed(a.acc + ((long long)pyw * W + pxw), v, a.ctr);
      }
    }
    __syncwarp();
  }
}

}  // namespace

cudaError_t launch_area(const Lattice& L, const FrameDev* d_frame, int W, int H, double m_tet, double unit,
                        unsigned long long* d_acc, float* d_out, DevCounters* ctr, cudaStream_t s) {
  const long long np = (long long)W * H;
  cudaError_t e = cudaMemsetAsync(d_acc, 0, sizeof(unsigned long long) * np, s);
  if (e != cudaSuccess) return e;
  AreaArgs a;
  a.L = L;
  a.frame = d_frame;
  a.m_tet = m_tet;
  a.inv_unit = 1.0 / unit;
  a.acc = d_acc;
  a.ctr = ctr;
  long long blocks = (6LL * L.n_particles + kAreaThreads - 1) / kAreaThreads;
  if (blocks > 152LL * 16) blocks = 152LL * 16;
  k_area<<<(unsigned)(blocks < 1 ? 1 : blocks), kAreaThreads, 0, s>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_fixed_finalize(d_acc, np, unit, false, d_out, s);
}

}  // namespace lt
