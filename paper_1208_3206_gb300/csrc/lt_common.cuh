// lt_common.cuh -- device-side building blocks shared by every kernel of the
// column-density renderer: lattice addressing, cube projection and the
// per-tetrahedron form of rho_t * dl_t used by the raster passes.
//
// The projection of Eq. 6 (Sec. 3.2) adds rho_t * dl_t(ray) for every
// tetrahedron t, rho_t = m / |V_t| (Eq. 3, 9). For a straight ray, dl_t is
// piecewise linear across the image and |V_t| cancels:
//
//  * Orthographic view. dl_t(x) / |V_t| is a pyramid over the convex hull of
//    the four projected vertices with unit integral: apex at the projected
//    vertex that lies inside the triangle of the other three, or at the
//    crossing of the two projected diagonals, apex height 3 / area(hull).
//    So rho_t * dl_t(x) = m * pyramid(x): only the projected vertex positions
//    enter. In pixel units the pyramid is min over hull edges (j,k) of
//        6 m * orient(v_j, v_k, x) / (orient(v_j, v_k, v_l1) * orient(v_j, v_k, v_l2)),
//    {l1, l2} the other two vertices (orient = 2D signed double area).
//  * Perspective view. Under (X, Y, Z) -> (X/Z, Y/Z, 1/Z) planes stay planes
//    and every ray becomes a line of constant image position, so the ray
//    parameter interval [1/w_hi, 1/w_lo] is the w-extent of the mapped
//    tetrahedron, whose volume is |V| / (Z0 Z1 Z2 Z3). Hence
//        rho_t * dl_t = m kx ky |d| pyramid'(x) / (Z0 Z1 Z2 Z3 * w_lo * w_hi),
//    pyramid' the same construction on the perspective-projected vertices,
//    |d| the length of the pixel's ray direction (x, y, 1). w_lo and w_hi
//    are the lower and upper depth surfaces of the mapped tetrahedron.
//
// Both are exact rewritings of rho * dl (no approximation); the volume is
// never divided by, which keeps sheet-like tetrahedra at caustics well
// conditioned in FP32. The form has a finite limit as V -> 0 (a sheet of the
// same mass), so tetrahedra with V == 0 exactly, which contribute nothing,
// are skipped explicitly through the build pass's zero-volume mask.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace lt {

// Connectivity of the six tetrahedra of a cube (Sec. 4.1); corner n of cube
// (i, j, k) is lattice point (i + (n & 1), j + ((n >> 1) & 1), k + ((n >> 2) & 1)).
__host__ __device__ constexpr int tet_corner(int s, int c) {
  return (s == 0) ? (c == 0 ? 1 : c == 1 ? 0 : c == 2 ? 2 : 4)
       : (s == 1) ? (c == 0 ? 3 : c == 1 ? 1 : c == 2 ? 2 : 4)
       : (s == 2) ? (c == 0 ? 3 : c == 1 ? 5 : c == 2 ? 1 : 4)
       : (s == 3) ? (c == 0 ? 3 : c == 1 ? 6 : c == 2 ? 5 : 4)
       : (s == 4) ? (c == 0 ? 3 : c == 1 ? 2 : c == 2 ? 6 : 4)
                  : (c == 0 ? 3 : c == 1 ? 7 : c == 2 ? 5 : 6);
}

// Latched device error bits (combined with atomicOr).
enum : unsigned {
  kErrCapacity = 1u,
  kErrNonFinite = 2u,
  kErrBehindEye = 4u,
  kErrRange = 8u,
  kErrBounds = 16u,  // an index check of a build with LT_CHECK_BOUNDS failed
};

// Device counters, one block of them per context.
struct DevCounters {
  unsigned errors;
  unsigned pad;
  unsigned long long nonfinite;
  unsigned long long behind_eye;
  unsigned long long degenerate;
  unsigned long long fp64_fallbacks;
  unsigned long long inverted;
  unsigned long long range_overflow;
  unsigned long long work_next;   // persistent raster work counter
  unsigned long long total_entries;
  unsigned long long exact_fragments;  // fragments re-evaluated in FP64
  unsigned long long queue_overflow;   // ill-conditioned fragments kept in FP32 (queue full)
  unsigned long long resample_intervals;  // (tetrahedron, grid line) pairs with a positive length
  unsigned long long resample_pieces;     // their pieces in separate slabs
  unsigned long long area_pairs;          // lt_render_area: (tetrahedron, pixel) pairs walked
  unsigned long long area_fp64_pairs;     // of them, clipped in FP64 (thin hulls)
  unsigned long long exact_tile_max;      // most ill-conditioned fragments of one tile (queued or not)
};

// Snapshot description.
struct Lattice {
  const void* pos;  // float4 or half4 per particle, n_snap arrays back to back
  int fmt;          // 0 float4 wrapped positions, 1 half4 offsets in cell units
  int N;
  float box, h, half_box;
  long long n_particles;  // N^3 (< 2^31)
  // per (snapshot, cube): bit s set when tetrahedron s has zero volume (such
  // a tetrahedron contributes nothing; written by the build pass)
  const unsigned char* degen;
  // unsigned division by N as a multiply-high and two shifts (Granlund and
  // Montgomery, "Division by invariant integers using multiplication", 1994,
  // Fig. 4.1): q = (t + ((n - t) >> s1)) >> s2, t = umulhi(div_m, n)
  unsigned div_m;
  int div_s1, div_s2;
};

// Host: fill the division constants for divisor N >= 1 (exact for every
// 32-bit dividend).
inline void lattice_set_divisor(Lattice& L, int N) {
  int l = 0;
  while ((1ull << l) < (unsigned long long)N) ++l;  // l = ceil(log2 N)
  L.div_m = (unsigned)((((1ull << l) - (unsigned long long)N) << 32) / (unsigned long long)N + 1ull);
  L.div_s1 = l < 1 ? l : 1;
  L.div_s2 = l > 1 ? l - 1 : 0;
}

__device__ __forceinline__ unsigned div_n(const Lattice& L, unsigned n) {
  const unsigned t = __umulhi(L.div_m, n);
  return (t + ((n - t) >> L.div_s1)) >> L.div_s2;
}

// Index checks of a debugging build (compiled with -DLT_CHECK_BOUNDS): a
// failed check latches kErrBounds and the access is skipped; the default
// build compiles them away.
#ifdef LT_CHECK_BOUNDS
#define LT_IN_BOUNDS(cond, err) ((cond) ? true : (atomicOr((err), kErrBounds), false))
#else
#define LT_IN_BOUNDS(cond, err) true
#endif

// True when tetrahedron s of `cube` in snapshot `snap` has zero volume.
__device__ __forceinline__ bool tet_degenerate(const Lattice& L, int snap, long long cube, int s) {
  return L.degen && ((__ldg(L.degen + (long long)snap * L.n_particles + cube) >> s) & 1u);
}

// Lattice indices of a cube (= of its corner-0 particle) from its id.
__device__ __forceinline__ void cube_ijk(const Lattice& L, long long cube, int& i, int& j, int& k) {
  const unsigned c = (unsigned)cube;
  const unsigned q = div_n(L, c);
  const unsigned N = (unsigned)L.N;
  i = (int)(c - q * N);
  const unsigned q2 = div_n(L, q);
  j = (int)(q - q2 * N);
  k = (int)q2;
}

// One view in kernel form.
struct FrameDev {
  int persp, W, H, wrap;
  int snapshot, tiles_x, tiles_y, tile;
  long long tile_base;  // first global tile index of this frame
  float r[3], u[3], f[3], eye[3];
  float sx, sy, ox, oy;   // ortho: pixel = dot(axis, P) * s + o
  float kx, ky, cx, cy;   // persp: pixel = (X / Z) * k + c in camera coordinates
  float near_z;           // perspective: vertices must have Z > near_z
  // Projected position of cube (i, j, k)'s Lagrangian corner as an affine
  // function of the lattice index, component c = ah[c][0] + i ah[c][1] +
  // j ah[c][2] + k ah[c][3] plus the same with al. The ah parts are integer
  // multiples of one power of two that keep every partial sum below 2^24
  // of it, so that sum is exact in FP32; al carries the remainder.
  // Orthographic: c = 0, 1 are pixel coordinates. Perspective: camera X, Y, Z.
  float ah[3][4], al[3][4];
  float kxh, kxl, kyh, kyl;  // perspective pixel scales as float-float pairs
  float K;                // value scale in accumulator units (see lt_api.cu)
  float inv6K;            // 1 / (6 K)
  float tan_x, tan_y;     // perspective image-plane half extents at unit distance
  double unit;            // accumulator unit -> column density
  double pix_area;        // pixel area for the frame mass
  // double-precision view for the exact evaluation of ill-conditioned fragments
  double rd[3], ud[3], fd[3], eyed[3];
  double lod[2], pxd[2];  // ortho window origin and pixel size (world units)
  double tand[2];         // perspective tan(fov/2) in x and y
  double m_tet;           // mass of one tetrahedron
  float sigma_units;      // mean column density in accumulator units (2^frac_bits)
  float pad_;
  // hybrid near/far rendering (perspective): when > 0, the square of the
  // radius around the eye beyond which a cube counts as far (see cube_far)
  double near_r2;
};

// ---------------------------------------------------------------------------
// Lattice addressing (Eq. 8) and the unwrapped corner positions.

__device__ __forceinline__ long long particle_id(int i, int j, int k, int N) {
  // N^3 < 2^31: the in-snapshot index fits in 32 bits
  return (long long)(unsigned)(i + N * (j + N * k));
}

// Minimum-image displacement of a wrapped coordinate p from its wrapped
// lattice point q (both in [0, box)). Each branch is a single FP32 subtraction
// of operands within a factor of two of each other where it matters
// (q +- box is exact for lattice points), so the displacement is the FP32
// rounding of the exact value even for particles that crossed the periodic
// boundary.
__device__ __forceinline__ float min_image(float p, float q, float box, float half_box) {
  const float d0 = p - q;
  return d0 > half_box ? p - (q + box) : (d0 < -half_box ? p - (q - box) : d0);
}

// Displacement of the particle at corner n of cube (i, j, k) from its own
// Lagrangian point. ok = false for non-finite data.
__device__ __forceinline__ float3 load_disp(const Lattice& L, long long snap_off, int i, int j, int k, int n,
                                            bool& ok) {
  const int a = n & 1, b = (n >> 1) & 1, c = (n >> 2) & 1;
  int ii = i + a, jj = j + b, kk = k + c;
  const int N = L.N;
  int im = ii == N ? 0 : ii, jm = jj == N ? 0 : jj, km = kk == N ? 0 : kk;
  long long id = snap_off + particle_id(im, jm, km, N);
  if (L.fmt == 0) {
    float4 p = __ldg(reinterpret_cast<const float4*>(L.pos) + id);
    const float dx = min_image(p.x, (float)im * L.h, L.box, L.half_box);
    const float dy = min_image(p.y, (float)jm * L.h, L.box, L.half_box);
    const float dz = min_image(p.z, (float)km * L.h, L.box, L.half_box);
    ok = ok && isfinite(p.x) && isfinite(p.y) && isfinite(p.z);
    return make_float3(dx, dy, dz);
  }
  const uint2 raw = __ldg(reinterpret_cast<const uint2*>(L.pos) + id);
  __half2 xy = *reinterpret_cast<const __half2*>(&raw.x);
  __half2 zw = *reinterpret_cast<const __half2*>(&raw.y);
  float2 fxy = __half22float2(xy);
  float fz = __low2float(zw);
  ok = ok && isfinite(fxy.x) && isfinite(fxy.y) && isfinite(fz);
  return make_float3(fxy.x * L.h, fxy.y * L.h, fz * L.h);
}

// One corner of cube (i, j, k) as a local offset from the cube's Lagrangian
// corner 0 (box units): lattice offset plus displacement.
__device__ __forceinline__ float3 load_corner(const Lattice& L, long long snap_off, int i, int j, int k, int n,
                                              bool& ok) {
  const float3 d = load_disp(L, snap_off, i, j, k, n, ok);
  const int a = n & 1, b = (n >> 1) & 1, c = (n >> 2) & 1;
  return make_float3((float)a * L.h + d.x, (float)b * L.h + d.y, (float)c * L.h + d.z);
}

// Hybrid near/far rendering: a cube is far when its corner-0 particle
// (unwrapped about its lattice point, in FP64) lies at least sqrt(near_r2)
// from the eye; never when near_r2 == 0. Every kernel that splits by it
// uses this one test, so each cube is drawn exactly once.
__device__ __forceinline__ bool cube_far(const Lattice& L, const FrameDev& F, long long cube) {
  if (!(F.near_r2 > 0.0)) return false;
  const unsigned c = (unsigned)cube;
  const int N = L.N;
  const int i = (int)(c % (unsigned)N), j = (int)((c / (unsigned)N) % (unsigned)N), k = (int)(c / ((unsigned)N * N));
  const float4 p = __ldg(reinterpret_cast<const float4*>(L.pos) + (long long)F.snapshot * L.n_particles + cube);
  const double h = (double)L.box / N, box = (double)L.box;
  const double pp[3] = {p.x, p.y, p.z};
  const int ix[3] = {i, j, k};
  // explicitly rounded operations (no fused multiply-add), so that the
  // test rounds like a plain evaluation of the same expression
  double e[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const double lq = __dmul_rn((double)ix[q], h);
    double d = __dsub_rn(pp[q], lq);
    if (d > 0.5 * box) d = __dsub_rn(d, box);
    else if (d < -0.5 * box) d = __dadd_rn(d, box);
    e[q] = __dsub_rn(__dadd_rn(lq, d), F.eyed[q]);
  }
  const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(e[0], e[0]), __dmul_rn(e[1], e[1])), __dmul_rn(e[2], e[2]));
  return !(r2 < F.near_r2);
}

// The eight corners of a cube projected to pixel coordinates, relative to
// the projection (ax, ay) of the cube's Lagrangian corner 0.
struct CubeProj {
  float x[8], y[8];
  float dw[8];   // perspective: 1/Z_n - 1/Z_anchor
  float z[8];    // perspective: Z_n (camera depth)
  float axh, axl, ayh, ayl;  // anchor pixel coordinate as hi + lo
  float w0;      // perspective: 1 / Z_anchor
  float xmin, xmax, ymin, ymax;  // relative bounding box of the 8 corners
};

// Lattice-affine anchor component as (hi, lo); hi is exact (see FrameDev).
__device__ __forceinline__ void anchor_affine(const FrameDev& F, int c, int i, int j, int k, float& hi, float& lo) {
  hi = fmaf((float)k, F.ah[c][3], fmaf((float)j, F.ah[c][2], fmaf((float)i, F.ah[c][1], F.ah[c][0])));
  lo = fmaf((float)k, F.al[c][3], fmaf((float)j, F.al[c][2], fmaf((float)i, F.al[c][1], F.al[c][0])));
}

// Approximate reciprocal (the hardware's, within a couple of ulp) for
// quantities whose rounding the fragment error model absorbs.
__device__ __forceinline__ float fast_rcp(float x) { return __fdividef(1.0f, x); }

// Float-float (Xh + Xl) / (Zh + Zl) * (kh + kl) + c0 -> (hi, lo); rz is an
// approximate 1 / Zh. One Newton step makes the high quotient faithful, so
// the FMA residual Xh - q Zh is exact.
__device__ __forceinline__ void ff_project(float Xh, float Xl, float Zh, float Zl, float rz, float kh, float kl,
                                           float c0, float& hi, float& lo) {
  const float q0 = Xh * rz;
  const float q = fmaf(fmaf(-q0, Zh, Xh), rz, q0);
  float r = fmaf(-q, Zh, Xh);  // exact residual of the division
  r = fmaf(-q, Zl, Xl) + r;
  const float ql = r * rz;
  const float p = kh * q;
  float e = fmaf(kh, q, -p);   // exact product error
  e = fmaf(kh, ql, e);
  e = fmaf(kl, q, e);
  const float s = p + c0;      // two-sum of p and c0
  const float bb = s - p;
  const float err = (p - (s - bb)) + (c0 - bb);
  hi = s;
  lo = err + e;
}

// Pixel coordinate relative to a cube copy's anchor (exact to ~1e-9 px for
// the pixel counts of one frame).
__device__ __forceinline__ float rel_coord(int p, int shift, float ah, float al) {
  return ((float)(p - shift) - ah) - al;
}

// Returns true when the cube can be drawn. A perspective cube entirely behind
// the eye plane is culled (no ray reaches it); one straddling the plane
// cannot be projected and sets straddle (callers count and report it).
template <bool PERSP>
__device__ __forceinline__ bool project_cube(const Lattice& L, const FrameDev& F, long long cube, CubeProj& P,
                                             bool& finite_ok, bool* straddle = nullptr) {
  int i, j, k;
  cube_ijk(L, cube, i, j, k);
  const long long snap_off = (long long)F.snapshot * L.n_particles;
  bool ok = true;
  if (!PERSP) {
    anchor_affine(F, 0, i, j, k, P.axh, P.axl);
    anchor_affine(F, 1, i, j, k, P.ayh, P.ayl);
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      float3 l = load_corner(L, snap_off, i, j, k, n, ok);
      P.x[n] = (F.r[0] * l.x + F.r[1] * l.y + F.r[2] * l.z) * F.sx;
      P.y[n] = (F.u[0] * l.x + F.u[1] * l.y + F.u[2] * l.z) * F.sy;
    }
  } else {
    float Xh, Xl, Yh, Yl, Zh, Zl;
    anchor_affine(F, 0, i, j, k, Xh, Xl);
    anchor_affine(F, 1, i, j, k, Yh, Yl);
    anchor_affine(F, 2, i, j, k, Zh, Zl);
    const float X0 = Xh + Xl, Y0 = Yh + Yl, Z0 = Zh + Zl;
    bool front = Z0 > F.near_z;
    int n_front = front ? 1 : 0;
    if (front) {
      const float rz = fast_rcp(Zh);
      ff_project(Xh, Xl, Zh, Zl, rz, F.kxh, F.kxl, F.cx, P.axh, P.axl);
      ff_project(Yh, Yl, Zh, Zl, rz, F.kyh, F.kyl, F.cy, P.ayh, P.ayl);
    }
    const float iZ0 = fast_rcp(Z0);
    P.w0 = iZ0;
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      float3 l = load_corner(L, snap_off, i, j, k, n, ok);
      const float dX = F.r[0] * l.x + F.r[1] * l.y + F.r[2] * l.z;
      const float dY = F.u[0] * l.x + F.u[1] * l.y + F.u[2] * l.z;
      const float dZ = F.f[0] * l.x + F.f[1] * l.y + F.f[2] * l.z;
      const float Zn = Z0 + dZ;
      front = front && (Zn > F.near_z);
      n_front += Zn > F.near_z ? 1 : 0;
      const float inv = fast_rcp(Zn * Z0);
      // X_n/Z_n - X0/Z0 = (dX Z0 - X0 dZ) / (Z_n Z0), free of cancellation
      P.x[n] = (dX * Z0 - X0 * dZ) * inv * F.kx;
      P.y[n] = (dY * Z0 - Y0 * dZ) * inv * F.ky;
      P.dw[n] = -dZ * inv;
      P.z[n] = Zn;
    }
    if (!front) {
      finite_ok = finite_ok && ok;
      if (straddle) *straddle = ok && n_front > 0;
      return false;
    }
  }
  finite_ok = finite_ok && ok;
  if (!ok) return false;
  float xmn = P.x[0], xmx = P.x[0], ymn = P.y[0], ymx = P.y[0];
#pragma unroll
  for (int n = 1; n < 8; ++n) {
    xmn = fminf(xmn, P.x[n]); xmx = fmaxf(xmx, P.x[n]);
    ymn = fminf(ymn, P.y[n]); ymx = fmaxf(ymx, P.y[n]);
  }
  P.xmin = xmn; P.xmax = xmx; P.ymin = ymn; P.ymax = ymx;
  return true;
}

// Corner n (0..7) of column c of row s of the connectivity table, for a
// run-time row index (rows 0..4 packed 12 bits each, row 5 separately).
__device__ __forceinline__ int tet_corner_dyn(int s, int c) {
  constexpr unsigned long long P =
      (unsigned long long)tet_corner(0, 0) | ((unsigned long long)tet_corner(0, 1) << 3) |
      ((unsigned long long)tet_corner(0, 2) << 6) | ((unsigned long long)tet_corner(0, 3) << 9) |
      ((unsigned long long)tet_corner(1, 0) << 12) | ((unsigned long long)tet_corner(1, 1) << 15) |
      ((unsigned long long)tet_corner(1, 2) << 18) | ((unsigned long long)tet_corner(1, 3) << 21) |
      ((unsigned long long)tet_corner(2, 0) << 24) | ((unsigned long long)tet_corner(2, 1) << 27) |
      ((unsigned long long)tet_corner(2, 2) << 30) | ((unsigned long long)tet_corner(2, 3) << 33) |
      ((unsigned long long)tet_corner(3, 0) << 36) | ((unsigned long long)tet_corner(3, 1) << 39) |
      ((unsigned long long)tet_corner(3, 2) << 42) | ((unsigned long long)tet_corner(3, 3) << 45) |
      ((unsigned long long)tet_corner(4, 0) << 48) | ((unsigned long long)tet_corner(4, 1) << 51) |
      ((unsigned long long)tet_corner(4, 2) << 54) | ((unsigned long long)tet_corner(4, 3) << 57);
  constexpr unsigned R5 = (unsigned)tet_corner(5, 0) | ((unsigned)tet_corner(5, 1) << 3) |
                          ((unsigned)tet_corner(5, 2) << 6) | ((unsigned)tet_corner(5, 3) << 9);
  return s < 5 ? (int)((P >> (12 * s + 3 * c)) & 7ull) : (int)((R5 >> (3 * c)) & 7u);
}

// The four vertices of tetrahedron s of a cube, projected like project_cube.
struct TetProj {
  float x[4], y[4], dw[4], z[4];
  float axh, axl, ayh, ayl, w0;
};

// Returns false for non-finite input or a tetrahedron not entirely in front
// of a perspective eye (those cubes are counted by the bin pass).
template <bool PERSP>
__device__ __forceinline__ bool project_tet(const Lattice& L, const FrameDev& F, long long cube, int s, TetProj& P) {
  int i, j, k;
  cube_ijk(L, cube, i, j, k);
  const long long snap_off = (long long)F.snapshot * L.n_particles;
  bool ok = true;
  if (!PERSP) {
    anchor_affine(F, 0, i, j, k, P.axh, P.axl);
    anchor_affine(F, 1, i, j, k, P.ayh, P.ayl);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float3 l = load_corner(L, snap_off, i, j, k, tet_corner_dyn(s, c), ok);
      P.x[c] = (F.r[0] * l.x + F.r[1] * l.y + F.r[2] * l.z) * F.sx;
      P.y[c] = (F.u[0] * l.x + F.u[1] * l.y + F.u[2] * l.z) * F.sy;
      P.dw[c] = 0.f;
      P.z[c] = 1.f;
    }
    P.w0 = 0.f;
    return ok;
  }
  float Xh, Xl, Yh, Yl, Zh, Zl;
  anchor_affine(F, 0, i, j, k, Xh, Xl);
  anchor_affine(F, 1, i, j, k, Yh, Yl);
  anchor_affine(F, 2, i, j, k, Zh, Zl);
  const float X0 = Xh + Xl, Y0 = Yh + Yl, Z0 = Zh + Zl;
  bool front = Z0 > F.near_z;
  const float rz = fast_rcp(Zh);
  ff_project(Xh, Xl, Zh, Zl, rz, F.kxh, F.kxl, F.cx, P.axh, P.axl);
  ff_project(Yh, Yl, Zh, Zl, rz, F.kyh, F.kyl, F.cy, P.ayh, P.ayl);
  P.w0 = fast_rcp(Z0);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const float3 l = load_corner(L, snap_off, i, j, k, tet_corner_dyn(s, c), ok);
    const float dX = F.r[0] * l.x + F.r[1] * l.y + F.r[2] * l.z;
    const float dY = F.u[0] * l.x + F.u[1] * l.y + F.u[2] * l.z;
    const float dZ = F.f[0] * l.x + F.f[1] * l.y + F.f[2] * l.z;
    const float Zn = Z0 + dZ;
    front = front && (Zn > F.near_z);
    const float inv = fast_rcp(Zn * Z0);
    P.x[c] = (dX * Z0 - X0 * dZ) * inv * F.kx;
    P.y[c] = (dY * Z0 - Y0 * dZ) * inv * F.ky;
    P.dw[c] = -dZ * inv;
    P.z[c] = Zn;
  }
  return ok && front;
}

// ---------------------------------------------------------------------------
// Per-tetrahedron setup.

struct TetRaster {
  // value(X, Y) = max(0, min_e a[e] X + b[e] Y + c[e]) (ortho, accumulator units)
  float a[4], b[4], c[4];
  // perspective depth surface: M = max(pa0 X + pb0 Y + pc0, pa1 X + pb1 Y + pc1),
  // value = T / (M (M + g T)), T the pyramid above
  float pa[2], pb[2], pc[2];
  float g;
  float xmin, xmax, ymin, ymax;  // relative bounding box
  // steepness |e|^2 / min(|o1|, |o2|) of each edge (0 for unused slots): the
  // FP32 round-off of an edge's value grows in proportion to it
  float st[4];
  float hmax;    // upper bound of the value over the tetrahedron (accumulator units)
  float vscale;  // perspective: bound of d value / d T (1 / w_min^2); 1 orthographic
};

__device__ __forceinline__ float cross2(float ax, float ay, float bx, float by) { return ax * by - ay * bx; }

// Conditionally swap two scalars.
__device__ __forceinline__ void cswap(bool s, float& p, float& q) {
  const float tp = p, tq = q;
  p = s ? tq : tp;
  q = s ? tp : tq;
}

// One hull edge (j, k) with the other two vertices l1, l2, in canonical
// coordinates; writes f_e = sigma * w * orient(v_j, v_k, x) with
// w = W / |o1 o2| (W = 6 K, or 6 K / (Z0 Z1 Z2 Z3) in perspective).
__device__ __forceinline__ void edge_fn(float xj, float yj, float ex, float ey, float o1, float o2, float Wn,
                                        float tiny, float& a, float& b, float& c) {
  const float prod = fmaxf(fabsf(o1 * o2), tiny);
  float w = __fdividef(Wn, prod);  // prod is far below 2^126
  w = (o1 + o2) < 0.0f ? -w : w;
  const bool dead = (o1 == 0.0f) && (o2 == 0.0f);  // zero-length edge or flat hull
  a = dead ? 0.0f : -ey * w;
  b = dead ? 0.0f : ex * w;
  c = dead ? __int_as_float(0x7f800000) : (ey * xj - ex * yj) * w;
}

// Plane of the mapped face (p, q, r) in (X, Y, w) space, w relative to the anchor.
__device__ __forceinline__ bool face_plane(float xp, float yp, float wp, float xq, float yq, float wq, float xr,
                                           float yr, float wr, float& pa, float& pb, float& pc) {
  const float ux = xq - xp, uy = yq - yp, uw = wq - wp;
  const float vx = xr - xp, vy = yr - yp, vw = wr - wp;
  const float nw = ux * vy - uy * vx;
  const float nx = uy * vw - uw * vy;
  const float ny = uw * vx - ux * vw;
  // a face seen nearly edge-on has an unreliable FP32 slope: treat as vertical
  if (!(fabsf(nw) > 1e-5f * (fabsf(ux * vy) + fabsf(uy * vx)))) return false;
  const float inw = fast_rcp(nw);
  pa = -nx * inw;
  pb = -ny * inw;
  pc = wp - pa * xp - pb * yp;
  return true;
}

// Canonical labelling of a projected tetrahedron. The signed areas
// c_i = (-1)^i orient(vertices other than i) sum to zero; same-sign pairs are
// the diagonals of a convex quadrilateral hull (two of each sign, "case B"),
// and a lone sign marks the vertex inside the triangle of the other three
// ("case A"). Vertices are reordered so that the diagonals are (0,1) | (2,3),
// or the inner vertex is 3.
struct TetCanon {
  float x[4], y[4], w[4];
  int perm[4];                 // canonical position -> original vertex slot
  bool caseB;
  float d1x, d1y, d2x, d2y, d3x, d3y;
  float D12, D13, D23, O123;   // orient(0,1,2), orient(0,1,3), orient(0,2,3), orient(1,2,3)
  float S;                     // sum |c_i| = 4 * area(hull)
};

__device__ __forceinline__ void cswapi(bool s, int& p, int& q) {
  const int tp = p, tq = q;
  p = s ? tq : tp;
  q = s ? tp : tq;
}

__device__ __forceinline__ bool tet_canon(float x0, float y0, float x1, float y1, float x2, float y2, float x3,
                                          float y3, float w0, float w1, float w2, float w3, TetCanon& k) {
  const float ax = x1 - x0, ay = y1 - y0, bx = x2 - x0, by = y2 - y0, cx = x3 - x0, cy = y3 - y0;
  const float ab = cross2(ax, ay, bx, by), ac = cross2(ax, ay, cx, cy), bc = cross2(bx, by, cx, cy);
  float c1 = -bc, c2 = ac, c3 = -ab;
  const float c0 = -(c1 + c2 + c3);
  const float S = fabsf(c0) + fabsf(c1) + fabsf(c2) + fabsf(c3);
  if (!(S > 0.0f)) return false;
  if (c0 < 0.0f) { c1 = -c1; c2 = -c2; c3 = -c3; }
  const int t1 = c1 > 0.0f, t2 = c2 > 0.0f, t3 = c3 > 0.0f;
  const int npos = t1 + t2 + t3;
  const bool caseB = npos == 1;
  const int p = t1 ? 1 : (t2 ? 2 : 3);
  const int apex = npos == 0 ? 0 : (!t1 ? 1 : (!t2 ? 2 : 3));
  const bool s12 = caseB && p == 2;
  const bool s13 = (caseB && p == 3) || (!caseB && apex == 1);
  const bool s23 = !caseB && apex == 2;
  const bool s03 = !caseB && apex == 0;
  int i0 = 0, i1 = 1, i2 = 2, i3 = 3;
  cswap(s12, x1, x2); cswap(s12, y1, y2); cswap(s12, w1, w2); cswapi(s12, i1, i2);
  cswap(s13, x1, x3); cswap(s13, y1, y3); cswap(s13, w1, w3); cswapi(s13, i1, i3);
  cswap(s23, x2, x3); cswap(s23, y2, y3); cswap(s23, w2, w3); cswapi(s23, i2, i3);
  cswap(s03, x0, x3); cswap(s03, y0, y3); cswap(s03, w0, w3); cswapi(s03, i0, i3);
  k.x[0] = x0; k.x[1] = x1; k.x[2] = x2; k.x[3] = x3;
  k.y[0] = y0; k.y[1] = y1; k.y[2] = y2; k.y[3] = y3;
  k.w[0] = w0; k.w[1] = w1; k.w[2] = w2; k.w[3] = w3;
  k.perm[0] = i0; k.perm[1] = i1; k.perm[2] = i2; k.perm[3] = i3;
  k.caseB = caseB;
  k.d1x = x1 - x0; k.d1y = y1 - y0;
  k.d2x = x2 - x0; k.d2y = y2 - y0;
  k.d3x = x3 - x0; k.d3y = y3 - y0;
  k.D12 = cross2(k.d1x, k.d1y, k.d2x, k.d2y);
  k.D13 = cross2(k.d1x, k.d1y, k.d3x, k.d3y);
  k.D23 = cross2(k.d2x, k.d2y, k.d3x, k.d3y);
  k.O123 = k.D12 + k.D23 - k.D13;
  k.S = S;
  return true;
}

// Hull edge of slot e in canonical indices: start j, edge vector, and the
// orientations o1, o2 of the other two vertices against it.
//   slot 0: (0,2) | 1,3    slot 1: (1,2) | 0,3
//   slot 2: case B (1,3) | 0,2, case A (0,1) | 2,3
//   slot 3: case B (0,3) | 1,2, case A unused
struct EdgeRef {
  int j, k, l1, l2;
  float ex, ey, o1, o2;
};

__device__ __forceinline__ EdgeRef edge_ref(const TetCanon& K, int e) {
  EdgeRef r;
  if (e == 0) {
    r.j = 0; r.k = 2; r.l1 = 1; r.l2 = 3; r.ex = K.d2x; r.ey = K.d2y; r.o1 = -K.D12; r.o2 = K.D23;
  } else if (e == 1) {
    r.j = 1; r.k = 2; r.l1 = 0; r.l2 = 3; r.ex = K.d2x - K.d1x; r.ey = K.d2y - K.d1y; r.o1 = K.D12; r.o2 = K.O123;
  } else if (e == 2) {
    if (K.caseB) {
      r.j = 1; r.k = 3; r.l1 = 0; r.l2 = 2; r.ex = K.d3x - K.d1x; r.ey = K.d3y - K.d1y; r.o1 = K.D13; r.o2 = -K.O123;
    } else {
      r.j = 0; r.k = 1; r.l1 = 2; r.l2 = 3; r.ex = K.d1x; r.ey = K.d1y; r.o1 = K.D12; r.o2 = K.D13;
    }
  } else {
    r.j = 0; r.k = 3; r.l1 = 1; r.l2 = 2; r.ex = K.d3x; r.ey = K.d3y; r.o1 = -K.D13; r.o2 = -K.D23;
  }
  return r;
}

__device__ __forceinline__ float sel4(const float* v, int i) {
  return i == 0 ? v[0] : (i == 1 ? v[1] : (i == 2 ? v[2] : v[3]));
}

// Build the raster form of one tetrahedron from its four projected vertices
// (relative pixel coordinates). Kn = 6 K (ortho) or 6 K / (Z0 Z1 Z2 Z3)
// (perspective); wa = 1/Z of the anchor (perspective). Returns false for a
// projection of zero area.
template <bool PERSP>
__device__ __forceinline__ bool tet_setup(float x0, float y0, float x1, float y1, float x2, float y2, float x3,
                                          float y3, float w0, float w1, float w2, float w3, float Kn, float wa,
                                          float invKn, TetRaster& t) {
  t.xmin = fminf(fminf(x0, x1), fminf(x2, x3));
  t.xmax = fmaxf(fmaxf(x0, x1), fmaxf(x2, x3));
  t.ymin = fminf(fminf(y0, y1), fminf(y2, y3));
  t.ymax = fmaxf(fmaxf(y0, y1), fmaxf(y2, y3));
  TetCanon K;
  if (!tet_canon(x0, y0, x1, y1, x2, y2, x3, y3, w0, w1, w2, w3, K)) return false;
  const float tiny = K.S * K.S * 1e-12f;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const EdgeRef r = edge_ref(K, e);
    edge_fn(sel4(K.x, r.j), sel4(K.y, r.j), r.ex, r.ey, r.o1, r.o2, Kn, tiny, t.a[e], t.b[e], t.c[e]);
    const float omin = fminf(fabsf(r.o1), fabsf(r.o2));
    t.st[e] = __fdividef(r.ex * r.ex + r.ey * r.ey, fmaxf(omin, tiny));
  }
  if (!K.caseB) {
    t.a[3] = 0.0f;
    t.b[3] = 0.0f;
    t.c[3] = __int_as_float(0x7f800000);
    t.st[3] = 0.0f;
  }
  // pyramid apex value 2 Kn / S; the perspective depth factor is at most 1 / w_min^2
  t.hmax = __fdividef(2.0f * Kn, K.S);
  t.vscale = 1.0f;
  if (PERSP) {
    const float wmin = wa + fminf(fminf(w0, w1), fminf(w2, w3));
    t.vscale = fast_rcp(wmin * wmin);
    t.hmax = t.hmax * t.vscale;
  }
  if (PERSP) {
    const float* X = K.x;
    const float* Y = K.y;
    const float* W = K.w;
    const float C0 = fabsf(K.O123), C1 = fabsf(K.D23), C2 = fabsf(K.D13), C3 = fabsf(K.D12);
    // Q > 0: the (0,1) diagonal (case B) / the outer face (case A) is the lower w surface
    const float Q = K.caseB ? (C2 * W[2] + C3 * W[3]) - (C0 * W[0] + C1 * W[1])
                            : C3 * W[3] - (C0 * W[0] + C1 * W[1] + C2 * W[2]);
    bool ok1, ok2;
    float pa0 = 0.f, pb0 = 0.f, pc0 = 0.f, pa1 = 0.f, pb1 = 0.f, pc1 = 0.f;
    if (!K.caseB) {
      ok1 = face_plane(X[0], Y[0], W[0], X[1], Y[1], W[1], X[2], Y[2], W[2], pa0, pb0, pc0);
      ok2 = ok1;
      pa1 = pa0; pb1 = pb0; pc1 = pc0;
    } else {
      const bool low01 = Q > 0.0f;
      const int ip = low01 ? 0 : 2, iq = low01 ? 1 : 3, ir = low01 ? 2 : 0, is = low01 ? 3 : 1;
      const float px = sel4(X, ip), py = sel4(Y, ip), pw = sel4(W, ip);
      const float qx = sel4(X, iq), qy = sel4(Y, iq), qw = sel4(W, iq);
      ok1 = face_plane(px, py, pw, qx, qy, qw, sel4(X, ir), sel4(Y, ir), sel4(W, ir), pa0, pb0, pc0);
      ok2 = face_plane(px, py, pw, qx, qy, qw, sel4(X, is), sel4(Y, is), sel4(W, is), pa1, pb1, pc1);
    }
    if (!ok1 && !ok2) return false;
    if (!ok1) { pa0 = pa1; pb0 = pb1; pc0 = pc1; }
    if (!ok2) { pa1 = pa0; pb1 = pb0; pc1 = pc0; }
    // sigma = -1 when the single outer face is the upper surface (case A)
    const float sg = (!K.caseB && Q < 0.0f) ? -1.0f : 1.0f;
    t.pa[0] = sg * pa0; t.pb[0] = sg * pb0; t.pc[0] = sg * (pc0 + wa);
    t.pa[1] = sg * pa1; t.pb[1] = sg * pb1; t.pc[1] = sg * (pc1 + wa);
    // the w-extent at the apex is 2|Q|/S and the pyramid apex value is 2 Kn / S
    t.g = fabsf(Q) * invKn;
  }
  return true;
}

// Pixel span [lo, hi] (relative X) of row terms where every edge function is
// >= 0, widened by a small margin so that rounding never drops a pixel.
__device__ __forceinline__ void row_span(const TetRaster& t, const float* erow, float& lo, float& hi) {
  lo = -3.0e38f;
  hi = 3.0e38f;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const float a = t.a[e];
    const float xb = -erow[e] / a;
    if (a > 0.0f) lo = fmaxf(lo, xb);
    else if (a < 0.0f) hi = fminf(hi, xb);
    else if (erow[e] < 0.0f) hi = -3.0e38f;
  }
  lo -= 1e-3f;
  hi += 1e-3f;
}

// Add a non-negative value q (accumulator units) to a pixel's 64-bit
// fixed-point sum in shared memory. Integer sums are exact and associative,
// so the image does not depend on the order of the adds. A value that cannot
// be converted (2^63 units or more, or not a number) and an add that carries
// the sum past 2^64 latch kErrRange and are counted: the atomic returns the
// sum before the add, so a wrap is seen by the add that causes it.
__device__ __forceinline__ void accum_fixed(unsigned long long* acc, float q, DevCounters* ctr) {
  constexpr float k2p63 = 9223372036854775808.0f;
  if (q < k2p63) {
    // values below 2^32 units (nearly all) convert through 32 bits: the
    // 64-bit conversion runs on the FP64 pipe, which GB300 keeps narrow
    const unsigned long long u =
        q < 4294967040.0f ? (unsigned long long)__float2uint_rn(q) : __float2ull_rn(q);
    if (u) {
      const unsigned long long old = atomicAdd(acc, u);
      if (old > ~0ull - u) {
        atomicOr(&ctr->errors, kErrRange);
        atomicAdd(&ctr->range_overflow, 1ull);
      }
    }
  } else if (!(q <= 0.0f)) {
    atomicOr(&ctr->errors, kErrRange);
    atomicAdd(&ctr->range_overflow, 1ull);
  }
}

// Exact value of rho_t * dl_t (Eq. 3, 6, 9) for tetrahedron s of `cube` at
// pixel (px, py) of the copy shifted by (sx, sy) periods, in FP64 from the
// stored positions: the ray through the pixel centre clipped against the four
// face planes. Used for the rare fragments whose FP32 evaluation is
// ill-conditioned. Returns the value in column-density units divided by the
// pixel's ray-direction length for perspective frames (the factor the tile
// applies when it stores the pixel).
__device__ __noinline__ static double exact_fragment(const Lattice& L, const FrameDev& F, long long cube, int s, int sx, int sy, int px,
                                 int py, double m) {
  const int N = L.N;
  const int i = (int)(cube % N), j = (int)((cube / N) % N), k = (int)(cube / ((long long)N * N));
  const long long soff = (long long)F.snapshot * L.n_particles;
  const double h = (double)L.box / N, box = (double)L.box;
  double v[4][3];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int n = tet_corner_dyn(s, c);
    const int a = n & 1, b = (n >> 1) & 1, cc = (n >> 2) & 1;
    const int ii = i + a, jj = j + b, kk = k + cc;
    const int im = ii == N ? 0 : ii, jm = jj == N ? 0 : jj, km = kk == N ? 0 : kk;
    const long long id = soff + particle_id(im, jm, km, N);
    double d[3];
    if (L.fmt == 0) {
      const float4 p = __ldg(reinterpret_cast<const float4*>(L.pos) + id);
      const double pp[3] = {p.x, p.y, p.z};
      const int ix[3] = {im, jm, km};
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        double dd = pp[q] - ix[q] * h;
        if (dd > 0.5 * box) dd -= box;
        else if (dd < -0.5 * box) dd += box;
        d[q] = dd;
      }
    } else {
      bool ok = true;
      const float3 df = load_disp(L, soff, i, j, k, n, ok);
      d[0] = df.x; d[1] = df.y; d[2] = df.z;
    }
    v[c][0] = (i + a) * h + d[0];
    v[c][1] = (j + b) * h + d[1];
    v[c][2] = (k + cc) * h + d[2];
  }
  // signed volume (Eq. 9) and density (Eq. 3)
  double e1[3], e2[3], e3[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    e1[q] = v[1][q] - v[0][q];
    e2[q] = v[2][q] - v[0][q];
    e3[q] = v[3][q] - v[0][q];
  }
  const double V = (e1[0] * (e2[1] * e3[2] - e2[2] * e3[1]) + e1[1] * (e2[2] * e3[0] - e2[0] * e3[2]) +
                    e1[2] * (e2[0] * e3[1] - e2[1] * e3[0])) / 6.0;
  if (V == 0.0) return 0.0;
  // pixel ray
  double o[3], dir[3];
  bool half = F.persp != 0;
  if (!half) {
    const double a = F.lod[0] + ((double)px - (double)sx * F.W + 0.5) * F.pxd[0];
    const double b = F.lod[1] + ((double)py - (double)sy * F.H + 0.5) * F.pxd[1];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      o[q] = a * F.rd[q] + b * F.ud[q];
      dir[q] = F.fd[q];
    }
  } else {
    const double xt = F.tand[0] * (2.0 * ((double)px + 0.5) / F.W - 1.0);
    const double yt = F.tand[1] * (2.0 * ((double)py + 0.5) / F.H - 1.0);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      o[q] = F.eyed[q];
      dir[q] = F.fd[q] + xt * F.rd[q] + yt * F.ud[q];
    }
  }
  const double dl = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
  // clip t (point o + t dir) against the four outward half-spaces
  double t_in = half ? 0.0 : -1e300, t_out = 1e300;
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const double* A = v[(f + 1) & 3];
    const double* B = v[(f + 2) & 3];
    const double* C = v[(f + 3) & 3];
    const double u1[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
    const double u2[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
    double nn[3] = {u1[1] * u2[2] - u1[2] * u2[1], u1[2] * u2[0] - u1[0] * u2[2], u1[0] * u2[1] - u1[1] * u2[0]};
    const double side = nn[0] * (v[f][0] - A[0]) + nn[1] * (v[f][1] - A[1]) + nn[2] * (v[f][2] - A[2]);
    if (side > 0.0) { nn[0] = -nn[0]; nn[1] = -nn[1]; nn[2] = -nn[2]; }
    const double den = nn[0] * dir[0] + nn[1] * dir[1] + nn[2] * dir[2];
    const double num = nn[0] * (A[0] - o[0]) + nn[1] * (A[1] - o[1]) + nn[2] * (A[2] - o[2]);
    if (den > 0.0) t_out = fmin(t_out, num / den);
    else if (den < 0.0) t_in = fmax(t_in, num / den);
    else if (num < 0.0) return 0.0;
  }
  if (!(t_out > t_in)) return 0.0;
  const double chord = (t_out - t_in) * dl;
  const double val = m / fabs(V) * chord;
  return half ? val / dl : val;
}

// One tetrahedron in FP64, relative to its cube's corner-0 Lagrangian point.
struct TetF64 {
  double v[4][3];
  double n[4][3];  // outward face normals (face f opposite vertex f)
  double d[4];     // plane offsets: inside when n . p <= d
  double V;        // signed volume (Eq. 9)
};

__device__ __forceinline__ void tet_f64(const Lattice& L, long long soff, int i, int j, int k, int s, bool& ok,
                                        TetF64& t) {
  const int N = L.N;
  const double h = (double)L.box / N, box = (double)L.box;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int n = tet_corner_dyn(s, c);
    const int a = n & 1, b = (n >> 1) & 1, cc = (n >> 2) & 1;
    const int ii = i + a, jj = j + b, kk = k + cc;
    const int im = ii == N ? 0 : ii, jm = jj == N ? 0 : jj, km = kk == N ? 0 : kk;
    double dd[3];
    if (L.fmt == 0) {
      const float4 p = __ldg(reinterpret_cast<const float4*>(L.pos) + soff + particle_id(im, jm, km, N));
      ok = ok && isfinite(p.x) && isfinite(p.y) && isfinite(p.z);
      const double pp[3] = {p.x, p.y, p.z};
      const int ix[3] = {im, jm, km};
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        double e = pp[q] - ix[q] * h;  // minimum image of the displacement
        if (e > 0.5 * box) e -= box;
        else if (e < -0.5 * box) e += box;
        dd[q] = e;
      }
    } else {
      const float3 df = load_disp(L, soff, i, j, k, n, ok);
      dd[0] = df.x; dd[1] = df.y; dd[2] = df.z;
    }
    t.v[c][0] = a * h + dd[0];
    t.v[c][1] = b * h + dd[1];
    t.v[c][2] = cc * h + dd[2];
  }
  const double e1[3] = {t.v[1][0] - t.v[0][0], t.v[1][1] - t.v[0][1], t.v[1][2] - t.v[0][2]};
  const double e2[3] = {t.v[2][0] - t.v[0][0], t.v[2][1] - t.v[0][1], t.v[2][2] - t.v[0][2]};
  const double e3[3] = {t.v[3][0] - t.v[0][0], t.v[3][1] - t.v[0][1], t.v[3][2] - t.v[0][2]};
  t.V = (e1[0] * (e2[1] * e3[2] - e2[2] * e3[1]) + e1[1] * (e2[2] * e3[0] - e2[0] * e3[2]) +
         e1[2] * (e2[0] * e3[1] - e2[1] * e3[0])) / 6.0;
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const double* A = t.v[(f + 1) & 3];
    const double* B = t.v[(f + 2) & 3];
    const double* C = t.v[(f + 3) & 3];
    const double u1[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
    const double u2[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
    double nn[3] = {u1[1] * u2[2] - u1[2] * u2[1], u1[2] * u2[0] - u1[0] * u2[2], u1[0] * u2[1] - u1[1] * u2[0]};
    const double side = nn[0] * (t.v[f][0] - A[0]) + nn[1] * (t.v[f][1] - A[1]) + nn[2] * (t.v[f][2] - A[2]);
    if (side > 0.0) { nn[0] = -nn[0]; nn[1] = -nn[1]; nn[2] = -nn[2]; }
    t.n[f][0] = nn[0]; t.n[f][1] = nn[1]; t.n[f][2] = nn[2];
    t.d[f] = nn[0] * A[0] + nn[1] * A[1] + nn[2] * A[2];
  }
}

// Error model of a fragment's FP32 value (accumulator units). Every hull edge
// e gets a bound e_e on its FP32 edge function f_e:
//   * the rounding of the projected vertex positions, absolute: the edge
//     moves by up to delta pixels, changing f_e by up to its slope
//     (|a_e| + |b_e|) times delta. Thin projected slivers have huge slopes;
//   * the round-off of the edge's coefficients, relative, about kFragErr
//     times the edge's steepness |e|^2 / min(|o1|, |o2|) times |f_e|;
//   * the round-off of evaluating a X + b Y + c, absolute: kEvalErr times
//     |a X| + |b Y| + |c|.
// The pyramid is the minimum over the edges, and the edge that is smallest in
// FP32 need not be the smallest in exact arithmetic: the true minimum lies in
// [min (f_e - e_e), min (f_e + e_e)]. The FP32 value max(min f, 0) may be off
// by its distance to the far end of that interval, scaled in perspective by
// d value / d T = 1 / (M + g T)^2. A fragment is recomputed exactly when that
// could exceed kFragTol of max(value, mean column density); a pixel just
// outside the FP32 hull that the bounds could move inside is one of them.
constexpr float kFragErr = 1e-5f;
constexpr float kFragTol = 1e-5f;
constexpr float kEvalErr = 4.0f / 16777216.0f;  // four ulp of the terms of a X + b Y + c

// Vertex position uncertainty (pixels) of a tetrahedron whose vertices lie
// within R pixels of its cube's anchor (R includes, in perspective, the
// depth terms of the projection): about four ulp of R from the displacement
// and projection arithmetic (eight with the perspective's approximate
// reciprocals), plus the tile-relative subtraction.
__device__ __forceinline__ float vertex_uncertainty(float R, bool persp) {
  // orthographic: 2^-21 R + 2^-19; perspective (approximate reciprocals): 2^-20 R + 2^-19
  return R * (persp ? (1.0f / 1048576.0f) : (1.0f / 2097152.0f)) + (1.0f / 524288.0f);
}

__device__ __forceinline__ float max_edge_slope(const TetRaster& t) {
  return fmaxf(fmaxf(fabsf(t.a[0]) + fabsf(t.b[0]), fabsf(t.a[1]) + fabsf(t.b[1])),
               fmaxf(fabsf(t.a[2]) + fabsf(t.b[2]), fabsf(t.a[3]) + fabsf(t.b[3])));
}

// Largest evaluation round-off of the edge functions over the bounding box
// (pixel coordinates up to R in magnitude).
__device__ __forceinline__ float max_eval_error(const TetRaster& t, float R) {
  float m = 0.0f;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const float ab = fabsf(t.a[e]) + fabsf(t.b[e]);
    if (ab > 0.0f) m = fmaxf(m, kEvalErr * fmaf(ab, R, fabsf(t.c[e])));
  }
  return m;
}

// True when some fragment of a set-up tetrahedron may need the exact path:
// with A the largest position term, C the largest evaluation term and B v the
// relative term over values v <= hmax (doubled: an edge within its bound of
// the minimum can hold up to about twice the minimum's value), some v has
// A + 2 B v + C > kFragTol max(v, sigma). Below sigma that needs
// A + 2 B min(hmax, sigma) + C > kFragTol sigma; above it, 2 B >= kFragTol.
__device__ __forceinline__ bool may_need_exact(const TetRaster& t, float sigma_units, float delta) {
  const float stmax = fmaxf(fmaxf(t.st[0], t.st[1]), fmaxf(t.st[2], t.st[3]));
  const float R = fmaxf(fmaxf(fabsf(t.xmin), fabsf(t.xmax)), fmaxf(fabsf(t.ymin), fabsf(t.ymax)));
  const float A = max_edge_slope(t) * delta * t.vscale, B = stmax * kFragErr;
  const float C = max_eval_error(t, R) * t.vscale;
  // written so that a non-finite coefficient (an extreme sliver) also flags
  return !(A + 2.0f * B * fminf(t.hmax, sigma_units) + C <= kFragTol * sigma_units) || !(B < 0.25f) ||
         (t.hmax > sigma_units && 2.0f * B >= kFragTol);
}

// True when the vertex uncertainty could move a pixel whose value matters
// across the FP32 hull boundary (steep thin slivers): such a tetrahedron has
// its whole bounding box visited.
__device__ __forceinline__ bool may_miss_fragments(const TetRaster& t, float sigma_units, float delta) {
  return !(max_edge_slope(t) * delta * t.vscale <= kFragTol * sigma_units);
}

// Bound e_e of one edge function's FP32 value f at pixel (X, Y); 0 for an
// unused slot (a = b = 0, a constant large c).
__device__ __forceinline__ float edge_error(float f, float a, float b, float c, float st, float X, float Y,
                                            float delta) {
  const float ab = fabsf(a) + fabsf(b);
  if (ab == 0.0f) return 0.0f;
  return fmaf(ab, delta, fmaf(kFragErr * st, fabsf(f), kEvalErr * (fabsf(a * X) + fabsf(b * Y) + fabsf(c))));
}

// Exact-path decision for one candidate pixel of a flagged tetrahedron: f the
// four edge functions at pixel (X, Y), a, b, c, st their coefficients and
// steepness, dvdT the perspective factor (1 orthographic), v the FP32 value.
__device__ __forceinline__ bool fragment_needs_exact(float f0, float f1, float f2, float f3, float4 a, float4 b,
                                                     float4 c, float4 st, float X, float Y, float delta, float dvdT,
                                                     float v, float sigma_units) {
  const float e0 = edge_error(f0, a.x, b.x, c.x, st.x, X, Y, delta);
  const float e1 = edge_error(f1, a.y, b.y, c.y, st.y, X, Y, delta);
  const float e2 = edge_error(f2, a.z, b.z, c.z, st.z, X, Y, delta);
  const float e3 = edge_error(f3, a.w, b.w, c.w, st.w, X, Y, delta);
  if (f0 != f0 || f1 != f1 || f2 != f2 || f3 != f3) return true;  // non-finite edge function: evaluate exactly
  const float lo = fminf(fminf(f0 - e0, f1 - e1), fminf(f2 - e2, f3 - e3));
  const float hi = fminf(fminf(f0 + e0, f1 + e1), fminf(f2 + e2, f3 + e3));
  if (!(hi > 0.0f) && hi == hi) return false;  // outside for certain
  const float T = fmaxf(fminf(fminf(f0, f1), fminf(f2, f3)), 0.0f);
  const float dev = fmaxf(T - fmaxf(lo, 0.0f), fmaxf(hi, 0.0f) - T);
  // written so that a non-finite bound also takes the exact path
  return !(dev * dvdT <= kFragTol * fmaxf(v, sigma_units));
}

// Number of periodic copies: shift range s in [s0, s1] such that the span
// [a + s P, b + s P] overlaps [lo, hi].
__device__ __forceinline__ void shift_range(float a, float b, float lo, float hi, float P, bool wrap, int& s0,
                                            int& s1) {
  if (!wrap) { s0 = 0; s1 = 0; return; }
  s0 = (int)ceilf((lo - b) / P);
  s1 = (int)floorf((hi - a) / P);
}

}  // namespace lt
