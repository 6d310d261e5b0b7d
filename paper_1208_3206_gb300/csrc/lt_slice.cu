// lt_slice.cu -- the total density of overlapping streams (Eq. 4) and the
// number of streams (Sec. 3.2) on a plane z = z0 of the periodic box, at the
// centres of an n x n grid over the box: the paper's 2D density slices
// through the tessellation.
//
// A point's total density is the sum of rho_t = m / |V_t| (Eq. 3) over the
// tetrahedra t that contain it (any periodic copy); its stream count is the
// number of them. One thread per lattice cube: a cube whose z-range does not
// reach the plane (or a periodic copy of it) returns at once. For each of the
// other cubes' six tetrahedra, in FP64 relative to the cube's Lagrangian
// corner:
//   * the cross-section with the plane, bounded by the crossings of the six
//     edges, gives the slice points to test;
//   * each candidate point is inside when it lies on the inner side of all
//     four face planes (a point on a face counts, like for the closed
//     tetrahedron);
//   * q_t is added to the point's 64-bit fixed-point sum with a global
//     integer atomic, so the slice does not depend on the order of the adds.
// A second kernel converts the sums to float.
#include "lt_internal.h"

namespace lt {

struct SliceArgs {
  Lattice L;
  int snapshot, n, weight;
  double z0, gs, m_tet, inv_unit;
  unsigned long long* acc;  // [n][n] fixed-point sums
  DevCounters* ctr;
};

__global__ void __launch_bounds__(128) k_slice(SliceArgs a) {
  const int N = a.L.N, n = a.n;
  const double h = (double)a.L.box / N, box = (double)a.L.box, gs = a.gs;
  const long long soff = (long long)a.snapshot * a.L.n_particles;
  for (long long cube = (long long)blockIdx.x * blockDim.x + threadIdx.x; cube < a.L.n_particles;
       cube += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    cube_ijk(a.L, cube, i, j, k);
    // the eight corners in FP64, relative to the cube's Lagrangian corner
    double cv[8][3];
    bool ok = true;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int ca = c & 1, cb = (c >> 1) & 1, cc = (c >> 2) & 1;
      const int ii = i + ca, jj = j + cb, kk = k + cc;
      const int im = ii == N ? 0 : ii, jm = jj == N ? 0 : jj, km = kk == N ? 0 : kk;
      double dd[3];
      if (a.L.fmt == 0) {
        const float4 p = __ldg(reinterpret_cast<const float4*>(a.L.pos) + soff + particle_id(im, jm, km, N));
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
        const float3 df = load_disp(a.L, soff, i, j, k, c, ok);
        dd[0] = df.x; dd[1] = df.y; dd[2] = df.z;
      }
      cv[c][0] = ca * h + dd[0];
      cv[c][1] = cb * h + dd[1];
      cv[c][2] = cc * h + dd[2];
    }
    if (!ok) continue;
    double zmn = cv[0][2], zmx = cv[0][2];
#pragma unroll
    for (int c = 1; c < 8; ++c) {
      zmn = fmin(zmn, cv[c][2]);
      zmx = fmax(zmx, cv[c][2]);
    }
    const double qx = i * h, qy = j * h, qz = k * h;
    // periodic copies of the plane that cross the cube
    const long long p0 = (long long)ceil((qz + zmn - a.z0) / box), p1 = (long long)floor((qz + zmx - a.z0) / box);
    if (p0 > p1) continue;
    const unsigned zmask = a.L.degen ? (unsigned)__ldg(a.L.degen + soff + cube) : 0u;
    for (int s = 0; s < 6; ++s) {
      if ((zmask >> s) & 1u) continue;  // zero volume: contributes nothing
      double v[4][3];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int cn = tet_corner_dyn(s, c);
        v[c][0] = cv[cn][0]; v[c][1] = cv[cn][1]; v[c][2] = cv[cn][2];
      }
      const double e1[3] = {v[1][0] - v[0][0], v[1][1] - v[0][1], v[1][2] - v[0][2]};
      const double e2[3] = {v[2][0] - v[0][0], v[2][1] - v[0][1], v[2][2] - v[0][2]};
      const double e3[3] = {v[3][0] - v[0][0], v[3][1] - v[0][1], v[3][2] - v[0][2]};
      const double V = (e1[0] * (e2[1] * e3[2] - e2[2] * e3[1]) + e1[1] * (e2[2] * e3[0] - e2[0] * e3[2]) +
                        e1[2] * (e2[0] * e3[1] - e2[1] * e3[0])) / 6.0;
      if (V == 0.0) continue;
      const double q = a.weight == 0 ? a.m_tet / fabs(V) : 1.0;
      double nrm[4][3], off[4];
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
        nrm[f][0] = nn[0]; nrm[f][1] = nn[1]; nrm[f][2] = nn[2];
        off[f] = nn[0] * A[0] + nn[1] * A[1] + nn[2] * A[2];
      }
      for (long long pc = p0; pc <= min(p1, p0 + 3); ++pc) {
        const double zr = a.z0 + (double)pc * box - qz;  // the plane, relative to the cube
        // bounding box of the cross-section: vertices on the plane and the
        // crossings of the edges that span it
        double xmn = 1e300, xmx = -1e300, ymn = 1e300, ymx = -1e300;
#pragma unroll
        for (int c1 = 0; c1 < 4; ++c1) {
          if (v[c1][2] == zr) {
            xmn = fmin(xmn, v[c1][0]); xmx = fmax(xmx, v[c1][0]);
            ymn = fmin(ymn, v[c1][1]); ymx = fmax(ymx, v[c1][1]);
          }
#pragma unroll
          for (int c2 = c1 + 1; c2 < 4; ++c2) {
            const double za = v[c1][2] - zr, zb = v[c2][2] - zr;
            if ((za < 0.0 && zb > 0.0) || (za > 0.0 && zb < 0.0)) {
              const double t = za / (za - zb);
              const double x = v[c1][0] + t * (v[c2][0] - v[c1][0]), y = v[c1][1] + t * (v[c2][1] - v[c1][1]);
              xmn = fmin(xmn, x); xmx = fmax(xmx, x);
              ymn = fmin(ymn, y); ymx = fmax(ymx, y);
            }
          }
        }
        if (!(xmn <= xmx)) continue;
        // slice points (unwrapped indices) whose centre can lie in the
        // cross-section; the bounds are widened by a hair for rounding
        const double eps = 1e-9;
        const long long A0 = (long long)ceil((qx + xmn) / gs - 0.5 - eps), A1 = (long long)floor((qx + xmx) / gs - 0.5 + eps);
        const long long B0 = (long long)ceil((qy + ymn) / gs - 0.5 - eps), B1 = (long long)floor((qy + ymx) / gs - 0.5 + eps);
        for (long long bb = B0; bb <= min(B1, B0 + 4LL * n); ++bb) {
          const double y = ((double)bb + 0.5) * gs - qy;
          const long long bw = ((bb % n) + n) % n;
          for (long long aa = A0; aa <= min(A1, A0 + 4LL * n); ++aa) {
            const double x = ((double)aa + 0.5) * gs - qx;
            bool inside = true;
#pragma unroll
            for (int f = 0; f < 4; ++f)
              inside = inside && (nrm[f][0] * x + nrm[f][1] * y + nrm[f][2] * zr <= off[f]);
            if (!inside) continue;
            const long long aw = ((aa % n) + n) % n;
            const double u = q * a.inv_unit;
            unsigned long long* cell = a.acc + (bw * n + aw);
            if (u < 9.2e18) {
              const unsigned long long add = (unsigned long long)__double2ull_rn(u);
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
  }
}

__global__ void k_slice_finalize(const unsigned long long* __restrict__ acc, long long np, double unit,
                                 float* __restrict__ out) {
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (long long)gridDim.x * blockDim.x)
    out[p] = (float)((double)acc[p] * unit);
}

cudaError_t launch_slice(const Lattice& L, int snapshot, int n, int weight, double z0, double m_tet, double unit,
                         unsigned long long* d_acc, float* d_out, DevCounters* ctr, cudaStream_t s) {
  const long long np = (long long)n * n;
  cudaError_t e = cudaMemsetAsync(d_acc, 0, sizeof(unsigned long long) * np, s);
  if (e != cudaSuccess) return e;
  SliceArgs a;
  a.L = L;
  a.snapshot = snapshot;
  a.n = n;
  a.weight = weight;
  a.z0 = z0;
  a.gs = (double)L.box / n;
  a.m_tet = m_tet;
  a.inv_unit = 1.0 / unit;
  a.acc = d_acc;
  a.ctr = ctr;
  long long blocks = (L.n_particles + 127) / 128;
  if (blocks > 152LL * 64) blocks = 152LL * 64;
  k_slice<<<(unsigned)(blocks < 1 ? 1 : blocks), 128, 0, s>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  long long fb = (np + 255) / 256;
  if (fb > 152LL * 32) fb = 152LL * 32;
  k_slice_finalize<<<(unsigned)fb, 256, 0, s>>>(d_acc, np, unit, d_out);
  return cudaGetLastError();
}

}  // namespace lt
