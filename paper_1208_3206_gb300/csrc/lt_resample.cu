// lt_resample.cu -- resampling of the tetrahedral tessellation onto a
// periodic n x n x n grid (Sec. 4.3, Eq. 10-12) and the stream-count field
// (Sec. 3.2).
//
// Cell (a, b, c) of edge g = box / n receives, from every tetrahedron t,
// q_t times the length of the part of the cell's central line along z
// (x = (a + 1/2) g, y = (b + 1/2) g) that lies inside t and inside the
// cell's slab [c g, (c + 1) g): the slab-wise form of the paper's
// resampling, in which each slab is a projection of the tetrahedra clipped
// to that slab. q_t = rho_t = m / |V_t| (Eq. 3) gives rho dl, the paper's
// estimate of the cell's mass over its face area; q_t = 1 gives the summed
// stream length, which over g is the mean number of streams on the line.
//
// The columns are the pixels of an orthographic view along z over the
// periodic box window, so the project-and-bin pass of lt_bin.cu lists each
// screen tile's cubes. One CTA per tile; each warp takes 32 of the tile's
// tetrahedra at a time:
//   * one lane per tetrahedron forms its four vertices in FP64, relative to
//     its cube's Lagrangian corner (lattice offsets plus minimum-image
//     displacements), its signed volume (Eq. 9), its outward face planes
//     (with the reciprocal of each plane's z slope) and the columns its
//     bounding box reaches, and leaves them in shared memory;
//   * then every (tetrahedron, periodic copy) in turn is walked by the whole
//     warp, 32 columns of the tile at a time: the interval of z where the
//     column's line is inside all four half-spaces, the exact entry and exit
//     points, in FP64;
//   * the interval's overlap with every slab it crosses, times q_t, added to
//     the cell as a 64-bit fixed-point integer with a global atomic. Integer
//     sums do not depend on the order of the adds, so the grid is bitwise
//     reproducible.
// A second kernel converts the integer grid to float.
#include "lt_internal.h"

namespace lt {

struct ResampleArgs {
  Lattice L;
  const FrameDev* frame;  // orthographic view along z over the box window, n x n pixels
  const unsigned long long* off;
  const unsigned* list;
  unsigned long long list_cap;
  int n, weight, tile;
  double gs;           // cell edge box / n
  double m_tet;        // mass of one tetrahedron
  double inv_unit;     // accumulator units per (q x length)
  unsigned long long* acc;  // [n][n][n] fixed-point cells
  DevCounters* ctr;
};

constexpr int kResampleThreads = 128;

// One tetrahedron of the current batch, as the warp's lanes read it.
struct ResampleTet {
  double nx[4], ny[4], d[4], inz[4];  // face planes: inside when nx x + ny y + nz z <= d; inz = 1 / nz (0: vertical face)
  double q;                           // rho (density weighting) or 1
  double qx, qy, qz;                  // the cube's Lagrangian corner
  long long A0, A1, B0, B1;           // unwrapped columns whose line can meet the tetrahedron
  long long sa0, sb0;                 // first periodic copy reaching the tile
  int nsa, ncopies;                   // copies along x, and in all
};

__global__ void __launch_bounds__(kResampleThreads) k_resample(ResampleArgs a) {
  __shared__ ResampleTet tets[kResampleThreads];
  const FrameDev& F = *a.frame;
  const long long tg = blockIdx.x;
  const int T = a.tile;
  const int tyi = (int)(tg / F.tiles_x), txi = (int)(tg - (long long)tyi * F.tiles_x);
  const int tx0 = txi * T, ty0 = tyi * T;
  const int tx1 = min(tx0 + T, a.n) - 1, ty1 = min(ty0 + T, a.n) - 1;
  unsigned long long e0 = a.off[tg], e1 = a.off[tg + 1];
  if (e1 > a.list_cap) {
    if (threadIdx.x == 0) atomicOr(&a.ctr->errors, kErrCapacity);
    e0 = min(e0, a.list_cap);
    e1 = a.list_cap;
  }
  const long long ntet = 6LL * (long long)(e1 - e0);
  const long long soff = (long long)F.snapshot * a.L.n_particles;
  const int N = a.L.N, n = a.n;
  const double gs = a.gs, inv_gs = 1.0 / a.gs, h = (double)a.L.box / N;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  ResampleTet* wt = tets + warp * 32;
  unsigned long long n_int = 0, n_piece = 0;
  for (long long tb = (long long)warp * 32; tb < ntet; tb += (long long)nw * 32) {
    // ---- one tetrahedron per lane: FP64 planes and the columns it can reach
    const long long tau = tb + lane;
    int ncopies = 0;
    if (tau < ntet) {
      const unsigned long long li = e0 + (unsigned long long)(tau / 6);
      const int s = (int)(tau % 6);
      const long long cube = LT_IN_BOUNDS(li < e1, &a.ctr->errors) ? (long long)a.list[li] : 0;
      if (!tet_degenerate(a.L, F.snapshot, cube, s)) {  // zero volume: contributes nothing
        int i, j, k;
        cube_ijk(a.L, cube, i, j, k);
        bool ok = true;
        TetF64 t;
        tet_f64(a.L, soff, i, j, k, s, ok, t);
        if (ok && t.V != 0.0) {
          ResampleTet& r = wt[lane];
#pragma unroll
          for (int f = 0; f < 4; ++f) {
            r.nx[f] = t.n[f][0];
            r.ny[f] = t.n[f][1];
            r.d[f] = t.d[f];
            r.inz[f] = t.n[f][2] != 0.0 ? 1.0 / t.n[f][2] : 0.0;
          }
          r.q = a.weight == 0 ? a.m_tet / fabs(t.V) : 1.0;
          r.qx = i * h;
          r.qy = j * h;
          r.qz = k * h;
          double xmn = t.v[0][0], xmx = xmn, ymn = t.v[0][1], ymx = ymn;
#pragma unroll
          for (int c = 1; c < 4; ++c) {
            xmn = fmin(xmn, t.v[c][0]); xmx = fmax(xmx, t.v[c][0]);
            ymn = fmin(ymn, t.v[c][1]); ymx = fmax(ymx, t.v[c][1]);
          }
          r.A0 = (long long)ceil((r.qx + xmn) * inv_gs - 0.5);
          r.A1 = (long long)floor((r.qx + xmx) * inv_gs - 0.5);
          r.B0 = (long long)ceil((r.qy + ymn) * inv_gs - 0.5);
          r.B1 = (long long)floor((r.qy + ymx) * inv_gs - 0.5);
          if (r.A0 <= r.A1 && r.B0 <= r.B1) {
            // periodic copies of the column ranges that reach the tile
            const long long sa0 = (long long)floor((double)(r.A0 - tx1 + n - 1) / n);
            const long long sa1 = min((long long)floor((double)(r.A1 - tx0) / n), sa0 + 7);
            const long long sb0 = (long long)floor((double)(r.B0 - ty1 + n - 1) / n);
            const long long sb1 = min((long long)floor((double)(r.B1 - ty0) / n), sb0 + 7);
            r.sa0 = sa0;
            r.sb0 = sb0;
            r.nsa = (int)max(0LL, sa1 - sa0 + 1);
            r.ncopies = r.nsa * (int)max(0LL, sb1 - sb0 + 1);
            ncopies = r.ncopies;
          }
        }
      }
    }
    __syncwarp();
    // ---- every (tetrahedron, copy) in turn: the warp's lanes take its columns
    unsigned todo = __ballot_sync(0xffffffffu, ncopies > 0);
    while (todo) {
      const int src = __ffs(todo) - 1;
      todo &= todo - 1u;
      const ResampleTet& r = wt[src];
      for (int cp = 0; cp < r.ncopies; ++cp) {
        const long long sa = r.sa0 + cp % r.nsa, sb = r.sb0 + cp / r.nsa;
        const long long al = max(r.A0 - sa * n, (long long)tx0), ah = min(r.A1 - sa * n, (long long)tx1);
        const long long bl = max(r.B0 - sb * n, (long long)ty0), bh = min(r.B1 - sb * n, (long long)ty1);
        if (al > ah || bl > bh) continue;
        const int wa = (int)(ah - al + 1);
        const int nc = wa * (int)(bh - bl + 1);
        for (int p = lane; p < nc; p += 32) {
          const int rb = p / wa;
          const long long aa = al + (p - rb * wa), bb = bl + rb;
          // the column's line (x, y, z), relative to the cube's corner
          const double x = ((double)(aa + sa * n) + 0.5) * gs - r.qx;
          const double y = ((double)(bb + sb * n) + 0.5) * gs - r.qy;
          double z_in = -1e300, z_out = 1e300;
          bool empty = false;
#pragma unroll
          for (int f = 0; f < 4; ++f) {
            const double rr = fma(-r.ny[f], y, fma(-r.nx[f], x, r.d[f]));
            const double iz = r.inz[f];
            if (iz > 0.0) z_out = fmin(z_out, rr * iz);
            else if (iz < 0.0) z_in = fmax(z_in, rr * iz);
            else if (rr < 0.0) empty = true;
          }
          if (empty || !(z_out > z_in)) continue;
          ++n_int;
          const double zl = r.qz + z_in, zh = r.qz + z_out;
          long long c = (long long)floor(zl * inv_gs);
          for (int guard = 0; guard < 1 << 20 && (double)c * gs < zh; ++guard, ++c) {
            const double lo = fmax(zl, (double)c * gs), hi = fmin(zh, (double)(c + 1) * gs);
            if (!(hi > lo)) continue;
            ++n_piece;
            const double u = r.q * (hi - lo) * a.inv_unit;
            const long long cw = ((c % n) + n) % n;
            unsigned long long* cell = a.acc + ((cw * n + bb) * n + aa);
            if (u < 9.2e18) {
              const unsigned long long add = (unsigned long long)__double2ull_rn(u);
              if (add) {
                const unsigned long long old = atomicAdd(cell, add);
                if (old > ~0ull - add) {
                  atomicOr(&a.ctr->errors, kErrRange);
                  atomicAdd(&a.ctr->range_overflow, 1ull);
                }
              }
            } else {
              atomicOr(&a.ctr->errors, kErrRange);
              atomicAdd(&a.ctr->range_overflow, 1ull);
            }
          }
        }
      }
    }
    __syncwarp();
  }
  const unsigned long long wi = __reduce_add_sync(0xffffffffu, (unsigned)n_int);
  const unsigned long long wp = __reduce_add_sync(0xffffffffu, (unsigned)n_piece);
  if (lane == 0) {
    if (wi) atomicAdd(&a.ctr->resample_intervals, wi);
    if (wp) atomicAdd(&a.ctr->resample_pieces, wp);
  }
}

__global__ void k_resample_finalize(const unsigned long long* __restrict__ acc, long long cells, double unit,
                                    float* __restrict__ out) {
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < cells; p += (long long)gridDim.x * blockDim.x)
    out[p] = (float)((double)acc[p] * unit);
}

cudaError_t launch_resample(const Lattice& L, const FrameDev* d_frame, long long n_tiles, int tile,
                            const unsigned long long* d_off, const unsigned* d_list, unsigned long long list_cap, int n,
                            int weight, double m_tet, double unit, unsigned long long* d_acc, float* d_out,
                            DevCounters* ctr, cudaStream_t s) {
  const long long cells = (long long)n * n * n;
  cudaError_t e = cudaMemsetAsync(d_acc, 0, sizeof(unsigned long long) * cells, s);
  if (e != cudaSuccess) return e;
  ResampleArgs a;
  a.L = L;
  a.frame = d_frame;
  a.off = d_off;
  a.list = d_list;
  a.list_cap = list_cap;
  a.n = n;
  a.weight = weight;
  a.tile = tile;
  a.gs = (double)L.box / n;
  a.m_tet = m_tet;
  a.inv_unit = 1.0 / unit;
  a.acc = d_acc;
  a.ctr = ctr;
  k_resample<<<(unsigned)n_tiles, kResampleThreads, 0, s>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  long long blocks = (cells + 255) / 256;
  if (blocks > 152LL * 32) blocks = 152LL * 32;
  k_resample_finalize<<<(unsigned)blocks, 256, 0, s>>>(d_acc, cells, unit, d_out);
  return cudaGetLastError();
}

}  // namespace lt
