// lt_build.cu -- per-tetrahedron signed volume (Eq. 9) and density (Eq. 3)
// for every cube of every snapshot, tetrahedra generated on the fly from the
// lattice index (Sec. 3.1, Sec. 4.1). FP32 determinant on local edge vectors,
// recomputed in FP64 when |V| falls below 1e-6 of a lattice cell (sheet-like
// tetrahedra at caustics).
#include "lt_internal.h"

namespace lt {

__device__ __forceinline__ void warp_add_u64(unsigned long long* dst, unsigned v) {
  const unsigned tot = __reduce_add_sync(0xffffffffu, v);
  if ((threadIdx.x & 31) == 0 && tot) atomicAdd(dst, (unsigned long long)tot);
}

__global__ void __launch_bounds__(256) k_build_tets(Lattice L, int n_snap, double m, float* __restrict__ rho_out,
                                                     unsigned char* __restrict__ degen, DevCounters* __restrict__ ctr) {
  const long long ncube = L.n_particles;
  const long long total = ncube * n_snap;
  // FP32 determinant error is about 3 * 2^-24 * |e|^3 / |V| relative; below
  // 0.1 h^3 (0.6 of an undeformed tetrahedron) that could exceed 1e-5, so the
  // volume is recomputed in FP64 from the exact displacements
  const float thr = 0.1f * L.h * L.h * L.h;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < total; base += (long long)gridDim.x * blockDim.x) {
    const long long gid = base + threadIdx.x;
    unsigned n_nonfinite = 0, n_degen = 0, n_fb = 0, n_inv = 0;
    if (gid < total) {
      const int snap = (int)(gid / ncube);
      const long long cube = gid - (long long)snap * ncube;
      const int N = L.N;
      const int i = (int)(cube % N), j = (int)((cube / N) % N), k = (int)(cube / ((long long)N * N));
      const long long soff = (long long)snap * L.n_particles;
      float3 d[8];
      bool ok0 = true, ok = true;
      d[0] = load_disp(L, soff, i, j, k, 0, ok0);
#pragma unroll
      for (int n = 1; n < 8; ++n) d[n] = load_disp(L, soff, i, j, k, n, ok);
      // exact displacement in FP64 (for the fallback): the FP32 one rounds
      // when |d| exceeds the position's own precision range
      auto disp64 = [&](int n, int c) -> double {
        const int ci = (i + (n & 1)) % N, cj = (j + ((n >> 1) & 1)) % N, ck = (k + ((n >> 2) & 1)) % N;
        if (L.fmt != 0) return (double)(c == 0 ? d[n].x : c == 1 ? d[n].y : d[n].z);  // exact already
        const float4 p4 = __ldg(reinterpret_cast<const float4*>(L.pos) + soff + particle_id(ci, cj, ck, N));
        const double pv = (double)(c == 0 ? p4.x : c == 1 ? p4.y : p4.z);
        const int im = c == 0 ? ci : c == 1 ? cj : ck;
        double dd = pv - (double)im * (double)L.h;
        const double bx = (double)L.box;
        if (dd > 0.5 * bx) dd -= bx;
        else if (dd < -0.5 * bx) dd += bx;
        return dd;
      };
      n_nonfinite = ok0 ? 0u : 1u;  // each particle is corner 0 of exactly one cube
      unsigned zero_mask = 0;
#pragma unroll
      for (int s = 0; s < 6; ++s) {
        const int n0 = tet_corner(s, 0), n1 = tet_corner(s, 1), n2 = tet_corner(s, 2), n3 = tet_corner(s, 3);
        // edge vectors: displacement differences plus exact lattice offsets
        const float h = L.h;
        const float ax = (d[n1].x - d[n0].x) + (float)((n1 & 1) - (n0 & 1)) * h;
        const float ay = (d[n1].y - d[n0].y) + (float)(((n1 >> 1) & 1) - ((n0 >> 1) & 1)) * h;
        const float az = (d[n1].z - d[n0].z) + (float)(((n1 >> 2) & 1) - ((n0 >> 2) & 1)) * h;
        const float bx = (d[n2].x - d[n0].x) + (float)((n2 & 1) - (n0 & 1)) * h;
        const float by = (d[n2].y - d[n0].y) + (float)(((n2 >> 1) & 1) - ((n0 >> 1) & 1)) * h;
        const float bz = (d[n2].z - d[n0].z) + (float)(((n2 >> 2) & 1) - ((n0 >> 2) & 1)) * h;
        const float cx = (d[n3].x - d[n0].x) + (float)((n3 & 1) - (n0 & 1)) * h;
        const float cy = (d[n3].y - d[n0].y) + (float)(((n3 >> 1) & 1) - ((n0 >> 1) & 1)) * h;
        const float cz = (d[n3].z - d[n0].z) + (float)(((n3 >> 2) & 1) - ((n0 >> 2) & 1)) * h;
        const float V = (ax * (by * cz - bz * cy) + ay * (bz * cx - bx * cz) + az * (bx * cy - by * cx)) * (1.0f / 6.0f);
        double Vd = (double)V;
        if (fabsf(V) < thr) {
          const double hd = (double)h;
          const double d0x = disp64(n0, 0), d0y = disp64(n0, 1), d0z = disp64(n0, 2);
          const double eax = (disp64(n1, 0) - d0x) + ((n1 & 1) - (n0 & 1)) * hd;
          const double eay = (disp64(n1, 1) - d0y) + (((n1 >> 1) & 1) - ((n0 >> 1) & 1)) * hd;
          const double eaz = (disp64(n1, 2) - d0z) + (((n1 >> 2) & 1) - ((n0 >> 2) & 1)) * hd;
          const double ebx = (disp64(n2, 0) - d0x) + ((n2 & 1) - (n0 & 1)) * hd;
          const double eby = (disp64(n2, 1) - d0y) + (((n2 >> 1) & 1) - ((n0 >> 1) & 1)) * hd;
          const double ebz = (disp64(n2, 2) - d0z) + (((n2 >> 2) & 1) - ((n0 >> 2) & 1)) * hd;
          const double ecx = (disp64(n3, 0) - d0x) + ((n3 & 1) - (n0 & 1)) * hd;
          const double ecy = (disp64(n3, 1) - d0y) + (((n3 >> 1) & 1) - ((n0 >> 1) & 1)) * hd;
          const double ecz = (disp64(n3, 2) - d0z) + (((n3 >> 2) & 1) - ((n0 >> 2) & 1)) * hd;
          Vd = (eax * (eby * ecz - ebz * ecy) + eay * (ebz * ecx - ebx * ecz) + eaz * (ebx * ecy - eby * ecx)) / 6.0;
          ++n_fb;
        }
        if (Vd == 0.0) {
          ++n_degen;
          zero_mask |= 1u << s;
        }
        if (Vd > 0.0) ++n_inv;
        if (rho_out) {
          const float rho = (Vd == 0.0 || !(ok && ok0)) ? 0.0f : (float)(m / fabs(Vd));
          rho_out[(long long)snap * 6 * ncube + 6 * cube + s] = rho;
        }
      }
      degen[gid] = (unsigned char)zero_mask;
    }
    warp_add_u64(&ctr->nonfinite, n_nonfinite);
    warp_add_u64(&ctr->degenerate, n_degen);
    warp_add_u64(&ctr->fp64_fallbacks, n_fb);
    warp_add_u64(&ctr->inverted, n_inv);
    if (n_nonfinite) atomicOr(&ctr->errors, kErrNonFinite);
  }
}

cudaError_t launch_build_tets(const Lattice& L, int n_snap, double m, float* rho_out, unsigned char* degen,
                              DevCounters* ctr, cudaStream_t s) {
  const long long total = L.n_particles * n_snap;
  long long blocks = (total + 255) / 256;
  if (blocks > 152LL * 64) blocks = 152LL * 64;
  if (blocks < 1) blocks = 1;
  k_build_tets<<<(unsigned)blocks, 256, 0, s>>>(L, n_snap, m, rho_out, degen, ctr);
  return cudaGetLastError();
}

}  // namespace lt
