// lt_bin.cu -- project-and-bin pass: for every (frame, cube) the screen
// tiles overlapped by the cube's projected bounding box; warp-aggregated
// per-tile counts (the count pass also keeps each cube's tile rectangle, so
// the scatter does not project again), a device exclusive scan, a scatter of
// cube ids into per-tile lists, and the (frame, tile) work list ordered by
// descending list length (bucketed by log2 of the length).
#include "lt_internal.h"

namespace lt {

// Tile intervals of one image axis touched by pixel span [p0, p1]; with a
// periodic window the span is wrapped, giving at most two intervals.
__device__ __forceinline__ int axis_tiles(int p0, int p1, int Wp, int T, int ntiles, bool wrap, int* lo, int* hi) {
  if (!wrap) {
    const int a = max(p0, 0), b = min(p1, Wp - 1);
    if (a > b) return 0;
    lo[0] = a / T; hi[0] = b / T;
    return 1;
  }
  if (p1 < p0) return 0;
  if (p1 - p0 + 1 >= Wp - T) {  // wide enough that wrapped copies could share a tile
    lo[0] = 0; hi[0] = ntiles - 1;
    return 1;
  }
  const int s = (int)floorf((float)p0 / (float)Wp);
  int q0 = p0 - s * Wp, q1 = p1 - s * Wp;
  if (q0 >= Wp) { q0 -= Wp; q1 -= Wp; }
  if (q0 < 0) { q0 += Wp; q1 += Wp; }
  if (q1 < Wp) {
    lo[0] = q0 / T; hi[0] = q1 / T;
    return 1;
  }
  lo[0] = q0 / T; hi[0] = ntiles - 1;
  lo[1] = 0; hi[1] = (q1 - Wp) / T;
  return 2;
}

__device__ __forceinline__ int clamp_pix(float v) { return (int)fminf(fmaxf(v, -1.0e9f), 1.0e9f); }

// Tiles of one cube: up to 2 x 2 rectangles of tiles.
struct CubeTiles {
  int nx, ny;
  int xlo[2], xhi[2], ylo[2], yhi[2];
  int cntx, cnty;
};

__device__ __forceinline__ bool cube_tiles(const Lattice& L, const FrameDev& F, long long cube, CubeTiles& ct,
                                           bool& finite_ok, bool& behind) {
  CubeProj P;
  bool projected;
  bool straddle = false;
  if (F.persp) projected = project_cube<true>(L, F, cube, P, finite_ok, &straddle);
  else projected = project_cube<false>(L, F, cube, P, finite_ok);
  behind = straddle;
  ct.cntx = ct.cnty = 0;
  if (!projected) return false;
  const float ax = P.axh + P.axl, ay = P.ayh + P.ayl;
  const int p0x = clamp_pix(ceilf(ax + P.xmin - 1e-3f)), p1x = clamp_pix(floorf(ax + P.xmax + 1e-3f));
  const int p0y = clamp_pix(ceilf(ay + P.ymin - 1e-3f)), p1y = clamp_pix(floorf(ay + P.ymax + 1e-3f));
  const bool wrap = F.wrap != 0;
  ct.nx = axis_tiles(p0x, p1x, F.W, F.tile, F.tiles_x, wrap, ct.xlo, ct.xhi);
  ct.ny = axis_tiles(p0y, p1y, F.H, F.tile, F.tiles_y, wrap, ct.ylo, ct.yhi);
  if (ct.nx == 0 || ct.ny == 0) return false;
  ct.cntx = (ct.xhi[0] - ct.xlo[0] + 1) + (ct.nx > 1 ? ct.xhi[1] - ct.xlo[1] + 1 : 0);
  ct.cnty = (ct.yhi[0] - ct.ylo[0] + 1) + (ct.ny > 1 ? ct.yhi[1] - ct.ylo[1] + 1 : 0);
  return true;
}

__device__ __forceinline__ long long cube_tile_at(const CubeTiles& ct, const FrameDev& F, int r) {
  const int iy = r / ct.cntx, ix = r - iy * ct.cntx;
  const int n0x = ct.xhi[0] - ct.xlo[0] + 1, n0y = ct.yhi[0] - ct.ylo[0] + 1;
  const int tx = ix < n0x ? ct.xlo[0] + ix : ct.xlo[1] + (ix - n0x);
  const int ty = iy < n0y ? ct.ylo[0] + iy : ct.ylo[1] + (iy - n0y);
  return F.tile_base + (long long)ty * F.tiles_x + tx;
}

// The count pass keeps each (frame, cube)'s tiles as one 32-bit descriptor
// so that the scatter pass need not project the cube again: first tile x and
// y (12 bits each, below 4095) and the tile counts minus one (4 bits each).
// A cube with no tiles, and one whose tiles do not fit the form (two
// periodic intervals, more than 16 tiles along an axis), get a sentinel;
// the scatter projects the latter again.
constexpr unsigned kDescNone = 0xFFFFFFFFu, kDescAgain = 0xFFFFFFFEu;  // both have the y field 0xFFF

__device__ __forceinline__ unsigned encode_tiles(bool have, const CubeTiles& ct) {
  if (!have) return kDescNone;
  if (ct.nx != 1 || ct.ny != 1) return kDescAgain;
  const int cx = ct.xhi[0] - ct.xlo[0] + 1, cy = ct.yhi[0] - ct.ylo[0] + 1;
  if (ct.xlo[0] >= 4095 || ct.ylo[0] >= 4095 || cx > 16 || cy > 16) return kDescAgain;
  return (unsigned)ct.xlo[0] | ((unsigned)ct.ylo[0] << 12) | ((unsigned)(cx - 1) << 24) | ((unsigned)(cy - 1) << 28);
}

__device__ __forceinline__ void decode_tiles(unsigned d, CubeTiles& ct) {
  ct.nx = ct.ny = 1;
  ct.xlo[0] = (int)(d & 0xFFFu);
  ct.ylo[0] = (int)((d >> 12) & 0xFFFu);
  ct.cntx = (int)((d >> 24) & 15u) + 1;
  ct.cnty = (int)(d >> 28) + 1;
  ct.xhi[0] = ct.xlo[0] + ct.cntx - 1;
  ct.yhi[0] = ct.ylo[0] + ct.cnty - 1;
}

template <bool SCATTER>
__global__ void __launch_bounds__(256) k_bin(Lattice L, const FrameDev* __restrict__ frames,
                                             const unsigned long long* __restrict__ off, unsigned* __restrict__ cnt,
                                             unsigned* __restrict__ list, unsigned long long capacity,
                                             unsigned* __restrict__ desc, DevCounters* __restrict__ ctr) {
  const FrameDev& F = frames[blockIdx.y];
  const long long ncube = L.n_particles;
  const unsigned lane = threadIdx.x & 31;
  unsigned* fdesc = desc ? desc + (long long)blockIdx.y * ncube : nullptr;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < ncube; base += (long long)gridDim.x * blockDim.x) {
    const long long cube = base + threadIdx.x;
    CubeTiles ct;
    bool finite_ok = true, behind = false;
    bool have = false;
    if (cube < ncube) {
      if (SCATTER && fdesc) {
        const unsigned d = fdesc[cube];
        if (d == kDescAgain) {
          have = cube_tiles(L, F, cube, ct, finite_ok, behind);
        } else if (d != kDescNone) {
          decode_tiles(d, ct);
          have = true;
        }
      } else {
        // hybrid rendering: far cubes are drawn as splats, not binned
        have = !cube_far(L, F, cube) && cube_tiles(L, F, cube, ct, finite_ok, behind);
        if (!SCATTER && fdesc) fdesc[cube] = encode_tiles(have, ct);
      }
    }
    if (!SCATTER) {
      const unsigned nb = __reduce_add_sync(0xffffffffu, behind ? 1u : 0u);
      if (lane == 0 && nb) {
        atomicAdd(&ctr->behind_eye, (unsigned long long)nb);
        atomicOr(&ctr->errors, kErrBehindEye);
      }
      if (!finite_ok) atomicOr(&ctr->errors, kErrNonFinite);
    }
    const int mine = have ? ct.cntx * ct.cnty : 0;
    for (int r = 0;; ++r) {
      const bool act = r < mine;
      const unsigned am = __ballot_sync(0xffffffffu, act);
      if (!am) break;
      if (act) {
        const long long t = cube_tile_at(ct, F, r);
        const unsigned grp = __match_any_sync(am, (unsigned long long)t);
        const int leader = __ffs(grp) - 1;
        const unsigned rank = __popc(grp & ((1u << lane) - 1u));
        if (!SCATTER) {
          if ((int)lane == leader) atomicAdd(&cnt[t], (unsigned)__popc(grp));
        } else {
          unsigned b = 0;
          if ((int)lane == leader) b = atomicAdd(&cnt[t], (unsigned)__popc(grp));
          b = __shfl_sync(grp, b, leader);
          const unsigned long long pos = off[t] + b + rank;
          if (pos < capacity) list[pos] = (unsigned)cube;
          else atomicOr(&ctr->errors, kErrCapacity);
        }
      }
    }
  }
}

static unsigned bin_blocks(long long ncube) {
  long long b = (ncube + 255) / 256;
  if (b > 4096) b = 4096;
  return (unsigned)(b < 1 ? 1 : b);
}

cudaError_t launch_bin_count(const Lattice& L, const FrameDev* d_frames, int n_frames, unsigned* d_count,
                             unsigned* d_desc, DevCounters* ctr, cudaStream_t s) {
  dim3 grid(bin_blocks(L.n_particles), n_frames);
  k_bin<false><<<grid, 256, 0, s>>>(L, d_frames, nullptr, d_count, nullptr, 0, d_desc, ctr);
  return cudaGetLastError();
}

cudaError_t launch_bin_scatter(const Lattice& L, const FrameDev* d_frames, int n_frames,
                               const unsigned long long* d_off, unsigned* d_cursor, unsigned* d_list,
                               unsigned long long capacity, unsigned* d_desc, DevCounters* ctr, cudaStream_t s) {
  dim3 grid(bin_blocks(L.n_particles), n_frames);
  k_bin<true><<<grid, 256, 0, s>>>(L, d_frames, d_off, d_cursor, d_list, capacity, d_desc, ctr);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Exclusive scan of 32-bit counts into 64-bit offsets (n + 1 entries, the last
// one the total). Block of 1024 threads x 4 items; block totals are scanned
// by the same kernel recursively.

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr long long kScanTile = kScanThreads * kScanItems;

template <typename T>
__device__ __forceinline__ unsigned long long block_exclusive_scan(unsigned long long v, unsigned long long* warp_sums,
                                                                   unsigned long long& total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned long long x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[wid] = x;
  __syncthreads();
  if (wid == 0) {
    unsigned long long w = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0ull;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    warp_sums[lane] = w;
  }
  __syncthreads();
  total = warp_sums[(blockDim.x >> 5) - 1];
  const unsigned long long before = wid > 0 ? warp_sums[wid - 1] : 0ull;
  return before + x - v;
}

template <typename TIn>
__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const TIn* __restrict__ in, long long n,
                                                             unsigned long long* __restrict__ out,
                                                             unsigned long long* __restrict__ block_sums) {
  __shared__ unsigned long long ws[32];
  const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
  unsigned long long v[kScanItems];
  unsigned long long sum = 0;
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    v[q] = (base + q < n) ? (unsigned long long)in[base + q] : 0ull;
    sum += v[q];
  }
  unsigned long long total;
  unsigned long long ex = block_exclusive_scan<unsigned long long>(sum, ws, total);
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    if (base + q < n) out[base + q] = ex;
    ex += v[q];
  }
  if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

__global__ void k_scan_add(unsigned long long* __restrict__ out, long long n,
                           const unsigned long long* __restrict__ block_off) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += block_off[i / kScanTile];
}

__global__ void k_scan_total(unsigned long long* __restrict__ out, long long n, const unsigned* __restrict__ cnt) {
  if (threadIdx.x == 0 && blockIdx.x == 0) out[n] = (n > 0 ? out[n - 1] + cnt[n - 1] : 0ull);
}

size_t scan_tmp_words(long long n) {
  size_t words = 0;
  long long m = n;
  while (m > 1) {
    const long long nb = (m + kScanTile - 1) / kScanTile;
    words += 2 * nb + 2;
    m = nb;
  }
  return words + 4;
}

// Recursive exclusive scan of a 64-bit array (used for the block totals).
static cudaError_t scan_u64(const unsigned long long* in, long long n, unsigned long long* out,
                            unsigned long long* tmp, cudaStream_t s) {
  const long long nb = (n + kScanTile - 1) / kScanTile;
  unsigned long long* sums = tmp;
  unsigned long long* sums_off = tmp + nb + 1;
  k_scan_tiles<unsigned long long><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, out, sums);
  if (nb > 1) {
    cudaError_t e = scan_u64(sums, nb, sums_off, tmp + 2 * nb + 2, s);
    if (e != cudaSuccess) return e;
    k_scan_add<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out, n, sums_off);
  }
  return cudaGetLastError();
}

cudaError_t launch_scan(const unsigned* d_count, long long n, unsigned long long* d_off, unsigned long long* d_tmp,
                        cudaStream_t s) {
  const long long nb = (n + kScanTile - 1) / kScanTile;
  unsigned long long* sums = d_tmp;
  unsigned long long* sums_off = d_tmp + nb + 1;
  k_scan_tiles<unsigned><<<(unsigned)nb, kScanThreads, 0, s>>>(d_count, n, d_off, sums);
  if (nb > 1) {
    cudaError_t e = scan_u64(sums, nb, sums_off, d_tmp + 2 * nb + 2, s);
    if (e != cudaSuccess) return e;
    k_scan_add<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(d_off, n, sums_off);
  }
  k_scan_total<<<1, 32, 0, s>>>(d_off, n, d_count);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Work list: every global tile, longest lists first (33 log2 buckets).

constexpr int kBuckets = 34;

__device__ __forceinline__ int len_bucket(unsigned long long len) {
  // bucket 0 holds the longest lists; empty tiles go last
  if (len == 0) return kBuckets - 1;
  const int lg = 63 - __clzll(len);  // 0..32
  return 32 - min(lg, 32);
}

__global__ void k_bucket_hist(const unsigned long long* __restrict__ off, long long n, unsigned* __restrict__ hist) {
  __shared__ unsigned h[kBuckets];
  for (int i = threadIdx.x; i < kBuckets; i += blockDim.x) h[i] = 0;
  __syncthreads();
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    atomicAdd(&h[len_bucket(off[t + 1] - off[t])], 1u);
  __syncthreads();
  for (int i = threadIdx.x; i < kBuckets; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[i], h[i]);
}

__global__ void k_bucket_scan(unsigned* __restrict__ hist) {
  // hist[0..kBuckets) -> exclusive offsets in hist[kBuckets..2 kBuckets), cursors zeroed
  if (threadIdx.x == 0) {
    unsigned acc = 0;
    for (int i = 0; i < kBuckets; ++i) {
      hist[kBuckets + i] = acc;
      acc += hist[i];
      hist[i] = 0;
    }
  }
}

__global__ void k_bucket_scatter(const unsigned long long* __restrict__ off, long long n, unsigned* __restrict__ hist,
                                 unsigned long long* __restrict__ work) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int b = len_bucket(off[t + 1] - off[t]);
    const unsigned pos = hist[kBuckets + b] + atomicAdd(&hist[b], 1u);
    work[pos] = (unsigned long long)t;
  }
}

cudaError_t launch_worklist(const unsigned long long* d_off, long long n_tiles, unsigned* d_hist,
                            unsigned long long* d_work, cudaStream_t s) {
  cudaMemsetAsync(d_hist, 0, sizeof(unsigned) * 2 * kBuckets, s);
  long long blocks = (n_tiles + 255) / 256;
  if (blocks > 2048) blocks = 2048;
  k_bucket_hist<<<(unsigned)blocks, 256, 0, s>>>(d_off, n_tiles, d_hist);
  k_bucket_scan<<<1, 32, 0, s>>>(d_hist);
  k_bucket_scatter<<<(unsigned)blocks, 256, 0, s>>>(d_off, n_tiles, d_hist, d_work);
  return cudaGetLastError();
}

}  // namespace lt
