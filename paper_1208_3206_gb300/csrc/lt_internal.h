// lt_internal.h -- host-side declarations shared by the library's .cu files.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lt_common.cuh"

namespace lt {

// ---- lt_build.cu: volumes, densities and position checks of every tetrahedron.
cudaError_t launch_build_tets(const Lattice& L, int n_snap, double m, float* rho_out, unsigned char* degen,
                              DevCounters* ctr, cudaStream_t s);

// ---- lt_bin.cu
// d_desc (may be null): per (frame, cube) tile descriptors, written by the
// count pass and read by the scatter
cudaError_t launch_bin_count(const Lattice& L, const FrameDev* d_frames, int n_frames, unsigned* d_count,
                             unsigned* d_desc, DevCounters* ctr, cudaStream_t s);
cudaError_t launch_scan(const unsigned* d_count, long long n, unsigned long long* d_off, unsigned long long* d_tmp,
                        cudaStream_t s);
size_t scan_tmp_words(long long n);
cudaError_t launch_bin_scatter(const Lattice& L, const FrameDev* d_frames, int n_frames,
                               const unsigned long long* d_off, unsigned* d_cursor, unsigned* d_list,
                               unsigned long long capacity, unsigned* d_desc, DevCounters* ctr, cudaStream_t s);
cudaError_t launch_worklist(const unsigned long long* d_off, long long n_tiles, unsigned* d_hist,
                            unsigned long long* d_work, cudaStream_t s);

// ---- lt_raster.cu
struct RasterArgs {
  Lattice L;
  const FrameDev* frames;
  const unsigned long long* off;
  const unsigned* list;
  const unsigned long long* work;
  long long n_items;
  float* image;
  long long image_stride;  // floats per frame (W * H)
  double* mass_tile;       // per global tile
  DevCounters* ctr;
  int tile;
  unsigned long long* xq;  // exact-evaluation queue, xq_cap entries per CTA
  unsigned xq_cap;
  unsigned long long list_cap;  // entries the cube lists hold (reads are clamped to it)
};
cudaError_t launch_raster(const RasterArgs& a, int ctas, int threads, int any_persp, cudaStream_t s);
int raster_max_ctas_per_sm(int threads, int tile, int any_persp);
constexpr int kRasterMaxCtasPerSm = 4;     // CTAs per SM the exact queue is sized for
constexpr unsigned kExactQueuePerPixel = 64;  // queued fragments per CTA and tile: 64 per pixel of the tile
cudaError_t launch_count_fragments(const RasterArgs& a, unsigned long long* d_counts, int n_frames, int ctas,
                                   int threads, cudaStream_t s);
cudaError_t launch_mass_reduce(const double* mass_tile, long long tpf, int n_frames, double* d_mass,
                               cudaStream_t s);
cudaError_t launch_atomic(const Lattice& L, const FrameDev* d_frames, long long stride, int n_frames, float* image,
                          DevCounters* ctr, cudaStream_t s);

// ---- lt_resample.cu: resampling onto a periodic n^3 grid (q = rho: weight 0,
// q = 1: weight 1) from the bins of an orthographic view along z whose
// pixels are the grid's columns.
cudaError_t launch_resample(const Lattice& L, const FrameDev* d_frame, long long n_tiles, int tile,
                            const unsigned long long* d_off, const unsigned* d_list, unsigned long long list_cap, int n,
                            int weight, double m_tet, double unit, unsigned long long* d_acc, float* d_out,
                            DevCounters* ctr, cudaStream_t s);

// ---- lt_slice.cu: total density (weight 0) or stream count (weight 1) at
// the centres of an n x n grid on the plane z = z0.
cudaError_t launch_slice(const Lattice& L, int snapshot, int n, int weight, double z0, double m_tet, double unit,
                         unsigned long long* d_acc, float* d_out, DevCounters* ctr, cudaStream_t s);

// ---- lt_centroids.cu: centroid splats of one orthographic frame.
// `add`: add to d_out instead of overwriting it. With F.near_r2 > 0 only
// the far cubes (cube_far) are drawn.
cudaError_t launch_centroids(const Lattice& L, const FrameDev* d_frame, int W, int H, double m_tet, double unit,
                             unsigned long long* d_acc, float* d_out, bool add, DevCounters* ctr, cudaStream_t s);
// 64-bit fixed-point sums (units of `unit`) to float, overwriting or adding to d_out.
cudaError_t launch_fixed_finalize(const unsigned long long* d_acc, long long np, double unit, bool add, float* d_out,
                                  cudaStream_t s);

// ---- lt_area.cu: area-averaged pixels of one orthographic frame.
cudaError_t launch_area(const Lattice& L, const FrameDev* d_frame, int W, int H, double m_tet, double unit,
                        unsigned long long* d_acc, float* d_out, DevCounters* ctr, cudaStream_t s);

// ---- lt_backward.cu
cudaError_t launch_backward(const Lattice& L, const FrameDev* d_frames, long long stride, int n_frames, int n_snap,
                            const float* dLdI, float* corner_grad, cudaStream_t s);
cudaError_t launch_gather_grad(const Lattice& L, int n_snap, const float* corner_grad, float* dLdpos,
                               cudaStream_t s);

}  // namespace lt
