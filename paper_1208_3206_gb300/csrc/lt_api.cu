// lt_api.cu -- the C ABI (include/lt.h): context, argument checks, buffer
// management, the project-bin / render pipeline, CUDA-graph capture and the
// autotuner. All heavy work is in the kernels of lt_build.cu, lt_bin.cu,
// lt_raster.cu and lt_backward.cu.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "../../include/lt.h"
#include "lt_internal.h"

using lt::DevCounters;
using lt::FrameDev;
using lt::Lattice;

struct lt_ctx {
  int device = 0;
  int num_sms = 1;
  lt_config cfg{};
  // registered lattice
  bool have_lattice = false;
  Lattice L{};
  int n_snap = 0;
  double total_mass = 0.0;
  // frames of the last lt_project_bin
  int n_frames = 0;
  int W = 0, H = 0, tile = 16;
  bool any_persp = false;
  FrameDev* d_frames = nullptr;
  size_t frames_cap = 0;
  FrameDev* h_frames = nullptr;  // pinned staging
  size_t h_frames_cap = 0;
  FrameDev* d_frames_aux = nullptr;  // lt_render_atomic
  size_t frames_aux_cap = 0;
  // bins
  long long n_tiles = 0;
  size_t tiles_cap = 0;
  unsigned* d_count = nullptr;
  unsigned* d_cursor = nullptr;
  unsigned long long* d_off = nullptr;
  unsigned long long* d_work = nullptr;
  double* d_mass_tile = nullptr;
  unsigned long long* d_xq = nullptr;  // exact-evaluation queues of the raster CTAs
  size_t xq_cap = 0;
  unsigned long long* d_scan_tmp = nullptr;
  size_t scan_tmp_cap = 0;
  unsigned* d_list = nullptr;
  unsigned long long list_cap = 0;
  unsigned long long entries = 0;
  unsigned* d_hist = nullptr;
  unsigned* d_desc = nullptr;  // per (frame, cube) tile descriptors of the bin pass (null above the budget)
  size_t desc_cap = 0;
  bool binned = false;
  // counters
  DevCounters* d_ctr = nullptr;
  DevCounters* h_ctr = nullptr;  // pinned
  unsigned long long* d_frag = nullptr;
  size_t frag_cap = 0;
  unsigned long long* h_u64 = nullptr;  // pinned scratch
  // zero-volume tetrahedra: one bit per tetrahedron, a byte per (snapshot, cube)
  unsigned char* d_degen = nullptr;
  size_t degen_cap = 0;
  // resampling: fixed-point cells
  unsigned long long* d_racc = nullptr;
  size_t racc_cap = 0;
  // slices: fixed-point points
  unsigned long long* d_sacc = nullptr;
  size_t sacc_cap = 0;
  // centroid splats: the frame and fixed-point pixels
  FrameDev* d_frame_cen = nullptr;
  size_t frame_cen_cap = 0;
  unsigned long long* d_cacc = nullptr;
  size_t cacc_cap = 0;
  // backward
  float* d_corner_grad = nullptr;
  size_t corner_grad_cap = 0;
  // graph
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  int graph_kernels = 0;
  FrameDev* d_frames_graph = nullptr;  // the graph's own copy of its frames
  size_t frames_graph_cap = 0;
  // set when a buffer the graph captured is reallocated or the lattice is
  // registered again: lt_graph_launch then refuses to replay
  bool graph_stale = false;
  // host-side latched error
  lt_status latched = LT_OK;
};

namespace {

#define LT_CUDA(call)                                  \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) {                           \
      fprintf(stderr, "liblt: %s failed: %s\n", #call, cudaGetErrorString(e_)); \
      return LT_ERR_CUDA;                              \
    }                                                  \
  } while (0)

constexpr size_t kDescBudgetBytes = (size_t)16 << 30;  // tile descriptors kept up to 16 GiB

lt_config default_config() {
  lt_config c;
  c.tile = 16;
  c.raster_threads = 256;
  c.ctas_per_sm = 0;
  c.frac_bits = 28;
  return c;
}

bool valid_config(const lt_config& c) {
  const bool tile_ok = c.tile == 0 || c.tile == 8 || c.tile == 16 || c.tile == 32 || c.tile == 64;
  const bool thr_ok = c.raster_threads == 0 || (c.raster_threads >= 64 && c.raster_threads <= 256 &&
                                                c.raster_threads % 32 == 0);
  const bool cps_ok = c.ctas_per_sm >= 0 && c.ctas_per_sm <= 32;
  const bool fb_ok = c.frac_bits == 0 || (c.frac_bits >= 8 && c.frac_bits <= 62);
  return tile_ok && thr_ok && cps_ok && fb_ok;
}

lt_config resolved(const lt_config& c) {
  lt_config d = default_config();
  if (c.tile) d.tile = c.tile;
  if (c.raster_threads) d.raster_threads = c.raster_threads;
  if (c.ctas_per_sm) d.ctas_per_sm = c.ctas_per_sm;
  if (c.frac_bits) d.frac_bits = c.frac_bits;
  return d;
}

template <typename T>
lt_status grow(T** p, size_t* cap, size_t n) {
  if (*cap >= n && *p) return LT_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  if (n == 0) n = 1;
  if (cudaMalloc((void**)p, n * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return LT_ERR_NOMEM;
  }
  *cap = n;
  return LT_OK;
}

// grow() for a buffer a captured graph may use: a reallocation makes the
// graph stale (its kernels hold the old address).
template <typename T>
lt_status grow_c(lt_ctx* ctx, T** p, size_t* cap, size_t n) {
  if (*cap >= n && *p) return LT_OK;
  ctx->graph_stale = true;
  return grow(p, cap, n);
}

lt_status grow_pinned(FrameDev** p, size_t* cap, size_t n) {
  if (*cap >= n && *p) return LT_OK;
  if (*p) cudaFreeHost(*p);
  *p = nullptr;
  *cap = 0;
  if (cudaMallocHost((void**)p, n * sizeof(FrameDev)) != cudaSuccess) {
    cudaGetLastError();
    return LT_ERR_NOMEM;
  }
  *cap = n;
  return LT_OK;
}

bool is_capturing(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &st) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return st != cudaStreamCaptureStatusNone;
}

void norm3(double* v) {
  const double n = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  v[0] /= n; v[1] /= n; v[2] /= n;
}

void cross3(const double* a, const double* b, double* o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

// Split v (double) into a float-float pair.
void split_ff(double v, float* hi, float* lo) {
  *hi = (float)v;
  *lo = (float)(v - (double)*hi);
}

// Anchor component base + i gi + j gj + k gk over the lattice 0 <= i, j, k < N
// as hi parts on a common power-of-two quantum q (every partial sum of
// hi terms is an integer multiple of q below 2^24 q, hence exact in FP32)
// plus lo remainders.
void split_affine(double base, double gi, double gj, double gk, int N, float* h, float* l) {
  const double B = fabs(base) + (double)N * (fabs(gi) + fabs(gj) + fabs(gk)) + 1e-300;
  const int e = (int)ceil(log2(B));
  const double q = ldexp(1.0, e - 23);
  const double v[4] = {base, gi, gj, gk};
  for (int c = 0; c < 4; ++c) {
    const double hv = nearbyint(v[c] / q) * q;
    h[c] = (float)hv;
    l[c] = (float)(v[c] - hv);
  }
}

// Camera -> kernel form. Returns false for an invalid camera.
bool make_frame(const lt_camera& c, const lt_ctx* ctx, int snapshot, int tile, int frame_index, FrameDev& F) {
  if (c.type != LT_ORTHO && c.type != LT_PERSP) return false;
  if (c.W < 1 || c.H < 1 || c.W > 65536 || c.H > 65536) return false;
  // hybrid near/far rendering: perspective views only
  if (!(c.near_radius >= 0.0) || !(c.near_radius < 1e150) || (c.near_radius > 0.0 && c.type != LT_PERSP)) return false;
  double f[3] = {c.fwd[0], c.fwd[1], c.fwd[2]}, up[3] = {c.up[0], c.up[1], c.up[2]};
  if (!(f[0] * f[0] + f[1] * f[1] + f[2] * f[2] > 0)) return false;
  norm3(f);
  double r[3], u[3];
  cross3(up, f, r);
  if (!(r[0] * r[0] + r[1] * r[1] + r[2] * r[2] > 1e-24)) return false;
  norm3(r);
  cross3(f, r, u);
  memset(&F, 0, sizeof F);
  F.persp = c.type == LT_PERSP;
  F.W = c.W;
  F.H = c.H;
  F.wrap = (!F.persp) && c.wrap;
  F.snapshot = snapshot;
  F.tile = tile;
  F.tiles_x = (c.W + tile - 1) / tile;
  F.tiles_y = (c.H + tile - 1) / tile;
  F.tile_base = (long long)frame_index * F.tiles_x * F.tiles_y;
  for (int q = 0; q < 3; ++q) {
    F.r[q] = (float)r[q];
    F.u[q] = (float)u[q];
    F.f[q] = (float)f[q];
    F.eye[q] = (float)c.eye[q];
  }
  const int N = ctx->L.N;
  const double box = ctx->L.box, M = ctx->total_mass;
  const double h = box / N;
  const double m = M / (6.0 * (double)N * N * N);
  const double scale_bits = ldexp(1.0, ctx->cfg.frac_bits);
  if (!F.persp) {
    const double lx = (double)c.hi[0] - c.lo[0], ly = (double)c.hi[1] - c.lo[1];
    if (!(lx > 0) || !(ly > 0)) return false;
    const double sx = c.W / lx, sy = c.H / ly;
    F.sx = (float)sx;
    F.sy = (float)sy;
    F.ox = (float)(-c.lo[0] * sx - 0.5);
    F.oy = (float)(-c.lo[1] * sy - 0.5);
    // pixel coordinates of lattice point (i, j, k) h: (axis . q) s - lo s - 1/2
    split_affine(-c.lo[0] * sx - 0.5, h * r[0] * sx, h * r[1] * sx, h * r[2] * sx, N, F.ah[0], F.al[0]);
    split_affine(-c.lo[1] * sy - 0.5, h * u[0] * sy, h * u[1] * sy, h * u[2] * sy, N, F.ah[1], F.al[1]);
    split_affine(0.0, 0.0, 0.0, 0.0, N, F.ah[2], F.al[2]);
    const double sigma = M / (lx * ly);  // mean column density of the window
    const double scale = scale_bits / sigma;
    F.K = (float)(m * sx * sy * scale);
    F.unit = sigma / scale_bits;
    F.pix_area = lx * ly / ((double)c.W * c.H);
  } else {
    if (!(c.fov_y_deg > 0.0f && c.fov_y_deg < 179.0f)) return false;
    const double ty = tan(0.5 * c.fov_y_deg * M_PI / 180.0);
    const double tx = ty * c.W / c.H;
    F.tan_x = (float)tx;
    F.tan_y = (float)ty;
    F.tand[0] = tx;
    F.tand[1] = ty;
    F.kx = (float)(c.W / (2.0 * tx));
    F.ky = (float)(c.H / (2.0 * ty));
    split_ff(c.W / (2.0 * tx), &F.kxh, &F.kxl);
    split_ff(c.H / (2.0 * ty), &F.kyh, &F.kyl);
    // camera coordinates of lattice point (i, j, k) h: axis . (q - eye)
    const double* ax3[3] = {r, u, f};
    for (int a = 0; a < 3; ++a) {
      const double* v = ax3[a];
      const double base = -(v[0] * c.eye[0] + v[1] * c.eye[1] + v[2] * c.eye[2]);
      split_affine(base, h * v[0], h * v[1], h * v[2], N, F.ah[a], F.al[a]);
    }
    F.cx = (float)(0.5 * c.W - 0.5);
    F.cy = (float)(0.5 * c.H - 0.5);
    F.near_z = (float)(1e-6 * box);
    const double sigma = M / (box * box);  // mean density times box depth
    const double scale = scale_bits / sigma;
    F.K = (float)(m * (double)F.kx * (double)F.ky * scale);
    F.unit = sigma / scale_bits;
    F.pix_area = (2.0 * tx / c.W) * (2.0 * ty / c.H);
  }
  F.inv6K = (float)(1.0 / (6.0 * (double)F.K));
  for (int q = 0; q < 3; ++q) {
    F.rd[q] = r[q];
    F.ud[q] = u[q];
    F.fd[q] = f[q];
    F.eyed[q] = c.eye[q];
  }
  if (!F.persp) {
    F.lod[0] = c.lo[0];
    F.lod[1] = c.lo[1];
    F.pxd[0] = ((double)c.hi[0] - c.lo[0]) / c.W;
    F.pxd[1] = ((double)c.hi[1] - c.lo[1]) / c.H;
  }
  F.m_tet = m;
  F.sigma_units = (float)scale_bits;
  F.near_r2 = c.near_radius > 0.0 ? c.near_radius * c.near_radius : 0.0;
  return true;
}

lt_status take_device_errors(lt_ctx* ctx) {
  if (cudaMemcpy(ctx->h_ctr, ctx->d_ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return LT_ERR_CUDA;
  }
  const unsigned e = ctx->h_ctr->errors;
  if (e) {
    unsigned zero = 0;
    cudaMemcpy(&ctx->d_ctr->errors, &zero, sizeof zero, cudaMemcpyHostToDevice);
  }
  if (e & lt::kErrNonFinite) return LT_ERR_NONFINITE;
  if (e & lt::kErrCapacity) return LT_ERR_CAPACITY;
  if (e & lt::kErrBehindEye) return LT_ERR_BEHIND_EYE;
  if (e & lt::kErrRange) return LT_ERR_RANGE;
  if (e & lt::kErrBounds) return LT_ERR_BOUNDS;
  return LT_OK;
}

// Frames from host cameras into ctx->h_frames (pinned). Same image size for all.
lt_status prepare_frames(lt_ctx* ctx, const lt_camera* cams, int n_frames, const int* frame_snapshot, int tile,
                         int* W, int* H, bool* any_persp) {
  if (!cams || n_frames < 1) return LT_ERR_ARG;
  lt_status st = grow_pinned(&ctx->h_frames, &ctx->h_frames_cap, (size_t)n_frames);
  if (st != LT_OK) return st;
  *W = cams[0].W;
  *H = cams[0].H;
  *any_persp = false;
  for (int f = 0; f < n_frames; ++f) {
    const int snap = frame_snapshot ? frame_snapshot[f] : 0;
    if (snap < 0 || snap >= ctx->n_snap) return LT_ERR_ARG;
    if (cams[f].W != *W || cams[f].H != *H) return LT_ERR_ARG;
    if (!make_frame(cams[f], ctx, snap, tile, f, ctx->h_frames[f])) return LT_ERR_ARG;
    *any_persp = *any_persp || cams[f].type == LT_PERSP;
  }
  return LT_OK;
}

// Launches of the bin pass after the frames are on the device.
lt_status bin_launches(lt_ctx* ctx, cudaStream_t s, bool allow_sync) {
  const long long n = ctx->n_tiles;
  LT_CUDA(cudaMemsetAsync(ctx->d_count, 0, sizeof(unsigned) * n, s));
  LT_CUDA(lt::launch_bin_count(ctx->L, ctx->d_frames, ctx->n_frames, ctx->d_count, ctx->d_desc, ctx->d_ctr, s));
  LT_CUDA(lt::launch_scan(ctx->d_count, n, ctx->d_off, ctx->d_scan_tmp, s));
  if (allow_sync) {
    LT_CUDA(cudaMemcpyAsync(ctx->h_u64, ctx->d_off + n, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    LT_CUDA(cudaStreamSynchronize(s));
    const unsigned long long total = ctx->h_u64[0];
    ctx->entries = total;
    if (total > ctx->list_cap) {
      size_t cap = ctx->list_cap;
      lt_status st = grow_c(ctx, &ctx->d_list, &cap, (size_t)(total + total / 8 + 1024));
      if (st != LT_OK) return st;
      ctx->list_cap = cap;
    }
  }
  LT_CUDA(cudaMemsetAsync(ctx->d_cursor, 0, sizeof(unsigned) * n, s));
  LT_CUDA(lt::launch_bin_scatter(ctx->L, ctx->d_frames, ctx->n_frames, ctx->d_off, ctx->d_cursor, ctx->d_list,
                                 ctx->list_cap, ctx->d_desc, ctx->d_ctr, s));
  LT_CUDA(lt::launch_worklist(ctx->d_off, n, ctx->d_hist, ctx->d_work, s));
  return LT_OK;
}

lt_status ensure_tiles(lt_ctx* ctx, long long n) {
  lt_status st;
  size_t c;
  if ((size_t)n > ctx->tiles_cap) {
    c = 0;
    if ((st = grow_c(ctx, &ctx->d_count, &c, (size_t)n)) != LT_OK) return st;
    c = 0;
    if ((st = grow_c(ctx, &ctx->d_cursor, &c, (size_t)n)) != LT_OK) return st;
    c = 0;
    if ((st = grow_c(ctx, &ctx->d_off, &c, (size_t)n + 1)) != LT_OK) return st;
    c = 0;
    if ((st = grow_c(ctx, &ctx->d_work, &c, (size_t)n)) != LT_OK) return st;
    c = 0;
    if ((st = grow_c(ctx, &ctx->d_mass_tile, &c, (size_t)n)) != LT_OK) return st;
    ctx->tiles_cap = (size_t)n;
  }
  const size_t words = lt::scan_tmp_words(n);
  if ((st = grow_c(ctx, &ctx->d_scan_tmp, &ctx->scan_tmp_cap, words)) != LT_OK) return st;
  const size_t xq = (size_t)ctx->num_sms * lt::kRasterMaxCtasPerSm * lt::kExactQueuePerPixel * ctx->cfg.tile *
                    ctx->cfg.tile;
  if ((st = grow_c(ctx, &ctx->d_xq, &ctx->xq_cap, xq)) != LT_OK) return st;
  return LT_OK;
}

lt_status project_bin_impl(lt_ctx* ctx, const lt_camera* cams, int n_frames, const int* frame_snapshot,
                           cudaStream_t s, bool upload_only) {
  if (!ctx) return LT_ERR_ARG;
  if (!ctx->have_lattice) return LT_ERR_STATE;
  const int tile = ctx->cfg.tile;
  int W, H;
  bool any_persp;
  lt_status st = prepare_frames(ctx, cams, n_frames, frame_snapshot, tile, &W, &H, &any_persp);
  if (st != LT_OK) return st;
  if ((st = grow(&ctx->d_frames, &ctx->frames_cap, (size_t)n_frames)) != LT_OK) return st;
  const long long tpf = (long long)ctx->h_frames[0].tiles_x * ctx->h_frames[0].tiles_y;
  const long long n_tiles = tpf * n_frames;
  if ((st = ensure_tiles(ctx, n_tiles)) != LT_OK) return st;
  // tile descriptors of the bin pass: 4 bytes per (frame, cube), kept only
  // below a memory budget (above it the scatter projects every cube again)
  const size_t n_desc = (size_t)n_frames * (size_t)ctx->L.n_particles;
  if (n_desc * sizeof(unsigned) <= kDescBudgetBytes) {
    if (grow_c(ctx, &ctx->d_desc, &ctx->desc_cap, n_desc) != LT_OK) {
      ctx->d_desc = nullptr;
      ctx->desc_cap = 0;
    }
  } else if (ctx->d_desc) {
    ctx->graph_stale = true;
    cudaFree(ctx->d_desc);
    ctx->d_desc = nullptr;
    ctx->desc_cap = 0;
  }
  LT_CUDA(cudaMemcpyAsync(ctx->d_frames, ctx->h_frames, sizeof(FrameDev) * n_frames, cudaMemcpyHostToDevice, s));
  ctx->n_frames = n_frames;
  ctx->W = W;
  ctx->H = H;
  ctx->tile = tile;
  ctx->any_persp = any_persp;
  ctx->n_tiles = n_tiles;
  ctx->binned = true;
  if (upload_only) return LT_OK;
  return bin_launches(ctx, s, !is_capturing(s));
}

lt_status render_impl(lt_ctx* ctx, float* d_image, double* d_mass, cudaStream_t s) {
  lt::RasterArgs a;
  a.L = ctx->L;
  a.frames = ctx->d_frames;
  a.off = ctx->d_off;
  a.list = ctx->d_list;
  a.work = ctx->d_work;
  a.n_items = ctx->n_tiles;
  a.image = d_image;
  a.image_stride = (long long)ctx->W * ctx->H;
  a.mass_tile = ctx->d_mass_tile;
  a.ctr = ctx->d_ctr;
  a.tile = ctx->tile;
  a.xq = ctx->d_xq;
  a.xq_cap = lt::kExactQueuePerPixel * (unsigned)(ctx->tile * ctx->tile);
  a.list_cap = ctx->list_cap;
  const int threads = ctx->cfg.raster_threads;
  int cps = ctx->cfg.ctas_per_sm;
  const int fit = lt::raster_max_ctas_per_sm(threads, ctx->tile, ctx->any_persp);
  if (fit < 1) return LT_ERR_ARG;  // CTA shape exceeds the SM's registers or shared memory
  if (cps <= 0 || cps > fit) cps = fit;
  if (cps > lt::kRasterMaxCtasPerSm) cps = lt::kRasterMaxCtasPerSm;  // the exact queues are sized for this
  long long ctas = (long long)ctx->num_sms * cps;
  if (ctas > ctx->n_tiles) ctas = ctx->n_tiles;
  if (ctas < 1) ctas = 1;
  LT_CUDA(cudaMemsetAsync(&ctx->d_ctr->work_next, 0, sizeof(unsigned long long), s));
  LT_CUDA(lt::launch_raster(a, (int)ctas, threads, ctx->any_persp ? 1 : 0, s));
  if (d_mass) {
    LT_CUDA(lt::launch_mass_reduce(ctx->d_mass_tile, ctx->n_tiles / ctx->n_frames, ctx->n_frames, d_mass, s));
  }
  return LT_OK;
}

// Centroid splats of one view into d_image (overwritten, or added to when
// `add`): the frame staged through the pinned memory (the call waits for
// the copy to leave it, since the staging is shared with the other entry
// points), 64-bit fixed-point sums in the context.
lt_status centroids_impl(lt_ctx* ctx, const lt_camera& cam, int snapshot, float* d_image, bool add, cudaStream_t s) {
  FrameDev F;
  if (!make_frame(cam, ctx, snapshot, ctx->cfg.tile, 0, F)) return LT_ERR_ARG;
  lt_status st = grow(&ctx->d_frame_cen, &ctx->frame_cen_cap, 1);
  if (st != LT_OK) return st;
  const size_t np = (size_t)cam.W * cam.H;
  if ((st = grow(&ctx->d_cacc, &ctx->cacc_cap, np)) != LT_OK) return st;
  if ((st = grow_pinned(&ctx->h_frames, &ctx->h_frames_cap, 1)) != LT_OK) return st;
  ctx->h_frames[0] = F;
  LT_CUDA(cudaMemcpyAsync(ctx->d_frame_cen, ctx->h_frames, sizeof(FrameDev), cudaMemcpyHostToDevice, s));
  // the fixed-point unit is the frame's: 2^-frac_bits of its mean column density
  LT_CUDA(lt::launch_centroids(ctx->L, ctx->d_frame_cen, cam.W, cam.H, F.m_tet, F.unit, ctx->d_cacc, d_image, add,
                               ctx->d_ctr, s));
  LT_CUDA(cudaStreamSynchronize(s));
  return LT_OK;
}

}  // namespace

extern "C" {

const char* lt_status_str(lt_status s) {
  switch (s) {
    case LT_OK: return "ok";
    case LT_ERR_ARG: return "invalid argument";
    case LT_ERR_CUDA: return "CUDA runtime error";
    case LT_ERR_CAPACITY: return "bin list capacity exceeded";
    case LT_ERR_NONFINITE: return "non-finite particle position";
    case LT_ERR_BEHIND_EYE: return "vertex at or behind the perspective eye plane";
    case LT_ERR_RANGE: return "fixed-point accumulator range exceeded";
    case LT_ERR_STATE: return "calls made out of order";
    case LT_ERR_NOMEM: return "device allocation failed";
    case LT_ERR_BOUNDS: return "index check failed (bounds-checking build)";
  }
  return "unknown status";
}

lt_status lt_create(lt_ctx** out, const lt_config* cfg) {
  if (!out) return LT_ERR_ARG;
  *out = nullptr;
  if (cfg && !valid_config(*cfg)) return LT_ERR_ARG;
  lt_ctx* ctx = new (std::nothrow) lt_ctx();
  if (!ctx) return LT_ERR_NOMEM;
  ctx->cfg = resolved(cfg ? *cfg : lt_config{});
  if (cudaGetDevice(&ctx->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return LT_ERR_CUDA;
  }
  if (cudaMalloc((void**)&ctx->d_ctr, sizeof(DevCounters)) != cudaSuccess ||
      cudaMallocHost((void**)&ctx->h_ctr, sizeof(DevCounters)) != cudaSuccess ||
      cudaMallocHost((void**)&ctx->h_u64, 64 * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMalloc((void**)&ctx->d_hist, 2 * 64 * sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    lt_destroy(ctx);
    return LT_ERR_NOMEM;
  }
  if (cudaMemset(ctx->d_ctr, 0, sizeof(DevCounters)) != cudaSuccess) {
    lt_destroy(ctx);
    return LT_ERR_CUDA;
  }
  *out = ctx;
  return LT_OK;
}

void lt_destroy(lt_ctx* ctx) {
  if (!ctx) return;
  if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
  if (ctx->graph) cudaGraphDestroy(ctx->graph);
  cudaFree(ctx->d_frames);
  cudaFree(ctx->d_frames_aux);
  cudaFree(ctx->d_frames_graph);
  cudaFree(ctx->d_count);
  cudaFree(ctx->d_cursor);
  cudaFree(ctx->d_off);
  cudaFree(ctx->d_work);
  cudaFree(ctx->d_mass_tile);
  cudaFree(ctx->d_xq);
  cudaFree(ctx->d_scan_tmp);
  cudaFree(ctx->d_list);
  cudaFree(ctx->d_hist);
  cudaFree(ctx->d_desc);
  cudaFree(ctx->d_ctr);
  cudaFree(ctx->d_frag);
  cudaFree(ctx->d_corner_grad);
  cudaFree(ctx->d_racc);
  cudaFree(ctx->d_sacc);
  cudaFree(ctx->d_frame_cen);
  cudaFree(ctx->d_cacc);
  cudaFree(ctx->d_degen);
  if (ctx->h_ctr) cudaFreeHost(ctx->h_ctr);
  if (ctx->h_u64) cudaFreeHost(ctx->h_u64);
  if (ctx->h_frames) cudaFreeHost(ctx->h_frames);
  delete ctx;
}

lt_status lt_set_config(lt_ctx* ctx, const lt_config* cfg) {
  if (!ctx || !cfg || !valid_config(*cfg)) return LT_ERR_ARG;
  ctx->cfg = resolved(*cfg);
  return LT_OK;
}

lt_status lt_get_config(const lt_ctx* ctx, lt_config* out) {
  if (!ctx || !out) return LT_ERR_ARG;
  *out = ctx->cfg;
  return LT_OK;
}

lt_status lt_build_tets(lt_ctx* ctx, const void* d_pos, int pos_fmt, int N, float box, double total_mass,
                        int n_snapshots, float* d_rho, lt_stream stream) {
  if (!ctx || !d_pos) return LT_ERR_ARG;
  if (N < 1 || (long long)N * N * N > (1LL << 31) - 1) return LT_ERR_ARG;
  if (!(box > 0.0f) || !(total_mass > 0.0) || n_snapshots < 1) return LT_ERR_ARG;
  if (pos_fmt != LT_POS_F32X4 && pos_fmt != LT_POS_F16_OFFSETS) return LT_ERR_ARG;
  const size_t align = pos_fmt == LT_POS_F32X4 ? 16 : 8;
  if (((uintptr_t)d_pos) % align) return LT_ERR_ARG;
  if (6LL * N * N * N * n_snapshots > (1LL << 40)) return LT_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  Lattice L;
  L.pos = d_pos;
  L.fmt = pos_fmt;
  L.N = N;
  L.box = box;
  L.h = box / (float)N;
  L.half_box = 0.5f * box;
  L.n_particles = (long long)N * N * N;
  lt::lattice_set_divisor(L, N);
  lt_status st = grow(&ctx->d_degen, &ctx->degen_cap, (size_t)L.n_particles * n_snapshots);
  if (st != LT_OK) return st;
  L.degen = ctx->d_degen;
  ctx->L = L;
  ctx->graph_stale = true;  // a graph captured the previous lattice
  ctx->n_snap = n_snapshots;
  ctx->total_mass = total_mass;
  ctx->have_lattice = true;
  ctx->binned = false;
  LT_CUDA(cudaMemsetAsync(&ctx->d_ctr->nonfinite, 0, sizeof(unsigned long long) * 5, s));
  const double m = total_mass / (6.0 * (double)N * N * N);
  LT_CUDA(lt::launch_build_tets(L, n_snapshots, m, d_rho, ctx->d_degen, ctx->d_ctr, s));
  return LT_OK;
}

lt_status lt_project_bin(lt_ctx* ctx, const lt_camera* cams, int n_frames, const int* frame_snapshot,
                         lt_stream stream) {
  return project_bin_impl(ctx, cams, n_frames, frame_snapshot, (cudaStream_t)stream, false);
}

lt_status lt_render_tiles(lt_ctx* ctx, float* d_image, double* d_mass, lt_stream stream) {
  if (!ctx || !d_image) return LT_ERR_ARG;
  if (!ctx->binned) return LT_ERR_STATE;
  return render_impl(ctx, d_image, d_mass, (cudaStream_t)stream);
}

lt_status lt_render_atomic(lt_ctx* ctx, const lt_camera* cams, int n_frames, const int* frame_snapshot,
                           float* d_image, lt_stream stream) {
  if (!ctx || !d_image) return LT_ERR_ARG;
  if (!ctx->have_lattice) return LT_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  int W, H;
  bool any_persp;
  lt_status st = prepare_frames(ctx, cams, n_frames, frame_snapshot, ctx->cfg.tile, &W, &H, &any_persp);
  if (st != LT_OK) return st;
  if ((st = grow(&ctx->d_frames_aux, &ctx->frames_aux_cap, (size_t)n_frames)) != LT_OK) return st;
  LT_CUDA(cudaMemcpyAsync(ctx->d_frames_aux, ctx->h_frames, sizeof(FrameDev) * n_frames, cudaMemcpyHostToDevice, s));
  LT_CUDA(lt::launch_atomic(ctx->L, ctx->d_frames_aux, (long long)W * H, n_frames, d_image, ctx->d_ctr, s));
  // the pinned staging is reused by the next call: make sure the copy has left it
  LT_CUDA(cudaStreamSynchronize(s));
  return LT_OK;
}

lt_status lt_count_fragments(lt_ctx* ctx, long long* h_counts, lt_stream stream) {
  if (!ctx || !h_counts) return LT_ERR_ARG;
  if (!ctx->binned) return LT_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  lt_status st = grow(&ctx->d_frag, &ctx->frag_cap, (size_t)ctx->n_frames);
  if (st != LT_OK) return st;
  LT_CUDA(cudaMemsetAsync(ctx->d_frag, 0, sizeof(unsigned long long) * ctx->n_frames, s));
  LT_CUDA(cudaMemsetAsync(&ctx->d_ctr->work_next, 0, sizeof(unsigned long long), s));
  lt::RasterArgs a;
  a.L = ctx->L;
  a.frames = ctx->d_frames;
  a.off = ctx->d_off;
  a.list = ctx->d_list;
  a.work = ctx->d_work;
  a.n_items = ctx->n_tiles;
  a.image = nullptr;
  a.image_stride = 0;
  a.mass_tile = nullptr;
  a.ctr = ctx->d_ctr;
  a.tile = ctx->tile;
  a.xq = nullptr;  // counting queues nothing
  a.xq_cap = 0;
  a.list_cap = ctx->list_cap;
  long long ctas = (long long)ctx->num_sms * 4;
  if (ctas > ctx->n_tiles) ctas = ctx->n_tiles;
  LT_CUDA(lt::launch_count_fragments(a, ctx->d_frag, ctx->n_frames, (int)ctas, 256, s));
  std::vector<unsigned long long> tmp(ctx->n_frames);
  LT_CUDA(cudaMemcpyAsync(tmp.data(), ctx->d_frag, sizeof(unsigned long long) * ctx->n_frames,
                          cudaMemcpyDeviceToHost, s));
  LT_CUDA(cudaStreamSynchronize(s));
  for (int f = 0; f < ctx->n_frames; ++f) h_counts[f] = (long long)tmp[f];
  return LT_OK;
}

lt_status lt_render_backward(lt_ctx* ctx, const float* d_dL_dimage, float* d_dL_dpos, lt_stream stream) {
  if (!ctx || !d_dL_dimage || !d_dL_dpos) return LT_ERR_ARG;
  if (!ctx->binned) return LT_ERR_STATE;
  // adjoint of orthographic views only; any_persp describes the frames of the
  // last bin (the pinned staging of h_frames is reused by lt_render_atomic)
  if (ctx->any_persp) return LT_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n = (size_t)ctx->n_snap * ctx->L.n_particles * 24;
  lt_status st = grow(&ctx->d_corner_grad, &ctx->corner_grad_cap, n);
  if (st != LT_OK) return st;
  LT_CUDA(lt::launch_backward(ctx->L, ctx->d_frames, (long long)ctx->W * ctx->H, ctx->n_frames, ctx->n_snap,
                              d_dL_dimage, ctx->d_corner_grad, s));
  LT_CUDA(lt::launch_gather_grad(ctx->L, ctx->n_snap, ctx->d_corner_grad, d_dL_dpos, s));
  return LT_OK;
}

lt_status lt_resample(lt_ctx* ctx, int n, int weight, int snapshot, float* d_grid, lt_stream stream) {
  if (!ctx || !d_grid || n < 1 || n > 2048 || (weight != LT_WEIGHT_DENSITY && weight != LT_WEIGHT_STREAMS))
    return LT_ERR_ARG;
  if (!ctx->have_lattice) return LT_ERR_STATE;
  if (snapshot < 0 || snapshot >= ctx->n_snap) return LT_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  // the grid's columns are the pixels of an orthographic view along z over
  // the periodic box window: pixel (a, b) is centred on column (a, b)
  lt_camera cam;
  memset(&cam, 0, sizeof cam);
  cam.type = LT_ORTHO;
  cam.fwd[2] = 1.0;
  cam.up[1] = 1.0;
  cam.hi[0] = cam.hi[1] = ctx->L.box;
  cam.W = cam.H = n;
  cam.wrap = 1;
  const int snaps[1] = {snapshot};
  lt_status st = project_bin_impl(ctx, &cam, 1, snaps, s, false);
  if (st != LT_OK) return st;
  const size_t cells = (size_t)n * n * n;
  if ((st = grow(&ctx->d_racc, &ctx->racc_cap, cells)) != LT_OK) return st;
  const double box = ctx->L.box, gs = box / n;
  const int N = ctx->L.N;
  const double m_tet = ctx->total_mass / (6.0 * (double)N * N * N);
  // fixed-point unit: 2^-frac_bits of the mean cell (mean density times g,
  // or one stream times g)
  const double mean_cell = weight == LT_WEIGHT_DENSITY ? ctx->total_mass / (box * box * box) * gs : gs;
  const double unit = mean_cell / ldexp(1.0, ctx->cfg.frac_bits);
  LT_CUDA(cudaMemsetAsync(&ctx->d_ctr->resample_intervals, 0, 2 * sizeof(unsigned long long), s));
  LT_CUDA(lt::launch_resample(ctx->L, ctx->d_frames, ctx->n_tiles, ctx->tile, ctx->d_off, ctx->d_list, ctx->list_cap,
                              n, weight, m_tet, unit, ctx->d_racc, d_grid, ctx->d_ctr, s));
  return LT_OK;
}

lt_status lt_slice(lt_ctx* ctx, int n, int weight, int snapshot, double z0, float* d_img, lt_stream stream) {
  if (!ctx || !d_img || n < 1 || n > 32768 || (weight != LT_WEIGHT_DENSITY && weight != LT_WEIGHT_STREAMS) ||
      !isfinite(z0))
    return LT_ERR_ARG;
  if (!ctx->have_lattice) return LT_ERR_STATE;
  if (snapshot < 0 || snapshot >= ctx->n_snap) return LT_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t np = (size_t)n * n;
  lt_status st = grow(&ctx->d_sacc, &ctx->sacc_cap, np);
  if (st != LT_OK) return st;
  const double box = ctx->L.box;
  const int N = ctx->L.N;
  const double m_tet = ctx->total_mass / (6.0 * (double)N * N * N);
  // fixed-point unit: 2^-frac_bits of the mean density, or of one stream
  const double scale = weight == LT_WEIGHT_DENSITY ? ctx->total_mass / (box * box * box) : 1.0;
  const double unit = scale / ldexp(1.0, ctx->cfg.frac_bits);
  LT_CUDA(lt::launch_slice(ctx->L, snapshot, n, weight, z0, m_tet, unit, ctx->d_sacc, d_img, ctx->d_ctr, s));
  return LT_OK;
}

lt_status lt_render_centroids(lt_ctx* ctx, const lt_camera* cam, int snapshot, float* d_image, lt_stream stream) {
  if (!ctx || !cam || !d_image) return LT_ERR_ARG;
  if (!ctx->have_lattice) return LT_ERR_STATE;
  if (snapshot < 0 || snapshot >= ctx->n_snap) return LT_ERR_ARG;
  return centroids_impl(ctx, *cam, snapshot, d_image, false, (cudaStream_t)stream);
}

lt_status lt_render_area(lt_ctx* ctx, const lt_camera* cam, int snapshot, float* d_image, lt_stream stream) {
  if (!ctx || !cam || !d_image) return LT_ERR_ARG;
  if (!ctx->have_lattice) return LT_ERR_STATE;
  if (snapshot < 0 || snapshot >= ctx->n_snap || cam->type != LT_ORTHO) return LT_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  FrameDev F;
  if (!make_frame(*cam, ctx, snapshot, ctx->cfg.tile, 0, F)) return LT_ERR_ARG;
  lt_status st = grow(&ctx->d_frame_cen, &ctx->frame_cen_cap, 1);
  if (st != LT_OK) return st;
  const size_t np = (size_t)cam->W * cam->H;
  if ((st = grow(&ctx->d_cacc, &ctx->cacc_cap, np)) != LT_OK) return st;
  if ((st = grow_pinned(&ctx->h_frames, &ctx->h_frames_cap, 1)) != LT_OK) return st;
  ctx->h_frames[0] = F;
  LT_CUDA(cudaMemcpyAsync(ctx->d_frame_cen, ctx->h_frames, sizeof(FrameDev), cudaMemcpyHostToDevice, s));
  LT_CUDA(cudaMemsetAsync(&ctx->d_ctr->area_pairs, 0, 2 * sizeof(unsigned long long), s));
  // the fixed-point unit is the frame's: 2^-frac_bits of its mean column density
  LT_CUDA(lt::launch_area(ctx->L, ctx->d_frame_cen, cam->W, cam->H, F.m_tet, F.unit, ctx->d_cacc, d_image, ctx->d_ctr,
                          s));
  LT_CUDA(cudaStreamSynchronize(s));
  return LT_OK;
}

lt_status lt_render_hybrid(lt_ctx* ctx, const lt_camera* cam, int snapshot, double near_radius, float* d_image,
                           lt_stream stream) {
  if (!ctx || !cam || !d_image) return LT_ERR_ARG;
  if (!ctx->have_lattice) return LT_ERR_STATE;
  if (snapshot < 0 || snapshot >= ctx->n_snap || cam->type != LT_PERSP || !(near_radius > 0.0)) return LT_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  lt_camera c = *cam;
  c.near_radius = near_radius;
  const int snaps[1] = {snapshot};
  // the near cubes: exact projection
  lt_status st = project_bin_impl(ctx, &c, 1, snaps, s, false);
  if (st != LT_OK) return st;
  if ((st = render_impl(ctx, d_image, nullptr, s)) != LT_OK) return st;
  // the far cubes: centroid splats, added to the image
  return centroids_impl(ctx, c, snapshot, d_image, true, s);
}

lt_status lt_graph_build(lt_ctx* ctx, const lt_camera* cams, int n_frames, const int* frame_snapshot,
                         float* d_image, double* d_mass, lt_stream stream) {
  if (!ctx || !d_image) return LT_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (s == 0) return LT_ERR_ARG;  // capture needs a created stream
  // uncaptured pass: upload frames, size the bins
  lt_status st = project_bin_impl(ctx, cams, n_frames, frame_snapshot, s, false);
  if (st != LT_OK) return st;
  const unsigned long long want = ctx->entries + ctx->entries / 4 + 4096;
  if (want > ctx->list_cap) {
    size_t cap = ctx->list_cap;
    if ((st = grow(&ctx->d_list, &cap, (size_t)want)) != LT_OK) return st;
    ctx->list_cap = cap;
    // the reallocation dropped the lists just built: bin again, so that direct
    // renders of these frames stay valid
    if ((st = bin_launches(ctx, s, true)) != LT_OK) return st;
  }
  // the graph keeps its own copy of the frames, so that later direct calls
  // (which upload theirs into d_frames) leave its views unchanged
  if ((st = grow(&ctx->d_frames_graph, &ctx->frames_graph_cap, (size_t)n_frames)) != LT_OK) return st;
  LT_CUDA(cudaMemcpyAsync(ctx->d_frames_graph, ctx->d_frames, sizeof(FrameDev) * n_frames, cudaMemcpyDeviceToDevice,
                          s));
  LT_CUDA(cudaStreamSynchronize(s));
  if (ctx->graph_exec) { cudaGraphExecDestroy(ctx->graph_exec); ctx->graph_exec = nullptr; }
  if (ctx->graph) { cudaGraphDestroy(ctx->graph); ctx->graph = nullptr; }
  FrameDev* const direct_frames = ctx->d_frames;
  ctx->d_frames = ctx->d_frames_graph;
  LT_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  lt_status st2 = bin_launches(ctx, s, false);
  if (st2 == LT_OK) st2 = render_impl(ctx, d_image, d_mass, s);
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(s, &g);
  ctx->d_frames = direct_frames;
  if (st2 != LT_OK) {
    if (g) cudaGraphDestroy(g);
    return st2;
  }
  if (ce != cudaSuccess) {
    cudaGetLastError();
    return LT_ERR_CUDA;
  }
  ctx->graph = g;
  size_t n_nodes = 0;
  LT_CUDA(cudaGraphGetNodes(g, nullptr, &n_nodes));
  std::vector<cudaGraphNode_t> nodes(n_nodes);
  LT_CUDA(cudaGraphGetNodes(g, nodes.data(), &n_nodes));
  ctx->graph_kernels = 0;
  for (size_t q = 0; q < n_nodes; ++q) {
    cudaGraphNodeType ty;
    if (cudaGraphNodeGetType(nodes[q], &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++ctx->graph_kernels;
  }
  LT_CUDA(cudaGraphInstantiate(&ctx->graph_exec, g, 0));
  ctx->graph_stale = false;
  return LT_OK;
}

lt_status lt_graph_launch(lt_ctx* ctx, lt_stream stream) {
  if (!ctx) return LT_ERR_ARG;
  if (!ctx->graph_exec || ctx->graph_stale) return LT_ERR_STATE;
  LT_CUDA(cudaGraphLaunch(ctx->graph_exec, (cudaStream_t)stream));
  return LT_OK;
}

lt_status lt_autotune(lt_ctx* ctx, const lt_camera* cams, int n_frames, const int* frame_snapshot,
                      float* d_image, int reps, lt_config* best, lt_stream stream) {
  if (!ctx || !d_image || reps < 1) return LT_ERR_ARG;
  if (!ctx->have_lattice) return LT_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  const lt_config base = ctx->cfg;
  const int tiles[] = {16, 32, 64};
  const int threads[] = {128, 256};
  float best_ms = 1e30f;
  lt_config best_cfg = base;
  cudaEvent_t e0, e1;
  LT_CUDA(cudaEventCreate(&e0));
  LT_CUDA(cudaEventCreate(&e1));
  lt_status result = LT_OK;
  for (int ti : tiles) {
    for (int th : threads) {
      lt_config c = base;
      c.tile = ti;
      c.raster_threads = th;
      c.ctas_per_sm = 0;
      if (lt::raster_max_ctas_per_sm(th, ti, 1) < 1 || lt::raster_max_ctas_per_sm(th, ti, 0) < 1) continue;
      ctx->cfg = c;
      lt_status st = project_bin_impl(ctx, cams, n_frames, frame_snapshot, s, false);
      if (st == LT_OK) st = render_impl(ctx, d_image, nullptr, s);
      if (st != LT_OK) { result = st; break; }
      cudaEventRecord(e0, s);
      for (int r = 0; r < reps && st == LT_OK; ++r) {
        st = project_bin_impl(ctx, cams, n_frames, frame_snapshot, s, false);
        if (st == LT_OK) st = render_impl(ctx, d_image, nullptr, s);
      }
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess || st != LT_OK) { result = st != LT_OK ? st : LT_ERR_CUDA; break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best_ms) {
        best_ms = ms;
        best_cfg = c;
      }
    }
    if (result != LT_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->cfg = result == LT_OK ? best_cfg : base;
  ctx->binned = false;
  if (best) *best = ctx->cfg;
  return result;
}

lt_status lt_sync(lt_ctx* ctx, lt_stream stream) {
  if (!ctx) return LT_ERR_ARG;
  LT_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  return take_device_errors(ctx);
}

lt_status lt_get_stats(lt_ctx* ctx, lt_stats* out) {
  if (!ctx || !out) return LT_ERR_ARG;
  LT_CUDA(cudaDeviceSynchronize());
  lt_status st = take_device_errors(ctx);
  const DevCounters& c = *ctx->h_ctr;
  memset(out, 0, sizeof *out);
  out->tets = ctx->have_lattice ? 6 * ctx->L.n_particles : 0;
  out->entries = (long long)ctx->entries;
  out->capacity = (long long)ctx->list_cap;
  out->degenerate = (long long)c.degenerate;
  out->fp64_fallbacks = (long long)c.fp64_fallbacks;
  out->inverted = (long long)c.inverted;
  out->nonfinite = (long long)c.nonfinite;
  out->behind_eye = (long long)c.behind_eye;
  out->range_overflow = (long long)c.range_overflow;
  out->exact_fragments = (long long)c.exact_fragments;
  out->queue_overflow = (long long)c.queue_overflow;
  out->resample_intervals = (long long)c.resample_intervals;
  out->resample_pieces = (long long)c.resample_pieces;
  out->area_pairs = (long long)c.area_pairs;
  out->area_fp64_pairs = (long long)c.area_fp64_pairs;
  out->exact_tile_max = (long long)c.exact_tile_max;
  out->n_frames = ctx->n_frames;
  out->tile = ctx->tile;
  out->graph_kernels = ctx->graph_kernels;
  return st;
}

}  // extern "C"
