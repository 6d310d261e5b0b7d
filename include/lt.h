/*
 * lt.h -- C ABI of the GB300 column-density renderer for the Lagrangian
 * tetrahedral tessellation of a periodic particle lattice
 * (Kaehler, Hahn & Abel, "A Novel Approach to Visualizing Dark Matter
 * Simulations", arXiv:1208.3206).
 *
 * What the library computes (Sec. 3.2, Eq. 6 with the density of Eq. 3):
 * for every pixel of every requested frame,
 *
 *     I(pixel) = sum over tetrahedra t of rho_t * dl_t(pixel),
 *
 * rho_t = m / |V_t| the constant density of tetrahedron t (V_t from Eq. 9),
 * m = total_mass / (6 N^3), and dl_t(pixel) the length of the ray through the
 * pixel centre inside t. The tetrahedra are the six per cube of the initial
 * N^3 particle lattice (Sec. 3.1, connectivity table of Sec. 4.1), built on
 * the fly from the particle id <-> lattice index map (Eq. 8); no
 * connectivity is stored.
 *
 * Conventions shared by every entry point:
 *   - Device pointers are CUDA device memory owned by the caller; the
 *     library never frees or keeps a pointer it did not allocate, except the
 *     position buffer registered by lt_build_tets, which must stay valid and
 *     unchanged in shape until the next lt_build_tets or lt_destroy.
 *   - Host pointers are read during the call only.
 *   - Calls are asynchronous on the given stream (0 = legacy default
 *     stream) unless stated otherwise. Errors the device detects (capacity
 *     overflow, non-finite positions, vertices behind a perspective eye,
 *     accumulator range) are latched in the context and returned by the next
 *     synchronising call (lt_get_stats, lt_sync).
 *   - Every function returns an lt_status and never aborts the process.
 *   - A context is used by one host thread at a time.
 *
 * Layouts:
 *   - positions, LT_POS_F32X4: float4 (x, y, z, unused) per particle, id
 *     order i + N (j + N k) (Eq. 8), wrapped into [0, box)^3; n_snapshots
 *     arrays of N^3 particles back to back.
 *   - positions, LT_POS_F16_OFFSETS: 4 halves (dx, dy, dz, unused) per
 *     particle, the displacement from the particle's lattice point in units
 *     of the lattice spacing box / N (not wrapped).
 *   - images: float [n_frames][H][W], row py along the camera's up axis,
 *     pixel (px, py) centred at ((px + 1/2) / W, (py + 1/2) / H) of the view.
 *   - tetrahedron id: 6 * (i + N (j + N k)) + s, s the row of the
 *     connectivity table of Sec. 4.1 for cube (i, j, k).
 */
#ifndef LT_H_
#define LT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* lt_stream; /* a cudaStream_t */

typedef enum {
  LT_OK = 0,
  LT_ERR_ARG = 1,         /* invalid argument: null pointer, bad size or enum */
  LT_ERR_CUDA = 2,        /* a CUDA runtime call failed */
  LT_ERR_CAPACITY = 3,    /* a bin list outgrew its reserved capacity */
  LT_ERR_NONFINITE = 4,   /* a particle position is NaN or infinite */
  LT_ERR_BEHIND_EYE = 5,  /* a cube straddles the eye plane of a perspective frame */
  LT_ERR_RANGE = 6,       /* a pixel exceeded the 64-bit fixed-point accumulator range (see frac_bits) */
  LT_ERR_STATE = 7,       /* calls made out of order (e.g. render before bin) */
  LT_ERR_NOMEM = 8,       /* device allocation failed */
  LT_ERR_BOUNDS = 9       /* an index check failed (only in a build with LT_CHECK_BOUNDS) */
} lt_status;

typedef enum { LT_POS_F32X4 = 0, LT_POS_F16_OFFSETS = 1 } lt_pos_format;
typedef enum { LT_WEIGHT_DENSITY = 0, LT_WEIGHT_STREAMS = 1 } lt_resample_weight;
typedef enum { LT_ORTHO = 0, LT_PERSP = 1 } lt_camera_type;

/* One view. right = normalize(up x fwd), up' = fwd x right.
 * LT_ORTHO: rays along fwd through the window [lo, hi] of the (right, up')
 *   coordinates of world points; wrap != 0 makes the window periodic (every
 *   periodic copy of a tetrahedron is drawn; use a window one box wide).
 * LT_PERSP: rays from eye (half-lines); vertical field of view fov_y_deg,
 *   square pixels. A cube entirely behind the eye plane is not drawn (no ray
 *   reaches it); a cube straddling the eye plane cannot be projected and
 *   latches LT_ERR_BEHIND_EYE.
 * The view is set up in double precision on the host; each cube's projected
 * anchor point is carried to the kernels with about 2^-37 relative error, so
 * pixel positions are exact to well below a millionth of a pixel. */
typedef struct {
  int type;
  double eye[3];
  double fwd[3];
  double up[3];
  double fov_y_deg;
  double lo[2];
  double hi[2];
  int W, H;
  int wrap;
  /* hybrid near/far rendering (perspective only, 0 = off): with r > 0 the
   * exact raster (lt_project_bin, lt_render_tiles, graphs) draws only the
   * cubes whose corner-0 particle lies within r of the eye, and
   * lt_render_centroids only the others; lt_render_hybrid draws both */
  double near_radius;
} lt_camera;

/* Tuning knobs (lt_autotune fills them; zero fields take defaults). */
typedef struct {
  int tile;           /* screen tile edge in pixels: 8, 16, 32 or 64 (default 16) */
  int raster_threads; /* threads per raster CTA: 64..256, multiple of 32 (default 256) */
  int ctas_per_sm;    /* persistent raster CTAs per SM (default: occupancy limit) */
  int frac_bits;      /* fixed-point fraction bits relative to the mean column density sigma, 8..62
                         (default 28): each pixel is summed in a 64-bit integer that resolves
                         2^-frac_bits sigma and holds values below 2^(64 - frac_bits) sigma; a pixel
                         that would pass that latches LT_ERR_RANGE */
} lt_config;

typedef struct {
  long long tets;            /* tetrahedra per snapshot, 6 N^3 */
  long long entries;         /* (tile, cube) bin entries of the last lt_project_bin */
  long long capacity;        /* reserved bin entries */
  long long degenerate;      /* tetrahedra with V == 0 found by lt_build_tets */
  long long fp64_fallbacks;  /* volumes recomputed in FP64 by lt_build_tets */
  long long inverted;        /* tetrahedra with V > 0 (orientation flipped vs t = 0) */
  long long nonfinite;       /* non-finite positions seen */
  long long behind_eye;      /* cubes skipped because they straddle a perspective eye plane */
  long long range_overflow;  /* pixels that left the accumulator range */
  long long exact_fragments; /* ill-conditioned fragments re-evaluated in FP64 (cumulative) */
  long long queue_overflow;  /* such fragments left in FP32 because a CTA's queue (64 per pixel of a tile) was full */
  long long resample_intervals; /* lt_resample: (tetrahedron, grid line) pairs of positive length, last call */
  long long resample_pieces;    /* lt_resample: their pieces in separate slabs (cell adds), last call */
  long long area_pairs;         /* lt_render_area: (tetrahedron, pixel) pairs walked, last call */
  long long area_fp64_pairs;    /* lt_render_area: of them, clipped in FP64 (hulls under 1/20 pixel wide, or an
                                   apex within 1e-3 pixel of a hull edge) */
  long long exact_tile_max;     /* most ill-conditioned fragments found in one tile since lt_create (the queue
                                   holds 64 per pixel of a tile) */
  int n_frames;              /* frames of the last lt_project_bin */
  int tile;                  /* tile edge in use */
  int graph_kernels;         /* kernel nodes in the graph of the last lt_graph_build */
  int pad;
} lt_stats;

typedef struct lt_ctx lt_ctx;

/* Create a context bound to the current CUDA device. cfg may be NULL.
 * Ownership: the context owns every scratch buffer it allocates (bins,
 * offsets, work queue, counters); lt_destroy frees them. */
lt_status lt_create(lt_ctx** out, const lt_config* cfg);
void lt_destroy(lt_ctx* ctx);

/* Replace the tuning knobs (takes effect at the next lt_project_bin). */
lt_status lt_set_config(lt_ctx* ctx, const lt_config* cfg);
lt_status lt_get_config(const lt_ctx* ctx, lt_config* out);

/*
 * lt_build_tets -- Sec. 3.1 / Sec. 4.1 (tessellation and per-tetrahedron
 * volume and density, Eq. 8, 9 and 3).
 * Registers n_snapshots position arrays at d_pos (layout above, caller
 * owned, read by every later call) for a lattice of N^3 particles in a
 * periodic box of edge `box` holding `total_mass`. Checks every position
 * for finiteness and computes, for every tetrahedron of every snapshot, the
 * signed volume V (FP32 from displacement differences, recomputed in FP64
 * when |V| < 0.1 of a lattice cell, where the FP32 error bound would pass
 * 1e-5; this covers every near-degenerate sheet tetrahedron at caustics) and
 * rho = m / |V| (0 when V == 0). Tetrahedra with V == 0 are marked in a
 * context-owned mask (one byte per cube and snapshot) and contribute nothing
 * to any later render. If d_rho is not NULL it receives rho as float
 * [n_snapshots][6 N^3] (tetrahedron id order).
 * Errors: LT_ERR_ARG (N < 1, N^3 > 2^31, box <= 0, total_mass <= 0,
 * n_snapshots < 1, unknown pos_fmt, misaligned d_pos); non-finite positions
 * latch LT_ERR_NONFINITE.
 */
lt_status lt_build_tets(lt_ctx* ctx, const void* d_pos, int pos_fmt, int N, float box, double total_mass,
                        int n_snapshots, float* d_rho, lt_stream stream);

/*
 * lt_project_bin -- project-and-bin pass (the screen-space counterpart of
 * the rasterisation step of Sec. 4.4).
 * For each of n_frames views cams[f] (host array) of snapshot
 * frame_snapshot[f] (host array, NULL = snapshot 0 for every frame), bins
 * every lattice cube into the screen tiles its projected bounding box
 * overlaps: warp-aggregated per-tile counts, a device exclusive scan, then a
 * scatter of cube ids into per-tile lists. Also orders the (frame, tile) work
 * items by descending list length for the raster pass.
 * Outside stream capture the call synchronises once to size the lists
 * (growing the context's buffers as needed). Inside stream capture it uses
 * the reserved capacity and latches LT_ERR_CAPACITY if it is exceeded.
 * Errors: LT_ERR_STATE (no lt_build_tets), LT_ERR_ARG (n_frames < 1, bad
 * camera, snapshot out of range, W or H < 1 or > 65536).
 */
lt_status lt_project_bin(lt_ctx* ctx, const lt_camera* cams, int n_frames, const int* frame_snapshot,
                         lt_stream stream);

/*
 * lt_render_tiles -- the projection of Eq. 6 for every frame of the last
 * lt_project_bin. One persistent launch; each CTA takes (frame, tile) work
 * items, accumulates rho_t * dl_t of every tetrahedron of the tile's cubes
 * into on-chip fixed-point integer sums (so the image is bit-reproducible
 * whatever the order), and stores every pixel once. Fragments whose FP32
 * value may be off by more than 1e-5 of max(value, mean column density)
 * (thin slivers, steep edges) are re-evaluated exactly in FP64 by clipping
 * the pixel ray against the four faces; tetrahedra with V == 0 contribute
 * nothing. A graph replay whose lists outgrew their capacity draws only the
 * entries the lists hold and latches LT_ERR_CAPACITY.
 * d_image: float [n_frames][H][W] (caller owned). d_mass (may be NULL):
 * double [n_frames], per frame the sum of pixel values times the pixel area
 * (orthographic: window area / (W H); perspective: area on the image plane
 * at unit distance), reduced in a fixed order.
 * Errors: LT_ERR_STATE (no lt_project_bin), LT_ERR_ARG (null d_image).
 */
lt_status lt_render_tiles(lt_ctx* ctx, float* d_image, double* d_mass, lt_stream stream);

/*
 * lt_render_atomic -- the plain form of Eq. 6: one thread per lattice cube
 * over all frames, every fragment added to the image with a float atomic
 * (order dependent in the last bits). Same arithmetic per tetrahedron as
 * lt_render_tiles; it needs no bins. d_image must be zeroed by the caller.
 * Errors: LT_ERR_STATE (no lt_build_tets), LT_ERR_ARG.
 */
lt_status lt_render_atomic(lt_ctx* ctx, const lt_camera* cams, int n_frames, const int* frame_snapshot,
                           float* d_image, lt_stream stream);

/*
 * lt_count_fragments -- number of (tetrahedron, pixel) pairs with a positive
 * chord in each frame of the last lt_project_bin (the work unit of the
 * benchmark). Synchronises; h_counts: host long long [n_frames].
 */
lt_status lt_count_fragments(lt_ctx* ctx, long long* h_counts, lt_stream stream);

/*
 * lt_render_backward -- adjoint of lt_render_tiles (the derivative of
 * Eq. 6 with respect to particle positions). Given dL/dI as float
 * [n_frames][H][W] for the frames of the last lt_project_bin, writes
 * dL/d(position) as float [n_snapshots][N^3][3] into d_dL_dpos (overwritten,
 * caller owned). Deterministic: per-tetrahedron gradients are gathered per
 * particle in a fixed order, no float atomics.
 * Errors: LT_ERR_STATE, LT_ERR_ARG.
 */
lt_status lt_render_backward(lt_ctx* ctx, const float* d_dL_dimage, float* d_dL_dpos, lt_stream stream);

/*
 * lt_resample -- resampling onto a periodic grid (Sec. 4.3, Eq. 10-12) and
 * the stream-count field (Sec. 3.2).
 * For snapshot `snapshot` of the registered lattice, fills d_grid (float
 * [n][n][n], index (c n + b) n + a, caller owned) with, for every cell
 * (a, b, c) of edge g = box / n, the sum over tetrahedra t of q_t times the
 * length of the part of the cell's central line along z, x = (a + 1/2) g,
 * y = (b + 1/2) g, that lies inside t and inside the slab [c g, (c + 1) g)
 * (every periodic copy of t counts). weight LT_WEIGHT_DENSITY: q_t = rho_t
 * (Eq. 3), so a cell holds rho dl, its mass over its face area;
 * LT_WEIGHT_STREAMS: q_t = 1, so a cell over g is the mean number of streams
 * on its line. Each (tetrahedron, line) interval is found exactly in FP64 by
 * clipping the line against the four face planes; the cells are summed as
 * 64-bit fixed-point integers (2^-frac_bits of the mean cell), so the grid
 * is bitwise reproducible. Tetrahedra with V == 0 contribute nothing.
 * Uses the project-and-bin pass with an orthographic view along z whose
 * pixels are the grid's columns, so it replaces the frames and bins of the
 * last lt_project_bin (render or count afterwards only after a new
 * lt_project_bin), synchronises once to size the bins, and keeps an n^3
 * array of 64-bit cells in the context.
 * Errors: LT_ERR_STATE (no lt_build_tets), LT_ERR_ARG (null d_grid, n < 1 or
 * n > 2048, unknown weight, snapshot out of range), LT_ERR_NOMEM; a cell
 * leaving the fixed-point range latches LT_ERR_RANGE.
 */
lt_status lt_resample(lt_ctx* ctx, int n, int weight, int snapshot, float* d_grid, lt_stream stream);

/*
 * lt_slice -- a 2D slice of the total density of overlapping streams (Sec.
 * 3.2, Eq. 4) or of the number of streams, on the plane z = z0 of the
 * periodic box.
 * For snapshot `snapshot` of the registered lattice, fills d_img (float
 * [n][n], index b n + a, caller owned) with, at the point
 * ((a + 1/2) box / n, (b + 1/2) box / n, z0), the sum over the tetrahedra
 * that contain it (every periodic copy counts) of rho_t = m / |V_t|
 * (LT_WEIGHT_DENSITY: the total density) or of 1 (LT_WEIGHT_STREAMS: the
 * number of streams). The containment test is done in FP64 against the four
 * face planes; a point on a face counts for both tetrahedra sharing it.
 * Sums are 64-bit fixed point in units of 2^-frac_bits of the mean density
 * (of one stream: counts are exact), so the slice is bitwise reproducible.
 * Tetrahedra with V == 0 contribute nothing. Asynchronous; leaves the bins
 * of the last lt_project_bin untouched; keeps an n^2 array of 64-bit sums in
 * the context.
 * Errors: LT_ERR_STATE (no lt_build_tets), LT_ERR_ARG (null d_img, n < 1 or
 * n > 32768, unknown weight, z0 not finite, snapshot out of range),
 * LT_ERR_NOMEM; a point leaving the fixed-point range latches LT_ERR_RANGE.
 */
lt_status lt_slice(lt_ctx* ctx, int n, int weight, int snapshot, double z0, float* d_img, lt_stream stream);

/*
 * lt_render_centroids -- the centroid rendering of Sec. 4.2 for one view:
 * every tetrahedron of snapshot `snapshot` is drawn as a 2D kernel on a
 * billboard through its centroid c_T = (v0 + v1 + v2 + v3) / 4, facing the
 * view direction, scaled with (m / rho_T)^(1/3) = |V_T|^(1/3) and carrying
 * the tetrahedron's mass m. The paper leaves the kernel's form and the scale
 * factor open; this library takes the 2D M4 cubic spline with unit integral
 * and smoothing length h = |V_T|^(1/3) (support radius 2h). A pixel (centre
 * sample) adds m W(d, h) for each billboard its ray crosses, d the distance
 * of the crossing from the centroid, over the cosine of the ray's angle to
 * the view direction (1 for orthographic views): an estimate of the column
 * density. Perspective billboards behind the eye are not drawn; a periodic
 * orthographic window draws every periodic copy. With cam->near_radius > 0
 * only the cubes beyond it are drawn (the far part of lt_render_hybrid).
 * Pixels are summed as 64-bit fixed-point integers (2^-frac_bits of the mean
 * column density), so the image is bitwise reproducible. Tetrahedra with
 * V == 0 carry no splat.
 * d_image: float [H][W] (caller owned, overwritten). Synchronises (the view
 * is staged through the context's pinned memory); keeps an H x W array of
 * 64-bit sums in the context; leaves the bins of lt_project_bin untouched.
 * Errors: LT_ERR_STATE (no lt_build_tets), LT_ERR_ARG (null pointer,
 * invalid camera, snapshot out of range), LT_ERR_NOMEM; a pixel leaving the
 * fixed-point range, or a splat covering more than 2^31 pixels of the window
 * (which is then left out), latches LT_ERR_RANGE.
 */
lt_status lt_render_centroids(lt_ctx* ctx, const lt_camera* cam, int snapshot, float* d_image, lt_stream stream);

/*
 * lt_render_area -- area-averaged pixels of one orthographic view (Sec. 3.2,
 * Eq. 6 integrated over each pixel): pixel (x, y) holds the mean of the
 * column density over its square (the window split into W x H equal
 * squares) rather than its value at the pixel centre, so features thinner
 * than a pixel keep their projected mass in the pixels they cross. Each
 * tetrahedron's chord is integrated exactly: it is linear on the triangles
 * joining the projected apex to the edges of the projected hull, and
 * rho_t times the chord at the apex is 3 m / (hull area). A periodic window
 * draws every periodic copy. Pixels are summed as 64-bit fixed-point integers
 * (2^-frac_bits of the mean column density), so the image is bitwise
 * reproducible and the frame mass is the projected mass up to that rounding.
 * Tetrahedra with V == 0 carry nothing. lt_stats.area_pairs counts the
 * (tetrahedron, pixel) pairs walked.
 * d_image: float [H][W] (caller owned, overwritten). Synchronises; keeps an
 * H x W array of 64-bit sums in the context; leaves the bins of
 * lt_project_bin untouched.
 * Errors: LT_ERR_STATE (no lt_build_tets), LT_ERR_ARG (null pointer, invalid
 * or perspective camera, snapshot out of range), LT_ERR_NOMEM; a pixel
 * leaving the fixed-point range, or a tetrahedron covering more than 2^31
 * pixels of the window (which is then left out), latches LT_ERR_RANGE.
 */
lt_status lt_render_area(lt_ctx* ctx, const lt_camera* cam, int snapshot, float* d_image, lt_stream stream);

/*
 * lt_render_hybrid -- hybrid near/far rendering of one perspective view
 * (Sec. 6, Fig. "LargeScale"): the cubes whose corner-0 particle lies within
 * near_radius (> 0) of the eye are drawn by the exact projection of Eq. 6
 * (lt_project_bin + lt_render_tiles), the other cubes' tetrahedra as
 * centroid splats (lt_render_centroids); d_image (float [H][W], caller
 * owned) receives the sum. Replaces the frames and bins of the last
 * lt_project_bin; synchronises.
 * Errors: as lt_project_bin and lt_render_centroids; LT_ERR_ARG for an
 * orthographic view or near_radius <= 0.
 */
lt_status lt_render_hybrid(lt_ctx* ctx, const lt_camera* cam, int snapshot, double near_radius, float* d_image,
                           lt_stream stream);

/*
 * lt_graph_build / lt_graph_launch -- capture lt_project_bin followed by
 * lt_render_tiles for the given frames into a CUDA graph owned by the
 * context, and replay it. lt_graph_build runs the pass once uncaptured to
 * size the bins (reserving 25 % headroom), then captures on `stream`.
 * Replays re-read the registered positions, so new snapshot contents
 * (same shape) may be written between launches. Capacity overflow during a
 * replay latches LT_ERR_CAPACITY. The graph keeps its own copy of its
 * frames: direct calls made after lt_graph_build do not change its views.
 * A later lt_build_tets, or a direct call that has to reallocate a buffer
 * the graph uses (more frames or tiles, longer lists), makes the graph stale:
 * lt_graph_launch then returns LT_ERR_STATE until lt_graph_build runs again.
 */
lt_status lt_graph_build(lt_ctx* ctx, const lt_camera* cams, int n_frames, const int* frame_snapshot,
                         float* d_image, double* d_mass, lt_stream stream);
lt_status lt_graph_launch(lt_ctx* ctx, lt_stream stream);

/*
 * lt_autotune -- time lt_project_bin + lt_render_tiles for the given
 * frames over a small grid of tile sizes (16, 32, 64) and raster CTA shapes
 * (128, 256 threads) (CUDA
 * events, `reps` timed repetitions each after one warm-up), keep the
 * fastest in the context and report it in *best (may be NULL).
 * Synchronises. d_image: scratch float [n_frames][H][W].
 */
lt_status lt_autotune(lt_ctx* ctx, const lt_camera* cams, int n_frames, const int* frame_snapshot,
                      float* d_image, int reps, lt_config* best, lt_stream stream);

/*
 * lt_frame_mass_static -- the per-frame mass of images the caller already
 * holds: for each frame, the sum of its pixel values times pixel_area, in
 * FP64 and in a fixed order (the reduction lt_render_tiles does for
 * d_mass). The paper has no counterpart: it exists for callers that must
 * not allocate device memory, for example one whose memory pool owns all
 * free device memory, or one that must not hit the implicit device
 * synchronisation an allocation or a free can cause. It allocates nothing
 * and needs no context.
 *
 * d_image: float [n_frames][H][W] (caller owned, read only). d_mass: double
 * [n_frames] (caller owned, overwritten). pixel_area > 0: one value for all
 * frames (orthographic: window area / (W H); perspective: the image-plane
 * pixel area at unit distance, as lt_render_tiles uses). Asynchronous on
 * `stream`.
 *
 * Scratch: one static device array per GPU of 155,648 bytes (128 frames x
 * 152 partial sums). It needs no initialisation: every partial is written
 * before it is read. Because it is shared, calls that can run at the same
 * time on one device (several streams or host threads) race on it and give
 * wrong sums: order them (one stream, or events between streams).
 * The first call on each device looks up the scratch address with that
 * device current; make that first call before any stream capture begins.
 *
 * Errors: LT_ERR_ARG (null pointer, n_frames, W or H < 1, pixel_area not a
 * positive finite number), LT_ERR_CAPACITY (n_frames > 128: split the
 * frames over several calls), LT_ERR_CUDA (symbol lookup or launch failed).
 */
lt_status lt_frame_mass_static(const float* d_image, int n_frames, int W, int H, double pixel_area, double* d_mass,
                               lt_stream stream);

/* Wait for the stream, then return (and clear) the first latched device error. */
lt_status lt_sync(lt_ctx* ctx, lt_stream stream);

/* Synchronise and read counters; returns the first latched error (and clears it). */
lt_status lt_get_stats(lt_ctx* ctx, lt_stats* out);

/* Static string for a status code. */
const char* lt_status_str(lt_status s);

#ifdef __cplusplus
}
#endif
#endif /* LT_H_ */
