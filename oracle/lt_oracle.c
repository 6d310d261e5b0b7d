/*
 * FP64 CPU oracle for the line-of-sight projection of the Lagrangian
 * tetrahedral tessellation (Kaehler, Hahn & Abel, arXiv:1208.3206).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plain definition that the
 * GPU path is checked against. Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it; the product library never does.
 * It shares no code, header, table or constant with the CUDA sources.
 *
 * What it computes, step by step in the paper's order:
 *   - the particle id <-> lattice index map, Eq. 8 (Sec. 4.1);
 *   - the six tetrahedra of each lattice cube from the connectivity table of
 *     Sec. 4.1 / Fig. "TetraSplit" (Sec. 3.1);
 *   - the signed volume, Eq. 9, and the per-tetrahedron density m / |V|,
 *     Eq. 3 (Sec. 3.2);
 *   - the line-of-sight projection q_proj = sum_i q_i * dl_i, Eq. 6
 *     (Sec. 3.2), with dl_i the exact length of the pixel ray inside
 *     tetrahedron i, found by clipping the ray against the four face planes.
 *   - the gradient of that projection with respect to particle positions,
 *     by differentiating rho_i * dl_i directly (density through the volume,
 *     chord through the entry and exit face planes).
 *   - area-averaged pixels of orthographic views (orc_render_area): the
 *     mean of Eq. 6 over each pixel's square, each tetrahedron's chord
 *     integrated exactly over its piecewise-linear pieces.
 *
 * Readings where the paper is silent:
 *   - corner n of a cube is lattice point (i+(n&1), j+((n>>1)&1), k+((n>>2)&1));
 *   - the lattice is periodic: N^3 cubes, corner indices taken mod N, each
 *     vertex unwrapped to the minimum image of its Lagrangian position;
 *   - m = total_mass / (6 N^3) for every tetrahedron;
 *   - a pixel's value is the projection along the ray through its centre;
 *   - a tetrahedron with V == 0 exactly contributes nothing;
 *   - orthographic windows may be periodic in both image axes (wrap), in
 *     which case every periodic copy of a tetrahedron is drawn; perspective
 *     views draw the single unwrapped copy of the lattice;
 *   - an area-averaged pixel splits the window into W x H equal squares,
 *     pixel (px, py) covering [px, px + 1) x [py, py + 1) in pixel units;
 *   - the tetrahedron is closed: a ray lying exactly in the plane of a face
 *     parallel to it counts the segment it shares with the face (the value
 *     there is the upper one-sided limit of a jump).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Connectivity of the six tetrahedra inside one cube (Sec. 4.1). */
static const int CUBE_TETS[6][4] = {
    {1, 0, 2, 4}, {3, 1, 2, 4}, {3, 5, 1, 4}, {3, 6, 5, 4}, {3, 2, 6, 4}, {3, 7, 5, 6}};

typedef struct {
  int type;           /* 0 orthographic, 1 perspective */
  double eye[3];      /* perspective eye position */
  double fwd[3];      /* viewing direction (need not be unit) */
  double up[3];       /* up hint (need not be unit or orthogonal) */
  double fov_y_deg;   /* perspective vertical field of view */
  double lo[2], hi[2];/* orthographic window in (right, up) coordinates */
  int W, H;           /* image size in pixels */
  int wrap;           /* orthographic only: window is periodic */
} orc_camera;

enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_BEHIND_EYE = 2 };

/* ---------- small vector helpers ---------- */
static void sub3(const double* a, const double* b, double* o) {
  o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2];
}
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double* a, const double* b, double* o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}
static void normalize3(double* a) {
  double n = sqrt(dot3(a, a));
  a[0] /= n; a[1] /= n; a[2] /= n;
}

/* ---------- camera frame ---------- */
typedef struct {
  int persp, W, H, wrap;
  double eye[3], r[3], u[3], f[3];
  double tan_x, tan_y;
  double lo[2], hi[2];
} frame_t;

static int frame_init(const orc_camera* c, frame_t* fr) {
  if (c->W <= 0 || c->H <= 0) return ORC_ERR_ARG;
  fr->persp = c->type == 1;
  fr->W = c->W; fr->H = c->H;
  fr->wrap = (!fr->persp) && c->wrap;
  memcpy(fr->eye, c->eye, sizeof fr->eye);
  memcpy(fr->f, c->fwd, sizeof fr->f);
  normalize3(fr->f);
  cross3(c->up, fr->f, fr->r); /* right = up x forward */
  normalize3(fr->r);
  cross3(fr->f, fr->r, fr->u); /* true up = forward x right */
  fr->tan_y = tan(0.5 * c->fov_y_deg * M_PI / 180.0);
  fr->tan_x = fr->tan_y * (double)c->W / (double)c->H;
  fr->lo[0] = c->lo[0]; fr->lo[1] = c->lo[1];
  fr->hi[0] = c->hi[0]; fr->hi[1] = c->hi[1];
  return ORC_OK;
}

/* Continuous pixel coordinate of a world point: pixel px has its centre at
 * fx == px. Returns 0 if the point is not in front of a perspective eye. */
static int to_pixel(const frame_t* fr, const double* X, double* fx, double* fy) {
  if (!fr->persp) {
    double a = dot3(fr->r, X), b = dot3(fr->u, X);
    *fx = (a - fr->lo[0]) / (fr->hi[0] - fr->lo[0]) * fr->W - 0.5;
    *fy = (b - fr->lo[1]) / (fr->hi[1] - fr->lo[1]) * fr->H - 0.5;
    return 1;
  }
  double c[3];
  sub3(X, fr->eye, c);
  double z = dot3(fr->f, c);
  if (!(z > 0.0)) return 0;
  double xt = dot3(fr->r, c) / z, yt = dot3(fr->u, c) / z;
  *fx = (xt / fr->tan_x + 1.0) * 0.5 * fr->W - 0.5;
  *fy = (yt / fr->tan_y + 1.0) * 0.5 * fr->H - 0.5;
  return 1;
}

/* Ray through the centre of (unwrapped) pixel (px, py): origin o, unit
 * direction d. Orthographic rays are full lines, perspective rays start at
 * the eye. */
static void pixel_ray(const frame_t* fr, long px, long py, double* o, double* d) {
  if (!fr->persp) {
    double a = fr->lo[0] + (px + 0.5) * (fr->hi[0] - fr->lo[0]) / fr->W;
    double b = fr->lo[1] + (py + 0.5) * (fr->hi[1] - fr->lo[1]) / fr->H;
    for (int q = 0; q < 3; ++q) { o[q] = a * fr->r[q] + b * fr->u[q]; d[q] = fr->f[q]; }
    return;
  }
  double xt = fr->tan_x * (2.0 * (px + 0.5) / fr->W - 1.0);
  double yt = fr->tan_y * (2.0 * (py + 0.5) / fr->H - 1.0);
  for (int q = 0; q < 3; ++q) { o[q] = fr->eye[q]; d[q] = fr->f[q] + xt * fr->r[q] + yt * fr->u[q]; }
  normalize3(d);
}

/* ---------- tessellation ---------- */

/* Unwrapped corner position: Lagrangian point of lattice index (ii,jj,kk)
 * (not reduced mod N) plus the minimum-image displacement of the particle
 * stored at that index mod N. Particle id follows Eq. 8 with d0 = d1 = N. */
static void corner_position(const double* pos, int N, double box, long ii, long jj, long kk, double* v) {
  long i = ii % N, j = jj % N, k = kk % N;
  long id = i + (long)N * (j + (long)N * k);
  double h = box / N;
  double q[3] = {ii * h, jj * h, kk * h};
  for (int a = 0; a < 3; ++a) {
    double dd = pos[3 * id + a] - q[a];
    dd -= box * nearbyint(dd / box);
    v[a] = q[a] + dd;
  }
}

/* Vertices of tetrahedron s of cube (i,j,k), in the table's order. */
static void tet_vertices(const double* pos, int N, double box, long i, long j, long k, int s, double v[4][3]) {
  for (int c = 0; c < 4; ++c) {
    int n = CUBE_TETS[s][c];
    corner_position(pos, N, box, i + (n & 1), j + ((n >> 1) & 1), k + ((n >> 2) & 1), v[c]);
  }
}

/* Signed volume, Eq. 9. */
static double tet_volume(double v[4][3]) {
  double a[3], b[3], c[3], bc[3];
  sub3(v[1], v[0], a); sub3(v[2], v[0], b); sub3(v[3], v[0], c);
  cross3(b, c, bc);
  return dot3(a, bc) / 6.0;
}

/* Exact chord of the ray o + s d (|d| = 1) through the tetrahedron: clip
 * against the four face planes. s starts at -inf for a full line and at 0
 * for a half-line. Optionally reports which face bounds the entry / exit. */
static double ray_chord(double v[4][3], const double* o, const double* d, int halfline, int* f_in,
                        int* f_out, double* s_in_out, double* s_out_out) {
  double s_in = halfline ? 0.0 : -INFINITY, s_out = INFINITY;
  int fin = -1, fout = -1;
  for (int i = 0; i < 4; ++i) {
    const double *a = v[(i + 1) & 3], *b = v[(i + 2) & 3], *c = v[(i + 3) & 3];
    double e1[3], e2[3], n[3], t[3];
    sub3(b, a, e1); sub3(c, a, e2);
    cross3(e1, e2, n);
    sub3(v[i], a, t);
    if (dot3(n, t) > 0.0) { n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2]; } /* outward */
    double ao[3];
    sub3(a, o, ao);
    double den = dot3(n, d), num = dot3(n, ao); /* inside: s * den <= num */
    if (den > 0.0) {
      double s = num / den;
      if (s < s_out) { s_out = s; fout = i; }
    } else if (den < 0.0) {
      double s = num / den;
      if (s > s_in) { s_in = s; fin = i; }
    } else if (num < 0.0) {
      return 0.0;
    }
  }
  if (f_in) *f_in = fin;
  if (f_out) *f_out = fout;
  if (s_in_out) *s_in_out = s_in;
  if (s_out_out) *s_out_out = s_out;
  return s_out > s_in ? s_out - s_in : 0.0;
}

/* Range of periodic image shifts (in units of W) that bring the pixel span
 * [a, b] into overlap with [lo, hi]. */
static void shift_range(long a, long b, long lo, long hi, long period, int wrap, long* s0, long* s1) {
  if (!wrap) { *s0 = 0; *s1 = 0; return; }
  /* need a + s*period <= hi and b + s*period >= lo */
  double lo_s = ceil((double)(lo - b) / period), hi_s = floor((double)(hi - a) / period);
  *s0 = (long)lo_s; *s1 = (long)hi_s;
}

/* Pixel bounding box of a tetrahedron: pixels whose centres lie inside the
 * bounding box of the projected vertices. Returns 1 on success, 0 when the
 * tetrahedron lies entirely behind a perspective eye (no ray reaches it; the
 * box is empty), -1 when it straddles the eye plane (cannot be projected). */
static int tet_pixel_box(const frame_t* fr, double v[4][3], long* x0, long* x1, long* y0, long* y1) {
  double mnx = INFINITY, mxx = -INFINITY, mny = INFINITY, mxy = -INFINITY;
  int behind = 0;
  for (int c = 0; c < 4; ++c) {
    double fx, fy;
    if (!to_pixel(fr, v[c], &fx, &fy)) { ++behind; continue; }
    if (fx < mnx) mnx = fx;
    if (fx > mxx) mxx = fx;
    if (fy < mny) mny = fy;
    if (fy > mxy) mxy = fy;
  }
  if (behind == 4) { *x0 = 1; *x1 = 0; *y0 = 1; *y1 = 0; return 0; }
  if (behind) return -1;
  *x0 = (long)ceil(mnx); *x1 = (long)floor(mxx);
  *y0 = (long)ceil(mny); *y1 = (long)floor(mxy);
  return 1;
}

static int num_threads(int req) {
#ifdef _OPENMP
  return req > 0 ? req : omp_get_max_threads();
#else
  (void)req;
  return 1;
#endif
}

/*
 * Column-density image(s). crops[4*c .. 4*c+3] = (x0, y0, w, h) of crop c in
 * pixel coordinates of the W x H frame; out holds the crops one after the
 * other, each row-major [h][w]. n_frag (optional) receives the number of
 * (tetrahedron, pixel) pairs with a positive chord inside the crops, and
 * n_degen (optional) the number of tetrahedra with V == 0.
 */
/* The projection over the cubes listed in `sel` (nsel of them), or over
 * every cube when sel is NULL. */
static int render_cubes(const double* pos, int N, double box, double total_mass, const orc_camera* cam,
                        const int* crops, int ncrops, const long long* sel, long nsel, double* out,
                        long long* n_frag, long long* n_degen, int nthreads) {
  frame_t fr;
  if (N <= 0 || box <= 0 || ncrops <= 0 || frame_init(cam, &fr) != ORC_OK) return ORC_ERR_ARG;
  long total = 0;
  long* coff = (long*)malloc(sizeof(long) * (ncrops + 1));
  coff[0] = 0;
  for (int c = 0; c < ncrops; ++c) coff[c + 1] = coff[c] + (long)crops[4 * c + 2] * crops[4 * c + 3];
  total = coff[ncrops];
  int T = num_threads(nthreads);
  double* bufs = (double*)calloc((size_t)T * total, sizeof(double));
  long long* frags = (long long*)calloc(T, sizeof(long long));
  long long* degen = (long long*)calloc(T, sizeof(long long));
  int* errs = (int*)calloc(T, sizeof(int));
  const double m = total_mass / (6.0 * (double)N * N * N);
  const long ncubes = sel ? nsel : (long)N * N * N;

#pragma omp parallel num_threads(T)
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    double* img = bufs + (size_t)tid * total;
#pragma omp for schedule(static)
    for (long q = 0; q < ncubes; ++q) {
      const long cube = sel ? (long)sel[q] : q;
      if (cube < 0 || cube >= (long)N * N * N) { errs[tid] = ORC_ERR_ARG; continue; }
      long i = cube % N, j = (cube / N) % N, k = cube / ((long)N * N);
      for (int s = 0; s < 6; ++s) {
        double v[4][3];
        tet_vertices(pos, N, box, i, j, k, s, v);
        double V = tet_volume(v);
        if (V == 0.0) { degen[tid]++; continue; }
        double rho = m / fabs(V); /* Eq. 3 */
        long bx0, bx1, by0, by1;
        if (tet_pixel_box(&fr, v, &bx0, &bx1, &by0, &by1) < 0) { errs[tid] = ORC_ERR_BEHIND_EYE; continue; }
        if (bx0 > bx1 || by0 > by1) continue;
        for (int c = 0; c < ncrops; ++c) {
          long cx0 = crops[4 * c], cy0 = crops[4 * c + 1];
          long cx1 = cx0 + crops[4 * c + 2] - 1, cy1 = cy0 + crops[4 * c + 3] - 1;
          long sx0, sx1, sy0, sy1;
          shift_range(bx0, bx1, cx0, cx1, fr.W, fr.wrap, &sx0, &sx1);
          shift_range(by0, by1, cy0, cy1, fr.H, fr.wrap, &sy0, &sy1);
          for (long sy = sy0; sy <= sy1; ++sy)
            for (long sx = sx0; sx <= sx1; ++sx) {
              /* pixel (px + sx W, py + sy H) of the frame sees this copy through
               * the unwrapped pixel (px, py) */
              long px0 = bx0 > cx0 - sx * fr.W ? bx0 : cx0 - sx * fr.W;
              long px1 = bx1 < cx1 - sx * fr.W ? bx1 : cx1 - sx * fr.W;
              long py0 = by0 > cy0 - sy * fr.H ? by0 : cy0 - sy * fr.H;
              long py1 = by1 < cy1 - sy * fr.H ? by1 : cy1 - sy * fr.H;
              for (long py = py0; py <= py1; ++py)
                for (long px = px0; px <= px1; ++px) {
                  double o[3], d[3];
                  pixel_ray(&fr, px, py, o, d);
                  double dl = ray_chord(v, o, d, fr.persp, NULL, NULL, NULL, NULL);
                  if (dl > 0.0) {
                    long X = px + sx * fr.W - cx0, Y = py + sy * fr.H - cy0;
                    img[coff[c] + Y * crops[4 * c + 2] + X] += rho * dl; /* Eq. 6 */
                    frags[tid]++;
                  }
                }
            }
        }
      }
    }
  }
  /* fixed-order reduction of the per-thread images */
  memset(out, 0, sizeof(double) * total);
  long long nf = 0, nd = 0;
  int err = ORC_OK;
  for (int t = 0; t < T; ++t) {
    const double* img = bufs + (size_t)t * total;
    for (long p = 0; p < total; ++p) out[p] += img[p];
    nf += frags[t];
    nd += degen[t];
    if (errs[t]) err = errs[t];
  }
  if (n_frag) *n_frag = nf;
  if (n_degen) *n_degen = nd;
  free(bufs); free(frags); free(degen); free(errs); free(coff);
  return err;
}

int orc_render(const double* pos, int N, double box, double total_mass, const orc_camera* cam,
               const int* crops, int ncrops, double* out, long long* n_frag, long long* n_degen,
               int nthreads) {
  return render_cubes(pos, N, box, total_mass, cam, crops, ncrops, NULL, 0, out, n_frag, n_degen, nthreads);
}

/* The same projection restricted to the listed cubes (ids i + N (j + N k)),
 * for tests that need a few pixels of a large lattice: the caller picks every
 * cube that can reach them. */
int orc_render_subset(const double* pos, int N, double box, double total_mass, const orc_camera* cam,
                      const int* crops, int ncrops, const long long* cubes, long ncubes, double* out,
                      long long* n_frag, long long* n_degen, int nthreads) {
  if (!cubes || ncubes < 0) return ORC_ERR_ARG;
  return render_cubes(pos, N, box, total_mass, cam, crops, ncrops, cubes, ncubes, out, n_frag, n_degen, nthreads);
}

/* Per-tetrahedron signed volume (Eq. 9) and density (Eq. 3), tetrahedron
 * id = 6 * cube + s with cube = i + N (j + N k). rho = 0 when V == 0. */
int orc_tets(const double* pos, int N, double box, double total_mass, double* vol, double* rho) {
  if (N <= 0 || box <= 0) return ORC_ERR_ARG;
  const double m = total_mass / (6.0 * (double)N * N * N);
  const long ncubes = (long)N * N * N;
#pragma omp parallel for schedule(static)
  for (long cube = 0; cube < ncubes; ++cube) {
    long i = cube % N, j = (cube / N) % N, k = cube / ((long)N * N);
    for (int s = 0; s < 6; ++s) {
      double v[4][3];
      tet_vertices(pos, N, box, i, j, k, s, v);
      double V = tet_volume(v);
      vol[6 * cube + s] = V;
      rho[6 * cube + s] = V == 0.0 ? 0.0 : m / fabs(V);
    }
  }
  return ORC_OK;
}

/* d s / d a for the crossing s of the ray with the plane of face (a, b, c)
 * when vertex a moves: the plane moves by lambda_a(X) * delta at the crossing
 * point X, so ds = lambda_a(X) (n . delta) / (n . d). Adds scale * that to g. */
static void add_crossing_grad(const double* a, const double* b, const double* c, const double* X,
                              const double* d, double scale, double* g) {
  double e1[3], e2[3], n[3], bx[3], cx[3], t[3];
  sub3(b, a, e1); sub3(c, a, e2);
  cross3(e1, e2, n);
  sub3(b, X, bx); sub3(c, X, cx);
  cross3(bx, cx, t);
  double lam = dot3(t, n) / dot3(n, n);
  double den = dot3(n, d);
  for (int q = 0; q < 3; ++q) g[q] += scale * lam * n[q] / den;
}

/*
 * Gradient of L with respect to particle positions, given dL/dI for every
 * pixel of the full W x H frame (row-major). For each (tetrahedron, pixel)
 * pair with a positive chord: d(rho dl) = dl d rho + rho d dl, with
 * d rho / d v = -(rho / V) dV/dv (Eq. 3 and 9) and dl = s_out - s_in moving
 * with the exit and entry face planes.
 */
int orc_grad(const double* pos, int N, double box, double total_mass, const orc_camera* cam,
             const double* dLdI, double* grad, int nthreads) {
  frame_t fr;
  if (N <= 0 || box <= 0 || frame_init(cam, &fr) != ORC_OK) return ORC_ERR_ARG;
  const long np = (long)N * N * N;
  int T = num_threads(nthreads);
  double* bufs = (double*)calloc((size_t)T * np * 3, sizeof(double));
  int* errs = (int*)calloc(T, sizeof(int));
  const double m = total_mass / (6.0 * (double)N * N * N);
#pragma omp parallel num_threads(T)
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    double* G = bufs + (size_t)tid * np * 3;
#pragma omp for schedule(static)
    for (long cube = 0; cube < np; ++cube) {
      long i = cube % N, j = (cube / N) % N, k = cube / ((long)N * N);
      for (int s = 0; s < 6; ++s) {
        double v[4][3];
        tet_vertices(pos, N, box, i, j, k, s, v);
        double V = tet_volume(v);
        if (V == 0.0) continue;
        double rho = m / fabs(V);
        /* dV/dv_c for the table order (Eq. 9) */
        double a[3], b[3], c[3], dV[4][3];
        sub3(v[1], v[0], a); sub3(v[2], v[0], b); sub3(v[3], v[0], c);
        cross3(b, c, dV[1]); cross3(c, a, dV[2]); cross3(a, b, dV[3]);
        for (int q = 0; q < 3; ++q) {
          dV[1][q] /= 6.0; dV[2][q] /= 6.0; dV[3][q] /= 6.0;
          dV[0][q] = -(dV[1][q] + dV[2][q] + dV[3][q]);
        }
        long ids[4];
        for (int cc = 0; cc < 4; ++cc) {
          int n = CUBE_TETS[s][cc];
          long ii = (i + (n & 1)) % N, jj = (j + ((n >> 1) & 1)) % N, kk = (k + ((n >> 2) & 1)) % N;
          ids[cc] = ii + (long)N * (jj + (long)N * kk);
        }
        long bx0, bx1, by0, by1;
        if (tet_pixel_box(&fr, v, &bx0, &bx1, &by0, &by1) < 0) { errs[tid] = ORC_ERR_BEHIND_EYE; continue; }
        if (bx0 > bx1 || by0 > by1) continue;
        long sx0, sx1, sy0, sy1;
        shift_range(bx0, bx1, 0, fr.W - 1, fr.W, fr.wrap, &sx0, &sx1);
        shift_range(by0, by1, 0, fr.H - 1, fr.H, fr.wrap, &sy0, &sy1);
        for (long sy = sy0; sy <= sy1; ++sy)
          for (long sx = sx0; sx <= sx1; ++sx) {
            long px0 = bx0 > -sx * fr.W ? bx0 : -sx * fr.W;
            long px1 = bx1 < fr.W - 1 - sx * fr.W ? bx1 : fr.W - 1 - sx * fr.W;
            long py0 = by0 > -sy * fr.H ? by0 : -sy * fr.H;
            long py1 = by1 < fr.H - 1 - sy * fr.H ? by1 : fr.H - 1 - sy * fr.H;
            for (long py = py0; py <= py1; ++py)
              for (long px = px0; px <= px1; ++px) {
                double o[3], d[3], s_in, s_out;
                int fin, fout;
                pixel_ray(&fr, px, py, o, d);
                double dl = ray_chord(v, o, d, fr.persp, &fin, &fout, &s_in, &s_out);
                if (!(dl > 0.0)) continue;
                double g = dLdI[(py + sy * fr.H) * (long)fr.W + (px + sx * fr.W)];
                if (g == 0.0) continue;
                double gv[4][3];
                memset(gv, 0, sizeof gv);
                for (int cc = 0; cc < 4; ++cc)
                  for (int q = 0; q < 3; ++q) gv[cc][q] = -dl * rho / V * dV[cc][q];
                /* chord through the exit (+) and entry (-) face planes */
                for (int side = 0; side < 2; ++side) {
                  int f = side == 0 ? fout : fin;
                  if (f < 0) continue; /* half-line start at the eye does not move */
                  double sgn = side == 0 ? rho : -rho;
                  double sv = side == 0 ? s_out : s_in;
                  double X[3] = {o[0] + sv * d[0], o[1] + sv * d[1], o[2] + sv * d[2]};
                  int fa = (f + 1) & 3, fb = (f + 2) & 3, fc = (f + 3) & 3;
                  add_crossing_grad(v[fa], v[fb], v[fc], X, d, sgn, gv[fa]);
                  add_crossing_grad(v[fb], v[fc], v[fa], X, d, sgn, gv[fb]);
                  add_crossing_grad(v[fc], v[fa], v[fb], X, d, sgn, gv[fc]);
                }
                for (int cc = 0; cc < 4; ++cc)
                  for (int q = 0; q < 3; ++q) G[3 * ids[cc] + q] += g * gv[cc][q];
              }
          }
      }
    }
  }
  memset(grad, 0, sizeof(double) * np * 3);
  int err = ORC_OK;
  for (int t = 0; t < T; ++t) {
    const double* G = bufs + (size_t)t * np * 3;
    for (long p = 0; p < np * 3; ++p) grad[p] += G[p];
    if (errs[t]) err = errs[t];
  }
  free(bufs); free(errs);
  return err;
}

/* ---------- entry points used by the oracle's own pins ---------- */

/* Chord of one ray through one tetrahedron (v: 4 x 3 doubles). */
double orc_chord(const double* v12, const double* o, const double* d, int halfline) {
  double v[4][3];
  memcpy(v, v12, sizeof v);
  double dn[3] = {d[0], d[1], d[2]};
  normalize3(dn);
  return ray_chord(v, o, dn, halfline, NULL, NULL, NULL, NULL);
}

/* Vertices (4 x 3) of tetrahedron s of cube (i, j, k) after unwrapping. */
int orc_tet_vertices(const double* pos, int N, double box, int i, int j, int k, int s, double* out12) {
  if (N <= 0 || s < 0 || s > 5) return ORC_ERR_ARG;
  double v[4][3];
  tet_vertices(pos, N, box, i, j, k, s, v);
  memcpy(out12, v, sizeof v);
  return ORC_OK;
}

/* Projection (Eq. 6) of an arbitrary set of tetrahedra with given constant
 * densities, full W x H frame, same pixel and ray conventions as orc_render
 * (no periodic copies). */
int orc_render_soup(const double* verts /* [n][4][3] */, const double* dens, long n, const orc_camera* cam,
                    double* out) {
  frame_t fr;
  if (frame_init(cam, &fr) != ORC_OK) return ORC_ERR_ARG;
  memset(out, 0, sizeof(double) * fr.W * fr.H);
  for (long t = 0; t < n; ++t) {
    double v[4][3];
    memcpy(v, verts + 12 * t, sizeof v);
    long x0, x1, y0, y1;
    const int pb = tet_pixel_box(&fr, v, &x0, &x1, &y0, &y1);
    if (pb < 0) return ORC_ERR_BEHIND_EYE;
    if (pb == 0) continue;
    if (x0 < 0) x0 = 0;
    if (y0 < 0) y0 = 0;
    if (x1 > fr.W - 1) x1 = fr.W - 1;
    if (y1 > fr.H - 1) y1 = fr.H - 1;
    for (long py = y0; py <= y1; ++py)
      for (long px = x0; px <= x1; ++px) {
        double o[3], d[3];
        pixel_ray(&fr, px, py, o, d);
        out[py * fr.W + px] += dens[t] * ray_chord(v, o, d, fr.persp, NULL, NULL, NULL, NULL);
      }
  }
  return ORC_OK;
}

/*
 * Resampling onto a periodic n x n x n grid over the box (Sec. 4.3,
 * Eq. 10-12). Cell (a, b, c), of edge g = box / n, receives from every
 * tetrahedron T_i the value q_i dl, where dl is the length of the part of
 * the cell's central line along z (x = (a + 1/2) g, y = (b + 1/2) g) that
 * lies inside both T_i and the cell's slab [c g, (c + 1) g). Eq. 12: the
 * front- and back-face terms of Eq. 10 and 11 add up to exactly this.
 *   weight 0: q_i = rho_i (Eq. 3). The cell holds rho dl, the paper's
 *             estimate A rho dl of its mass divided by the face area A.
 *   weight 1: q_i = 1. The cell holds the summed stream length; divided by
 *             g, that is the mean number of streams on its central line
 *             (Sec. 3.2).
 * out: [n][n][n], index (c n + b) n + a. Tetrahedra with V == 0 contribute
 * nothing.
 */
int orc_resample(const double* pos, int N, double box, double total_mass, int n, int weight, double* out,
                 int nthreads) {
  if (N <= 0 || box <= 0 || n <= 0 || (weight != 0 && weight != 1)) return ORC_ERR_ARG;
  const long cells = (long)n * n * n;
  const int T = num_threads(nthreads);
  double* bufs = (double*)calloc((size_t)T * cells, sizeof(double));
  const double m = total_mass / (6.0 * (double)N * N * N);
  const double g = box / n;
  const long ncubes = (long)N * N * N;
#pragma omp parallel num_threads(T)
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    double* grid = bufs + (size_t)tid * cells;
#pragma omp for schedule(static)
    for (long cube = 0; cube < ncubes; ++cube) {
      long i = cube % N, j = (cube / N) % N, k = cube / ((long)N * N);
      for (int s = 0; s < 6; ++s) {
        double v[4][3];
        tet_vertices(pos, N, box, i, j, k, s, v);
        double V = tet_volume(v);
        if (V == 0.0) continue;
        const double q = weight == 0 ? m / fabs(V) : 1.0;
        double xmin = v[0][0], xmax = v[0][0], ymin = v[0][1], ymax = v[0][1];
        for (int c = 1; c < 4; ++c) {
          xmin = fmin(xmin, v[c][0]); xmax = fmax(xmax, v[c][0]);
          ymin = fmin(ymin, v[c][1]); ymax = fmax(ymax, v[c][1]);
        }
        /* columns whose central line can meet the tetrahedron (unwrapped indices) */
        const long a0 = (long)ceil(xmin / g - 0.5), a1 = (long)floor(xmax / g - 0.5);
        const long b0 = (long)ceil(ymin / g - 0.5), b1 = (long)floor(ymax / g - 0.5);
        for (long b = b0; b <= b1; ++b)
          for (long a = a0; a <= a1; ++a) {
            const double o[3] = {((double)a + 0.5) * g, ((double)b + 0.5) * g, 0.0};
            const double d[3] = {0.0, 0.0, 1.0};
            double z_in, z_out;
            if (!(ray_chord(v, o, d, 0, NULL, NULL, &z_in, &z_out) > 0.0)) continue;
            const long aw = ((a % n) + n) % n, bw = ((b % n) + n) % n;
            for (long c = (long)floor(z_in / g); (double)c * g < z_out; ++c) {
              const double lo = fmax(z_in, (double)c * g), hi = fmin(z_out, (double)(c + 1) * g);
              if (hi > lo) grid[((((c % n) + n) % n) * n + bw) * n + aw] += q * (hi - lo);
            }
          }
      }
    }
  }
  memset(out, 0, sizeof(double) * cells);
  for (int t = 0; t < T; ++t) {
    const double* grid = bufs + (size_t)t * cells;
    for (long p = 0; p < cells; ++p) out[p] += grid[p];
  }
  free(bufs);
  return ORC_OK;
}

/*
 * Point evaluation of the overlapping-streams density (Sec. 3.2, Eq. 4-5):
 * for each point p (pts[3 P], in box coordinates, any period), the sum over
 * the tetrahedra T_i containing p (any periodic copy) of q_i, with
 * q_i = rho_i (weight 0: the total density rho_tot(p) of Eq. 4) or 1
 * (weight 1: the number of streams at p). Every (point, tetrahedron) pair is
 * tested, so it is meant for small point sets (slices, grid centres of small
 * grids). Points exactly on a face count for both sides.
 */
int orc_point_density(const double* pos, int N, double box, double total_mass, const double* pts, long P,
                      int weight, double* out, int nthreads) {
  if (N <= 0 || box <= 0 || P < 0 || (weight != 0 && weight != 1)) return ORC_ERR_ARG;
  const int T = num_threads(nthreads);
  double* bufs = (double*)calloc((size_t)T * (P > 0 ? P : 1), sizeof(double));
  const double m = total_mass / (6.0 * (double)N * N * N);
  const long ncubes = (long)N * N * N;
#pragma omp parallel num_threads(T)
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    double* acc = bufs + (size_t)tid * (P > 0 ? P : 1);
#pragma omp for schedule(static)
    for (long cube = 0; cube < ncubes; ++cube) {
      long i = cube % N, j = (cube / N) % N, k = cube / ((long)N * N);
      for (int s = 0; s < 6; ++s) {
        double v[4][3];
        tet_vertices(pos, N, box, i, j, k, s, v);
        const double V = tet_volume(v);
        if (V == 0.0) continue;
        const double q = weight == 0 ? m / fabs(V) : 1.0;
        /* outward face planes: inside means n_f . (p - a_f) <= 0 for all f */
        double nrm[4][3], base[4][3];
        for (int f = 0; f < 4; ++f) {
          const double *a = v[(f + 1) & 3], *b = v[(f + 2) & 3], *c = v[(f + 3) & 3];
          double e1[3], e2[3], t[3];
          sub3(b, a, e1); sub3(c, a, e2);
          cross3(e1, e2, nrm[f]);
          sub3(v[f], a, t);
          if (dot3(nrm[f], t) > 0.0) { nrm[f][0] = -nrm[f][0]; nrm[f][1] = -nrm[f][1]; nrm[f][2] = -nrm[f][2]; }
          memcpy(base[f], a, sizeof base[f]);
        }
        double lo[3], hi[3];
        for (int c = 0; c < 3; ++c) {
          lo[c] = fmin(fmin(v[0][c], v[1][c]), fmin(v[2][c], v[3][c]));
          hi[c] = fmax(fmax(v[0][c], v[1][c]), fmax(v[2][c], v[3][c]));
        }
        for (long p = 0; p < P; ++p) {
          /* the periodic copy of the point nearest the tetrahedron's box */
          double x[3];
          int in_box = 1;
          for (int c = 0; c < 3; ++c) {
            double xc = pts[3 * p + c];
            xc -= box * floor((xc - lo[c]) / box);  /* into [lo, lo + box) */
            x[c] = xc;
            if (xc > hi[c]) in_box = 0;
          }
          if (!in_box) continue;
          int inside = 1;
          for (int f = 0; f < 4 && inside; ++f) {
            double t[3];
            sub3(x, base[f], t);
            if (dot3(nrm[f], t) > 0.0) inside = 0;
          }
          if (inside) acc[p] += q;
        }
      }
    }
  }
  memset(out, 0, sizeof(double) * (P > 0 ? P : 1));
  for (int t = 0; t < T; ++t)
    for (long p = 0; p < P; ++p) out[p] += bufs[(size_t)t * (P > 0 ? P : 1) + p];
  free(bufs);
  return ORC_OK;
}

/*
 * Centroid splats (Sec. 4.2): every tetrahedron T drawn as a 2D kernel on a
 * billboard through its centroid c_T = (v0 + v1 + v2 + v3) / 4 (its centre of
 * mass, the density being constant), facing the view direction, scaled with
 * (m / rho_T)^(1/3) = |V_T|^(1/3) and carrying its mass m. The paper names a
 * cubic-spline kernel and leaves its form and the scale factor open; this
 * oracle takes the 2D M4 cubic spline with unit integral and smoothing
 * length h_T = |V_T|^(1/3):
 *   W(r, h) = 10 / (7 pi h^2) * w(r / h),
 *   w(q) = 1 - 3/2 q^2 + 3/4 q^3 (q < 1), (2 - q)^3 / 4 (1 <= q < 2), 0 else.
 * The billboard holds surface density m W(d, h), d the distance from c_T to
 * the point where the pixel's ray crosses the billboard's plane, so the ray
 * picks up m W(d, h) / cos(theta), theta its angle to the view direction:
 *   orthographic: cos = 1 and d is the distance in the image plane;
 *   perspective: with camera coordinates (X, Y, Z) of c_T and the pixel's
 *     ray direction (xt, yt, 1), d = |(Z xt - X, Z yt - Y)| and
 *     1 / cos = |(xt, yt, 1)|. Billboards with Z <= 0 are not drawn.
 * A pixel holds the sum over tetrahedra (an estimate of the column density).
 * A periodic orthographic window draws every periodic copy, like
 * orc_render. Tetrahedra with V == 0 carry no splat.
 *
 * Hybrid near/far rendering (Sec. 6, Fig. "LargeScale"): with r_near > 0
 * (perspective views only), the cubes whose corner-0 particle lies within
 * r_near of the eye are drawn by the exact projection of Eq. 6 (the chords
 * of orc_render) and only the other cubes' tetrahedra as splats. r_near = 0
 * gives splats only. out: [H][W].
 */
static double spline_w(double q) {
  if (q < 1.0) return 1.0 - 1.5 * q * q + 0.75 * q * q * q;
  if (q < 2.0) { const double t = 2.0 - q; return 0.25 * t * t * t; }
  return 0.0;
}

int orc_hybrid(const double* pos, int N, double box, double total_mass, const orc_camera* cam, double r_near,
               double* out, int nthreads) {
  frame_t fr;
  if (N <= 0 || box <= 0 || !(r_near >= 0.0) || frame_init(cam, &fr) != ORC_OK) return ORC_ERR_ARG;
  if (r_near > 0.0 && !fr.persp) return ORC_ERR_ARG;
  const long npix = (long)fr.W * fr.H;
  const int T = num_threads(nthreads);
  double* bufs = (double*)calloc((size_t)T * npix, sizeof(double));
  int* errs = (int*)calloc(T, sizeof(int));
  const double m = total_mass / (6.0 * (double)N * N * N);
  const double dx = (fr.hi[0] - fr.lo[0]) / fr.W, dy = (fr.hi[1] - fr.lo[1]) / fr.H;
  const double ptx = 2.0 * fr.tan_x / fr.W, pty = 2.0 * fr.tan_y / fr.H;  /* perspective pixel size in tan units */
  const long ncubes = (long)N * N * N;
#pragma omp parallel num_threads(T)
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    double* img = bufs + (size_t)tid * npix;
#pragma omp for schedule(static)
    for (long cube = 0; cube < ncubes; ++cube) {
      long i = cube % N, j = (cube / N) % N, k = cube / ((long)N * N);
      int near = 0;
      if (r_near > 0.0) {
        double c0[3], e[3];
        corner_position(pos, N, box, i, j, k, c0);
        sub3(c0, fr.eye, e);
        near = dot3(e, e) < r_near * r_near;
      }
      for (int s = 0; s < 6; ++s) {
        double v[4][3];
        tet_vertices(pos, N, box, i, j, k, s, v);
        const double V = tet_volume(v);
        if (V == 0.0) continue;
        if (near) {
          /* exact projection (Eq. 6), as in orc_render */
          const double rho = m / fabs(V);
          long bx0, bx1, by0, by1;
          if (tet_pixel_box(&fr, v, &bx0, &bx1, &by0, &by1) < 0) { errs[tid] = ORC_ERR_BEHIND_EYE; continue; }
          if (bx0 < 0) bx0 = 0;
          if (by0 < 0) by0 = 0;
          if (bx1 > fr.W - 1) bx1 = fr.W - 1;
          if (by1 > fr.H - 1) by1 = fr.H - 1;
          for (long py = by0; py <= by1; ++py)
            for (long px = bx0; px <= bx1; ++px) {
              double o[3], d[3];
              pixel_ray(&fr, px, py, o, d);
              const double dl = ray_chord(v, o, d, fr.persp, NULL, NULL, NULL, NULL);
              if (dl > 0.0) img[py * fr.W + px] += rho * dl;
            }
          continue;
        }
        double c[3];
        for (int q = 0; q < 3; ++q) c[q] = 0.25 * (v[0][q] + v[1][q] + v[2][q] + v[3][q]);
        const double h = cbrt(fabs(V));
        const double norm = m * 10.0 / (7.0 * M_PI * h * h);
        if (!fr.persp) {
          const double a = dot3(fr.r, c), b = dot3(fr.u, c);  /* centroid in window coordinates */
          /* pixels whose centre lies within 2h of the centroid (unwrapped indices) */
          const long x0 = (long)ceil((a - 2.0 * h - fr.lo[0]) / dx - 0.5), x1 = (long)floor((a + 2.0 * h - fr.lo[0]) / dx - 0.5);
          const long y0 = (long)ceil((b - 2.0 * h - fr.lo[1]) / dy - 0.5), y1 = (long)floor((b + 2.0 * h - fr.lo[1]) / dy - 0.5);
          if (x0 > x1 || y0 > y1) continue;
          long sx0, sx1, sy0, sy1;
          shift_range(x0, x1, 0, fr.W - 1, fr.W, fr.wrap, &sx0, &sx1);
          shift_range(y0, y1, 0, fr.H - 1, fr.H, fr.wrap, &sy0, &sy1);
          for (long sy = sy0; sy <= sy1; ++sy)
            for (long sx = sx0; sx <= sx1; ++sx) {
              const long px0 = x0 > -sx * fr.W ? x0 : -sx * fr.W, px1 = x1 < fr.W - 1 - sx * fr.W ? x1 : fr.W - 1 - sx * fr.W;
              const long py0 = y0 > -sy * fr.H ? y0 : -sy * fr.H, py1 = y1 < fr.H - 1 - sy * fr.H ? y1 : fr.H - 1 - sy * fr.H;
              for (long py = py0; py <= py1; ++py)
                for (long px = px0; px <= px1; ++px) {
                  const double xw = fr.lo[0] + (px + 0.5) * dx, yw = fr.lo[1] + (py + 0.5) * dy;
                  const double r = sqrt((xw - a) * (xw - a) + (yw - b) * (yw - b));
                  const double w = spline_w(r / h);
                  if (w > 0.0) img[(py + sy * fr.H) * fr.W + (px + sx * fr.W)] += norm * w;
                }
            }
        } else {
          double e[3];
          sub3(c, fr.eye, e);
          const double Z = dot3(fr.f, e), X = dot3(fr.r, e), Y = dot3(fr.u, e);
          if (!(Z > 0.0)) continue;
          /* pixel centre xt = tan_x (2 (px + 1/2) / W - 1): the ray meets the billboard
           * at distance Z |xt - X/Z| along r; the support is |d| < 2h */
          const double cx = (X / Z / fr.tan_x + 1.0) * 0.5 * fr.W - 0.5, cy = (Y / Z / fr.tan_y + 1.0) * 0.5 * fr.H - 0.5;
          const double rx = 2.0 * h / Z / ptx, ry = 2.0 * h / Z / pty;
          long x0 = (long)ceil(cx - rx), x1 = (long)floor(cx + rx), y0 = (long)ceil(cy - ry), y1 = (long)floor(cy + ry);
          if (x0 < 0) x0 = 0;
          if (y0 < 0) y0 = 0;
          if (x1 > fr.W - 1) x1 = fr.W - 1;
          if (y1 > fr.H - 1) y1 = fr.H - 1;
          for (long py = y0; py <= y1; ++py)
            for (long px = x0; px <= x1; ++px) {
              const double xt = fr.tan_x * (2.0 * (px + 0.5) / fr.W - 1.0);
              const double yt = fr.tan_y * (2.0 * (py + 0.5) / fr.H - 1.0);
              const double ddx = Z * xt - X, ddy = Z * yt - Y;
              const double w = spline_w(sqrt(ddx * ddx + ddy * ddy) / h);
              if (w > 0.0) img[py * fr.W + px] += norm * w * sqrt(1.0 + xt * xt + yt * yt);
            }
        }
      }
    }
  }
  memset(out, 0, sizeof(double) * npix);
  int err = ORC_OK;
  for (int t = 0; t < T; ++t) {
    for (long p = 0; p < npix; ++p) out[p] += bufs[(size_t)t * npix + p];
    if (errs[t]) err = errs[t];
  }
  free(bufs);
  free(errs);
  return err;
}

/* Centroid splats of every tetrahedron: orc_hybrid with r_near = 0. */
int orc_centroids(const double* pos, int N, double box, double total_mass, const orc_camera* cam, double* out,
                  int nthreads) {
  return orc_hybrid(pos, N, box, total_mass, cam, 0.0, out, nthreads);
}

/*
 * Area-averaged pixels (orthographic views): each pixel holds the mean of the
 * column density (Eq. 6) over its square instead of the value at its
 * centre. For one tetrahedron the chord dl(x, y) is zero on the boundary of
 * the projected hull and linear on each triangle joining the apex -- the
 * projected vertex inside the triangle of the other three, or else the
 * crossing of the hull's two diagonals -- to a hull edge (the front and back
 * faces change there and nowhere else). So the integral over the pixel
 * square is, per triangle, the area of the triangle clipped to the square
 * times dl at the clipped polygon's centroid. dl at the apex is the depth of
 * the back surface minus that of the front one there. A periodic window
 * draws every periodic copy. out: [H][W].
 */
typedef struct { double x, y; } pt2;

/* Clip polygon p[n] (convex, counter-clockwise or not) to the half-plane
 * s * (x - x0) >= 0 (axis 0) or s * (y - y0) >= 0 (axis 1); returns the new
 * vertex count (at most n + 1). */
static int clip_half(const pt2* p, int n, int axis, double x0, double s, pt2* q) {
  int m = 0;
  for (int i = 0; i < n; ++i) {
    const pt2 a = p[i], b = p[(i + 1) % n];
    const double da = s * ((axis == 0 ? a.x : a.y) - x0), db = s * ((axis == 0 ? b.x : b.y) - x0);
    if (da >= 0.0) q[m++] = a;
    if ((da >= 0.0) != (db >= 0.0)) {
      const double t = da / (da - db);
      q[m].x = a.x + t * (b.x - a.x);
      q[m].y = a.y + t * (b.y - a.y);
      ++m;
    }
  }
  return m;
}

/* Integral over the square [x0, x1] x [y0, y1] of the linear function that is
 * h at A and 0 at B and C, restricted to triangle ABC. */
static double tri_square_integral(pt2 A, pt2 B, pt2 C, double h, double x0, double x1, double y0, double y1) {
  pt2 p[8], q[8];
  p[0] = A; p[1] = B; p[2] = C;
  int n = 3;
  n = clip_half(p, n, 0, x0, 1.0, q);
  n = clip_half(q, n, 0, x1, -1.0, p);
  n = clip_half(p, n, 1, y0, 1.0, q);
  n = clip_half(q, n, 1, y1, -1.0, p);
  if (n < 3) return 0.0;
  double area2 = 0.0, cx = 0.0, cy = 0.0;
  for (int i = 0; i < n; ++i) {
    const pt2 a = p[i], b = p[(i + 1) % n];
    const double cr = a.x * b.y - b.x * a.y;
    area2 += cr;
    cx += (a.x + b.x) * cr;
    cy += (a.y + b.y) * cr;
  }
  if (area2 == 0.0) return 0.0;
  cx /= 3.0 * area2;
  cy /= 3.0 * area2;
  /* barycentric weight of A at the centroid */
  const double den = (B.y - C.y) * (A.x - C.x) + (C.x - B.x) * (A.y - C.y);
  if (den == 0.0) return 0.0;
  const double la = ((B.y - C.y) * (cx - C.x) + (C.x - B.x) * (cy - C.y)) / den;
  return 0.5 * fabs(area2) * h * la;
}

static double orient2(pt2 a, pt2 b, pt2 c) { return (b.x - a.x) * (c.y - a.y) - (b.y - a.y) * (c.x - a.x); }

int orc_render_area(const double* pos, int N, double box, double total_mass, const orc_camera* cam, double* out,
                    int nthreads) {
  frame_t fr;
  if (N <= 0 || box <= 0 || frame_init(cam, &fr) != ORC_OK || fr.persp) return ORC_ERR_ARG;
  const long npix = (long)fr.W * fr.H;
  const int T = num_threads(nthreads);
  double* bufs = (double*)calloc((size_t)T * npix, sizeof(double));
  const double m = total_mass / (6.0 * (double)N * N * N);
  const double dx = (fr.hi[0] - fr.lo[0]) / fr.W, dy = (fr.hi[1] - fr.lo[1]) / fr.H;
  const long ncubes = (long)N * N * N;
#pragma omp parallel num_threads(T)
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    double* img = bufs + (size_t)tid * npix;
#pragma omp for schedule(static)
    for (long cube = 0; cube < ncubes; ++cube) {
      long i = cube % N, j = (cube / N) % N, k = cube / ((long)N * N);
      for (int s = 0; s < 6; ++s) {
        double v[4][3];
        tet_vertices(pos, N, box, i, j, k, s, v);
        const double V = tet_volume(v);
        if (V == 0.0) continue;
        const double rho = m / fabs(V);
        /* projected vertices in pixel units (pixel px covers [px, px + 1)) */
        pt2 P[4];
        for (int c = 0; c < 4; ++c) {
          P[c].x = (dot3(fr.r, v[c]) - fr.lo[0]) / dx;
          P[c].y = (dot3(fr.u, v[c]) - fr.lo[1]) / dy;
        }
        /* depth of each vertex along the view direction */
        double z[4];
        for (int c = 0; c < 4; ++c) z[c] = dot3(fr.f, v[c]);
        /* the apex, the hull (counter-clockwise) and the chord at the apex:
         * the depth of the back surface there minus that of the front one
         * (Eq. 6). A vertex inside the triangle of the other three, or on its
         * boundary (coincident projections, as for the undeformed lattice
         * seen along an axis), is the apex; the chord there runs from it to
         * the opposite face. */
        pt2 apex, hull[4];
        int nh = 0;
        int inner = -1;
        double chord = 0.0;
        for (int c = 0; c < 4 && inner < 0; ++c) {
          const int ia = (c + 1) & 3, ib = (c + 2) & 3, id = (c + 3) & 3;
          const pt2 a = P[ia], b = P[ib], d = P[id];
          const double o = orient2(a, b, d);
          if (o == 0.0) continue;
          /* barycentric coordinates of P[c] in triangle (a, b, d) */
          const double la = orient2(b, d, P[c]) / o, lb = orient2(d, a, P[c]) / o, ld = orient2(a, b, P[c]) / o;
          if (la >= 0.0 && lb >= 0.0 && ld >= 0.0) {
            inner = c;
            chord = fabs(z[c] - (la * z[ia] + lb * z[ib] + ld * z[id]));
          }
        }
        if (inner >= 0) {
          apex = P[inner];
          for (int c = 0; c < 4; ++c)
            if (c != inner) hull[nh++] = P[c];
          if (orient2(hull[0], hull[1], hull[2]) < 0.0) { pt2 t = hull[1]; hull[1] = hull[2]; hull[2] = t; }
        } else {
          /* convex quadrilateral: find the order in which 0-a and b-c are the diagonals */
          int a = -1;
          for (int c = 1; c < 4 && a < 0; ++c) {
            int o1 = c == 1 ? 2 : 1, o2 = 6 - c - o1;
            const double s1 = orient2(P[0], P[c], P[o1]), s2 = orient2(P[0], P[c], P[o2]);
            if ((s1 > 0.0 && s2 < 0.0) || (s1 < 0.0 && s2 > 0.0)) a = c;
          }
          if (a < 0) continue; /* no projected area */
          const int b1 = a == 1 ? 2 : 1, b2 = 6 - a - b1;
          /* diagonals P0-Pa and Pb1-Pb2 cross at the apex */
          const double d1x = P[a].x - P[0].x, d1y = P[a].y - P[0].y;
          const double d2x = P[b2].x - P[b1].x, d2y = P[b2].y - P[b1].y;
          const double den = d1x * d2y - d1y * d2x;
          if (den == 0.0) continue;
          const double t = ((P[b1].x - P[0].x) * d2y - (P[b1].y - P[0].y) * d2x) / den;
          const double u = ((P[b1].x - P[0].x) * d1y - (P[b1].y - P[0].y) * d1x) / den;
          apex.x = P[0].x + t * d1x;
          apex.y = P[0].y + t * d1y;
          /* the chord at the crossing runs between the two diagonal edges */
          chord = fabs((z[0] + t * (z[a] - z[0])) - (z[b1] + u * (z[b2] - z[b1])));
          hull[0] = P[0]; hull[1] = P[b1]; hull[2] = P[a]; hull[3] = P[b2];
          nh = 4;
          if (orient2(hull[0], hull[1], hull[2]) < 0.0) { pt2 t2 = hull[1]; hull[1] = hull[3]; hull[3] = t2; }
        }
        const double h = rho * chord;
        if (!(h > 0.0)) continue;
        double xmn = P[0].x, xmx = P[0].x, ymn = P[0].y, ymx = P[0].y;
        for (int c = 1; c < 4; ++c) {
          xmn = fmin(xmn, P[c].x); xmx = fmax(xmx, P[c].x);
          ymn = fmin(ymn, P[c].y); ymx = fmax(ymx, P[c].y);
        }
        const long x0 = (long)floor(xmn), x1 = (long)floor(xmx), y0 = (long)floor(ymn), y1 = (long)floor(ymx);
        long sx0, sx1, sy0, sy1;
        shift_range(x0, x1, 0, fr.W - 1, fr.W, fr.wrap, &sx0, &sx1);
        shift_range(y0, y1, 0, fr.H - 1, fr.H, fr.wrap, &sy0, &sy1);
        for (long sy = sy0; sy <= sy1; ++sy)
          for (long sx = sx0; sx <= sx1; ++sx) {
            const long px0 = x0 > -sx * fr.W ? x0 : -sx * fr.W, px1 = x1 < fr.W - 1 - sx * fr.W ? x1 : fr.W - 1 - sx * fr.W;
            const long py0 = y0 > -sy * fr.H ? y0 : -sy * fr.H, py1 = y1 < fr.H - 1 - sy * fr.H ? y1 : fr.H - 1 - sy * fr.H;
            for (long py = py0; py <= py1; ++py)
              for (long px = px0; px <= px1; ++px) {
                double sum = 0.0;
                for (int e = 0; e < nh; ++e)
                  sum += tri_square_integral(apex, hull[e], hull[(e + 1) % nh], h, (double)px, (double)px + 1.0,
                                             (double)py, (double)py + 1.0);
                img[(py + sy * fr.H) * fr.W + (px + sx * fr.W)] += sum;  /* area in pixels: the mean over the square */
              }
          }
      }
    }
  }
  memset(out, 0, sizeof(double) * npix);
  for (int t = 0; t < T; ++t)
    for (long p = 0; p < npix; ++p) out[p] += bufs[(size_t)t * npix + p];
  free(bufs);
  return ORC_OK;
}
