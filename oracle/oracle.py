"""ctypes front end of the FP64 oracle (lt_oracle.c).

TEST INFRASTRUCTURE ONLY. Positions come in as the product stores them
(float32 x, y, z per particle in id order, Eq. 8) and are promoted to float64
before any arithmetic; everything below runs in double precision.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

from . import build as _build

_lib = None


class _Cam(C.Structure):
    _fields_ = [
        ("type", C.c_int),
        ("eye", C.c_double * 3),
        ("fwd", C.c_double * 3),
        ("up", C.c_double * 3),
        ("fov_y_deg", C.c_double),
        ("lo", C.c_double * 2),
        ("hi", C.c_double * 2),
        ("W", C.c_int),
        ("H", C.c_int),
        ("wrap", C.c_int),
    ]


@dataclass
class Camera:
    """View description shared by the oracle and the GPU path.

    type: "ortho" or "persp". Orthographic rays run along `fwd` through the
    window [lo, hi] spanned by right = up x fwd and up' = fwd x right;
    perspective rays start at `eye`. Pixel (px, py) has its centre at
    ((px + 1/2)/W, (py + 1/2)/H) of the window (row py runs along up').
    """

    type: str
    W: int
    H: int
    eye: Sequence[float] = (0.0, 0.0, 0.0)
    fwd: Sequence[float] = (0.0, 0.0, 1.0)
    up: Sequence[float] = (0.0, 1.0, 0.0)
    fov_y_deg: float = 60.0
    lo: Sequence[float] = (0.0, 0.0)
    hi: Sequence[float] = (1.0, 1.0)
    wrap: bool = False

    def to_c(self) -> _Cam:
        c = _Cam()
        c.type = 1 if self.type == "persp" else 0
        c.eye[:] = [float(x) for x in self.eye]
        c.fwd[:] = [float(x) for x in self.fwd]
        c.up[:] = [float(x) for x in self.up]
        c.fov_y_deg = float(self.fov_y_deg)
        c.lo[:] = [float(x) for x in self.lo]
        c.hi[:] = [float(x) for x in self.hi]
        c.W, c.H = int(self.W), int(self.H)
        c.wrap = int(bool(self.wrap))
        return c

    @classmethod
    def from_dict(cls, d: dict) -> "Camera":
        return cls(**d)


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = C.CDLL(path)
        dp, ip, llp = C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_longlong)
        lib.orc_render.argtypes = [dp, C.c_int, C.c_double, C.c_double, C.POINTER(_Cam), ip, C.c_int,
                                   dp, llp, llp, C.c_int]
        lib.orc_render.restype = C.c_int
        lib.orc_tets.argtypes = [dp, C.c_int, C.c_double, C.c_double, dp, dp]
        lib.orc_tets.restype = C.c_int
        lib.orc_grad.argtypes = [dp, C.c_int, C.c_double, C.c_double, C.POINTER(_Cam), dp, dp, C.c_int]
        lib.orc_grad.restype = C.c_int
        lib.orc_chord.argtypes = [dp, dp, dp, C.c_int]
        lib.orc_chord.restype = C.c_double
        lib.orc_tet_vertices.argtypes = [dp, C.c_int, C.c_double, C.c_int, C.c_int, C.c_int, C.c_int, dp]
        lib.orc_tet_vertices.restype = C.c_int
        lib.orc_render_soup.argtypes = [dp, dp, C.c_long, C.POINTER(_Cam), dp]
        lib.orc_render_soup.restype = C.c_int
        lib.orc_resample.argtypes = [dp, C.c_int, C.c_double, C.c_double, C.c_int, C.c_int, dp, C.c_int]
        lib.orc_resample.restype = C.c_int
        lib.orc_point_density.argtypes = [dp, C.c_int, C.c_double, C.c_double, dp, C.c_long, C.c_int, dp, C.c_int]
        lib.orc_point_density.restype = C.c_int
        lib.orc_centroids.argtypes = [dp, C.c_int, C.c_double, C.c_double, C.POINTER(_Cam), dp, C.c_int]
        lib.orc_centroids.restype = C.c_int
        lib.orc_hybrid.argtypes = [dp, C.c_int, C.c_double, C.c_double, C.POINTER(_Cam), C.c_double, dp, C.c_int]
        lib.orc_hybrid.restype = C.c_int
        lib.orc_render_subset.argtypes = [dp, C.c_int, C.c_double, C.c_double, C.POINTER(_Cam), C.POINTER(C.c_int),
                                          C.c_int, C.POINTER(C.c_longlong), C.c_long, dp,
                                          C.POINTER(C.c_longlong), C.POINTER(C.c_longlong), C.c_int]
        lib.orc_render_subset.restype = C.c_int
        lib.orc_render_area.argtypes = [dp, C.c_int, C.c_double, C.c_double, C.POINTER(_Cam), dp, C.c_int]
        lib.orc_render_area.restype = C.c_int
        _lib = lib
    return _lib


def _pos64(pos: np.ndarray, N: int) -> np.ndarray:
    p = np.asarray(pos)
    p = p.reshape(N * N * N, -1)[:, :3]
    return np.ascontiguousarray(p, dtype=np.float64)


def _ptr(a: np.ndarray, t):
    return a.ctypes.data_as(C.POINTER(t))


def _cam(cam) -> Camera:
    return cam if isinstance(cam, Camera) else Camera.from_dict(cam)


def render_crops(pos, N: int, cam, crops: Sequence[Sequence[int]], box: float = 1.0,
                 total_mass: float = 1.0, nthreads: int = 0, cubes=None):
    """Render the listed crops (x0, y0, w, h) of the frame; returns
    (list of [h][w] float64 images, fragment count, degenerate count).
    `cubes`: optional cube ids (i + N (j + N k)) to draw instead of all of
    them; the caller must list every cube that can reach the crops."""
    lib = _load()
    cam = _cam(cam)
    p = _pos64(pos, N)
    cr = np.ascontiguousarray(np.asarray(crops, dtype=np.int32).reshape(-1, 4))
    sizes = [int(w) * int(h) for (_, _, w, h) in cr]
    out = np.zeros(sum(sizes), dtype=np.float64)
    nf, nd = C.c_longlong(0), C.c_longlong(0)
    cc = cam.to_c()
    if cubes is None:
        rc = lib.orc_render(_ptr(p, C.c_double), N, box, total_mass, C.byref(cc), _ptr(cr, C.c_int),
                            len(cr), _ptr(out, C.c_double), C.byref(nf), C.byref(nd), nthreads)
    else:
        sel = np.ascontiguousarray(np.asarray(cubes, dtype=np.int64).ravel())
        rc = lib.orc_render_subset(_ptr(p, C.c_double), N, box, total_mass, C.byref(cc), _ptr(cr, C.c_int),
                                   len(cr), _ptr(sel, C.c_longlong), len(sel), _ptr(out, C.c_double),
                                   C.byref(nf), C.byref(nd), nthreads)
    if rc != 0:
        raise RuntimeError(f"oracle render failed with code {rc}")
    imgs, o = [], 0
    for (_, _, w, h), s in zip(cr, sizes):
        imgs.append(out[o:o + s].reshape(int(h), int(w)))
        o += s
    return imgs, int(nf.value), int(nd.value)


def render(pos, N: int, cam, box: float = 1.0, total_mass: float = 1.0, nthreads: int = 0,
           return_counts: bool = False):
    """Full-frame FP64 column-density image [H][W] (Eq. 6 per pixel-centre ray)."""
    cam = _cam(cam)
    imgs, nf, nd = render_crops(pos, N, cam, [(0, 0, cam.W, cam.H)], box, total_mass, nthreads)
    if return_counts:
        return imgs[0], nf, nd
    return imgs[0]


def tet_volumes(pos, N: int, box: float = 1.0, total_mass: float = 1.0):
    """Signed volumes (Eq. 9) and densities (Eq. 3) of all 6 N^3 tetrahedra."""
    lib = _load()
    p = _pos64(pos, N)
    n = 6 * N ** 3
    vol = np.zeros(n, dtype=np.float64)
    rho = np.zeros(n, dtype=np.float64)
    rc = lib.orc_tets(_ptr(p, C.c_double), N, box, total_mass, _ptr(vol, C.c_double),
                      _ptr(rho, C.c_double))
    if rc != 0:
        raise RuntimeError(f"oracle tets failed with code {rc}")
    return vol, rho


def gradient(pos, N: int, cam, dLdI: np.ndarray, box: float = 1.0, total_mass: float = 1.0,
             nthreads: int = 0) -> np.ndarray:
    """dL/d(particle positions) [N^3][3] for a given dL/dI [H][W]."""
    lib = _load()
    cam = _cam(cam)
    p = _pos64(pos, N)
    g_img = np.ascontiguousarray(np.asarray(dLdI, dtype=np.float64).reshape(cam.H, cam.W))
    out = np.zeros((N ** 3, 3), dtype=np.float64)
    cc = cam.to_c()
    rc = lib.orc_grad(_ptr(p, C.c_double), N, box, total_mass, C.byref(cc), _ptr(g_img, C.c_double),
                      _ptr(out, C.c_double), nthreads)
    if rc != 0:
        raise RuntimeError(f"oracle grad failed with code {rc}")
    return out


def frame_mass(img: np.ndarray, cam) -> float:
    """Sum of pixel values times the orthographic pixel area."""
    cam = _cam(cam)
    area = (cam.hi[0] - cam.lo[0]) * (cam.hi[1] - cam.lo[1]) / (cam.W * cam.H)
    return float(np.sum(img, dtype=np.float64) * area)


def chord(verts, origin, direction, halfline: bool = False) -> float:
    """Exact length of the ray origin + s * direction inside one tetrahedron."""
    lib = _load()
    v = np.ascontiguousarray(np.asarray(verts, dtype=np.float64).reshape(4, 3))
    o = np.ascontiguousarray(np.asarray(origin, dtype=np.float64))
    d = np.ascontiguousarray(np.asarray(direction, dtype=np.float64))
    return float(lib.orc_chord(_ptr(v, C.c_double), _ptr(o, C.c_double), _ptr(d, C.c_double), int(halfline)))


def tet_vertices(pos, N: int, i: int, j: int, k: int, s: int, box: float = 1.0) -> np.ndarray:
    """Unwrapped vertices [4][3] of tetrahedron s of cube (i, j, k)."""
    lib = _load()
    p = _pos64(pos, N)
    out = np.zeros((4, 3), dtype=np.float64)
    rc = lib.orc_tet_vertices(_ptr(p, C.c_double), N, box, i, j, k, s, _ptr(out, C.c_double))
    if rc != 0:
        raise RuntimeError(f"oracle tet_vertices failed with code {rc}")
    return out


def render_soup(verts, dens, cam) -> np.ndarray:
    """Projection of arbitrary tetrahedra [n][4][3] with densities [n]."""
    lib = _load()
    cam = _cam(cam)
    v = np.ascontiguousarray(np.asarray(verts, dtype=np.float64).reshape(-1, 4, 3))
    d = np.ascontiguousarray(np.asarray(dens, dtype=np.float64).reshape(-1))
    out = np.zeros((cam.H, cam.W), dtype=np.float64)
    cc = cam.to_c()
    rc = lib.orc_render_soup(_ptr(v, C.c_double), _ptr(d, C.c_double), len(d), C.byref(cc),
                             _ptr(out, C.c_double))
    if rc != 0:
        raise RuntimeError(f"oracle render_soup failed with code {rc}")
    return out


def resample(pos, N: int, n: int, weight: str = "density", box: float = 1.0, total_mass: float = 1.0,
             nthreads: int = 0) -> np.ndarray:
    """Resampling onto a periodic n^3 grid (Sec. 4.3, Eq. 10-12): cell
    [c][b][a] holds the sum over tetrahedra of q dl, dl the length of the
    cell's central line along z inside the tetrahedron and the cell's slab;
    q = rho (weight "density") or 1 (weight "streams")."""
    lib = _load()
    p = _pos64(pos, N)
    w = {"density": 0, "streams": 1}[weight]
    out = np.zeros((n, n, n), dtype=np.float64)
    rc = lib.orc_resample(_ptr(p, C.c_double), N, box, total_mass, n, w, _ptr(out, C.c_double), nthreads)
    if rc != 0:
        raise RuntimeError(f"oracle resample failed with code {rc}")
    return out


def point_density(pos, N: int, points, weight: str = "density", box: float = 1.0, total_mass: float = 1.0,
                  nthreads: int = 0) -> np.ndarray:
    """Sum over the tetrahedra containing each point (Sec. 3.2, Eq. 4) of rho
    (weight "density": the total density) or 1 (weight "streams": the
    number of streams). points: [P][3] in box coordinates."""
    lib = _load()
    p = _pos64(pos, N)
    pts = np.ascontiguousarray(np.asarray(points, dtype=np.float64).reshape(-1, 3))
    w = {"density": 0, "streams": 1}[weight]
    out = np.zeros(max(1, pts.shape[0]), dtype=np.float64)
    rc = lib.orc_point_density(_ptr(p, C.c_double), N, box, total_mass, _ptr(pts, C.c_double), pts.shape[0], w,
                               _ptr(out, C.c_double), nthreads)
    if rc != 0:
        raise RuntimeError(f"oracle point_density failed with code {rc}")
    return out[:pts.shape[0]]


def centroids(pos, N: int, cam, box: float = 1.0, total_mass: float = 1.0, nthreads: int = 0) -> np.ndarray:
    """Centroid splats (Sec. 4.2) of every tetrahedron: the 2D M4 cubic
    spline of unit integral with smoothing length |V|^(1/3) on a billboard
    through the centroid facing the view, weighted by the tetrahedron's
    mass (perspective rays pick it up over the cosine of their angle to the
    view direction). Returns [H][W] float64."""
    lib = _load()
    cam = _cam(cam)
    p = _pos64(pos, N)
    out = np.zeros((cam.H, cam.W), dtype=np.float64)
    cc = cam.to_c()
    rc = lib.orc_centroids(_ptr(p, C.c_double), N, box, total_mass, C.byref(cc), _ptr(out, C.c_double), nthreads)
    if rc != 0:
        raise RuntimeError(f"oracle centroids failed with code {rc}")
    return out


def hybrid(pos, N: int, cam, r_near: float, box: float = 1.0, total_mass: float = 1.0,
           nthreads: int = 0) -> np.ndarray:
    """Hybrid near/far rendering of a perspective view: cubes whose corner-0
    particle lies within r_near of the eye by the exact projection (Eq. 6),
    the others' tetrahedra as centroid splats. Returns [H][W] float64."""
    lib = _load()
    cam = _cam(cam)
    p = _pos64(pos, N)
    out = np.zeros((cam.H, cam.W), dtype=np.float64)
    cc = cam.to_c()
    rc = lib.orc_hybrid(_ptr(p, C.c_double), N, box, total_mass, C.byref(cc), float(r_near), _ptr(out, C.c_double),
                        nthreads)
    if rc != 0:
        raise RuntimeError(f"oracle hybrid failed with code {rc}")
    return out


def render_area(pos, N: int, cam, box: float = 1.0, total_mass: float = 1.0, nthreads: int = 0) -> np.ndarray:
    """Area-averaged pixels of an orthographic view: each pixel holds the
    mean of the column density (Eq. 6) over its square. Returns [H][W]."""
    lib = _load()
    cam = _cam(cam)
    p = _pos64(pos, N)
    out = np.zeros((cam.H, cam.W), dtype=np.float64)
    cc = cam.to_c()
    rc = lib.orc_render_area(_ptr(p, C.c_double), N, box, total_mass, C.byref(cc), _ptr(out, C.c_double), nthreads)
    if rc != 0:
        raise RuntimeError(f"oracle render_area failed with code {rc}")
    return out
