"""Two further formulations of the projection, for tiny inputs only.

TEST INFRASTRUCTURE ONLY. Written independently of lt_oracle.c (own lattice
walk, own unwrapping, own camera rays, connectivity read from the table
printed in the paper, tests/golden/connectivity.txt), so that agreement with
the oracle pins its arithmetic:

  * `render_barycentric`: every (pixel, tetrahedron) pair; the chord is the
    length of the parameter interval on which all four barycentric
    coordinates of the ray point are >= 0 (the definition of "inside").
  * `render_cell_projection`: the front/back face form of Eq. 13 (Sec. 4.4):
    every face hit by the ray adds rho * |X - c| to a back-face sum or to a
    front-face sum, c the camera location; the pixel is back minus front.
  * `resample_barycentric`: the grid resampling of Sec. 4.3 with the same
    barycentric inside test along each cell column.
  * `centroids_bruteforce`: the centroid splats of Sec. 4.2 over every
    (pixel, tetrahedron, period) triple, in numpy.
  * `area_bruteforce`: area-averaged pixels of an orthographic view as the
    volume of each tetrahedron clipped to the prism of each pixel's square
    (the vertices of the eight-plane polytope by brute force over plane
    triples, its volume by a convex hull), times rho, over the pixel's area.

Both draw every periodic copy of every tetrahedron for periodic orthographic
windows by brute force over image-period shifts in [-2, 2].
"""
from __future__ import annotations

import math
import os

import numpy as np

_TABLE = None


def connectivity() -> np.ndarray:
    global _TABLE
    if _TABLE is None:
        path = os.path.join(os.path.dirname(__file__), "..", "tests", "golden", "connectivity.txt")
        rows = [list(map(int, ln.split())) for ln in open(path) if ln.strip() and not ln.startswith("#")]
        _TABLE = np.array(rows, dtype=np.int64)
    return _TABLE


def lattice_tets(pos, N: int, box: float = 1.0, total_mass: float = 1.0):
    """All tetrahedra of the periodic lattice: vertices [6N^3][4][3] and
    densities [6N^3], tetrahedron id = 6 * (i + N (j + N k)) + s."""
    p = np.asarray(pos, dtype=np.float64).reshape(N ** 3, -1)[:, :3]
    h = box / N
    tab = connectivity()
    verts = np.zeros((6 * N ** 3, 4, 3))
    t = 0
    for k in range(N):
        for j in range(N):
            for i in range(N):
                for s in range(6):
                    for c in range(4):
                        n = int(tab[s, c])
                        ii, jj, kk = i + (n & 1), j + ((n >> 1) & 1), k + ((n >> 2) & 1)
                        pid = (ii % N) + N * ((jj % N) + N * (kk % N))
                        q = np.array([ii, jj, kk], dtype=np.float64) * h
                        d = p[pid] - q
                        d = d - box * np.round(d / box)
                        verts[t, c] = q + d
                    t += 1
    a = verts[:, 1] - verts[:, 0]
    b = verts[:, 2] - verts[:, 0]
    c = verts[:, 3] - verts[:, 0]
    vol = np.einsum("ij,ij->i", a, np.cross(b, c)) / 6.0
    m = total_mass / (6.0 * N ** 3)
    with np.errstate(divide="ignore"):
        rho = np.where(vol != 0, m / np.abs(vol), 0.0)
    return verts, rho, vol


def _frame(cam):
    f = np.asarray(cam["fwd"], dtype=np.float64)
    f = f / np.linalg.norm(f)
    r = np.cross(np.asarray(cam["up"], dtype=np.float64), f)
    r = r / np.linalg.norm(r)
    u = np.cross(f, r)
    return r, u, f


def pixel_rays(cam):
    """Origins and unit directions [H*W][3] of all pixel-centre rays."""
    W, H = cam["W"], cam["H"]
    r, u, f = _frame(cam)
    px, py = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    px, py = px.ravel(), py.ravel()
    if cam["type"] == "ortho":
        lo, hi = cam["lo"], cam["hi"]
        a = lo[0] + px * (hi[0] - lo[0]) / W
        b = lo[1] + py * (hi[1] - lo[1]) / H
        o = a[:, None] * r + b[:, None] * u
        d = np.broadcast_to(f, o.shape).copy()
        return o, d, False
    ty = math.tan(math.radians(cam["fov_y_deg"]) / 2)
    tx = ty * W / H
    xt = tx * (2 * px / W - 1)
    yt = ty * (2 * py / H - 1)
    d = f + xt[:, None] * r + yt[:, None] * u
    d = d / np.linalg.norm(d, axis=1, keepdims=True)
    o = np.broadcast_to(np.asarray(cam["eye"], dtype=np.float64), d.shape).copy()
    return o, d, True


def _copies(cam):
    if cam["type"] == "ortho" and cam.get("wrap", False):
        r, u, _ = _frame(cam)
        pu = (cam["hi"][0] - cam["lo"][0]) * r
        pv = (cam["hi"][1] - cam["lo"][1]) * u
        return [sx * pu + sy * pv for sx in range(-2, 3) for sy in range(-2, 3)]
    return [np.zeros(3)]


def _chord_barycentric(v, o, d, halfline):
    M = np.vstack([v.T, np.ones(4)])  # columns are [v_i; 1]
    Minv = np.linalg.inv(M)
    lam0 = (Minv[:, :3] @ o.T) + Minv[:, 3:4]  # [4][P]
    mu = Minv[:, :3] @ d.T
    P = o.shape[0]
    lo = np.full(P, -np.inf if not halfline else 0.0)
    hi = np.full(P, np.inf)
    ok = np.ones(P, dtype=bool)
    for i in range(4):
        with np.errstate(divide="ignore", invalid="ignore"):
            s = -lam0[i] / mu[i]
        pos = mu[i] > 0
        neg = mu[i] < 0
        zer = mu[i] == 0
        lo = np.where(pos, np.maximum(lo, s), lo)
        hi = np.where(neg, np.minimum(hi, s), hi)
        ok &= ~(zer & (lam0[i] < 0))
    return np.where(ok & (hi > lo), hi - lo, 0.0)


def render_barycentric(pos, N: int, cam: dict, box: float = 1.0, total_mass: float = 1.0) -> np.ndarray:
    verts, rho, vol = lattice_tets(pos, N, box, total_mass)
    o, d, half = pixel_rays(cam)
    img = np.zeros(o.shape[0])
    for shift in _copies(cam):
        for t in range(len(rho)):
            if vol[t] == 0:
                continue
            img += rho[t] * _chord_barycentric(verts[t] + shift, o, d, half)
    return img.reshape(cam["H"], cam["W"])


def _face_hits(a, b, c, o, d):
    """Ray / triangle intersection (all rays against one triangle):
    parameter s and a hit mask (barycentric coordinates all >= 0)."""
    e1, e2 = b - a, c - a
    pvec = np.cross(d, e2)
    det = pvec @ e1
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / det
        tvec = o - a
        uu = np.einsum("ij,ij->i", tvec, pvec) * inv
        qvec = np.cross(tvec, e1)
        vv = np.einsum("ij,ij->i", qvec, d) * inv
        s = (qvec @ e2) * inv
    hit = (det != 0) & (uu >= 0) & (vv >= 0) & (uu + vv <= 1)
    return s, hit


def render_cell_projection(pos, N: int, cam: dict, box: float = 1.0, total_mass: float = 1.0,
                           far: float = 100.0) -> np.ndarray:
    verts, rho, vol = lattice_tets(pos, N, box, total_mass)
    o, d, half = pixel_rays(cam)
    # camera location c: the eye, or a point far behind the orthographic image plane
    c = o if half else o - far * d
    front = np.zeros(o.shape[0])
    back = np.zeros(o.shape[0])
    for shift in _copies(cam):
        for t in range(len(rho)):
            if vol[t] == 0:
                continue
            v = verts[t] + shift
            for i in range(4):
                a, b, cc = v[(i + 1) % 4], v[(i + 2) % 4], v[(i + 3) % 4]
                n = np.cross(b - a, cc - a)
                if n @ (v[i] - a) > 0:
                    n = -n  # outward normal
                s, hit = _face_hits(a, b, cc, o, d)
                if half:
                    hit &= s >= 0
                X = o + s[:, None] * d
                dist = np.linalg.norm(X - c, axis=1)
                facing = d @ n
                front += np.where(hit & (facing < 0), rho[t] * dist, 0.0)
                back += np.where(hit & (facing > 0), rho[t] * dist, 0.0)
    return (back - front).reshape(cam["H"], cam["W"])


def resample_barycentric(pos, N: int, n: int, weight: str = "density", box: float = 1.0,
                         total_mass: float = 1.0) -> np.ndarray:
    """Resampling onto the periodic n^3 grid (Sec. 4.3) by brute force: every
    (cell column, tetrahedron, period shift) triple; the segment of the
    column's central line inside the tetrahedron is the parameter interval on
    which all four barycentric coordinates are >= 0, then clipped to each
    slab. Cell [c][b][a] as in oracle.resample."""
    verts, rho, _ = lattice_tets(pos, N, box, total_mass)
    g = box / n
    out = np.zeros((n, n, n))
    cols = np.array([[(a + 0.5) * g, (b + 0.5) * g] for b in range(n) for a in range(n)])
    d = np.tile(np.array([[0.0, 0.0, 1.0]]), (cols.shape[0], 1))
    for t in range(verts.shape[0]):
        if rho[t] == 0.0:
            continue
        q = rho[t] if weight == "density" else 1.0
        v = verts[t]
        M = np.vstack([v.T, np.ones(4)])
        Minv = np.linalg.inv(M)
        for sy in range(-2, 3):
            for sx in range(-2, 3):
                o = np.column_stack([cols[:, 0] + sx * box, cols[:, 1] + sy * box, np.zeros(cols.shape[0])])
                lam0 = (Minv[:, :3] @ o.T) + Minv[:, 3:4]
                mu = Minv[:, :3] @ d.T
                lo = np.full(o.shape[0], -np.inf)
                hi = np.full(o.shape[0], np.inf)
                ok = np.ones(o.shape[0], dtype=bool)
                for i in range(4):
                    with np.errstate(divide="ignore", invalid="ignore"):
                        s = -lam0[i] / mu[i]
                    lo = np.where(mu[i] > 0, np.maximum(lo, s), lo)
                    hi = np.where(mu[i] < 0, np.minimum(hi, s), hi)
                    ok &= ~((mu[i] == 0) & (lam0[i] < 0))
                for p in np.nonzero(ok & (hi > lo))[0]:
                    a, b = p % n, p // n
                    for c in range(int(math.floor(lo[p] / g)), int(math.floor(hi[p] / g)) + 1):
                        seg = min(hi[p], (c + 1) * g) - max(lo[p], c * g)
                        if seg > 0:
                            out[c % n, b, a] += q * seg
    return out


def centroids_bruteforce(pos, N: int, W: int, H: int, lo=(0.0, 0.0), hi=(1.0, 1.0), box: float = 1.0,
                         total_mass: float = 1.0) -> np.ndarray:
    """Centroid splats for a periodic orthographic view along +z (right = +x,
    up = +y) over the window [lo, hi]: every (pixel, tetrahedron, image-period
    shift) triple, the 2D M4 cubic spline (unit integral) of smoothing length
    |V|^(1/3) at the centroid, times the tetrahedron's mass."""
    verts, _, vol = lattice_tets(pos, N, box, total_mass)
    m = total_mass / (6.0 * N ** 3)
    cen = verts.mean(axis=1)
    lx, ly = hi[0] - lo[0], hi[1] - lo[1]
    xs = lo[0] + (np.arange(W) + 0.5) * lx / W
    ys = lo[1] + (np.arange(H) + 0.5) * ly / H
    X, Y = np.meshgrid(xs, ys)  # [H][W]
    out = np.zeros((H, W))
    for t in range(len(vol)):
        if vol[t] == 0.0:
            continue
        h = abs(vol[t]) ** (1.0 / 3.0)
        norm = m * 10.0 / (7.0 * math.pi * h * h)
        for sy in range(-2, 3):
            for sx in range(-2, 3):
                r = np.hypot(X - (cen[t, 0] - sx * lx), Y - (cen[t, 1] - sy * ly)) / h
                w = np.where(r < 1.0, 1.0 - 1.5 * r ** 2 + 0.75 * r ** 3, np.where(r < 2.0, 0.25 * (2.0 - r) ** 3, 0.0))
                out += norm * w
    return out


def splats_perspective_bruteforce(verts, W: int, H: int, eye, fwd, up, fov_y_deg: float, total_mass: float,
                                  N: int) -> np.ndarray:
    """Perspective centroid splats of the given tetrahedra [n][4][3]: for every
    (pixel, tetrahedron), the ray through the pixel centre meets the
    billboard (through the centroid, normal to the view direction) at a point
    d from the centroid; the pixel adds m W(d, |V|^(1/3)) over the cosine of
    the ray's angle to the view direction."""
    f = np.asarray(fwd, dtype=np.float64)
    f = f / np.linalg.norm(f)
    r = np.cross(np.asarray(up, dtype=np.float64), f)
    r = r / np.linalg.norm(r)
    u = np.cross(f, r)
    ty = math.tan(math.radians(fov_y_deg) / 2.0)
    tx = ty * W / H
    xt = tx * (2.0 * (np.arange(W) + 0.5) / W - 1.0)
    yt = ty * (2.0 * (np.arange(H) + 0.5) / H - 1.0)
    XT, YT = np.meshgrid(xt, yt)
    e0 = np.asarray(eye, dtype=np.float64)
    m = total_mass / (6.0 * N ** 3)
    out = np.zeros((H, W))
    for v in verts:
        vol = np.dot(v[1] - v[0], np.cross(v[2] - v[0], v[3] - v[0])) / 6.0
        if vol == 0.0:
            continue
        c = v.mean(axis=0) - e0
        Z, X, Y = c @ f, c @ r, c @ u
        if Z <= 0.0:
            continue
        # the ray e0 + t (f + xt r + yt u) meets the plane through the centroid at t = Z
        d = np.hypot(Z * XT - X, Z * YT - Y)
        h = abs(vol) ** (1.0 / 3.0)
        q = d / h
        w = np.where(q < 1.0, 1.0 - 1.5 * q ** 2 + 0.75 * q ** 3, np.where(q < 2.0, 0.25 * (2.0 - q) ** 3, 0.0))
        out += m * 10.0 / (7.0 * math.pi * h * h) * w * np.sqrt(1.0 + XT ** 2 + YT ** 2)
    return out


def _clipped_volume(planes):
    """Volume of {p : n . p <= d for all (n, d) in planes} (bounded), from
    the feasible intersections of every plane triple."""
    from itertools import combinations
    from scipy.spatial import ConvexHull
    from scipy.spatial import QhullError
    n = np.array([q[0] for q in planes])
    d = np.array([q[1] for q in planes])
    pts = []
    for a, b, c in combinations(range(len(planes)), 3):
        M = n[[a, b, c]]
        if abs(np.linalg.det(M)) < 1e-14:
            continue
        x = np.linalg.solve(M, d[[a, b, c]])
        if np.all(n @ x <= d + 1e-12):
            pts.append(x)
    if len(pts) < 4:
        return 0.0
    try:
        return float(ConvexHull(np.array(pts)).volume)
    except QhullError:
        return 0.0


def area_bruteforce(pos, N: int, cam: dict, box: float = 1.0, total_mass: float = 1.0) -> np.ndarray:
    """Area-averaged pixels [H][W] of an orthographic view: for every
    (pixel, tetrahedron, period) triple, rho times the volume of the
    tetrahedron inside the prism over the pixel's square, over the square's
    area. Tiny inputs only."""
    verts, rho, vol = lattice_tets(pos, N, box, total_mass)
    r, u, _ = _frame(cam)
    W, H = cam["W"], cam["H"]
    lo, hi = np.asarray(cam["lo"], dtype=np.float64), np.asarray(cam["hi"], dtype=np.float64)
    dx, dy = (hi[0] - lo[0]) / W, (hi[1] - lo[1]) / H
    out = np.zeros((H, W))
    for t in range(len(verts)):
        if vol[t] == 0.0:
            continue
        v0 = verts[t]
        for shift in _copies(cam):
            v = v0 + shift
            # outward face planes of the tetrahedron
            faces = []
            for f in range(4):
                a, b, c = v[(f + 1) % 4], v[(f + 2) % 4], v[(f + 3) % 4]
                nrm = np.cross(b - a, c - a)
                if nrm @ (v[f] - a) > 0:
                    nrm = -nrm
                faces.append((nrm, float(nrm @ a)))
            a_, b_ = v @ r, v @ u
            x0 = max(0, int(math.floor((a_.min() - lo[0]) / dx)))
            x1 = min(W - 1, int(math.floor((a_.max() - lo[0]) / dx)))
            y0 = max(0, int(math.floor((b_.min() - lo[1]) / dy)))
            y1 = min(H - 1, int(math.floor((b_.max() - lo[1]) / dy)))
            for py in range(y0, y1 + 1):
                for px in range(x0, x1 + 1):
                    xa, xb = lo[0] + px * dx, lo[0] + (px + 1) * dx
                    ya, yb = lo[1] + py * dy, lo[1] + (py + 1) * dy
                    planes = faces + [(-r, -xa), (r, xb), (-u, -ya), (u, yb)]
                    out[py, px] += rho[t] * _clipped_volume(planes) / (dx * dy)
    return out
