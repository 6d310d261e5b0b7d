"""Cubes that can reach given pixels of an orthographic view along z through
the periodic box window (test helper).

A tetrahedron of cube (i, j, k) has its vertices at the cube's Lagrangian
corners plus their displacements, so in x it spans at most
[i h - B h, (i + 1) h + B h] with B the largest displacement component in
cells (and the same in y). A pixel centre outside that band, modulo the
box, cannot see the cube. One extra cell of margin covers rounding and
sub-pixel shifts of the rays."""
import numpy as np


def max_displacement_cells(pos, N: int, box: float = 1.0) -> float:
    p = np.asarray(pos, dtype=np.float64).reshape(N ** 3, -1)[:, :3]
    idx = np.arange(N ** 3)
    q = np.stack([idx % N, (idx // N) % N, idx // (N * N)], axis=1) * (box / N)
    d = p - q
    d -= box * np.round(d / box)
    return float(np.abs(d).max()) * N / box


def cubes_near_pixels(pos, N: int, W: int, H: int, pixels, box: float = 1.0, B=None) -> np.ndarray:
    """Sorted unique ids i + N (j + N k) of every cube that can reach any of
    the pixel centres `pixels` [(px, py), ...] of the [0, box)^2 window. B:
    the largest displacement component in cells, when the caller knows it
    (FP16 offsets hold it directly)."""
    if B is None:
        B = max_displacement_cells(pos, N, box)
    r = int(np.ceil(B)) + 2
    ids = set()
    ks = np.arange(N)
    for px, py in pixels:
        cx = (px + 0.5) / W * N
        cy = (py + 0.5) / H * N
        ii = np.arange(int(np.floor(cx)) - r, int(np.floor(cx)) + r + 1) % N
        jj = np.arange(int(np.floor(cy)) - r, int(np.floor(cy)) + r + 1) % N
        I, J, K = np.meshgrid(np.unique(ii), np.unique(jj), ks, indexing="ij")
        ids.update((I + N * (J + N * K)).ravel().tolist())
    return np.array(sorted(ids), dtype=np.int64)
