"""Central differences of an oracle loss when one particle moves: only the
48 tetrahedra of the 8 cubes around it change, so their image is re-rendered
alone (with the periodic copies of the box window) and swapped into the
full oracle image."""
import numpy as np

import oracle


def incident_tets(p, N):
    """Tetrahedron ids (6 cube + s) of the 8 cubes that have particle p as a corner."""
    i, j, k = p % N, (p // N) % N, p // (N * N)
    out = []
    for n in range(8):
        ci, cj, ck = (i - (n & 1)) % N, (j - ((n >> 1) & 1)) % N, (k - ((n >> 2) & 1)) % N
        cube = ci + N * (cj + N * ck)
        out.extend(6 * cube + s for s in range(6))
    return out


def local_image(pos64, N, tets, cam, box=1.0):
    """The oracle's image of the listed tetrahedra alone, with the periodic
    copies of the box window (shifts of one box in x and y)."""
    _, rho = oracle.tet_volumes(pos64, N)
    verts = []
    for t in tets:
        cube, s = divmod(t, 6)
        i, j, k = cube % N, (cube // N) % N, cube // (N * N)
        verts.append(oracle.tet_vertices(pos64, N, i, j, k, s))
    verts = np.array(verts)
    dens = rho[tets]
    allv, alld = [], []
    for dx in (-box, 0.0, box):
        for dy in (-box, 0.0, box):
            allv.append(verts + np.array([dx, dy, 0.0]))
            alld.append(dens)
    soup_cam = dict(cam)
    soup_cam["wrap"] = False
    return oracle.render_soup(np.concatenate(allv), np.concatenate(alld), soup_cam)
