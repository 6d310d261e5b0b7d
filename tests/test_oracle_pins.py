"""Pins of the FP64 oracle against facts fixed by the paper and by geometry.

Each test checks the oracle against something other than itself: the
connectivity table printed in the paper (tests/golden/connectivity.txt),
closed forms, invariants of the tessellation, or two independent brute-force
formulations. A plausible mistake in the oracle (a wrong corner numbering, a
dropped periodic copy, a sign error in an orientation, a wrong ray) breaks at
least one of them.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import bruteforce as bf
from lt_inputs import ZeldovichField, camera_dict, ortho_z


def lattice_positions(N, box=1.0, disp=None, dtype=np.float32):
    idx = np.arange(N ** 3)
    q = np.stack([idx % N, (idx // N) % N, idx // (N * N)], axis=1) * (box / N)
    x = q if disp is None else q + disp(q)
    x = np.mod(x, box)
    out = np.zeros((N ** 3, 4), dtype=dtype)
    out[:, :3] = x
    out[:, :3] = np.where(out[:, :3] >= dtype(box), dtype(0), out[:, :3])
    return out


def offset_window(W, H, box=1.0, off=(0.0123, 0.0457)):
    # a periodic window whose pixel centres avoid the lattice planes
    return camera_dict("ortho", W, H, fwd=(0, 0, 1), up=(0, 1, 0), lo=off,
                       hi=(off[0] + box, off[1] + box), wrap=True)


# ---------------------------------------------------------------------------
# Sec. 4.1 connectivity table (golden) and Eq. 9


def test_connectivity_table_tiles_the_cube():
    """The printed table with corner n -> (n&1, n>>1&1, n>>2&1) splits the
    unit cube into six tetrahedra of volume -1/6 that cover it exactly once."""
    tab = bf.connectivity()
    corners = np.array([[(n & 1), (n >> 1) & 1, (n >> 2) & 1] for n in range(8)], dtype=np.float64)
    rng = np.random.default_rng(0)
    pts = rng.random((20000, 3))
    inside = np.zeros(len(pts), dtype=int)
    for row in tab:
        v = corners[row]
        vol = np.dot(v[1] - v[0], np.cross(v[2] - v[0], v[3] - v[0])) / 6.0
        assert vol == pytest.approx(-1.0 / 6.0, abs=1e-15)
        M = np.vstack([v.T, np.ones(4)])
        lam = np.linalg.solve(M, np.vstack([pts.T, np.ones(len(pts))]))
        inside += np.all(lam >= 0, axis=0)
    assert np.all(inside == 1)


def test_oracle_tets_follow_golden_table():
    N, box = 3, 1.0
    pos = lattice_positions(N, box)
    tab = bf.connectivity()
    h = box / N
    for (i, j, k) in [(0, 0, 0), (2, 1, 0), (2, 2, 2)]:
        for s in range(6):
            v = oracle.tet_vertices(pos, N, i, j, k, s, box)
            want = [[(i + (n & 1)) * h, (j + ((n >> 1) & 1)) * h, (k + ((n >> 2) & 1)) * h] for n in tab[s]]
            np.testing.assert_allclose(v, want, atol=1e-7)


def test_signed_volumes_unperturbed_and_total():
    """Unperturbed: every tet has V = -h^3/6 (all six negative with this
    table). Deformed, periodic: the signed volumes still sum to -box^3."""
    N = 6
    vol, rho = oracle.tet_volumes(lattice_positions(N), N)
    np.testing.assert_allclose(vol, -1.0 / (6 * N ** 3), rtol=1e-6)
    np.testing.assert_allclose(rho, 1.0, rtol=1e-6)  # m / |V| with M = 1 in a unit box
    f = ZeldovichField.generate(16, -2.0, 6.0, 3)
    vol, rho = oracle.tet_volumes(f.positions(3.0), 16)
    assert (vol > 0).any()  # shell crossing inverts some tetrahedra
    assert vol.sum() == pytest.approx(-1.0, rel=1e-12)


# ---------------------------------------------------------------------------
# Eq. 6: chords and single tetrahedra


def test_corner_tet_chord_closed_form():
    """Tet (0,0,0),(a,0,0),(0,a,0),(0,0,a): chord along z at (x, y) is
    a - x - y inside the triangle, along x at (y, z) it is a - y - z."""
    a = 0.7
    v = [[0, 0, 0], [a, 0, 0], [0, a, 0], [0, 0, a]]
    rng = np.random.default_rng(1)
    for _ in range(200):
        x, y = rng.uniform(-0.2, 0.9, 2)
        want = max(0.0, a - x - y) if (x >= 0 and y >= 0) else 0.0
        assert oracle.chord(v, [x, y, -3.0], [0, 0, 1]) == pytest.approx(want, abs=1e-14)
        assert oracle.chord(v, [5.0, x, y], [-1, 0, 0]) == pytest.approx(
            max(0.0, a - x - y) if (x >= 0 and y >= 0) else 0.0, abs=1e-14)
    # a half-line that starts inside the tet only measures the part ahead
    assert oracle.chord(v, [0.1, 0.1, 0.2], [0, 0, 1], halfline=True) == pytest.approx(a - 0.2 - 0.2, abs=1e-14)


def test_corner_tet_image_closed_form():
    a = 0.6
    v = np.array([[[0, 0, 0], [a, 0, 0], [0, a, 0], [0, 0, a]]], dtype=np.float64)
    cam = camera_dict("ortho", 37, 41, fwd=(0, 0, 1), up=(0, 1, 0), lo=(-0.11, -0.07), hi=(0.71, 0.69))
    img = oracle.render_soup(v, [2.5], cam)
    xs = -0.11 + (np.arange(37) + 0.5) * (0.82 / 37)
    ys = -0.07 + (np.arange(41) + 0.5) * (0.76 / 41)
    X, Y = np.meshgrid(xs, ys)
    want = np.where((X >= 0) & (Y >= 0), 2.5 * np.maximum(0.0, a - X - Y), 0.0)
    np.testing.assert_allclose(img, want, atol=1e-13)


def test_single_tet_mass_converges():
    """Sum of rho * chord * pixel area -> rho |V| = m as the pixels shrink,
    with O(h^2) error (the chord is piecewise linear over the projection)."""
    rng = np.random.default_rng(7)
    v = rng.uniform(0.2, 0.8, (1, 4, 3))
    vol = abs(np.dot(v[0, 1] - v[0, 0], np.cross(v[0, 2] - v[0, 0], v[0, 3] - v[0, 0]))) / 6
    dens = 1.0 / vol  # unit mass
    errs = []
    for W in (50, 100, 200, 400):
        cam = camera_dict("ortho", W, W, fwd=(0.3, -0.2, 1.0), up=(0, 1, 0), lo=(-1.0, -1.0), hi=(1.5, 1.5))
        img = oracle.render_soup(v, [dens], cam)
        errs.append(abs(oracle.frame_mass(img, cam) - 1.0))
    assert errs[-1] < 1e-3
    assert errs[-1] < errs[0] / 10


# ---------------------------------------------------------------------------
# Lattices with known projections


def test_unperturbed_lattice_is_uniform_column_density():
    N = 8
    cam = offset_window(61, 53)
    img, nf, nd = oracle.render(lattice_positions(N), N, cam, return_counts=True)
    np.testing.assert_allclose(img, 1.0, rtol=1e-12)
    assert nd == 0
    assert nf == 4 * N * 61 * 53  # every z-ray crosses exactly 4 tets per cube
    # scaling with box and mass: column density = M / box^2
    box, M = 2.0, 3.0
    cam = offset_window(29, 31, box=box, off=(0.031, 0.077))
    img = oracle.render(lattice_positions(N, box), N, cam, box=box, total_mass=M)
    np.testing.assert_allclose(img, M / box ** 2, rtol=1e-12)


def test_translated_and_z_displaced_lattices_stay_uniform():
    """A uniform translation, or any displacement along the line of sight
    (even with shell crossing and inverted tetrahedra), leaves every column
    of the periodic box with the same mass."""
    N = 8
    cam = offset_window(47, 43)
    shift = lambda q: np.broadcast_to(np.array([0.31, 0.17, 0.4]), q.shape)
    img = oracle.render(lattice_positions(N, disp=shift, dtype=np.float64), N, cam)
    np.testing.assert_allclose(img, 1.0, rtol=1e-11)

    def dz(q):
        d = np.zeros_like(q)
        d[:, 2] = 0.25 * np.sin(2 * np.pi * q[:, 2]) + 0.1 * np.cos(2 * np.pi * q[:, 0]) * np.sin(2 * np.pi * q[:, 1])
        return d

    pos = lattice_positions(N, disp=dz)
    vol, _ = oracle.tet_volumes(pos, N)
    assert (vol > 0).any()
    img = oracle.render(pos, N, cam)
    np.testing.assert_allclose(img, 1.0, rtol=1e-10)


def _pancake(N, A):
    return lambda q: np.stack([-(A / (2 * np.pi)) * np.sin(2 * np.pi * q[:, 0]),
                               np.zeros(len(q)), np.zeros(len(q))], axis=1)


def test_pancake_closed_form_multistream():
    """1D Zel'dovich pancake x = q - A/(2 pi) sin(2 pi q): each lattice cube
    maps affinely onto [x_i, x_{i+1}], so the projection along z is exactly
    sum over cube columns containing x of 1 / (N |x_{i+1} - x_i|); A > 1 gives
    three streams and inverted tetrahedra."""
    N, A = 16, 2.5
    pos = lattice_positions(N, disp=_pancake(N, A))
    W, H = 200, 24
    cam = offset_window(W, H, off=(0.0031, 0.0123))
    img = oracle.render(pos, N, cam)
    # unwrapped column edges from the stored float32 positions
    h = 1.0 / N
    xs = []
    for i in range(N + 1):
        d = float(pos[i % N, 0]) - i * h
        d -= round(d)
        xs.append(i * h + d)
    px = 0.0031 + (np.arange(W) + 0.5) / W
    want = np.zeros(W)
    for i in range(N):
        a, b = sorted((xs[i], xs[i + 1]))
        for s in (-1, 0, 1):
            inside = (px >= a + s) & (px <= b + s)
            want += np.where(inside, 1.0 / (N * (b - a)), 0.0)
    assert want.max() > 3  # caustics
    streams = np.zeros(W, dtype=int)
    for i in range(N):
        a, b = sorted((xs[i], xs[i + 1]))
        for s in (-1, 0, 1):
            streams += (px >= a + s) & (px <= b + s)
    assert streams.max() == 3
    np.testing.assert_allclose(img, np.broadcast_to(want, (H, W)), rtol=1e-9)


def test_periodic_frame_mass_is_total_mass():
    f = ZeldovichField.generate(16, -2.0, 6.0, 11)
    pos = f.positions(1.5)
    errs = []
    for W in (128, 512):
        img = oracle.render(pos, 16, ortho_z(W, W))
        errs.append(abs(oracle.frame_mass(img, ortho_z(W, W)) - 1.0))
    assert errs[1] < 1e-3 and errs[1] < errs[0]


def test_perspective_unperturbed_lattice_is_box_chord():
    """Unperturbed lattice of mean density 1 seen from outside: each pixel is
    the length of its ray inside the unit box (slab intersection)."""
    N = 6
    pos = lattice_positions(N, dtype=np.float64)
    eye = np.array([2.3, 1.7, 2.9])
    cam = camera_dict("persp", 40, 36, eye=eye, fwd=np.array([0.5, 0.5, 0.5]) - eye, up=(0, 0, 1),
                      fov_y_deg=50.0)
    img = oracle.render(pos, N, cam)
    o, d, _ = bf.pixel_rays(cam)
    with np.errstate(divide="ignore"):
        t1 = (0.0 - o) / d
        t2 = (1.0 - o) / d
    tmin = np.minimum(t1, t2).max(axis=1)
    tmax = np.maximum(t1, t2).min(axis=1)
    want = np.maximum(0.0, tmax - np.maximum(tmin, 0.0)).reshape(36, 40)
    assert want.max() > 1.0
    np.testing.assert_allclose(img, want, atol=1e-12)


@pytest.mark.parametrize("view", ["ortho", "persp"])
def test_oracle_matches_bruteforce_formulations(view):
    N = 4
    f = ZeldovichField.generate(N, -2.0, 2.0, 7)
    pos = f.positions(1.8)
    if view == "ortho":
        cam = camera_dict("ortho", 24, 20, fwd=(0.2, 0.1, 1.0), up=(0, 1, 0), lo=(0.013, 0.021),
                          hi=(1.013, 1.021), wrap=False)
    else:
        eye = np.array([0.5, -1.6, 1.3])
        cam = camera_dict("persp", 22, 18, eye=eye, fwd=np.array([0.5, 0.5, 0.5]) - eye, up=(0, 0, 1),
                          fov_y_deg=55.0)
    a = oracle.render(pos, N, cam)
    b = bf.render_barycentric(pos, N, cam)
    c = bf.render_cell_projection(pos, N, cam)
    assert a.max() > 0
    np.testing.assert_allclose(a, b, atol=1e-12 * a.max())
    np.testing.assert_allclose(a, c, atol=1e-9 * a.max())


def test_oracle_matches_bruteforce_periodic_window():
    N = 3
    f = ZeldovichField.generate(N, -2.0, 1.5, 5)
    pos = f.positions(1.2)
    cam = offset_window(18, 16, off=(0.017, 0.029))
    a = oracle.render(pos, N, cam)
    b = bf.render_barycentric(pos, N, cam)
    np.testing.assert_allclose(a, b, atol=1e-12 * a.max())


# ---------------------------------------------------------------------------
# Gradient


def _fd_grad(pos, N, cam, target, comps, h=1e-6):
    def loss(p):
        img = oracle.render(p, N, cam)
        return float(np.sum((img - target) ** 2))

    base = pos[:, :3].astype(np.float64)
    out = []
    for (pid, a) in comps:
        pp = base.copy()
        pp[pid, a] += h
        lp = loss(pp)
        pp[pid, a] -= 2 * h
        lm = loss(pp)
        out.append((lp - lm) / (2 * h))
    return np.array(out)


@pytest.mark.parametrize("view", ["ortho", "persp"])
def test_gradient_matches_central_differences(view):
    N = 3
    f = ZeldovichField.generate(N, -2.0, 1.5, 9)
    pos = f.positions(1.4).astype(np.float64)
    if view == "ortho":
        cam = camera_dict("ortho", 26, 22, fwd=(0.15, -0.1, 1.0), up=(0, 1, 0), lo=(-0.1, -0.1),
                          hi=(1.1, 1.1), wrap=False)
    else:
        eye = np.array([1.9, 0.2, 1.4])
        cam = camera_dict("persp", 24, 20, eye=eye, fwd=np.array([0.5, 0.5, 0.5]) - eye, up=(0, 0, 1),
                          fov_y_deg=60.0)
    rng = np.random.default_rng(3)
    img = oracle.render(pos, N, cam)
    target = img + rng.normal(0, 0.3, img.shape)
    g = oracle.gradient(pos, N, cam, 2 * (img - target))
    comps = [(p, a) for p in range(N ** 3) for a in range(3)]
    fd = _fd_grad(pos, N, cam, target, comps)
    an = np.array([g[p, a] for (p, a) in comps])
    assert np.linalg.norm(an - fd) <= 1e-4 * np.linalg.norm(fd)


def test_gradient_along_orthographic_axis_vanishes():
    """Moving a vertex along the line of sight moves no mass between columns,
    so dI/dz = 0 for a projection along z."""
    N = 4
    f = ZeldovichField.generate(N, -2.0, 2.0, 13)
    pos = f.positions(1.6)
    cam = offset_window(32, 32)
    rng = np.random.default_rng(4)
    g = oracle.gradient(pos, N, cam, rng.normal(size=(32, 32)))
    assert np.abs(g[:, :2]).max() > 1e-3
    assert np.abs(g[:, 2]).max() <= 1e-10 * np.abs(g[:, :2]).max()


def test_local_difference_equals_full_render_difference():
    """The incident-tetrahedra image swap used for central differences of
    large frames reproduces differences of full oracle renders."""
    from fd_local import incident_tets, local_image
    N, W = 6, 48
    pos = ZeldovichField.generate(N, -2.5, 2.5, 1005).positions(2.0)
    tgt = ZeldovichField.generate(N, -2.5, 2.5, 2005).positions(2.0)
    cam = ortho_z(W, W)
    T = oracle.render(tgt, N, cam)
    I = oracle.render(pos, N, cam)
    pos64 = pos[:, :3].astype(np.float64)
    h = 1e-5
    for p in (0, N - 1, N ** 3 - 1, 77):
        tets = incident_tets(p, N)
        rest = I - local_image(pos64, N, tets, cam) - T
        for ax in range(3):
            pp = pos64.copy()
            pp[p, ax] += h
            up, Lp = local_image(pp, N, tets, cam), np.sum((oracle.render(pp, N, cam) - T) ** 2)
            pp[p, ax] -= 2 * h
            dn, Lm = local_image(pp, N, tets, cam), np.sum((oracle.render(pp, N, cam) - T) ** 2)
            local = np.sum((up - dn) * (up + dn + 2.0 * rest))
            assert local == pytest.approx(Lp - Lm, rel=1e-8, abs=1e-12 * max(1.0, abs(Lp)))


def test_chord_jumps_across_a_face_parallel_to_the_ray():
    """A face parallel to the view direction projects to a hull edge where the
    chord jumps; on the face itself the closed tetrahedron gives the upper
    one-sided limit. Corner tetrahedron (0,0,0), (a,0,0), (0,a,0), (0,0,a)
    seen along z: its face x = 0 contains the z axis, and for a ray at
    (x, y) with x, y >= 0 the chord is a - x - y."""
    a, y = 1.0, 0.25
    v = np.array([[0, 0, 0], [a, 0, 0], [0, a, 0], [0, 0, a]], dtype=np.float64)
    eps = 1e-9
    inside = oracle.chord(v, [eps, y, -3.0], [0, 0, 1])
    outside = oracle.chord(v, [-eps, y, -3.0], [0, 0, 1])
    on_face = oracle.chord(v, [0.0, y, -3.0], [0, 0, 1])
    assert inside == pytest.approx(a - y - eps, abs=1e-12)
    assert outside == 0.0
    assert on_face == pytest.approx(a - y, abs=1e-12)


# ---------------------------------------------------------------------------
# Resampling onto a grid (Sec. 4.3)


def test_resample_unperturbed_lattice_is_uniform():
    """One stream of density 1 everywhere: every cell holds rho g = g, in
    both weights (grids chosen so no central line lies on a cube face)."""
    N = 4
    idx = np.arange(N ** 3)
    pos = np.zeros((N ** 3, 4))
    pos[:, 0], pos[:, 1], pos[:, 2] = idx % N / N, (idx // N) % N / N, idx // (N * N) / N
    for n in (4, 8, 12):
        np.testing.assert_allclose(oracle.resample(pos, N, n, "density"), 1.0 / n, atol=1e-15)
        np.testing.assert_allclose(oracle.resample(pos, N, n, "streams"), 1.0 / n, atol=1e-15)


def test_resample_pancake_along_z_closed_form():
    """Displacement along z only, z = q_z - (A / 2 pi) sin(2 pi q_z) with
    A > 1 (shell crossing, three streams). Cube k of every column maps onto
    the box between z_k and z_{k+1}, with density h / |z_{k+1} - z_k|, so
    each slab's value is a sum of interval overlaps."""
    N, n, A = 8, 24, 1.6
    h, g = 1.0 / N, 1.0 / n
    idx = np.arange(N ** 3)
    i, j, k = idx % N, (idx // N) % N, idx // (N * N)
    pos = np.zeros((N ** 3, 4))
    pos[:, 0], pos[:, 1] = i * h, j * h
    pos[:, 2] = np.mod(k * h - A / (2 * np.pi) * np.sin(2 * np.pi * k * h), 1.0)
    zk = np.arange(N + 1) * h - A / (2 * np.pi) * np.sin(2 * np.pi * np.arange(N + 1) * h)
    dens, streams = np.zeros(n), np.zeros(n)
    for q in range(N):
        lo, hi = sorted((zk[q], zk[q + 1]))
        for c in range(-n, 2 * n):
            ov = max(0.0, min(hi, (c + 1) * g) - max(lo, c * g))
            dens[c % n] += h / (hi - lo) * ov
            streams[c % n] += ov
    assert streams.max() > 2.5 * g  # three streams somewhere
    np.testing.assert_allclose(oracle.resample(pos, N, n, "density"),
                               np.broadcast_to(dens[:, None, None], (n, n, n)), atol=1e-12)
    np.testing.assert_allclose(oracle.resample(pos, N, n, "streams"),
                               np.broadcast_to(streams[:, None, None], (n, n, n)), atol=1e-13)


def test_resample_columns_add_up_to_the_projection():
    """Summing a column's slabs gives its whole chord sum: the orthographic
    projection along z sampled at the same centres."""
    N, n = 8, 16
    pos = ZeldovichField.generate(N, -2.0, 3.0, 7).positions(1.8)
    r = oracle.resample(pos, N, n, "density")
    img = oracle.render(pos, N, ortho_z(n, n))
    np.testing.assert_allclose(r.sum(axis=0), img, atol=1e-12 * img.max())


def test_resample_matches_bruteforce_barycentric():
    """orc_resample against the barycentric brute force on a small random
    lattice (independent walk, unwrapping and inside test)."""
    N, n = 3, 6
    pos = ZeldovichField.generate(N, -2.0, 1.5, 11).positions(1.3).astype(np.float64)
    for weight in ("density", "streams"):
        a = oracle.resample(pos, N, n, weight)
        b = bf.resample_barycentric(pos, N, n, weight)
        np.testing.assert_allclose(a, b, atol=1e-12 * max(1.0, b.max()))


def test_point_density_uniform_and_pancake_closed_form():
    """Total density and stream count at points (Sec. 3.2, Eq. 4): one stream
    of density 1 for the unperturbed lattice; for the z-pancake, every stream
    k whose z-interval holds the point adds h / |z_{k+1} - z_k|."""
    rng = np.random.default_rng(17)
    pts = rng.random((300, 3))
    N = 4
    idx = np.arange(N ** 3)
    flat = np.zeros((N ** 3, 4))
    flat[:, 0], flat[:, 1], flat[:, 2] = idx % N / N, (idx // N) % N / N, idx // (N * N) / N
    np.testing.assert_allclose(oracle.point_density(flat, N, pts, "density"), 1.0, atol=1e-12)
    np.testing.assert_allclose(oracle.point_density(flat, N, pts, "streams"), 1.0, atol=0)
    N, A = 8, 1.6
    h = 1.0 / N
    ids = np.arange(N ** 3)
    i, j, k = ids % N, (ids // N) % N, ids // (N * N)
    pos = np.zeros((N ** 3, 4))
    pos[:, 0], pos[:, 1] = i * h, j * h
    pos[:, 2] = np.mod(k * h - A / (2 * np.pi) * np.sin(2 * np.pi * k * h), 1.0)
    zk = np.arange(N + 1) * h - A / (2 * np.pi) * np.sin(2 * np.pi * np.arange(N + 1) * h)
    want_d, want_s = np.zeros(len(pts)), np.zeros(len(pts))
    for q in range(N):
        lo, hi = sorted((zk[q], zk[q + 1]))
        for p, z in enumerate(pts[:, 2]):
            zz = z - np.floor(z - lo)  # the copy in [lo, lo + 1)
            if zz <= hi:
                want_d[p] += h / (hi - lo)
                want_s[p] += 1
    assert want_s.max() >= 3
    np.testing.assert_allclose(oracle.point_density(pos, N, pts, "density"), want_d, rtol=1e-12)
    np.testing.assert_allclose(oracle.point_density(pos, N, pts, "streams"), want_s, atol=0)


def test_point_density_matches_bruteforce_barycentric():
    """Against an independent barycentric inside test over all periodic
    copies of every tetrahedron."""
    N = 3
    pos = ZeldovichField.generate(N, -2.0, 1.5, 11).positions(1.3).astype(np.float64)
    verts, rho, _ = bf.lattice_tets(pos, N)
    pts = np.random.default_rng(5).random((200, 3))
    want_d, want_s = np.zeros(len(pts)), np.zeros(len(pts))
    shifts = np.array([[a, b, c] for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)], dtype=np.float64)
    for t in range(verts.shape[0]):
        if rho[t] == 0.0:
            continue
        Minv = np.linalg.inv(np.vstack([verts[t].T, np.ones(4)]))
        for sh in shifts:
            lam = Minv @ np.vstack([(pts + sh).T, np.ones(len(pts))])
            inside = (lam >= 0).all(axis=0)
            want_d[inside] += rho[t]
            want_s[inside] += 1
    np.testing.assert_allclose(oracle.point_density(pos, N, pts, "density"), want_d, rtol=1e-10)
    np.testing.assert_allclose(oracle.point_density(pos, N, pts, "streams"), want_s, atol=0)


@pytest.mark.parametrize("seed", [101, 202, 303, 404])
def test_oracle_matches_bruteforce_random_views(seed):
    """Seeded random lattices and views (orthographic in a random direction,
    or perspective from a random eye outside the box) against the
    barycentric brute force."""
    rng = np.random.default_rng(seed)
    N = 3
    pos = ZeldovichField.generate(N, -2.0, 1.5, seed).positions(float(rng.uniform(0.5, 2.0)))
    if seed % 2:
        fwd = rng.normal(size=3)
        fwd[2] = abs(fwd[2]) + 0.5
        cam = camera_dict("ortho", 20, 17, fwd=fwd, up=(0, 1, 0), lo=(-0.4, -0.4), hi=(1.4, 1.4), wrap=False)
    else:
        d = rng.normal(size=3)
        eye = np.array([0.5, 0.5, 0.5]) + 2.2 * d / np.linalg.norm(d)
        target = np.array([0.5, 0.5, 0.5]) + rng.uniform(-0.1, 0.1, 3)
        up = (0, 0, 1) if abs((target - eye)[2]) < 0.9 * np.linalg.norm(target - eye) else (0, 1, 0)
        cam = camera_dict("persp", 19, 16, eye=eye, fwd=target - eye, up=up, fov_y_deg=50.0)
    a = oracle.render(pos, N, cam)
    b = bf.render_barycentric(pos, N, cam)
    assert a.max() > 0
    np.testing.assert_allclose(a, b, atol=1e-11 * a.max())


@pytest.mark.parametrize("view", ["ortho_wrap", "persp"])
def test_render_crops_equal_slices_of_the_full_frame(view):
    """Several offset crops in one call (including ones that touch the frame
    edges and overlap each other) equal the same slices of the full-frame
    render: pins the crop offsets and the per-crop output layout that the
    sampled parity tests and the benchmark's CPU leg rely on."""
    N = 8
    pos = ZeldovichField.generate(N, -2.0, 3.0, 77).positions(1.7)
    if view == "ortho_wrap":
        cam = camera_dict("ortho", 61, 47, fwd=(0.2, -0.1, 1.0), up=(0, 1, 0), lo=(0.05, -0.1), hi=(1.05, 0.9),
                          wrap=True)
    else:
        cam = camera_dict("persp", 58, 64, eye=(0.5, -1.3, 0.9), fwd=(0.0, 1.8, -0.4), up=(0, 0, 1), fov_y_deg=55)
    full, nf_full, _ = oracle.render(pos, N, cam, return_counts=True)
    crops = [(0, 0, 61 if view == "ortho_wrap" else 58, 1), (3, 5, 17, 9), (40, 30, 18, 17), (10, 8, 21, 23),
             (0, 20, 7, 27), (33, 0, 1, 1)]
    imgs, nf, _ = oracle.render_crops(pos, N, cam, crops)
    assert len(imgs) == len(crops)
    for (x, y, w, h), got in zip(crops, imgs):
        assert got.shape == (h, w)
        np.testing.assert_array_equal(got, full[y:y + h, x:x + w])
    # fragments are counted per crop: the batched count is the sum of the
    # crops' own counts (overlapping crops count their shared pixels twice)
    assert nf == sum(oracle.render_crops(pos, N, cam, [c])[1] for c in crops)
    assert 0 < nf
    single, nf_one, _ = oracle.render_crops(pos, N, cam, [(0, 0, cam["W"], cam["H"])])
    np.testing.assert_array_equal(single[0], full)
    assert nf_one == nf_full


def test_centroid_kernel_has_unit_integral():
    """The 2D M4 cubic spline of the centroid splats integrates to 1 over the
    plane: one tetrahedron's splat carries its mass (midpoint rule on a fine
    polar grid, independent of the oracle)."""
    h = 0.37
    r = (np.arange(20000) + 0.5) * (2.0 * h / 20000)
    q = r / h
    w = np.where(q < 1.0, 1.0 - 1.5 * q ** 2 + 0.75 * q ** 3, 0.25 * (2.0 - q) ** 3)
    integral = float(np.sum(10.0 / (7.0 * math.pi * h * h) * w * 2.0 * math.pi * r) * (2.0 * h / 20000))
    assert abs(integral - 1.0) <= 1e-8


@pytest.mark.parametrize("N,W,lam,seed", [(1, 24, 0.0, 0), (2, 20, 0.6, 3), (3, 17, 1.1, 8)])
def test_centroids_match_bruteforce(N, W, lam, seed):
    """The oracle's splats against an independent numpy evaluation of every
    (pixel, tetrahedron, period) triple on tiny lattices, including the
    undeformed unit cube (N = 1) and a ragged window."""
    rng = np.random.default_rng(seed)
    # tiny lattices have no Zel'dovich modes below Nyquist: seeded random
    # displacements of up to lam / 3 of a cell instead
    pos = lattice_positions(N) if lam == 0.0 else lattice_positions(
        N, disp=lambda q: rng.uniform(-lam / 3, lam / 3, q.shape) / N)
    cam = ortho_z(W, W + 3)
    ref = bf.centroids_bruteforce(pos, N, W, W + 3)
    got = oracle.centroids(pos, N, cam)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_centroid_frame_mass_converges_to_total_mass():
    """Over the periodic box window the splats carry the whole mass: the
    pixel-centre sum times the pixel area tends to 1 as the pixels shrink
    relative to the splats."""
    N = 4
    pos = ZeldovichField.generate(N, -2.0, 2.0, 11).positions(0.8)
    errs = []
    for W in (16, 32, 64):
        img = oracle.centroids(pos, N, ortho_z(W, W))
        errs.append(abs(img.sum() / (W * W) - 1.0))
    assert errs[2] <= 1e-4
    assert errs[2] < errs[0]


def test_centroids_shift_with_the_particles():
    """Moving every particle by exactly one pixel along x moves the periodic
    image by one pixel."""
    N, W = 4, 32
    pos = ZeldovichField.generate(N, -2.0, 2.0, 12).positions(0.9).astype(np.float64)
    cam = ortho_z(W, W)
    a = oracle.centroids(pos, N, cam)
    moved = pos.copy()
    moved[:, 0] = np.mod(moved[:, 0] + 1.0 / W, 1.0)
    b = oracle.centroids(moved, N, cam)
    np.testing.assert_allclose(np.roll(a, 1, axis=1), b, rtol=1e-9, atol=1e-9)


def test_perspective_centroids_match_bruteforce():
    """Perspective splats against an independent numpy evaluation over every
    (pixel, tetrahedron) pair."""
    N = 3
    rng = np.random.default_rng(21)
    pos = lattice_positions(N, disp=lambda q: rng.uniform(-0.3, 0.3, q.shape) / N)
    cam = camera_dict("persp", 40, 34, eye=(0.4, -1.1, 0.7), fwd=(0.1, 1.5, -0.3), up=(0, 0, 1), fov_y_deg=50)
    verts, _, _ = bf.lattice_tets(pos, N)
    ref = bf.splats_perspective_bruteforce(verts, 40, 34, cam["eye"], cam["fwd"], cam["up"], 50.0, 1.0, N)
    got = oracle.centroids(pos, N, cam)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_hybrid_limits_and_split():
    """Hybrid near/far rendering: r_near beyond every cube is the exact
    projection, r_near = 0 the splats; in between, the near cubes' exact
    chords (through the tetrahedron-soup projection) plus the far cubes'
    splats (numpy), with near decided by the cube's corner-0 particle."""
    N = 4
    rng = np.random.default_rng(22)
    pos = lattice_positions(N, disp=lambda q: rng.uniform(-0.3, 0.3, q.shape) / N)
    cam = camera_dict("persp", 36, 30, eye=(0.5, -0.9, 0.55), fwd=(0.0, 1.0, 0.0), up=(0, 0, 1), fov_y_deg=55)
    np.testing.assert_array_equal(oracle.hybrid(pos, N, cam, 1e30), oracle.render(pos, N, cam))
    np.testing.assert_array_equal(oracle.hybrid(pos, N, cam, 0.0), oracle.centroids(pos, N, cam))
    r_near = 1.4
    verts, rho, _ = bf.lattice_tets(pos, N)
    p = np.asarray(pos, dtype=np.float64)[:, :3]
    idx = np.arange(N ** 3)
    q = np.stack([idx % N, (idx // N) % N, idx // (N * N)], axis=1) / N
    d = p - q
    d -= np.round(d)
    near_cube = np.linalg.norm(q + d - np.asarray(cam["eye"]), axis=1) < r_near
    near = np.repeat(near_cube, 6)
    assert 0 < near.sum() < near.size
    ref = oracle.render_soup(verts[near], rho[near], cam) + bf.splats_perspective_bruteforce(
        verts[~near], 36, 30, cam["eye"], cam["fwd"], cam["up"], 55.0, 1.0, N)
    np.testing.assert_allclose(oracle.hybrid(pos, N, cam, r_near), ref, rtol=1e-10, atol=1e-12)


def test_perspective_splats_keep_the_projected_mass():
    """A perspective splat carries m |dir| / Z^2 over the image plane (at unit
    distance), like the exact projection of the same tetrahedron to leading
    order in its size over its distance: the frame masses agree to about
    (h / Z)^2."""
    N = 8
    pos = ZeldovichField.generate(N, -2.0, 3.0, 23).positions(1.0)
    cam = camera_dict("persp", 96, 96, eye=(0.5, -2.0, 0.5), fwd=(0, 1, 0), up=(0, 0, 1), fov_y_deg=40)
    exact = oracle.render(pos, N, cam).sum()
    splat = oracle.centroids(pos, N, cam).sum()
    assert abs(splat / exact - 1.0) <= 3e-3


@pytest.mark.parametrize("N,W,H,lam,seed,oblique", [(2, 9, 7, 0.6, 3, False), (2, 11, 8, 0.9, 4, True),
                                                    (3, 7, 10, 1.1, 8, False)])
def test_area_pixels_match_polytope_volumes(N, W, H, lam, seed, oblique):
    """Area-averaged pixels against an independent formulation: rho times
    the volume of each tetrahedron clipped to the prism over each pixel's
    square (plane-triple vertices and a convex hull), for periodic and
    oblique windows on tiny randomly displaced lattices."""
    pytest.importorskip("scipy")
    rng = np.random.default_rng(seed)
    pos = lattice_positions(N, disp=lambda q: rng.uniform(-lam / 3, lam / 3, q.shape) / N)
    cam = (camera_dict("ortho", W, H, fwd=(0.3, -0.2, 1.0), up=(0, 1, 0), lo=(-0.2, 0.1), hi=(0.9, 1.2))
           if oblique else ortho_z(W, H))
    ref = bf.area_bruteforce(pos, N, cam)
    got = oracle.render_area(pos, N, cam)
    np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-10)


def test_area_pixels_of_the_undeformed_lattice_are_uniform():
    """Viewed along a lattice axis through the periodic box, the undeformed
    lattice (and any uniform translation of it) has column density equal to
    the mean everywhere: every area-averaged pixel is 1, whatever the pixel
    grid (here incommensurate with the lattice)."""
    N = 4
    for shift in (0.0, 0.0371):
        pos = lattice_positions(N, disp=lambda q: np.full(q.shape, shift), dtype=np.float64)
        img = oracle.render_area(pos, N, ortho_z(13, 9))
        np.testing.assert_allclose(img, 1.0, rtol=0, atol=1e-12)


def test_area_frame_mass_is_the_total_mass():
    """Over the periodic box window the area-averaged pixels hold the whole
    mass to rounding (each tetrahedron is integrated exactly), unlike
    pixel-centre sampling."""
    N, W = 8, 40
    pos = ZeldovichField.generate(N, -2.0, 3.0, 5).positions(1.2)
    img = oracle.render_area(pos, N, ortho_z(W, W + 7))
    assert abs(img.sum() / (W * (W + 7)) - 1.0) <= 1e-12
    assert img.min() > 0.0


def test_supersampled_pixel_centres_converge_to_the_area_mean():
    """Averaging pixel-centre samples over f x f sub-pixels converges to the
    area mean as f grows (second order away from the kinks of the chord
    function)."""
    N, W = 8, 32
    pos = ZeldovichField.generate(N, -2.0, 3.0, 5).positions(1.2)
    area = oracle.render_area(pos, N, ortho_z(W, W))
    errs = []
    for f in (8, 16, 32):
        s = oracle.render(pos, N, ortho_z(W * f, W * f)).reshape(W, f, W, f).mean(axis=(1, 3))
        errs.append(float(np.abs(s - area).max() / area.mean()))
    assert errs[2] <= 5e-3
    assert errs[2] < 0.5 * errs[1] < 0.5 * errs[0]


def test_render_over_the_cubes_near_a_pixel_equals_the_full_render():
    """The oracle's render restricted to the cubes that can reach some pixels
    (the offset bound of tests/near_cubes.py) equals the full render there,
    also for rays moved by a small fraction of a pixel; a subset that misses
    the reaching cubes does not."""
    from near_cubes import cubes_near_pixels
    N, W = 32, 128
    pos = ZeldovichField.generate(N, -2.0, 16.0, 321).positions(1.5)
    cam = ortho_z(W, W)
    full = oracle.render(pos, N, cam)
    picks = [(5, 7), (70, 61), (127, 0)]
    sel = cubes_near_pixels(pos, N, W, W, picks)
    assert 0 < len(sel) < N ** 3
    one = [(x, y, 1, 1) for x, y in picks]
    got = [r[0, 0] for r in oracle.render_crops(pos, N, cam, one, cubes=sel)[0]]
    np.testing.assert_array_equal(got, [full[y, x] for x, y in picks])
    eps = 1e-4 / W
    shifted = dict(cam, lo=(eps, -eps), hi=(1.0 + eps, 1.0 - eps))
    a = [r[0, 0] for r in oracle.render_crops(pos, N, shifted, one, cubes=sel)[0]]
    b = [r[0, 0] for r in oracle.render_crops(pos, N, shifted, one)[0]]
    np.testing.assert_array_equal(a, b)
    far = np.setdiff1d(np.arange(N ** 3), sel)
    assert all(r[0, 0] == 0.0 for r in oracle.render_crops(pos, N, cam, one, cubes=far)[0])
