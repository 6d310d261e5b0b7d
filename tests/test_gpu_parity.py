"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.

Tolerance (from the stated target): every pixel within 1e-4 of
max(pixel value, mean column density), the frame mass within 1e-6
(relative), and fragment counts within 1e-4 (relative; pixels whose centre
falls on a tetrahedron boundary to rounding may be counted on one side only).
"""
import math

import numpy as np
import pytest

import oracle
from lt_inputs import (ZeldovichField, camera_dict, config, decode_fp16_offsets, fp16_offsets, ortho_z,
                       sphere_cameras)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PIX_TOL = 1e-4
MASS_TOL = 1e-6


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1208_3206_gb300.render import Renderer
    return Renderer()


def pixel_error(img, ref, mean_cd=None):
    if mean_cd is None:
        nz = ref[ref > 0]
        mean_cd = nz.mean() if nz.size else 1.0
    return float((np.abs(img.astype(np.float64) - ref) / np.maximum(np.abs(ref), mean_cd)).max())


_FIELDS = {}


def field(N, n_index, k_cut, seed):
    key = (N, n_index, k_cut, seed)
    if key not in _FIELDS:
        _FIELDS[key] = ZeldovichField.generate(N, n_index, k_cut, seed)
    return _FIELDS[key]


def gpu_render(R, pos, N, cams, snaps=None, box=1.0, mass=1.0, atomic=False):
    p = torch.from_numpy(np.ascontiguousarray(pos)).cuda()
    R.build_tets(p, N, box, mass)
    if atomic:
        img = R.render_atomic(cams, snaps)
        m = None
    else:
        R.project_bin(cams, snaps)
        img, m = R.render_tiles(with_mass=True)
    R.sync()
    return img.cpu().numpy(), (None if m is None else m.cpu().numpy())


# ---------------------------------------------------------------------------


def test_small_ortho_config_matches_oracle(R):
    c = config("zel32_ortho256")
    f = field(c["N"], c["n_index"], c["k_cut"], c["seed"])
    pos = f.positions(c["lams"][0])
    cam = ortho_z(c["W"], c["H"])
    ref, nf_ref, _ = oracle.render(pos, c["N"], cam, return_counts=True)
    img, m = gpu_render(R, pos, c["N"], [cam])
    assert pixel_error(img[0], ref, 1.0) <= PIX_TOL
    assert abs(m[0] - oracle.frame_mass(ref, cam)) <= MASS_TOL * oracle.frame_mass(ref, cam)
    nf = R.count_fragments()[0]
    assert abs(nf - nf_ref) <= 1e-4 * nf_ref


def test_atomic_form_matches_oracle(R):
    c = config("zel32_ortho256")
    f = field(c["N"], c["n_index"], c["k_cut"], c["seed"])
    pos = f.positions(c["lams"][0])
    cam = ortho_z(c["W"], c["H"])
    ref = oracle.render(pos, c["N"], cam)
    img, _ = gpu_render(R, pos, c["N"], [cam], atomic=True)
    assert pixel_error(img[0], ref, 1.0) <= PIX_TOL


def test_bitwise_reproducible_across_runs_and_tiles(R):
    """Fixed-point accumulation makes every run of one configuration bitwise
    identical. Other tile sizes place the vertices relative to other tile
    origins (FP32 round-off of the last bits), so they agree to round-off."""
    f = field(32, -2.0, 16.0, 1001)
    pos = f.positions(2.5)
    cam = ortho_z(200, 184)
    for tile in (16, 32, 8):
        R.set_config(tile=tile)
        runs = [gpu_render(R, pos, 32, [cam])[0] for _ in range(3)]
        assert np.array_equal(runs[0], runs[1]) and np.array_equal(runs[0], runs[2])
        if tile == 16:
            base = runs[0]
        else:
            assert np.abs(runs[0] - base).max() <= 1e-5 * max(1.0, float(base.max()))
    R.set_config(tile=16)


def test_perspective_matches_oracle(R):
    N = 32
    f = field(N, -2.0, 16.0, 1003)
    cams = sphere_cameras(4, 160, 128)
    pos = np.concatenate([f.positions(1.0), f.positions(3.0)])
    snaps = [0, 1, 1, 0]
    img, m = gpu_render(R, pos, N, cams, snaps)
    for k, cam in enumerate(cams):
        ref = oracle.render(pos[snaps[k] * N ** 3:(snaps[k] + 1) * N ** 3], N, cam)
        assert pixel_error(img[k], ref) <= PIX_TOL, k
        # perspective frame mass: sum of pixels times the unit-distance pixel area
        ty = math.tan(math.radians(cam["fov_y_deg"]) / 2)
        tx = ty * cam["W"] / cam["H"]
        area = (2 * tx / cam["W"]) * (2 * ty / cam["H"])
        want = float(img[k].astype(np.float64).sum() * area)
        assert abs(m[k] - want) <= 1e-12 * abs(want)
        assert abs(m[k] - ref.sum() * area) <= MASS_TOL * ref.sum() * area


def test_perspective_atomic_matches_oracle(R):
    N = 16
    f = field(N, -2.0, 6.0, 77)
    cam = sphere_cameras(5, 96, 80)[2]
    pos = f.positions(2.0)
    ref = oracle.render(pos, N, cam)
    img, _ = gpu_render(R, pos, N, [cam], atomic=True)
    assert pixel_error(img[0], ref) <= PIX_TOL


def test_ragged_and_offset_windows(R):
    N = 16
    f = field(N, -2.0, 6.0, 5)
    pos = f.positions(2.2)
    cams = [
        camera_dict("ortho", 133, 71, fwd=(0, 0, 1), up=(0, 1, 0), lo=(0.1, -0.2), hi=(1.1, 0.8), wrap=True),
    ]
    ref = oracle.render(pos, N, cams[0])
    img, _ = gpu_render(R, pos, N, cams)
    assert pixel_error(img[0], ref, 1.0) <= PIX_TOL
    # non-periodic oblique window partially covering the box
    cam = camera_dict("ortho", 97, 113, fwd=(0.3, -0.4, 1.0), up=(0, 1, 0), lo=(-0.3, 0.2), hi=(0.9, 1.5))
    ref = oracle.render(pos, N, cam)
    img, _ = gpu_render(R, pos, N, [cam])
    assert pixel_error(img[0], ref, 1.0) <= PIX_TOL


def test_unperturbed_lattice_is_exactly_uniform(R):
    """Degenerate projections (vertical tetrahedron edges) everywhere."""
    N = 8
    idx = np.arange(N ** 3)
    pos = np.zeros((N ** 3, 4), np.float32)
    pos[:, 0], pos[:, 1], pos[:, 2] = idx % N, (idx // N) % N, idx // (N * N)
    pos[:, :3] /= N
    cam = camera_dict("ortho", 61, 53, fwd=(0, 0, 1), up=(0, 1, 0), lo=(0.0123, 0.0457), hi=(1.0123, 1.0457),
                      wrap=True)
    img, m = gpu_render(R, pos, N, [cam])
    assert np.abs(img[0] - 1.0).max() <= 1e-5
    assert abs(m[0] - 1.0) <= 1e-6


def test_tiny_lattices_and_images(R):
    rng = np.random.default_rng(8)
    for N, W, H in ((1, 7, 5), (2, 16, 16), (3, 1, 1), (4, 33, 17)):
        # random displacements of up to a third of a cell (the tiny lattices
        # have no Zel'dovich modes below Nyquist)
        idx = np.arange(N ** 3)
        q = np.stack([idx % N, (idx // N) % N, idx // (N * N)], axis=1) / N
        pos = np.zeros((N ** 3, 4), np.float32)
        pos[:, :3] = np.mod(q + rng.uniform(-0.33, 0.33, q.shape) / N, 1.0)
        cam = camera_dict("ortho", W, H, fwd=(0, 0, 1), up=(0, 1, 0), lo=(0.011, 0.023), hi=(1.011, 1.023),
                          wrap=True)
        ref = oracle.render(pos, N, cam)
        img, _ = gpu_render(R, pos, N, [cam])
        assert pixel_error(img[0], ref, 1.0) <= PIX_TOL, (N, W, H)


def test_camera_looking_away_gives_empty_frame(R):
    N = 8
    f = field(N, -2.0, 3.0, 9)
    pos = f.positions(1.0)
    cam = camera_dict("persp", 64, 64, eye=(0.5, 0.5, 3.0), fwd=(0, 0, 1), up=(0, 1, 0), fov_y_deg=40)
    img, m = gpu_render(R, pos, N, [cam])
    assert np.all(img == 0) and m[0] == 0.0


def test_fp16_offsets_match_oracle_on_decoded_positions(R):
    N = 32
    f = field(N, -2.5, 12.0, 1004)
    off = fp16_offsets(f.displacement(4.0), N)
    dec = decode_fp16_offsets(off, N)
    cam = ortho_z(256, 256)
    ref = oracle.render(dec, N, cam)
    img, _ = gpu_render(R, off, N, [cam])
    assert pixel_error(img[0], ref, 1.0) <= PIX_TOL


def test_graph_replay_equals_direct_render(R):
    N = 16
    f = field(N, -2.0, 6.0, 21)
    pos = torch.from_numpy(np.concatenate([f.positions(1.0), f.positions(2.0)])).cuda()
    cams = sphere_cameras(3, 96, 96) + [ortho_z(96, 96)]
    snaps = [0, 1, 0, 1]
    R.build_tets(pos, N)
    R.project_bin(cams, snaps)
    direct = R.render_tiles().clone()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        img = R.graph_build(cams, snaps)
        R.graph_launch()
        R.graph_launch()
        R.sync()
    torch.cuda.synchronize()
    assert torch.equal(img, direct)
    # building the graph grows the bin list for headroom; the direct bins of
    # the same frames must survive that
    again = R.render_tiles()
    R.sync()
    assert torch.equal(again, direct)


def test_error_paths(R):
    from paper_1208_3206_gb300._lib import LtError
    N = 8
    f = field(N, -2.0, 3.0, 9)
    pos = f.positions(1.0)
    bad = pos.copy()
    bad[17, 1] = np.nan
    p = torch.from_numpy(bad).cuda()
    R.build_tets(p, N)
    with pytest.raises(LtError) as e:
        R.sync()
    assert e.value.name == "LT_ERR_NONFINITE"
    # a vertex behind the perspective eye
    R.build_tets(torch.from_numpy(pos).cuda(), N)
    R.sync()
    cam = camera_dict("persp", 32, 32, eye=(0.5, 0.5, 0.5), fwd=(0, 0, 1), up=(0, 1, 0), fov_y_deg=60)
    R.project_bin([cam])
    with pytest.raises(LtError) as e:
        R.sync()
    assert e.value.name == "LT_ERR_BEHIND_EYE"
    # argument errors
    with pytest.raises(LtError):
        R.project_bin([camera_dict("ortho", 0, 8)])
    with pytest.raises(LtError):
        R.project_bin([ortho_z(8, 8)], frame_snapshot=[3])
    R.sync()


def test_build_tets_volumes_and_densities(R):
    N = 16
    f = field(N, -2.0, 6.0, 3)
    pos = f.positions(3.0)
    vol, rho = oracle.tet_volumes(pos, N)
    out = torch.empty(6 * N ** 3, dtype=torch.float32, device="cuda")
    R.build_tets(torch.from_numpy(pos).cuda(), N, rho_out=out)
    st = R.get_stats()
    got = out.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(got, rho, rtol=2e-4)
    assert st["inverted"] == int((vol > 0).sum())
    assert st["degenerate"] == int((vol == 0).sum())


@pytest.mark.parametrize("name", ["zel128_ortho1024"])
def test_mid_config_full_frame(R, name):
    c = config(name)
    f = field(c["N"], c["n_index"], c["k_cut"], c["seed"])
    pos = f.positions(c["lams"][0])
    cam = ortho_z(c["W"], c["H"])
    ref, nf_ref, _ = oracle.render(pos, c["N"], cam, return_counts=True)
    img, m = gpu_render(R, pos, c["N"], [cam])
    assert pixel_error(img[0], ref, 1.0) <= PIX_TOL
    mass_ref = oracle.frame_mass(ref, cam)
    assert abs(m[0] - mass_ref) <= MASS_TOL * mass_ref
    nf = R.count_fragments()[0]
    assert abs(nf - nf_ref) <= 1e-4 * nf_ref
    img_a, _ = gpu_render(R, pos, c["N"], [cam], atomic=True)
    assert pixel_error(img_a[0], ref, 1.0) <= PIX_TOL


def test_graph_replay_reports_bin_capacity_overflow():
    """A graph's bin lists are sized when it is built. Replaying it after the
    positions changed to a lattice that needs more list entries latches
    LT_ERR_CAPACITY: the scatter checks every write against the capacity and
    the raster reads only what the lists hold. (A fresh context, so that the
    lists are sized by this graph alone.)"""
    from paper_1208_3206_gb300._lib import LtError
    from paper_1208_3206_gb300.render import Renderer
    R = Renderer()
    N = 16
    f = field(N, -2.0, 6.0, 31)
    calm = torch.from_numpy(f.positions(0.05)).cuda()
    wild = torch.from_numpy(f.positions(4.0)).cuda()
    cams = [ortho_z(256, 256)]
    R.set_config(tile=8)
    pos = calm.clone()
    R.build_tets(pos, N)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        R.graph_build(cams)
        R.graph_launch()
        R.sync()
        need_calm = R.get_stats()["entries"]
        pos.copy_(wild)
        R.graph_launch()
        with pytest.raises(LtError) as e:
            R.sync()
    torch.cuda.synchronize()
    assert e.value.name == "LT_ERR_CAPACITY"
    # the same lattice binned directly fits (the pass sizes its lists)
    R.build_tets(wild, N)
    R.project_bin(cams)
    R.render_tiles()
    R.sync()
    assert R.get_stats()["entries"] > need_calm


def test_accumulator_range_overflow_is_reported():
    """Each pixel is summed in a 64-bit integer holding values below
    2^(64 - frac_bits) mean column densities. With frac_bits = 62 (4 sigma)
    the caustics of this frame (up to about 9 sigma) pass the range, and the
    add that wraps a pixel's sum latches LT_ERR_RANGE; with frac_bits = 59
    (32 sigma) the same frame fits and matches the oracle."""
    from paper_1208_3206_gb300._lib import LtError
    from paper_1208_3206_gb300.render import Renderer
    N, W = 32, 256
    pos = field(N, -2.0, 16.0, 1001).positions(4.0)
    cam = ortho_z(W, W)
    ref = oracle.render(pos, N, cam)
    assert 4.0 < ref.max() < 32.0
    R = Renderer(frac_bits=62)
    R.build_tets(torch.from_numpy(pos).cuda(), N)
    R.project_bin([cam])
    R.render_tiles()
    with pytest.raises(LtError) as e:
        R.sync()
    assert e.value.name == "LT_ERR_RANGE"
    assert R.get_stats()["range_overflow"] > 0
    R.set_config(frac_bits=59)
    R.project_bin([cam])
    img = R.render_tiles()
    R.sync()
    assert pixel_error(img[0].cpu().numpy(), ref, 1.0) <= PIX_TOL


def test_graph_keeps_its_frames_and_goes_stale_when_buffers_move():
    """A graph keeps its own copy of its views: a direct lt_project_bin with
    other cameras between replays does not change what the graph renders. A
    direct call that has to reallocate a buffer the graph captured (here:
    ten times the tiles), and a new lt_build_tets, make the graph stale, and
    lt_graph_launch refuses with LT_ERR_STATE until it is built again."""
    from paper_1208_3206_gb300._lib import LtError
    from paper_1208_3206_gb300.render import Renderer
    R = Renderer(tile=16)
    N = 16
    f = field(N, -2.0, 6.0, 21)
    pos = torch.from_numpy(np.concatenate([f.positions(1.0), f.positions(2.0)])).cuda()
    cams = sphere_cameras(2, 64, 64)
    R.build_tets(pos, N)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        img = R.graph_build(cams, [0, 1])
        R.graph_launch()
        R.sync()
        first = img.clone()
        # other views of the same size, binned directly: the graph's views stay
        R.project_bin(sphere_cameras(5, 64, 64)[3:5], [1, 0])
        R.render_tiles()
        R.graph_launch()
        R.sync()
        assert torch.equal(img, first)
        # many more tiles: the direct call reallocates the bins
        R.project_bin([ortho_z(640, 640)] * 4)
        with pytest.raises(LtError) as e:
            R.graph_launch()
        assert e.value.name == "LT_ERR_STATE"
        R.graph_build(cams, [0, 1], image=img)
        R.graph_launch()
        R.sync()
        assert torch.equal(img, first)
        R.build_tets(pos, N)
        with pytest.raises(LtError) as e:
            R.graph_launch()
        assert e.value.name == "LT_ERR_STATE"
    torch.cuda.synchronize()
