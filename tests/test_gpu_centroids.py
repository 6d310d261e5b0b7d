"""GPU parity of the centroid splats (lt_render_centroids, Sec. 4.2) and of
the hybrid near/far rendering (lt_render_hybrid, Sec. 6) against the FP64
oracle (oracle.centroids, oracle.hybrid) on the same seeded inputs: every
pixel within 1e-4 of max(pixel, mean column density), the frame mass within
1e-6.
The GPU forms each splat's centroid and scale in FP64 and evaluates the
spline in FP32 relative to the centroid's pixel, so its error is a few
1e-7 per splat plus the 64-bit fixed-point rounding."""
import numpy as np
import pytest

import oracle
from lt_inputs import ZeldovichField, camera_dict, config, ortho_z, sphere_cameras

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


def pixel_error(got, ref):
    nz = ref[ref > 0]
    mean = nz.mean() if nz.size else 1.0
    return float((np.abs(got.astype(np.float64) - ref) / np.maximum(np.abs(ref), mean)).max())


@pytest.mark.parametrize("N,W,H,lam,seed", [(16, 128, 128, 2.0, 31), (32, 256, 200, 1.5, 1001), (8, 61, 47, 1.2, 5)])
def test_centroids_match_oracle_periodic_window(R, N, W, H, lam, seed):
    pos = ZeldovichField.generate(N, -2.0, max(3.0, N / 2.0), seed).positions(lam)
    cam = ortho_z(W, H)
    ref = oracle.centroids(pos, N, cam)
    R.build_tets(torch.from_numpy(pos).cuda(), N)
    got = R.render_centroids(cam).cpu().numpy()
    R.sync()
    assert pixel_error(got, ref) <= PIX_TOL
    area = 1.0 / (W * H)
    assert abs(got.astype(np.float64).sum() * area - ref.sum() * area) <= MASS_TOL * ref.sum() * area


def test_centroids_oblique_window_and_reproducible(R):
    N = 16
    pos = ZeldovichField.generate(N, -2.0, 6.0, 44).positions(1.7)
    cam = camera_dict("ortho", 97, 81, fwd=(0.3, -0.2, 1.0), up=(0, 1, 0), lo=(-0.2, 0.1), hi=(0.9, 1.2))
    ref = oracle.centroids(pos, N, cam)
    R.build_tets(torch.from_numpy(pos).cuda(), N)
    a = R.render_centroids(cam).clone()
    b = R.render_centroids(cam)
    R.sync()
    assert torch.equal(a, b)
    assert pixel_error(a.cpu().numpy(), ref) <= PIX_TOL


def test_centroids_128_lattice_at_1024(R):
    c = config("zel128_ortho1024")
    N = c["N"]
    pos = ZeldovichField.generate(N, c["n_index"], c["k_cut"], c["seed"]).positions(c["lams"][0])
    cam = ortho_z(c["W"], c["H"])
    R.build_tets(torch.from_numpy(pos).cuda(), N)
    got = R.render_centroids(cam).cpu().numpy()
    R.sync()
    ref = oracle.centroids(pos, N, cam)
    assert pixel_error(got, ref) <= PIX_TOL
    area = 1.0 / (c["W"] * c["H"])
    assert abs(got.astype(np.float64).sum() * area - ref.sum() * area) <= MASS_TOL * ref.sum() * area


def test_near_radius_needs_a_perspective_view(R):
    from paper_1208_3206_gb300._lib import LtError
    from paper_1208_3206_gb300.render import Camera
    N = 8
    pos = ZeldovichField.generate(N, -2.0, 3.0, 9).positions(1.0)
    R.build_tets(torch.from_numpy(pos).cuda(), N)
    with pytest.raises(LtError) as e:
        R.render_centroids(Camera(**ortho_z(32, 32), near_radius=1.0))
    assert e.value.name == "LT_ERR_ARG"
    with pytest.raises(LtError) as e:
        R.render_hybrid(ortho_z(32, 32), 1.0)
    assert e.value.name == "LT_ERR_ARG"
    R.sync()


@pytest.mark.parametrize("N,W,lam,seed", [(16, 128, 2.0, 31), (32, 200, 1.5, 1001)])
def test_perspective_centroids_match_oracle(R, N, W, lam, seed):
    pos = ZeldovichField.generate(N, -2.0, max(3.0, N / 2.0), seed).positions(lam)
    for cam in sphere_cameras(3, W, W - 24)[:2]:
        ref = oracle.centroids(pos, N, cam)
        R.build_tets(torch.from_numpy(pos).cuda(), N)
        got = R.render_centroids(cam).cpu().numpy()
        R.sync()
        assert pixel_error(got, ref) <= PIX_TOL
        assert abs(got.astype(np.float64).sum() - ref.sum()) <= MASS_TOL * ref.sum()


@pytest.mark.parametrize("r_near", [1.6, 2.0, 2.4])
def test_hybrid_matches_oracle(R, r_near):
    """Hybrid near/far rendering (cubes within r_near of the eye by exact
    projection, the others as splats) against the oracle's, for spheres
    that split the box near, through and past its centre (cameras at
    distance 2 from it)."""
    N, W = 32, 160
    pos = ZeldovichField.generate(N, -2.0, 16.0, 1003).positions(2.0)
    cam = sphere_cameras(4, W, 128)[1]
    ref = oracle.hybrid(pos, N, cam, r_near)
    R.build_tets(torch.from_numpy(pos).cuda(), N)
    got = R.render_hybrid(cam, r_near).cpu().numpy()
    R.sync()
    assert pixel_error(got, ref) <= PIX_TOL
    assert abs(got.astype(np.float64).sum() - ref.sum()) <= MASS_TOL * ref.sum()


def test_near_radius_splits_the_exact_raster(R):
    """With a near radius the exact raster draws only the near cubes, and
    the centroid renderer only the far ones: near exact + far splats is the
    hybrid image; a radius beyond the whole box gives the plain render."""
    from paper_1208_3206_gb300.render import Camera
    N, W = 16, 96
    pos = ZeldovichField.generate(N, -2.0, 6.0, 61).positions(1.8)
    cam = dict(sphere_cameras(3, W, W)[2])
    R.build_tets(torch.from_numpy(pos).cuda(), N)
    R.project_bin([Camera(**cam, near_radius=100.0)])
    full_far = R.render_tiles()[0].clone()
    R.project_bin([Camera(**cam)])
    plain = R.render_tiles()[0].clone()
    R.project_bin([Camera(**cam, near_radius=2.0)])
    near = R.render_tiles()[0].clone()
    far = R.render_centroids(Camera(**cam, near_radius=2.0))
    hyb = R.render_hybrid(cam, 2.0)
    R.sync()
    assert torch.equal(full_far, plain)
    assert float((hyb - (near + far)).abs().max()) <= 1e-6 * float(hyb.max())
    ref = oracle.hybrid(pos, N, cam, 2.0)
    assert pixel_error(hyb.cpu().numpy(), ref) <= PIX_TOL
