"""GPU parity of the area-averaged pixels (lt_render_area) against the FP64
oracle (oracle.render_area) on the same seeded inputs: every pixel within
1e-4 of max(pixel, mean column density), the frame mass within 1e-6.
The GPU sets up each tetrahedron's pyramid in FP64 and evaluates each line
at the pixel's corner in float-float; the clip runs in FP32 (FP64 for hulls
thinner than 1/20 pixel), so its error is a few 1e-7 of the largest column
density in the pixel plus the 64-bit fixed-point rounding."""
import numpy as np
import pytest

import oracle
from lt_inputs import ZeldovichField, camera_dict, config, ortho_z

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


@pytest.mark.parametrize("N,W,H,lam,seed", [(16, 128, 128, 2.0, 31), (32, 256, 200, 1.5, 1001), (8, 61, 47, 1.2, 5),
                                            (32, 96, 96, 3.0, 77)])
def test_area_matches_oracle_periodic_window(R, N, W, H, lam, seed):
    pos = ZeldovichField.generate(N, -2.0, max(3.0, N / 2.0), seed).positions(lam)
    cam = ortho_z(W, H)
    ref = oracle.render_area(pos, N, cam)
    R.build_tets(torch.from_numpy(pos).cuda(), N)
    got = R.render_area(cam).cpu().numpy()
    R.sync()
    assert pixel_error(got, ref) <= PIX_TOL
    # the periodic window holds the whole mass
    assert abs(got.astype(np.float64).sum() / (W * H) - 1.0) <= MASS_TOL
    assert R.get_stats()["area_pairs"] > 0


def test_area_oblique_window_and_reproducible(R):
    N = 16
    pos = ZeldovichField.generate(N, -2.0, 6.0, 44).positions(1.7)
    cam = camera_dict("ortho", 97, 81, fwd=(0.3, -0.2, 1.0), up=(0, 1, 0), lo=(-0.2, 0.1), hi=(0.9, 1.2))
    ref = oracle.render_area(pos, N, cam)
    R.build_tets(torch.from_numpy(pos).cuda(), N)
    a = R.render_area(cam).clone()
    b = R.render_area(cam)
    R.sync()
    assert torch.equal(a, b)
    assert pixel_error(a.cpu().numpy(), ref) <= PIX_TOL
    assert abs(a.double().sum().item() - ref.sum()) <= MASS_TOL * ref.sum()


def test_area_undeformed_lattice_is_uniform(R):
    """Seen along a lattice axis the undeformed lattice projects with
    coincident vertices (the apex on the hull boundary): every area-averaged
    pixel is the mean column density 1."""
    N, W, H = 16, 53, 40
    idx = np.arange(N ** 3)
    pos = np.zeros((N ** 3, 4), dtype=np.float32)
    pos[:, 0], pos[:, 1], pos[:, 2] = idx % N, (idx // N) % N, idx // (N * N)
    pos[:, :3] /= N
    R.build_tets(torch.from_numpy(pos).cuda(), N)
    got = R.render_area(ortho_z(W, H)).cpu().numpy()
    R.sync()
    assert float(np.abs(got.astype(np.float64) - 1.0).max()) <= PIX_TOL


def test_area_128_lattice_at_1024(R):
    """The 128^3 workload at 1024^2 (eigenvalue 3 of the deformation): the
    whole frame's mass, and a central 256^2 crop against the oracle's render
    of a window with the same pixel edges."""
    c = config("zel128_ortho1024")
    N, W, H = c["N"], c["W"], c["H"]
    pos = ZeldovichField.generate(N, c["n_index"], c["k_cut"], c["seed"]).positions(c["lams"][0])
    R.build_tets(torch.from_numpy(pos).cuda(), N)
    got = R.render_area(ortho_z(W, H)).cpu().numpy()
    R.sync()
    assert abs(got.astype(np.float64).sum() / (W * H) - 1.0) <= MASS_TOL
    x0, y0, w = 384, 384, 256
    crop = camera_dict("ortho", w, w, fwd=(0, 0, 1), up=(0, 1, 0), lo=(x0 / W, y0 / H),
                       hi=((x0 + w) / W, (y0 + w) / H))
    ref = oracle.render_area(pos, N, crop)
    assert pixel_error(got[y0:y0 + w, x0:x0 + w], ref) <= PIX_TOL


def test_area_needs_an_orthographic_view(R):
    from paper_1208_3206_gb300._lib import LtError
    from lt_inputs import sphere_cameras
    N = 8
    pos = ZeldovichField.generate(N, -2.0, 3.0, 9).positions(1.0)
    R.build_tets(torch.from_numpy(pos).cuda(), N)
    with pytest.raises(LtError) as e:
        R.render_area(sphere_cameras(2, 32, 32)[0])
    assert e.value.name == "LT_ERR_ARG"
    R.sync()
