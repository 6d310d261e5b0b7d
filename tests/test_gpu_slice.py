"""GPU parity of the 2D slices (lt_slice): the total density of overlapping
streams (Eq. 4) and the number of streams (Sec. 3.2) at the centres of an
n x n grid on a plane z = z0, against the FP64 oracle (oracle.point_density)
on the same seeded inputs.

Tolerances: stream counts are integers and must match exactly; densities
within 1e-4 of max(value, mean density). Both sides test containment in
FP64 with the closed-tetrahedron rule, so points would differ only within
rounding of a face, which generic input does not reach.
"""
import numpy as np
import pytest

import oracle
from lt_inputs import ZeldovichField, decode_fp16_offsets, fp16_offsets

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DENS_TOL = 1e-4


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1208_3206_gb300.render import Renderer
    return Renderer()


def slice_points(n, z0, box=1.0):
    g = box / n
    a = (np.arange(n) + 0.5) * g
    X, Y = np.meshgrid(a, a)  # [b][a]
    return np.stack([X.ravel(), Y.ravel(), np.full(n * n, z0)], axis=1)


def check(got, ref, weight):
    got = got.astype(np.float64).ravel()
    if weight == "streams":
        assert np.array_equal(got, ref), np.abs(got - ref).max()
    else:
        err = np.abs(got - ref) / np.maximum(np.abs(ref), 1.0)
        assert float(err.max()) <= DENS_TOL


@pytest.mark.parametrize("weight", ["density", "streams"])
@pytest.mark.parametrize("N,n,lam,z0", [(16, 64, 2.5, 0.37), (8, 50, 1.8, 0.9123), (16, 33, 3.5, 1.21)])
def test_slice_matches_oracle(R, weight, N, n, lam, z0):
    pos = ZeldovichField.generate(N, -2.0, max(3.0, N / 2.0), 900 + N).positions(lam)
    R.build_tets(torch.from_numpy(pos).cuda(), N)
    got = R.slice(n, z0, weight)
    R.sync()
    ref = oracle.point_density(pos, N, slice_points(n, z0), weight)
    check(got.cpu().numpy(), ref, weight)


def test_slice_plane_is_periodic_and_reproducible(R):
    N, n = 16, 40
    pos = ZeldovichField.generate(N, -2.0, 8.0, 77).positions(2.2)
    R.build_tets(torch.from_numpy(pos).cuda(), N)
    a = R.slice(n, 0.4, "density").clone()
    b = R.slice(n, 1.4, "density").clone()
    c = R.slice(n, -0.6, "density")
    d = R.slice(n, 0.4, "density")
    R.sync()
    assert torch.equal(a, d)
    # the same plane one period away: the same tetrahedra, so the same sums
    # up to the rounding of the containment tests near faces
    assert float((a - b).abs().max()) <= DENS_TOL * max(1.0, float(a.max()))
    assert float((a - c).abs().max()) <= DENS_TOL * max(1.0, float(a.max()))


def test_slice_fp16_offsets(R):
    N, n = 16, 48
    f = ZeldovichField.generate(N, -2.5, 6.0, 1004)
    off = fp16_offsets(f.displacement(3.0), N)
    R.build_tets(torch.from_numpy(off).cuda(), N)
    got = R.slice(n, 0.55, "streams")
    R.sync()
    ref = oracle.point_density(decode_fp16_offsets(off, N), N, slice_points(n, 0.55), "streams")
    check(got.cpu().numpy(), ref, "streams")


def test_slice_128_lattice_at_512_sampled(R):
    """The 128^3 workload (deformation eigenvalue 3), a 512^2 slice at
    z = 0.5: 4096 seeded points against the oracle, both weightings."""
    from lt_inputs import config
    c = config("zel128_ortho1024")
    N, n, z0 = c["N"], 512, 0.5
    pos = ZeldovichField.generate(N, c["n_index"], c["k_cut"], c["seed"]).positions(c["lams"][0])
    R.build_tets(torch.from_numpy(pos).cuda(), N)
    dens = R.slice(n, z0, "density").cpu().numpy().ravel()
    streams = R.slice(n, z0, "streams").cpu().numpy().ravel()
    R.sync()
    pick = np.random.default_rng(6006).choice(n * n, size=4096, replace=False)
    pts = slice_points(n, z0)[pick]
    check(dens[pick], oracle.point_density(pos, N, pts, "density"), "density")
    check(streams[pick], oracle.point_density(pos, N, pts, "streams"), "streams")
    assert streams.min() >= 1.0  # every point of the box lies in at least one stream


def test_slice_errors(R):
    from paper_1208_3206_gb300._lib import LtError
    N = 8
    pos = ZeldovichField.generate(N, -2.0, 3.0, 9).positions(1.0)
    R.build_tets(torch.from_numpy(pos).cuda(), N)
    with pytest.raises(LtError) as e:
        R.slice(16, 0.5, "density", snapshot=2)
    assert e.value.name == "LT_ERR_ARG"
    with pytest.raises(LtError) as e:
        R.slice(8, float("nan"), "density")
    assert e.value.name == "LT_ERR_ARG"
    R.sync()
