"""GPU parity of the resampling onto a periodic grid and of the stream-count
field (lt_resample; Sec. 4.3, Eq. 10-12, Sec. 3.2) against the FP64 oracle
(oracle.resample), cell by cell, on the same seeded inputs.

Tolerance: every cell within 1e-4 of max(cell, mean cell), the grid's total
(times the cell face area: the mass in the density weighting) within 1e-6.
The GPU path clips each (tetrahedron, line) pair exactly in FP64 and sums in
64-bit fixed point, so the measured errors sit near the fixed-point
resolution (2^-28 of the mean cell per add).
"""
import numpy as np
import pytest

import oracle
from lt_inputs import ZeldovichField, decode_fp16_offsets, fp16_offsets

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CELL_TOL = 1e-4
SUM_TOL = 1e-6


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1208_3206_gb300.render import Renderer
    return Renderer()


def cell_error(got, ref):
    mean = float(np.mean(ref))
    return float((np.abs(got.astype(np.float64) - ref) / np.maximum(np.abs(ref), mean)).max())


def gpu_resample(R, pos, N, n, weight, snapshot=0):
    R.build_tets(torch.from_numpy(np.ascontiguousarray(pos)).cuda(), N)
    g = R.resample(n, weight, snapshot)
    R.sync()
    return g.cpu().numpy()


@pytest.mark.parametrize("weight", ["density", "streams"])
@pytest.mark.parametrize("N,n,lam,tile", [(16, 32, 2.5, 16), (8, 40, 1.8, 16), (8, 13, 1.2, 8), (12, 24, 3.0, 32)])
def test_resample_matches_oracle(R, weight, N, n, lam, tile):
    R.set_config(tile=tile)
    pos = ZeldovichField.generate(N, -2.0, max(3.0, N / 2.0), 700 + N).positions(lam)
    ref = oracle.resample(pos, N, n, weight)
    got = gpu_resample(R, pos, N, n, weight)
    assert got.shape == (n, n, n)
    assert cell_error(got, ref) <= CELL_TOL
    assert abs(got.astype(np.float64).sum() - ref.sum()) <= SUM_TOL * ref.sum()
    R.set_config(tile=16)


def test_resample_unperturbed_lattice_is_uniform(R):
    """An unperturbed lattice has density 1 and one stream everywhere: every
    cell holds exactly g (density times g, or one stream times g)."""
    N, n = 8, 24
    idx = np.arange(N ** 3)
    pos = np.zeros((N ** 3, 4), np.float32)
    pos[:, 0], pos[:, 1], pos[:, 2] = idx % N, (idx // N) % N, idx // (N * N)
    pos[:, :3] /= N
    for weight in ("density", "streams"):
        got = gpu_resample(R, pos, N, n, weight).astype(np.float64)
        assert np.abs(got - 1.0 / n).max() <= 1e-6 / n


def test_resample_second_snapshot_and_reproducibility(R):
    N, n = 16, 32
    f = ZeldovichField.generate(N, -2.0, 8.0, 812)
    pos = np.concatenate([f.positions(0.7), f.positions(2.9)])
    R.build_tets(torch.from_numpy(pos).cuda(), N)
    a = R.resample(n, "density", 1).clone()
    b = R.resample(n, "density", 1)
    R.sync()
    assert torch.equal(a, b)
    ref = oracle.resample(pos[N ** 3:], N, n, "density")
    assert cell_error(a.cpu().numpy(), ref) <= CELL_TOL


def test_resample_fp16_offsets(R):
    N, n = 16, 48
    f = ZeldovichField.generate(N, -2.5, 6.0, 1004)
    off = fp16_offsets(f.displacement(3.0), N)
    ref = oracle.resample(decode_fp16_offsets(off, N), N, n, "streams")
    got = gpu_resample(R, off, N, n, "streams")
    assert cell_error(got, ref) <= CELL_TOL


def test_resample_128_lattice_at_512(R):
    """The 128^3 workload (deformation eigenvalue 3) resampled onto 512^3
    cells: the whole grid against the oracle, and the mass in the density
    weighting."""
    from lt_inputs import config
    c = config("zel128_ortho1024")
    N, n = c["N"], 512
    pos = ZeldovichField.generate(N, c["n_index"], c["k_cut"], c["seed"]).positions(c["lams"][0])
    got = gpu_resample(R, pos, N, n, "density")
    ref = oracle.resample(pos, N, n, "density")
    assert cell_error(got, ref) <= CELL_TOL
    g2 = (1.0 / n) ** 2
    assert abs(got.astype(np.float64).sum() * g2 - ref.sum() * g2) <= SUM_TOL * ref.sum() * g2


def test_resample_errors(R):
    from paper_1208_3206_gb300._lib import LtError
    N = 8
    pos = ZeldovichField.generate(N, -2.0, 3.0, 9).positions(1.0)
    R.build_tets(torch.from_numpy(pos).cuda(), N)
    with pytest.raises(LtError) as e:
        R.resample(16, "density", snapshot=1)
    assert e.value.name == "LT_ERR_ARG"
    with pytest.raises(LtError) as e:
        R.resample(0, "density")
    assert e.value.name == "LT_ERR_ARG"
    R.sync()
