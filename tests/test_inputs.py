"""Checks of the seeded synthetic input generator (test tooling)."""
import numpy as np

from lt_inputs import ZeldovichField, fp16_offsets, decode_fp16_offsets, sphere_cameras, CONFIGS


def test_reproducible_and_wrapped():
    a = ZeldovichField.generate(16, -2.0, 6.0, 42).positions(2.0)
    b = ZeldovichField.generate(16, -2.0, 6.0, 42).positions(2.0)
    c = ZeldovichField.generate(16, -2.0, 6.0, 43).positions(2.0)
    assert a.dtype == np.float32 and a.shape == (16 ** 3, 4)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert a[:, :3].min() >= 0.0 and a[:, :3].max() < 1.0
    assert np.all(a[:, 3] == 0)


def test_max_deformation_eigenvalue_matches_finite_differences():
    N = 48
    f = ZeldovichField.generate(N, -2.5, 6.0, 5)
    psi = f.psi  # [3][k][j][i]
    h = 1.0 / N
    # axis b of q: x -> array axis 2, y -> 1, z -> 0
    ax = {0: 2, 1: 1, 2: 0}
    T = np.zeros((N ** 3, 3, 3))
    for a in range(3):
        for b in range(3):
            d = (np.roll(psi[a], -1, axis=ax[b]) - np.roll(psi[a], 1, axis=ax[b])) / (2 * h)
            T[:, a, b] = -d.ravel()
    T = 0.5 * (T + T.transpose(0, 2, 1))
    lam_fd = np.linalg.eigvalsh(T)[:, -1].max()
    assert abs(lam_fd - f.lambda0) < 0.1 * f.lambda0
    # the growth factor puts the maximum eigenvalue at the requested value
    assert f.growth_for(3.0) * f.lambda0 == 3.0 or abs(f.growth_for(3.0) * f.lambda0 - 3.0) < 1e-12


def test_power_spectrum_slope():
    N, n_idx = 64, -2.0
    f = ZeldovichField.generate(N, n_idx, 1e6, 9)  # no cutoff
    # density contrast delta = -div psi, spectrally
    k = np.fft.fftfreq(N, d=1.0 / N) * 2 * np.pi
    kz, ky, kx = np.meshgrid(k, k, k, indexing="ij")
    div = sum(1j * kk * np.fft.fftn(f.psi[a]) for a, kk in enumerate((kx, ky, kz)))
    p = np.abs(div) ** 2
    kmag = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    shells = [(4, 6), (12, 18)]
    pw = []
    for lo, hi in shells:
        m = (kmag >= lo * 2 * np.pi) & (kmag < hi * 2 * np.pi)
        pw.append((p[m].mean(), kmag[m].mean()))
    slope = np.log(pw[1][0] / pw[0][0]) / np.log(pw[1][1] / pw[0][1])
    assert abs(slope - n_idx) < 0.3


def test_fp16_offsets_roundtrip():
    f = ZeldovichField.generate(16, -2.0, 6.0, 1)
    d = f.displacement(2.0)
    off = fp16_offsets(d, 16)
    assert off.dtype == np.float16 and off.shape == (16 ** 3, 4)
    x = decode_fp16_offsets(off, 16)
    p = f.positions(2.0)[:, :3].astype(np.float64)
    err = np.abs((x - p + 0.5) % 1.0 - 0.5)
    assert err.max() < 2e-3 / 16  # half-ulp of float16 offsets of a few cells


def test_sphere_cameras_look_at_centre():
    cams = sphere_cameras(16, 64, 64)
    assert len(cams) == 16
    for c in cams:
        eye = np.array(c["eye"])
        assert abs(np.linalg.norm(eye - 0.5) - 2.0) < 1e-12
        f = np.array(c["fwd"])
        assert np.allclose(eye + f, 0.5)


def test_configs_are_complete():
    assert set(CONFIGS) == {"zel32_ortho256", "zel128_ortho1024", "zel256_persp2048x128",
                            "zel512_fp16_ortho4096", "zel64_grad512"}
    assert len(CONFIGS["zel256_persp2048x128"]["lams"]) == 8
