"""Seeded Zel'dovich particle lattices on a periodic box.

Recipe (test tooling, not part of the paper's method):
  * white noise from numpy.random.default_rng(seed), N^3 normals, indexed
    [k, j, i] so that the flattened order is the particle id i + N (j + N k);
  * Fourier transform, multiply by sqrt(P(k)), P(k) = k^n exp(-k^2 / k_c^2),
    k angular (2 pi times the integer wavenumber for a unit box);
    the k = 0 mode and the Nyquist planes are zeroed;
  * displacement psi_k = i k delta_k / k^2 (so that delta = -div psi);
  * growth factor D chosen so that D * max_q lambda_max(-d psi_a / d q_b)
    equals the requested deformation eigenvalue (shell crossing when > 1);
  * x = q + D psi, wrapped into [0, box), stored as float32 (x, y, z, 0).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

try:  # multi-threaded FFTs when scipy is present
    import scipy.fft as _fft

    def _rfftn(a):
        return _fft.rfftn(a, workers=-1)

    def _irfftn(a, s):
        return _fft.irfftn(a, s=s, workers=-1)
except Exception:  # pragma: no cover - numpy fallback
    def _rfftn(a):
        return np.fft.rfftn(a)

    def _irfftn(a, s):
        return np.fft.irfftn(a, s=s)


@dataclass
class ZeldovichField:
    """Displacement field psi (unit growth) on an N^3 lattice and its maximum
    deformation eigenvalue lambda0 (at unit growth)."""

    N: int
    box: float
    psi: np.ndarray  # [3][N][N][N] float64, components (x, y, z), indexed [k, j, i]
    lambda0: float

    @classmethod
    def generate(cls, N: int, n_index: float, k_cut_over_2pi: float, seed: int,
                 box: float = 1.0) -> "ZeldovichField":
        rng = np.random.default_rng(seed)
        white = rng.standard_normal((N, N, N))
        wk = _rfftn(white)
        del white
        two_pi = 2.0 * np.pi / box
        kz = (np.fft.fftfreq(N, d=1.0 / N) * two_pi)[:, None, None]
        ky = (np.fft.fftfreq(N, d=1.0 / N) * two_pi)[None, :, None]
        kx = (np.fft.rfftfreq(N, d=1.0 / N) * two_pi)[None, None, :]
        k2 = kx * kx + ky * ky + kz * kz
        kmag = np.sqrt(k2)
        kc = k_cut_over_2pi * 2.0 * np.pi
        with np.errstate(divide="ignore", invalid="ignore"):
            pk = np.where(k2 > 0, kmag ** n_index * np.exp(-k2 / (kc * kc)), 0.0)
        delta = wk * np.sqrt(pk)
        del wk, pk, kmag
        if N % 2 == 0:
            h = N // 2
            delta[h, :, :] = 0
            delta[:, h, :] = 0
            delta[:, :, h] = 0
        delta[0, 0, 0] = 0
        with np.errstate(divide="ignore", invalid="ignore"):
            inv_k2 = np.where(k2 > 0, 1.0 / k2, 0.0)
        kvec = (kx, ky, kz)
        psi = np.empty((3, N, N, N), dtype=np.float64)
        for a in range(3):
            psi[a] = _irfftn(1j * kvec[a] * delta * inv_k2, s=(N, N, N))
        # deformation tensor T_ab = -d psi_a / d q_b = k_a k_b delta / k^2
        comps = {}
        for a in range(3):
            for b in range(a, 3):
                comps[(a, b)] = _irfftn(kvec[a] * kvec[b] * delta * inv_k2, s=(N, N, N)).ravel()
        del delta, inv_k2
        lam = _max_eigenvalue(comps, N ** 3)
        return cls(N=N, box=box, psi=psi, lambda0=lam)

    def growth_for(self, lam_target: float) -> float:
        return float(lam_target) / self.lambda0

    def displacement(self, lam_target: float) -> np.ndarray:
        """Displacement D psi as [N^3][3] float64 in id order."""
        D = self.growth_for(lam_target)
        return (D * self.psi.reshape(3, -1)).T.copy()

    def positions(self, lam_target: float, dtype=np.float32) -> np.ndarray:
        """Wrapped particle positions [N^3][4] (x, y, z, 0) in id order."""
        return zeldovich_positions_from(self.displacement(lam_target), self.N, self.box, dtype)


def _lattice(N: int, box: float) -> np.ndarray:
    idx = np.arange(N ** 3, dtype=np.int64)
    i, j, k = idx % N, (idx // N) % N, idx // (N * N)
    return np.stack([i, j, k], axis=1).astype(np.float64) * (box / N)


def zeldovich_positions_from(disp: np.ndarray, N: int, box: float, dtype=np.float32) -> np.ndarray:
    x = _lattice(N, box) + disp
    x = np.mod(x, box)
    x = np.where(x >= box, x - box, x)
    out = np.zeros((N ** 3, 4), dtype=dtype)
    out[:, :3] = x.astype(dtype)
    # float32 rounding can land exactly on box: keep the stored value in [0, box)
    out[:, :3] = np.where(out[:, :3] >= dtype(box), dtype(0), out[:, :3])
    return out


def _max_eigenvalue(comps, n: int, chunk: int = 1 << 22) -> float:
    best = -np.inf
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        m = np.empty((e - s, 3, 3))
        for a in range(3):
            for b in range(a, 3):
                m[:, a, b] = comps[(a, b)][s:e]
                m[:, b, a] = comps[(a, b)][s:e]
        best = max(best, float(np.linalg.eigvalsh(m)[:, -1].max()))
    return best


def zeldovich_positions(N: int, n_index: float, k_cut_over_2pi: float, lam_target: float, seed: int,
                        box: float = 1.0) -> np.ndarray:
    """One snapshot: wrapped float32 positions [N^3][4]."""
    return ZeldovichField.generate(N, n_index, k_cut_over_2pi, seed, box).positions(lam_target)


def fp16_offsets(disp: np.ndarray, N: int, box: float = 1.0) -> np.ndarray:
    """Displacements as float16 offsets from the lattice point in cell units,
    padded to 4 halves (8 bytes) per particle."""
    out = np.zeros((N ** 3, 4), dtype=np.float16)
    out[:, :3] = (disp * (N / box)).astype(np.float16)
    return out


def decode_fp16_offsets(off: np.ndarray, N: int, box: float = 1.0) -> np.ndarray:
    """Wrapped float64 positions [N^3][3] that the float16 offsets encode."""
    x = _lattice(N, box) / (box / N) + off[:, :3].astype(np.float64)
    x = x * (box / N)
    return np.mod(x, box)
