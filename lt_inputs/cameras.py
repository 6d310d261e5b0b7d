"""Camera descriptions (plain dicts) understood by both the oracle and the
GPU binding. See oracle.Camera / paper_1208_3206_gb300.Camera for meaning."""
from __future__ import annotations

import math

import numpy as np


def camera_dict(type: str, W: int, H: int, eye=(0.0, 0.0, 0.0), fwd=(0.0, 0.0, 1.0), up=(0.0, 1.0, 0.0),
                fov_y_deg: float = 60.0, lo=(0.0, 0.0), hi=(1.0, 1.0), wrap: bool = False) -> dict:
    return dict(type=type, W=int(W), H=int(H), eye=tuple(float(x) for x in eye),
                fwd=tuple(float(x) for x in fwd), up=tuple(float(x) for x in up),
                fov_y_deg=float(fov_y_deg), lo=tuple(float(x) for x in lo),
                hi=tuple(float(x) for x in hi), wrap=bool(wrap))


def ortho_z(W: int, H: int, box: float = 1.0, wrap: bool = True) -> dict:
    """Orthographic projection along +z onto the periodic [0, box)^2 window."""
    return camera_dict("ortho", W, H, fwd=(0, 0, 1), up=(0, 1, 0), lo=(0, 0), hi=(box, box), wrap=wrap)


def sphere_cameras(n: int, W: int, H: int, radius: float = 2.0, fov_y_deg: float = 60.0,
                   center=(0.5, 0.5, 0.5)) -> list:
    """n perspective cameras on a Fibonacci sphere of the given radius around
    `center`, each looking at the centre; up = +z unless the view is within
    about 8 degrees of the z axis, then +y."""
    cams = []
    golden = math.pi * (3.0 - math.sqrt(5.0))
    c = np.asarray(center, dtype=np.float64)
    for i in range(n):
        z = 1.0 - 2.0 * (i + 0.5) / n
        r = math.sqrt(max(0.0, 1.0 - z * z))
        phi = golden * i
        eye = c + radius * np.array([r * math.cos(phi), r * math.sin(phi), z])
        fwd = c - eye
        fu = fwd / np.linalg.norm(fwd)
        up = (0.0, 0.0, 1.0) if abs(fu[2]) <= 0.99 else (0.0, 1.0, 0.0)
        cams.append(camera_dict("persp", W, H, eye=eye, fwd=fwd, up=up, fov_y_deg=fov_y_deg))
    return cams
