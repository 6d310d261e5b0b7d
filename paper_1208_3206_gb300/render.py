"""Python binding of liblt (include/lt.h): a Renderer owning one lt_ctx, with
methods named after the C entry points, and a torch.autograd.Function over
the forward render and its hand-written adjoint.

PyTorch supplies device memory and the current CUDA stream; every step of
the projection runs in the library's kernels. There is no CPU path.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field
from typing import Optional, Sequence

import torch

from . import _lib
from ._lib import LtCamera, LtConfig, LtStats, check

POS_F32X4 = 0
POS_F16_OFFSETS = 1


@dataclass
class Camera:
    """One view (see include/lt.h, lt_camera)."""

    type: str
    W: int
    H: int
    eye: Sequence[float] = (0.0, 0.0, 0.0)
    fwd: Sequence[float] = (0.0, 0.0, 1.0)
    up: Sequence[float] = (0.0, 1.0, 0.0)
    fov_y_deg: float = 60.0
    lo: Sequence[float] = (0.0, 0.0)
    hi: Sequence[float] = (1.0, 1.0)
    wrap: bool = False
    near_radius: float = 0.0

    def to_c(self) -> LtCamera:
        c = LtCamera()
        c.type = 1 if self.type == "persp" else 0
        c.eye[:] = [float(x) for x in self.eye]
        c.fwd[:] = [float(x) for x in self.fwd]
        c.up[:] = [float(x) for x in self.up]
        c.fov_y_deg = float(self.fov_y_deg)
        c.lo[:] = [float(x) for x in self.lo]
        c.hi[:] = [float(x) for x in self.hi]
        c.W, c.H = int(self.W), int(self.H)
        c.wrap = int(bool(self.wrap))
        c.near_radius = float(self.near_radius)
        return c


def _cams(cams) -> tuple:
    if isinstance(cams, (dict, Camera)):
        cams = [cams]
    cs = [c if isinstance(c, Camera) else Camera(**c) for c in cams]
    arr = (LtCamera * len(cs))(*[c.to_c() for c in cs])
    return cs, arr


def _snaps(frame_snapshot, n):
    if frame_snapshot is None:
        return None
    fs = list(frame_snapshot)
    if len(fs) != n:
        raise ValueError("frame_snapshot must have one entry per camera")
    return (C.c_int * n)(*[int(x) for x in fs])


def _stream() -> C.c_void_p:
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t: Optional[torch.Tensor]) -> C.c_void_p:
    return C.c_void_p(0 if t is None else t.data_ptr())


class Renderer:
    """Owner of one library context (lt_create / lt_destroy)."""

    def __init__(self, tile: int = 0, raster_threads: int = 0, ctas_per_sm: int = 0, frac_bits: int = 0):
        self._lib = _lib.load()
        if not torch.cuda.is_available():
            raise RuntimeError("paper_1208_3206_gb300 needs a CUDA device (no CPU path)")
        torch.cuda.init()
        cfg = LtConfig(tile, raster_threads, ctas_per_sm, frac_bits)
        h = C.c_void_p()
        check("lt_create", self._lib.lt_create(C.byref(h), C.byref(cfg)))
        self._h = h
        self._pos = None
        self.N = None
        self.n_snapshots = 0
        self._cams = []
        self._frame_snapshot = None

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.lt_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- configuration
    def set_config(self, tile=0, raster_threads=0, ctas_per_sm=0, frac_bits=0):
        cfg = LtConfig(tile, raster_threads, ctas_per_sm, frac_bits)
        check("lt_set_config", self._lib.lt_set_config(self._h, C.byref(cfg)))

    def get_config(self) -> dict:
        cfg = LtConfig()
        check("lt_get_config", self._lib.lt_get_config(self._h, C.byref(cfg)))
        return dict(tile=cfg.tile, raster_threads=cfg.raster_threads, ctas_per_sm=cfg.ctas_per_sm,
                    frac_bits=cfg.frac_bits)

    # -- lt_build_tets
    def build_tets(self, pos: torch.Tensor, N: int, box: float = 1.0, total_mass: float = 1.0,
                   rho_out: Optional[torch.Tensor] = None) -> None:
        """Register positions: float32 [S][N^3][4] (or [N^3][4]) wrapped
        positions, or float16 [S][N^3][4] offsets in cell units."""
        if not pos.is_cuda or not pos.is_contiguous():
            raise ValueError("positions must be a contiguous CUDA tensor")
        if pos.dtype == torch.float32:
            fmt = POS_F32X4
        elif pos.dtype == torch.float16:
            fmt = POS_F16_OFFSETS
        else:
            raise ValueError("positions must be float32 (x,y,z,pad) or float16 offsets")
        if pos.shape[-1] != 4 or pos.numel() % (4 * N ** 3):
            raise ValueError("positions must be [..., N^3, 4]")
        S = pos.numel() // (4 * N ** 3)
        if rho_out is not None and (rho_out.dtype != torch.float32 or rho_out.numel() != 6 * N ** 3 * S
                                    or not rho_out.is_cuda):
            raise ValueError("rho_out must be float32 CUDA [S][6 N^3]")
        check("lt_build_tets", self._lib.lt_build_tets(self._h, _ptr(pos), fmt, int(N), float(box),
                                                       float(total_mass), int(S), _ptr(rho_out), _stream()))
        self._pos = pos
        self.N = N
        self.box = box
        self.total_mass = total_mass
        self.n_snapshots = S

    # -- lt_project_bin
    def project_bin(self, cams, frame_snapshot=None) -> None:
        cs, arr = _cams(cams)
        fs = _snaps(frame_snapshot, len(cs))
        check("lt_project_bin", self._lib.lt_project_bin(self._h, arr, len(cs), fs, _stream()))
        self._cams = cs
        self._frame_snapshot = None if frame_snapshot is None else list(frame_snapshot)

    def _image(self, image, cams=None):
        cs = cams or self._cams
        F, H, W = len(cs), cs[0].H, cs[0].W
        if image is None:
            return torch.empty((F, H, W), dtype=torch.float32, device="cuda")
        if image.dtype != torch.float32 or not image.is_cuda or image.numel() != F * H * W or not image.is_contiguous():
            raise ValueError(f"image must be a contiguous float32 CUDA tensor with {F}x{H}x{W} elements")
        return image

    # -- lt_render_tiles
    def render_tiles(self, image: Optional[torch.Tensor] = None, mass: Optional[torch.Tensor] = None,
                     with_mass: bool = False):
        img = self._image(image)
        if mass is None and with_mass:
            mass = torch.empty(len(self._cams), dtype=torch.float64, device="cuda")
        check("lt_render_tiles", self._lib.lt_render_tiles(self._h, _ptr(img), _ptr(mass), _stream()))
        return (img, mass) if with_mass or mass is not None else img

    # -- lt_render_atomic
    def render_atomic(self, cams, frame_snapshot=None, image: Optional[torch.Tensor] = None):
        cs, arr = _cams(cams)
        img = self._image(image, cs)
        img.zero_()
        fs = _snaps(frame_snapshot, len(cs))
        check("lt_render_atomic", self._lib.lt_render_atomic(self._h, arr, len(cs), fs, _ptr(img), _stream()))
        return img

    # -- lt_count_fragments
    def count_fragments(self) -> list:
        out = (C.c_longlong * len(self._cams))()
        check("lt_count_fragments", self._lib.lt_count_fragments(self._h, out, _stream()))
        return [int(x) for x in out]

    # -- lt_render_backward
    def render_backward(self, dL_dimage: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        g = dL_dimage.contiguous().to(torch.float32)
        if out is None:
            out = torch.empty((self.n_snapshots, self.N ** 3, 3), dtype=torch.float32, device="cuda")
        check("lt_render_backward", self._lib.lt_render_backward(self._h, _ptr(g), _ptr(out), _stream()))
        return out

    # -- lt_resample
    def resample(self, n: int, weight: str = "density", snapshot: int = 0,
                 out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Resampling of one registered snapshot onto a periodic n^3 grid
        (float32 [n][n][n], index [c][b][a]): per cell, q dl along its
        central line in z inside its slab, q = rho ("density") or 1
        ("streams"). Replaces the frames and bins of the last project_bin."""
        w = {"density": 0, "streams": 1}[weight]
        if out is None:
            out = torch.empty((n, n, n), dtype=torch.float32, device="cuda")
        if out.dtype != torch.float32 or not out.is_cuda or out.numel() != n ** 3 or not out.is_contiguous():
            raise ValueError("out must be a contiguous float32 CUDA tensor with n^3 elements")
        check("lt_resample", self._lib.lt_resample(self._h, int(n), w, int(snapshot), _ptr(out), _stream()))
        self._cams = []
        return out

    # -- lt_slice
    def slice(self, n: int, z0: float, weight: str = "density", snapshot: int = 0,
              out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Total density ("density") or number of streams ("streams") at the
        centres of an n x n grid on the plane z = z0 (float32 [n][n], index
        [b][a])."""
        w = {"density": 0, "streams": 1}[weight]
        if out is None:
            out = torch.empty((n, n), dtype=torch.float32, device="cuda")
        if out.dtype != torch.float32 or not out.is_cuda or out.numel() != n * n or not out.is_contiguous():
            raise ValueError("out must be a contiguous float32 CUDA tensor with n^2 elements")
        check("lt_slice", self._lib.lt_slice(self._h, int(n), w, int(snapshot), float(z0), _ptr(out), _stream()))
        return out

    # -- lt_render_centroids
    def render_centroids(self, cam, snapshot: int = 0, image: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Centroid splats (Sec. 4.2) of one registered snapshot in one
        orthographic view: float32 [H][W]."""
        cs, arr = _cams([cam])
        c = cs[0]
        if image is None:
            image = torch.empty((c.H, c.W), dtype=torch.float32, device="cuda")
        if image.dtype != torch.float32 or not image.is_cuda or image.numel() != c.H * c.W or not image.is_contiguous():
            raise ValueError(f"image must be a contiguous float32 CUDA tensor with {c.H}x{c.W} elements")
        check("lt_render_centroids", self._lib.lt_render_centroids(self._h, arr, int(snapshot), _ptr(image), _stream()))
        return image

    # -- lt_render_area
    def render_area(self, cam, snapshot: int = 0, image: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Area-averaged pixels of one orthographic view: each pixel the mean
        column density (Eq. 6) over its square. float32 [H][W]."""
        cs, arr = _cams([cam])
        c = cs[0]
        if image is None:
            image = torch.empty((c.H, c.W), dtype=torch.float32, device="cuda")
        if image.dtype != torch.float32 or not image.is_cuda or image.numel() != c.H * c.W or not image.is_contiguous():
            raise ValueError(f"image must be a contiguous float32 CUDA tensor with {c.H}x{c.W} elements")
        check("lt_render_area", self._lib.lt_render_area(self._h, arr, int(snapshot), _ptr(image), _stream()))
        return image

    # -- lt_render_hybrid
    def render_hybrid(self, cam, near_radius: float, snapshot: int = 0,
                      image: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Hybrid near/far rendering of one perspective view: cubes within
        near_radius of the eye by exact projection, the others as centroid
        splats. float32 [H][W]."""
        cs, arr = _cams([cam])
        c = cs[0]
        if image is None:
            image = torch.empty((c.H, c.W), dtype=torch.float32, device="cuda")
        if image.dtype != torch.float32 or not image.is_cuda or image.numel() != c.H * c.W or not image.is_contiguous():
            raise ValueError(f"image must be a contiguous float32 CUDA tensor with {c.H}x{c.W} elements")
        check("lt_render_hybrid", self._lib.lt_render_hybrid(self._h, arr, int(snapshot), float(near_radius),
                                                             _ptr(image), _stream()))
        self._cams = []
        return image

    # -- graphs
    def graph_build(self, cams, frame_snapshot=None, image: Optional[torch.Tensor] = None,
                    mass: Optional[torch.Tensor] = None, stream: Optional[torch.cuda.Stream] = None):
        cs, arr = _cams(cams)
        img = self._image(image, cs)
        fs = _snaps(frame_snapshot, len(cs))
        st = stream or torch.cuda.current_stream()
        if st.cuda_stream == 0:
            raise ValueError("graph capture needs a non-default stream")
        check("lt_graph_build", self._lib.lt_graph_build(self._h, arr, len(cs), fs, _ptr(img), _ptr(mass),
                                                         C.c_void_p(st.cuda_stream)))
        self._cams = cs
        self._frame_snapshot = None if frame_snapshot is None else list(frame_snapshot)
        return img

    def graph_launch(self, stream: Optional[torch.cuda.Stream] = None) -> None:
        st = stream or torch.cuda.current_stream()
        check("lt_graph_launch", self._lib.lt_graph_launch(self._h, C.c_void_p(st.cuda_stream)))

    # -- autotuner
    def autotune(self, cams, frame_snapshot=None, reps: int = 2) -> dict:
        cs, arr = _cams(cams)
        img = self._image(None, cs)
        fs = _snaps(frame_snapshot, len(cs))
        best = LtConfig()
        check("lt_autotune", self._lib.lt_autotune(self._h, arr, len(cs), fs, _ptr(img), int(reps),
                                                   C.byref(best), _stream()))
        return dict(tile=best.tile, raster_threads=best.raster_threads, ctas_per_sm=best.ctas_per_sm,
                    frac_bits=best.frac_bits)

    # -- status
    def sync(self) -> None:
        check("lt_sync", self._lib.lt_sync(self._h, _stream()))

    def get_stats(self) -> dict:
        s = LtStats()
        check("lt_get_stats", self._lib.lt_get_stats(self._h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in LtStats._fields_}


# module-level names mirroring the C entry points
def lt_build_tets(r: Renderer, *a, **k):
    return r.build_tets(*a, **k)


def lt_project_bin(r: Renderer, *a, **k):
    return r.project_bin(*a, **k)


def lt_render_tiles(r: Renderer, *a, **k):
    return r.render_tiles(*a, **k)


def lt_render_backward(r: Renderer, *a, **k):
    return r.render_backward(*a, **k)


def lt_resample(r: Renderer, *a, **k):
    return r.resample(*a, **k)


def lt_slice(r: Renderer, *a, **k):
    return r.slice(*a, **k)


def lt_render_centroids(r: Renderer, *a, **k):
    return r.render_centroids(*a, **k)


def lt_render_area(r: Renderer, *a, **k):
    return r.render_area(*a, **k)


def lt_render_hybrid(r: Renderer, *a, **k):
    return r.render_hybrid(*a, **k)


def lt_frame_mass_static(image: torch.Tensor, pixel_area: float, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Per-frame mass (sum of pixels times pixel_area, FP64, fixed order) of a
    float32 CUDA image [F][H][W], through the library's allocation-free
    entry point (no context; its scratch is static device memory, so calls
    on one device must not overlap). `out`: float64 CUDA [F] (allocated here
    when None, by the caller's PyTorch)."""
    if image.dtype != torch.float32 or not image.is_cuda or not image.is_contiguous() or image.dim() != 3:
        raise ValueError("image must be a contiguous float32 CUDA tensor [F][H][W]")
    F, H, W = image.shape
    if out is None:
        out = torch.empty(F, dtype=torch.float64, device=image.device)
    if out.dtype != torch.float64 or not out.is_cuda or out.numel() != F or not out.is_contiguous():
        raise ValueError("out must be a contiguous float64 CUDA tensor with one entry per frame")
    lib = _lib.load()
    check("lt_frame_mass_static", lib.lt_frame_mass_static(_ptr(image), int(F), int(W), int(H), float(pixel_area),
                                                           _ptr(out), _stream()))
    return out


class LTRender(torch.autograd.Function):
    """image = LTRender.apply(pos, renderer, cams): forward through
    lt_build_tets + lt_project_bin + lt_render_tiles, backward through
    lt_render_backward (orthographic views). pos: float32 CUDA [N^3][4]."""

    @staticmethod
    def forward(ctx, pos, renderer: Renderer, cams, N: int, box: float = 1.0, total_mass: float = 1.0):
        p = pos.detach().contiguous()
        renderer.build_tets(p, N, box, total_mass)
        renderer.project_bin(cams)
        img = renderer.render_tiles()
        ctx.renderer = renderer
        ctx.pos_shape = pos.shape
        ctx.save_for_backward(p)
        return img

    @staticmethod
    def backward(ctx, g):
        (p,) = ctx.saved_tensors
        r = ctx.renderer
        if r._pos is None or r._pos.data_ptr() != p.data_ptr():
            raise RuntimeError("the renderer was re-bound to other positions before backward")
        gp = r.render_backward(g)
        out = torch.zeros(ctx.pos_shape, dtype=torch.float32, device=p.device)
        out.view(-1, 4)[:, :3] = gp.view(-1, 3)
        return out, None, None, None, None, None


def lt_render(pos: torch.Tensor, N: int, cams, renderer: Optional[Renderer] = None, box: float = 1.0,
              total_mass: float = 1.0) -> torch.Tensor:
    """Differentiable column-density render of one snapshot."""
    r = renderer or Renderer()
    return LTRender.apply(pos, r, cams, N, box, total_mass)
