"""GB300 column-density renderer for the Lagrangian tetrahedral tessellation
of a periodic dark-matter particle lattice (arXiv:1208.3206).

The compute path is liblt.so (hand-written sm_103a CUDA behind the C ABI of
include/lt.h); this package only marshals arguments. Importing the package
does not load the library; creating a Renderer does, and fails loudly if
the library has not been built.
"""
from ._build import build, LIB as LIB_PATH  # noqa: F401


def __getattr__(name):
    # lazy: the binding needs torch and the compiled library
    if name in ("Renderer", "Camera", "LTRender", "lt_render", "lt_build_tets", "lt_project_bin",
                "lt_render_tiles", "lt_render_backward"):
        from . import render

        return getattr(render, name)
    raise AttributeError(name)
