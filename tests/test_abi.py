"""The C ABI library loads and exports every entry point declared in
include/lt.h (no GPU needed, no compute calls)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:lt_status|void|const char\*)\s+(lt_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1208_3206_gb300 import _build, _lib
    _build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lt_build_tets", "lt_project_bin", "lt_render_tiles", "lt_render_backward"):
        assert required in names
    assert len(names) >= 16


def test_every_declared_symbol_is_exported(lib):
    from paper_1208_3206_gb300 import _lib
    names = declared_functions()
    assert sorted(_lib.EXPORTS) == names
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings_and_null_arguments(lib):
    for code in range(10):
        assert lib.lt_status_str(code)
    assert lib.lt_status_str(99) == b"unknown status"
    # argument checks happen before any CUDA call
    assert lib.lt_create(None, None) == 1
    assert lib.lt_build_tets(None, None, 0, 4, 1.0, 1.0, 1, None, None) == 1
    assert lib.lt_project_bin(None, None, 1, None, None) == 1
    assert lib.lt_render_tiles(None, None, None, None) == 1
    assert lib.lt_render_backward(None, None, None, None) == 1
    assert lib.lt_sync(None, None) == 1


def test_library_is_sm103a_only():
    from paper_1208_3206_gb300 import _build
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No CPU fallback: without the compiled library the binding raises."""
    from paper_1208_3206_gb300 import _build, _lib
    monkeypatch.setattr(_build, "LIB", str(tmp_path / "missing" / "liblt.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="liblt.so not found"):
        _lib.load()


def test_frame_mass_static_argument_checks(lib):
    """Argument and capacity errors come back before any CUDA call."""
    import ctypes as C
    fake = C.c_void_p(0x1000)  # never dereferenced: the checks return first
    assert lib.lt_frame_mass_static(None, 1, 4, 4, 1.0, fake, None) == 1
    assert lib.lt_frame_mass_static(fake, 0, 4, 4, 1.0, fake, None) == 1
    assert lib.lt_frame_mass_static(fake, 1, 4, 4, 0.0, fake, None) == 1
    assert lib.lt_frame_mass_static(fake, 1, 4, 4, float("nan"), fake, None) == 1
    assert lib.lt_frame_mass_static(fake, 129, 4, 4, 1.0, fake, None) == 3


def test_bounds_checking_build_compiles(tmp_path):
    """The debugging build with index checks (LT_CHECK_BOUNDS) stays
    compilable (compile only; the checks latch LT_ERR_BOUNDS when run)."""
    import subprocess
    from paper_1208_3206_gb300 import _build
    src = os.path.join(_build.CSRC, "lt_tile.cu")
    cmd = [_build._nvcc(), *_build.ARCH, *_build.FLAGS, "-DLT_CHECK_BOUNDS", "-c", src, "-o",
           str(tmp_path / "lt_tile_checked.o")]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr


def test_ctypes_structs_match_the_header(tmp_path):
    """The binding's ctypes mirrors of lt_camera, lt_config and lt_stats have
    the header's size and field offsets (compiled by the host C compiler
    against include/lt.h), so a field added on one side only fails here."""
    import shutil
    import subprocess

    from paper_1208_3206_gb300 import _lib

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"lt_camera": _lib.LtCamera, "lt_config": _lib.LtConfig, "lt_stats": _lib.LtStats}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "lt.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln.strip():
            a, b, v = ln.split()
            got[(a, b)] = int(v)
    for cname, py in structs.items():
        assert got[(cname, "size")] == C.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
