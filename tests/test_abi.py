"""C-ABI checks that need no GPU: the library loads, exports every entry point
include/dem.h declares, the ctypes structures match the C layout, and the
host-only calls behave."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dem.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2301_00611_gb300 import _build, dem
    _build.build()
    return dem.load_library()


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dem_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    from paper_2301_00611_gb300 import dem
    declared = _declared()
    assert len(declared) >= 20
    out = subprocess.run(["nm", "-D", "--defined-only", dem.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(dem_\w+)", out))
    missing = [d for d in declared if d not in exported]
    assert not missing, missing
    # the binding covers the same set
    assert sorted(dem.exported_symbols()) == declared


def test_struct_layout_matches_header(tmp_path):
    from paper_2301_00611_gb300 import dem
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "dem.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu\\n\", sizeof(dem_scene_desc),"
        " offsetof(dem_scene_desc, cuda_stream), offsetof(dem_scene_desc, device),"
        " sizeof(dem_stats), offsetof(dem_stats, stress), offsetof(dem_stats, packing_fraction));"
        "return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    vals = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                           check=True).stdout.split()]
    D, S = dem.SceneDesc, dem.Stats
    assert vals == [ctypes.sizeof(D), D.cuda_stream.offset, D.device.offset, ctypes.sizeof(S),
                    S.stress.offset, S.packing_fraction.offset]


def test_desc_defaults_and_version(lib):
    from paper_2301_00611_gb300 import dem
    d = dem.SceneDesc()
    lib.dem_scene_desc_init(ctypes.byref(d))
    assert d.damping == 0.2 and d.verlet_dist == -0.5 and d.precision == dem.DEM_FP64
    assert list(d.cell_h) == [1, 0, 0, 0, 1, 0, 0, 0, 1]
    assert d.device == -1 and d.cuda_stream is None
    assert "sm_103a" in dem.version()


def test_create_rejects_bad_descriptions_on_the_host(lib):
    """Descriptions that are invalid are refused before any CUDA call."""
    from paper_2301_00611_gb300 import dem
    d = dem.SceneDesc()
    lib.dem_scene_desc_init(ctypes.byref(d))
    d.periodic = 1
    d.cell_h[4] = -1.0  # an inverted cell (sheared cells are accepted, inverted ones not)
    h = ctypes.c_void_p()
    rc = lib.dem_scene_create(ctypes.byref(d), ctypes.byref(h))
    assert rc == 1 and not h.value
    assert b"positive determinant" in lib.dem_last_error(None)
    lib.dem_scene_desc_init(ctypes.byref(d))
    d.damping = 1.5
    assert lib.dem_scene_create(ctypes.byref(d), ctypes.byref(h)) == 1
    lib.dem_scene_desc_init(ctypes.byref(d))
    d.precision = dem.DEM_MIXED + 7
    assert lib.dem_scene_create(ctypes.byref(d), ctypes.byref(h)) == 10
    assert lib.dem_scene_create(None, ctypes.byref(h)) == 1


def test_product_path_never_imports_the_oracle():
    """The CUDA path must not route through the oracle: no package module imports it."""
    pkg = os.path.join(ROOT, "paper_2301_00611_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "dem_oracle" not in text and "liboracle" not in text, f
