"""Host-side checks of the C ABI that need no GPU: the library builds for sm_103a, loads, exports
every entry point include/gvx.h declares, and rejects invalid arguments before touching CUDA."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import paper_2312_02756_gb300 as gvx
    return gvx.load_library()


def _declared():
    src = open(os.path.join(ROOT, "include", "gvx.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return set(re.findall(r"\b(gvx_[a-z0-9_]+)\s*\(", src))


def test_exports_every_declared_symbol(lib):
    from paper_2312_02756_gb300 import _lib
    declared = _declared()
    assert declared == set(_lib.EXPORTS)
    for name in declared:
        assert getattr(lib, name) is not None


def test_version_and_status_strings(lib):
    assert re.match(rb"^\d+\.\d+\.\d+$", lib.gvx_version())
    for code in range(13):
        assert lib.gvx_status_string(code).startswith(b"GVX_")
    assert lib.gvx_status_string(12).startswith(b"GVX_ERR_BOUNDS")
    assert lib.gvx_status_string(99) == b"unknown gvx status"


def _lv(layout=0, ptrs=(0, 0, 0, 0)):
    from paper_2312_02756_gb300._lib import LV
    v = LV()
    v.layout = layout
    for k, p in enumerate(ptrs):
        v.c[k] = p
    return v


def test_mass_validation(lib):
    good = _lv(0, (64, 128, 192, 256))
    r = ctypes.byref
    assert lib.gvx_invariant_mass(r(good), r(good), 512, 10, 7, None) == 3   # dtype
    assert lib.gvx_invariant_mass(r(good), r(good), 512, -1, 0, None) == 2   # size
    assert lib.gvx_invariant_mass(r(good), r(good), 512, 0, 0, None) == 0    # n = 0: no-op
    assert lib.gvx_invariant_mass(None, r(good), 512, 10, 0, None) == 1      # null
    assert lib.gvx_invariant_mass(r(_lv(0)), r(good), 512, 10, 0, None) == 1
    assert lib.gvx_invariant_mass(r(good), r(good), None, 10, 0, None) == 1
    assert lib.gvx_invariant_mass(r(_lv(0, (64, 128, 196, 256))), r(good), 512, 10, 0, None) == 5
    assert lib.gvx_invariant_mass(r(good), r(good), 516, 10, 0, None) == 5   # misaligned out
    assert lib.gvx_invariant_mass(r(_lv(1, (48, 0, 0, 0))), r(good), 512, 10, 0, None) == 5
    assert lib.gvx_invariant_mass(r(_lv(2, (64, 0, 0, 0))), r(good), 512, 10, 0, None) == 4
    assert lib.gvx_invariant_mass_bwd(r(good), r(good), None, 512, r(good), None, 10, 0, None) == 1
    assert lib.gvx_invariant_mass_bwd(r(good), r(good), 4, 512, r(good), r(good), 10, 0, None) == 5


def test_boost_validation(lib):
    r = ctypes.byref
    v = _lv(0, (64, 128, 192, 256))
    beta = _lv(1, (8, 0, 0, 0))
    assert lib.gvx_boost(r(v), r(beta), 2, r(v), 10, 0, None) == 11          # stride
    assert lib.gvx_boost(r(v), r(_lv(0, (8, 16, 0, 0))), 1, r(v), 10, 0, None) == 1
    assert lib.gvx_boost(r(v), r(_lv(1, (4, 0, 0, 0))), 1, r(v), 10, 0, None) == 5
    assert lib.gvx_boost(r(v), r(beta), 1, r(v), 0, 0, None) == 0
    assert lib.gvx_boost_bwd(r(v), r(beta), 3, r(v), r(v), r(beta), 10, 0, None, 0, None) == 11


def test_jagged_validation(lib):
    r = ctypes.byref
    p = _lv(1, (256, 0, 0, 0))
    sums = _lv(1, (512, 0, 0, 0))
    ws_need = lib.gvx_event_pair_masses_workspace(1000)
    assert ws_need == 256 + 8 * ((1000 + 63) // 64)
    assert lib.gvx_event_pair_masses_workspace(0) == 0
    args = lambda n_ev, off, ws, wsb: (r(p), off, n_ev, 100, 1024, 2048, 50, r(sums), ws, wsb, None)
    assert lib.gvx_event_pair_masses(*args(-1, 64, 4096, ws_need)) == 2
    assert lib.gvx_event_pair_masses(*args(1000, None, 4096, ws_need)) == 1
    assert lib.gvx_event_pair_masses(*args(1000, 68, 4096, ws_need)) == 5
    assert lib.gvx_event_pair_masses(*args(1000, 64, 4096, ws_need - 8)) == 7
    assert lib.gvx_event_pair_masses(*args(1000, 64, None, ws_need)) == 7
    assert lib.gvx_event_pair_masses(*args(1000, 64, 4100, ws_need)) == 5
    # the adjoint: 256 bytes of header, then one int64 per tile of 14 events
    wb = lib.gvx_event_pair_masses_bwd_workspace(1000)
    assert wb == 256 + 8 * ((1000 + 13) // 14)
    assert lib.gvx_event_pair_masses_bwd_workspace(0) == 0
    bargs = lambda n_ev, ws, wsb: (r(p), 64, 128, n_ev, 100, 4096, 50, None, r(p), ws, wsb, None)
    assert lib.gvx_event_pair_masses_bwd(*bargs(1000, None, wb)) == 7
    assert lib.gvx_event_pair_masses_bwd(*bargs(1000, 4096, wb - 8)) == 7
    assert lib.gvx_event_pair_masses_bwd(*bargs(1000, 4104, wb)) == 5
    assert lib.gvx_event_pair_masses_bwd(*bargs(0, None, 0)) == 0  # nothing to do
    assert lib.gvx_event_pair_masses_set_shape(1000, 99) == 11
    n = lib.gvx_event_pair_masses_num_shapes()
    assert n >= 2
    te, nt = ctypes.c_int32(), ctypes.c_int32()
    for s in range(n):
        assert lib.gvx_event_pair_masses_shape(s, r(te), r(nt)) == 0
        assert 0 < te.value <= nt.value and nt.value % 32 == 0
    assert lib.gvx_event_pair_masses_shape(n, r(te), r(nt)) == 11
    assert lib.gvx_graph_launch(None, None) == 1
    assert lib.gvx_graph_destroy(None) == 0
    assert lib.gvx_device_status(None, None) == 1


def test_no_cpu_fallback_in_package():
    """The product path has no CPU or oracle route: the package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2312_02756_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"(import\s+oracle|from\s+oracle|liboracle|gvx_oracle)", src), f


def test_coordinate_and_transformation_validation(lib):
    """gvx_invariant_mass_cart, gvx_to_pxpypze and gvx_lorentz_apply reject bad coordinate codes,
    dtypes, sizes, null and misaligned pointers on the host (status codes of include/gvx.h)."""
    good = _lv(0, (64, 128, 192, 256))
    r = ctypes.byref
    ARG, SIZE, DTYPE, NULL, ALIGN = 11, 2, 3, 1, 5
    # pair masses in other coordinate systems: coords 1 (PxPyPzE), 2 (PxPyPzM), 3 (PtEtaPhiE)
    for coords in (1, 2, 3):
        assert lib.gvx_invariant_mass_cart(r(good), r(good), 512, 0, coords, 0, None) == 0
        assert lib.gvx_invariant_mass_cart(r(good), r(good), 512, -1, coords, 0, None) == SIZE
        assert lib.gvx_invariant_mass_cart(r(good), r(good), None, 10, coords, 0, None) == NULL
        assert lib.gvx_invariant_mass_cart(r(good), r(good), 516, 10, coords, 0, None) == ALIGN
        assert lib.gvx_invariant_mass_cart(r(good), r(good), 512, 10, coords, 9, None) == DTYPE
    assert lib.gvx_invariant_mass_cart(r(good), r(good), 512, 10, 4, 0, None) == ARG
    assert lib.gvx_invariant_mass_cart(r(good), r(good), 512, 10, -1, 0, None) == ARG
    # conversion: PtEtaPhiM (0), PxPyPzM (2), PtEtaPhiE (3); PxPyPzE (1) has nothing to convert
    for coords in (0, 2, 3):
        assert lib.gvx_to_pxpypze(r(good), r(good), 0, coords, 0, None) == 0
        assert lib.gvx_to_pxpypze(r(good), r(good), -3, coords, 0, None) == SIZE
        assert lib.gvx_to_pxpypze(None, r(good), 10, coords, 0, None) == NULL
        assert lib.gvx_to_pxpypze(r(good), r(_lv(0)), 10, coords, 0, None) == NULL
        assert lib.gvx_to_pxpypze(r(good), r(good), 10, coords, 5, None) == DTYPE
    assert lib.gvx_to_pxpypze(r(good), r(good), 10, 1, 0, None) == ARG
    assert lib.gvx_to_pxpypze(r(good), r(good), 10, 7, 0, None) == ARG
    # general transformation: l_stride 0 or 1, L aligned to a scalar (shared) or 16 bytes
    assert lib.gvx_lorentz_apply(ctypes.c_void_p(64), 2, r(good), r(good), 10, 0, None) == ARG
    assert lib.gvx_lorentz_apply(None, 0, r(good), r(good), 10, 0, None) == NULL
    assert lib.gvx_lorentz_apply(ctypes.c_void_p(72), 1, r(good), r(good), 10, 0, None) == ALIGN
    assert lib.gvx_lorentz_apply(ctypes.c_void_p(68), 0, r(good), r(good), 10, 0, None) == ALIGN
    assert lib.gvx_lorentz_apply(ctypes.c_void_p(64), 0, r(good), r(good), -1, 0, None) == SIZE


def test_python_coordinate_names():
    """The Python bindings name the coordinate systems; an unknown name is a ValueError."""
    import paper_2312_02756_gb300 as gvx
    assert gvx._coords_code("ptetaphie") == 3 and gvx._coords_code("pxpypze") == 1
    with pytest.raises(ValueError):
        gvx._coords_code("xyzt")


def test_debug_bounds_variant_compiles(tmp_path):
    """The GVX_DEBUG_BOUNDS variant of the jagged kernels (explicit index checks that record
    GVX_ERR_BOUNDS) compiles for sm_103a, and selecting it changes the library's file name (so
    the two builds never overwrite each other)."""
    import subprocess
    import sys
    from paper_2312_02756_gb300 import build as b
    b.generate_tables()
    for name in ("jagged.cu", "jagged_bwd.cu"):
        cmd = [b.nvcc(), *b.ARCH, *b.NVCC_FLAGS, "-DGVX_DEBUG_BOUNDS", "-c",
               os.path.join(b.CSRC, name), "-o", str(tmp_path / (name + ".o"))]
        subprocess.run(cmd, check=True, capture_output=True)
    code = "from paper_2312_02756_gb300 import build as b; print(b.LIB_PATH)"
    env = dict(os.environ, GVX_DEBUG_BOUNDS="1")
    out = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, check=True,
                         capture_output=True, text=True).stdout.strip()
    assert os.path.basename(out).startswith("libgvx_dbg_") and out != b.LIB_PATH
