"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every symbol that
include/i4d.h declares; host-only entry points behave (CPU only, no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2510_01119_gb300 import build, _lib
    build.build()
    return _lib.load()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "i4d.h")).read()
    return sorted(set(re.findall(r"^I4D_API\s+[\w\s\*]+?\b(i4d_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("i4d_slice_project", "i4d_bin_tiles", "i4d_render_fwd", "i4d_render_bwd", "i4d_adam_step",
                     "i4d_prune_points"):
        assert required in names
    assert len(names) >= 17


def test_binding_constants_match_the_header():
    from paper_2510_01119_gb300 import _lib
    text = open(os.path.join(ROOT, "include", "i4d.h")).read()
    const = {k: int(v) for k, v in re.findall(r"^#define (I4D_\w+) \(?(-?\d+)\)?", text, flags=re.M)}
    assert const["I4D_MAX_VIEWS"] == _lib.MAX_VIEWS
    assert const["I4D_GRAD2D_FLOATS"] == _lib.GRAD2D_FLOATS


def test_every_declared_symbol_is_exported(lib):
    from paper_2510_01119_gb300 import _lib
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert set(_lib.exported_names()) == set(declared_symbols())


def test_host_only_entry_points(lib):
    from paper_2510_01119_gb300 import _lib as L
    assert lib.i4d_version() == 1
    s = L.default_settings()
    assert abs(s.alpha_max - 0.99) < 1e-7 and abs(s.alpha_min - 1 / 255) < 1e-9 and s.q_max == 9.0
    v = L.make_views([(128, 96), (30, 17)])
    assert lib.i4d_total_tiles(ctypes.byref(v)) == 8 * 6 + 2 * 2
    assert lib.i4d_total_pixels(ctypes.byref(v)) == 128 * 96 + 30 * 17
    assert lib.i4d_param_floats(0) == 20 and lib.i4d_param_floats(3) == 68
    assert lib.i4d_param_floats(4) == -1
    assert L.i4d_bin_tiles_workspace_size(v, 2000, 1 << 16) > 0
    assert L.i4d_prune_workspace_size(1000, 3) == 0          # table size must be a power of two
    assert L.i4d_prune_workspace_size(1000, 1 << 12) > 0
    assert lib.i4d_status_string(-2) == b"capacity exceeded"


def test_argument_errors_are_reported_not_launched(lib):
    from paper_2510_01119_gb300 import _lib as L
    bad = L.make_views([(128, 96)], tile=(16, 16))
    bad.tile_w = 12                                         # unsupported tile
    g = L.Gaussians()
    g.n, g.sh_deg, g.mode = 10, 0, 0
    s = L.default_settings()
    rc = lib.i4d_slice_project(ctypes.byref(g), ctypes.byref(bad), None, ctypes.byref(s), None, None, None)
    assert rc == -1
    g.sh_deg = 7
    ok = L.make_views([(128, 96)])
    rc = lib.i4d_slice_project(ctypes.byref(g), ctypes.byref(ok), None, ctypes.byref(s), None, None, None)
    assert rc == -1
    assert lib.i4d_adam_step(None, None, None, None, 6, None, 0, None, 0.9, 0.999, 1e-15, None) == -1
    assert lib.i4d_loss(None, None, 10, 5, None, None, None) == -1
    # photometric loss: lambda outside [0, 1]; workspace too small
    fake = ctypes.c_void_p(16)
    assert lib.i4d_photometric_loss(ctypes.byref(ok), fake, fake, ctypes.c_float(1.5), fake, fake, None, fake,
                                    1 << 30, None) == -1
    assert lib.i4d_photometric_loss(ctypes.byref(ok), fake, fake, ctypes.c_float(0.2), fake, fake, None, fake,
                                    8, None) == -4
    assert L.i4d_photometric_loss_workspace_size(ok) >= 9 * 4 * 128 * 96
    # pruning inputs: no frames, non-positive lambda; a negative dynamic voxel edge
    assert lib.i4d_adaptive_voxel(fake, 0, 4, 4, fake, ctypes.c_float(1.0), fake, fake, 1 << 20, None) == -1
    assert lib.i4d_adaptive_voxel(fake, 2, 4, 4, fake, ctypes.c_float(0.0), fake, fake, 1 << 20, None) == -1
    assert lib.i4d_motion_masks(fake, 0, 4, 4, 8, 8, fake, None, fake, 1 << 20, None) == -1
    assert lib.i4d_motion_masks(fake, 2, 4, 4, 8, 8, fake, None, fake, 4, None) == -4
    assert L.i4d_motion_masks_workspace_size(3) >= 3 * 1024 and L.i4d_adaptive_voxel_workspace_size(3) >= 36
    # voxel_dynamic may be 0 (dynamic points unpruned) but not negative
    args = lambda vd: (fake, None, None, None, 100, ctypes.c_float(0.01), ctypes.c_float(vd), 1, 1 << 10, 100,
                       fake, fake, fake, fake, fake, fake, fake, fake, fake, 8, None)
    assert lib.i4d_prune_points_xyz(*args(-0.01)) == -1
    assert lib.i4d_prune_points_xyz(*args(0.0)) == -4            # accepted, then the workspace is too small


def test_no_cpu_fallback_without_library(tmp_path):
    from paper_2510_01119_gb300 import _lib as L
    saved = L._lib
    try:
        L._lib = None
        with pytest.raises(L.I4DError):
            L.load(str(tmp_path / "missing.so"))
    finally:
        L._lib = saved
