"""The C ABI without a GPU: the library loads, exports every symbol include/fbst.h declares, and its
host-only parameter derivation validates input and picks the documented sizes."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import paper_2512_08887_gb300 as fb
from paper_2512_08887_gb300 import _native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2512_08887_gb300.build import build
    build()
    return fb.load_library()


def _declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        with open(os.path.join(ROOT, "include", h)) as f:
            src = re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)
        names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(fbst_\w+)\s*\(", src, flags=re.M))
    return names


def test_every_declared_symbol_is_exported(lib):
    declared = _declared_functions()
    assert {"fbst_plan", "fbst_execute", "fbst_destroy", "fbst_czt", "fbst_toeplitz_apply"} <= declared
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(_native.SIGNATURES), "binding signatures out of sync with the header"


def test_status_strings(lib):
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert lib.fbst_status_string(code).decode().startswith(_native.STATUS_NAMES[code])


def test_derive_paper_sizes(lib):
    # C2: L = 2N = 512; temporal split in two halves of size 2N; spatial pow2(M+B-1) = 512;
    # GS circulant 2L; reconstruction halves of size L.
    info = fb.derive(fb.make_geometry("ula", 256), 256, fb.make_band(0.5))
    assert (info.L, info.P_time, info.S_time, info.P_space_x) == (512, 512, 2, 512)
    assert (info.P_gs, info.P_rec, info.S_rec) == (1024, 512, 2)
    assert (info.eps_num, info.eps_den, info.fb_num, info.fb_den) == (101, 100, 1, 2)
    assert abs(info.rho - 0.2) < 1e-15
    assert abs(info.delta - 1e-3 * 256 * 256) < 1e-9
    assert info.stage2 == fb.STAGE2["gs_ir1"]
    # Eq. (8) bound for a 256-element array at fb = 0.5: rho*(M-1) = 51 < N.
    assert abs(info.snapshot_bound - 0.2 * 255) < 1e-9 and not info.warn_snapshots
    # URA 32x32, fb = 0.3 (3/10).
    info = fb.derive(fb.make_geometry("ura", 32, 32), 512, fb.make_band(0.3))
    assert (info.L, info.P_space_x, info.P_space_y, info.fb_num, info.fb_den) == (1024, 64, 64, 3, 10)


def test_derive_warns_below_snapshot_bound(lib):
    info = fb.derive(fb.make_geometry("ula", 1024), 128, fb.make_band(0.6))
    assert info.warn_snapshots and info.snapshot_bound > 128


@pytest.mark.parametrize("kw,N", [
    (dict(geom=("ula", 8, 2)), 16),                         # linear array with my != 1
    (dict(band=dict(frac_bw=2.5)), 16),                     # fb outside (0, 2)
    (dict(band=dict(frac_bw=0.0)), 16),
    (dict(band=dict(epsilon=0.9)), 16),                     # epsilon < 1
    (dict(band=dict(gamma=(3, 2))), 15),                    # L = 22.5 not an integer
    (dict(band=dict(gamma=(1, 2))), 16),                    # L < N
    (dict(band=dict(delta=0.0)), 16),
    (dict(band=dict(max_blocks=0)), 16),
    (dict(band=dict(stage2="dense_fp32")), 0),              # N = 0
])
def test_derive_rejects_invalid(lib, kw, N):
    g = fb.make_geometry(*kw.get("geom", ("ula", 8)))
    b = fb.make_band(**{"frac_bw": 0.5, **kw.get("band", {})})
    with pytest.raises(fb.FBSTError) as e:
        fb.derive(g, N, b)
    assert e.value.status == -1


def test_derive_rejects_oversized_transforms(lib):
    with pytest.raises(fb.FBSTError) as e:
        fb.derive(fb.make_geometry("ula", 64), 2048, fb.make_band(0.5))  # P_gs = 8192
    assert e.value.status == -4


def test_rational_rounding(lib):
    info = fb.derive(fb.make_geometry("ula", 32), 128, fb.make_band(0.437, epsilon=1.0))
    assert (info.fb_num, info.fb_den, info.eps_num, info.eps_den) == (437, 1000, 1, 1)


def test_nulling_entry_points_check_arguments_before_any_cuda_call(lib):
    # The entry points of Eq. (14) reject missing handles and pointers on the host.
    h = C.c_void_p()
    arr = (C.c_int * 2)(1, 2)
    assert lib.fbst_null_create(None, None, arr, 2, 0, None) == -1
    assert lib.fbst_null_create(C.byref(h), None, arr, 2, 0, None) == -1 and not h.value
    assert lib.fbst_null_apply(None, None, None, 1, None) == -1
    assert lib.fbst_null_execute(None, None, None, 1, None) == -1
    assert lib.fbst_null_launch_count(None, 4) == 0
    assert lib.fbst_null_destroy(None) == 0


def test_generator_solver_field_is_checked(lib):
    for name in ("levinson", "superfast"):
        assert fb.derive(fb.make_geometry("ula", 8), 16, fb.make_band(0.5, generator_solver=name)).L == 32
    band = fb.make_band(0.5)
    band.generator_solver = 2
    with pytest.raises(fb.FBSTError) as e:
        fb.derive(fb.make_geometry("ula", 8), 16, band)
    assert e.value.status == -1


def test_trace_and_generator_entry_points_check_arguments_before_any_cuda_call(lib):
    assert lib.fbst_trace_stages(None, 4) == -1
    assert lib.fbst_trace_read(None, None, 0) == -1
    assert lib.fbst_solve_generators(None, 0, None, None) == -1


def test_positions_are_checked_before_any_cuda_call(lib):
    # fbst_plan_positions (Sec. IX) validates the element positions and the 2-D NUFFT's size on the
    # host, before it touches the device.
    def call(kind, mx, my, bx, by, pos):
        g = fb.make_geometry(kind, mx, my, bx, by)
        arr = (C.c_double * pos.size)(*pos.ravel().tolist())
        h = C.c_void_p()
        return lib.fbst_plan_positions(C.byref(h), C.byref(g), arr, mx * my, 16, bx * by,
                                       C.byref(fb.make_band(0.5)), None, None, None, None), h
    grid = np.stack([np.arange(8.0), np.zeros(8)], axis=1)
    bad = grid.copy()
    bad[3, 0] = np.inf
    assert call("ula", 8, 1, 8, 1, bad)[0] == -1                  # not finite
    bad = grid.copy()
    bad[2, 1] = 0.25
    assert call("ula", 8, 1, 8, 1, bad)[0] == -1                  # y off the axis of a linear array
    ura = np.zeros((4, 2))
    ura[1, 1] = np.nan
    r, h = call("ura", 2, 2, 2, 2, ura)
    assert r == -1 and not h.value                                # not finite, rectangular array
    assert call("ura", 2, 2, 128, 128, np.zeros((4, 2)))[0] == -4  # a 256 x 256 grid: beyond the 2-D kernel
