"""The C ABI: libwdd.so loads, exports every entry point include/wdd.h declares, the binding's
struct layouts match the C compiler's, and host-side validation errors need no GPU."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "wdd.h")


@pytest.fixture(scope="module")
def wdd():
    from paper_2212_01309_gb300 import build, wdd
    if not os.path.exists(wdd.LIB_PATH):
        build.build()
    wdd.lib()
    return wdd


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(wdd_[a-z_]+)\s*\(", text)))


def test_header_declares_expected_entry_points():
    names = declared_functions()
    for required in ("wdd_plan_create", "wdd_push_frames", "wdd_snapshot", "wdd_finalize",
                     "wdd_plan_destroy", "wdd_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(wdd):
    L = wdd.lib()
    for name in declared_functions():
        assert hasattr(L, name), name
    assert set(wdd.exported_symbols()) >= set(declared_functions())


def test_library_resolves_every_symbol_at_load(wdd):
    """A shared library links with undefined symbols; binding them all at load time catches an
    internal function that no translation unit defines."""
    ctypes.CDLL(wdd.LIB_PATH, mode=os.RTLD_NOW)


def test_status_strings(wdd):
    L = wdd.lib()
    assert L.wdd_status_string(0) == b"WDD_OK"
    assert L.wdd_status_string(4) == b"WDD_ERR_SCAN_INDEX"
    assert L.wdd_version() >> 16 == 0


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not available")
def test_struct_layout_matches_c(wdd, tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "wdd.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n\", sizeof(wdd_params),"
        " offsetof(wdd_params, rank_k), offsetof(wdd_params, det_center_y),"
        " offsetof(wdd_params, hbm_budget_bytes), sizeof(wdd_result), sizeof(wdd_plan_info),"
        " offsetof(wdd_params, overlap_pushes), offsetof(wdd_params, proj_cluster),"
        " offsetof(wdd_params, accum_segment), offsetof(wdd_params, accum_mode),"
        " offsetof(wdd_plan_info, proj_tensor), offsetof(wdd_params, scan_rotation_rad));"
        "return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True,
                                       check=True).stdout.split()))
    P = wdd.Params
    assert got == [ctypes.sizeof(P), P.rank_k.offset, P.det_center_y.offset,
                   P.hbm_budget_bytes.offset, ctypes.sizeof(wdd.Result),
                   ctypes.sizeof(wdd.PlanInfo), P.overlap_pushes.offset, P.proj_cluster.offset,
                   P.accum_segment.offset, P.accum_mode.offset, wdd.PlanInfo.proj_tensor.offset,
                   P.scan_rotation_rad.offset]


def test_invalid_params_rejected_on_host(wdd):
    L = wdd.lib()
    p = wdd.Params()
    assert L.wdd_params_default(ctypes.byref(p)) == 0
    h = ctypes.c_void_p()
    # zero geometry
    assert L.wdd_plan_create(ctypes.byref(p), ctypes.byref(h)) == wdd.ERR_INVALID_ARG
    assert b"positive" in L.wdd_last_error()
    p2 = wdd.make_params(scan_y=8, scan_x=8, scan_step_m=1e-10, det_y=16, det_x=16,
                         det_px_inv_m=1e9, voltage_v=3e5, semiconv_rad=0.02, rank_k=15)
    assert L.wdd_plan_create(ctypes.byref(p2), ctypes.byref(h)) == wdd.ERR_INVALID_ARG  # not square
    p3 = wdd.make_params(scan_y=8, scan_x=8, scan_step_m=1e-10, det_y=128, det_x=128,
                         det_px_inv_m=1e9, voltage_v=3e5, semiconv_rad=0.02,
                         rank_k=128 * 128, basis="fourier_full")
    assert L.wdd_plan_create(ctypes.byref(p3), ctypes.byref(h)) == wdd.ERR_UNSUPPORTED
    p4 = wdd.make_params(scan_y=8, scan_x=8, scan_step_m=1e-10, det_y=16, det_x=16,
                         det_px_inv_m=1e9, voltage_v=3e5, semiconv_rad=0.02, rank_k=16,
                         epsilon=-1.0)
    assert L.wdd_plan_create(ctypes.byref(p4), ctypes.byref(h)) == wdd.ERR_INVALID_ARG
    assert L.wdd_plan_create(None, ctypes.byref(h)) == wdd.ERR_INVALID_ARG
    assert L.wdd_push_frames(None, None, None, 0, None) == wdd.ERR_INVALID_ARG
    assert L.wdd_snapshot(None, None) == wdd.ERR_INVALID_ARG
    assert L.wdd_plan_destroy(None) == wdd.ERR_INVALID_ARG


def test_plan_footprint_without_gpu(wdd):
    """The footprint call validates like plan creation and sizes the plan without a GPU."""
    small = wdd.make_params(scan_y=32, scan_x=32, scan_step_m=1e-10, det_y=32, det_x=32,
                            det_px_inv_m=1e9, voltage_v=3e5, semiconv_rad=0.02, rank_k=64)
    big = wdd.make_params(scan_y=256, scan_x=256, scan_step_m=1e-10, det_y=128, det_x=128,
                          det_px_inv_m=1e9, voltage_v=3e5, semiconv_rad=0.02, rank_k=256,
                          precision="split", accum_depth=4096)
    a, b = wdd.plan_footprint(small), wdd.plan_footprint(big)
    assert 0 < a < b
    # W and H alone: 2 x S x K x 8 bytes
    assert b >= 2 * 65536 * 256 * 8
    bad = wdd.make_params(scan_y=32, scan_x=32, scan_step_m=1e-10, det_y=32, det_x=32,
                          det_px_inv_m=1e9, voltage_v=3e5, semiconv_rad=0.02, rank_k=63)
    with pytest.raises(wdd.WddError):
        wdd.plan_footprint(bad)


def test_classical_plan_footprint_and_validation_without_gpu(wdd):
    """The classical plan holds the scan spectrum and the Wiener kernel, S x N^2 complex64 each;
    its footprint and its parameter checks need no GPU."""
    kw = dict(scan_step_m=1e-10, det_px_inv_m=1e9, voltage_v=3e5, semiconv_rad=0.02, rank_k=1)
    p = wdd.make_params(scan_y=128, scan_x=128, det_y=128, det_x=128, **kw)
    b = wdd.offline_footprint(p)
    big = 2 * 128 * 128 * 128 * 128 * 8
    assert big <= b < big + (1 << 22)
    # against the live plan of the same geometry (the memory contrast of the comparison)
    live = wdd.plan_footprint(wdd.make_params(scan_y=128, scan_x=128, det_y=128, det_x=128,
                                              **dict(kw, rank_k=64)))
    assert live * 50 < b
    # a detector centre off pixel N/2 cannot be moved to pixel 0 by an integer roll
    off = wdd.make_params(scan_y=8, scan_x=8, det_y=32, det_x=32, det_center_y=15.5, **kw)
    with pytest.raises(wdd.WddError) as ei:
        wdd.offline_footprint(off)
    assert ei.value.status == wdd.ERR_UNSUPPORTED
    at_half = wdd.make_params(scan_y=8, scan_x=8, det_y=32, det_x=32, det_center_y=16.0,
                              det_center_x=16.0, **kw)
    assert wdd.offline_footprint(at_half) > 0
    for bad in (dict(epsilon=-1.0), dict(scan_rotation_rad=float("nan")),
                dict(frame_dtype=7)):
        q = wdd.make_params(scan_y=8, scan_x=8, det_y=32, det_x=32, **dict(kw, **bad))
        with pytest.raises(wdd.WddError) as ei:
            wdd.offline_footprint(q)
        assert ei.value.status == wdd.ERR_INVALID_ARG
    L = wdd.lib()
    h = ctypes.c_void_p()
    assert L.wdd_offline_plan_create(None, ctypes.byref(h)) == wdd.ERR_INVALID_ARG
    assert L.wdd_offline_reconstruct(None, None, None, None) == wdd.ERR_INVALID_ARG
    assert L.wdd_offline_plan_destroy(None) == wdd.ERR_INVALID_ARG


def test_probe_plan_validation_without_gpu(wdd):
    """The probe-reconstruction plan (the swapped deconvolution) refuses a missing object
    estimate and a rotated scan before touching the GPU."""
    import numpy as np
    kw = dict(scan_y=8, scan_x=8, scan_step_m=1e-10, det_y=32, det_x=32, det_px_inv_m=1e9,
              voltage_v=3e5, semiconv_rad=0.02, rank_k=1)
    L = wdd.lib()
    h = ctypes.c_void_p(1)
    p = wdd.make_params(**kw)
    assert L.wdd_offline_probe_plan_create(ctypes.byref(p), None, ctypes.byref(h)) == \
        wdd.ERR_INVALID_ARG
    assert h.value is None
    est = np.ones(64, dtype=np.complex64)
    rot = wdd.make_params(scan_rotation_rad=0.3, **kw)
    assert L.wdd_offline_probe_plan_create(ctypes.byref(rot), ctypes.c_void_p(est.ctypes.data),
                                           ctypes.byref(h)) == wdd.ERR_UNSUPPORTED
    bad = wdd.make_params(**dict(kw, epsilon=-1.0))
    assert L.wdd_offline_probe_plan_create(ctypes.byref(bad), ctypes.c_void_p(est.ctypes.data),
                                           ctypes.byref(h)) == wdd.ERR_INVALID_ARG
    # the Wiener update of a live plan from a recovered probe
    assert L.wdd_plan_set_probe(None, ctypes.c_void_p(est.ctypes.data)) == wdd.ERR_INVALID_ARG
    # merging an exported state
    assert L.wdd_merge_state(None, None, None, 0) == wdd.ERR_INVALID_ARG


def test_rotation_and_centre_validation_without_gpu(wdd):
    kw = dict(scan_y=8, scan_x=8, scan_step_m=1e-10, det_y=32, det_x=32, det_px_inv_m=1e9,
              voltage_v=3e5, semiconv_rad=0.02, rank_k=16)
    assert wdd.plan_footprint(wdd.make_params(scan_rotation_rad=1.2, **kw)) > 0
    with pytest.raises(wdd.WddError) as ei:
        wdd.plan_footprint(wdd.make_params(scan_rotation_rad=float("inf"), **kw))
    assert ei.value.status == wdd.ERR_INVALID_ARG
    L = wdd.lib()
    cy, cx = ctypes.c_double(), ctypes.c_double()
    assert L.wdd_detector_center(None, 1, 8, 8, 1, ctypes.byref(cy), ctypes.byref(cx),
                                 None) == wdd.ERR_INVALID_ARG
