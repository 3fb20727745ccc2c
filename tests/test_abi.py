"""The C-ABI library loads and exports every function include/vt.h declares
(no GPU needed: nothing here launches a kernel)."""

import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_names():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            with open(os.path.join(ROOT, "include", fn)) as f:
                names += re.findall(r"^VT_API\s+[\w\s\*]*?\b(vt_\w+)\s*\(", f.read(), flags=re.M)
    return names


def test_header_declares_the_boundary():
    names = set(_header_names())
    for required in ("vt_pyramid_build", "vt_gradients", "vt_klt_track", "vt_fb_check", "vt_pyramid_level",
                     "vt_pyramid_free", "vt_status_str"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import paper_2607_01757_gb300 as vt

    lib = C.CDLL(vt.LIB_PATH)
    missing = [n for n in _header_names() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(vt.header_functions()) == set(_header_names())


def test_status_strings_and_version():
    import paper_2607_01757_gb300 as vt

    assert vt.vt_status_str(vt.VT_OK) == "VT_OK"
    assert "invalid argument" in vt.vt_status_str(vt.VT_ERR_ARG)
    assert "sm_103a" in vt.vt_version()


def test_argument_errors_need_no_device():
    """Invalid arguments are rejected on the host before any CUDA call."""
    import paper_2607_01757_gb300 as vt

    lib = C.CDLL(vt.LIB_PATH)
    lib.vt_klt_track.restype = C.c_int
    lib.vt_pyramid_build.restype = C.c_int
    out = C.c_void_p()
    # w = 0, null image, too many levels
    assert lib.vt_pyramid_build(C.c_void_p(1), 0, 10, 10, 1, 0, None, C.byref(out)) == vt.VT_ERR_ARG
    assert lib.vt_pyramid_build(None, 10, 10, 10, 1, 0, None, C.byref(out)) == vt.VT_ERR_ARG
    assert lib.vt_pyramid_build(C.c_void_p(1), 10, 10, 10, 9, 0, None, C.byref(out)) == vt.VT_ERR_ARG
    assert lib.vt_pyramid_build(C.c_void_p(1), 10, 10, 5, 1, 0, None, C.byref(out)) == vt.VT_ERR_ARG
    # null pyramids
    assert lib.vt_klt_track(None, None, None, 0, None, 21, 4, 30, C.c_float(0.01), None, None, None, None) \
        == vt.VT_ERR_ARG
    lib.vt_fb_check.restype = C.c_int
    assert lib.vt_fb_check(None, None, None, None, -1, C.c_float(0.5), None, None) == vt.VT_ERR_ARG


@pytest.mark.parametrize("win", [9, 15, 21, 31])
def test_supported_windows_match_header(win):
    import paper_2607_01757_gb300 as vt

    with open(os.path.join(ROOT, "include", "vt.h")) as f:
        m = re.search(r"#define VT_SUPPORTED_WINDOWS \{([^}]*)\}", f.read())
    assert win in [int(t) for t in m.group(1).split(",")]
    assert win in vt.SUPPORTED_WINDOWS


def test_stereo_gate_argument_errors_need_no_device():
    import paper_2607_01757_gb300 as vt

    f = vt.vt_stereo_gate
    rig = vt.StereoRig((460.0, 460.0, 375.5, 239.5), (460.0, 460.0, 375.5, 239.5), t=(-0.11, 0.0, 0.0))
    prm = vt.GateParams()
    from paper_2607_01757_gb300.vt import _lib as lib

    one = C.c_void_p(16)
    call = lambda n, r, p, pl=one, st=one: lib.vt_stereo_gate(pl, one, None, n, C.byref(r), C.byref(p), None, st,
                                                            None, None)  # noqa: E731
    assert call(0, rig.c(), prm.c()) == vt.VT_OK  # n == 0 launches nothing
    assert call(-1, rig.c(), prm.c()) == vt.VT_ERR_ARG
    assert call(5, rig.c(), prm.c(), pl=None) == vt.VT_ERR_ARG
    assert call(5, rig.c(), prm.c(), st=None) == vt.VT_ERR_ARG
    bad = rig.c()
    bad.kl[0] = 0.0
    assert call(5, bad, prm.c()) == vt.VT_ERR_ARG
    bad = rig.c()
    bad.R[4] = float("nan")
    assert call(5, bad, prm.c()) == vt.VT_ERR_ARG
    for p in (vt.GateParams(min_disp=-1.0), vt.GateParams(z_min=5.0, z_max=1.0), vt.GateParams(max_reproj=-0.1),
              vt.GateParams(z_min=float("nan"))):
        assert call(5, rig.c(), p.c()) == vt.VT_ERR_ARG
    with pytest.raises(vt.VTError):
        f(np.zeros((3, 2), np.float32), np.zeros((3, 2), np.float32), rig, vt.GateParams(min_disp=-2.0),
          np.zeros(3, np.uint8), stream=0)


def test_bookkeeping_and_detector_argument_errors_need_no_device():
    import paper_2607_01757_gb300 as vt
    from paper_2607_01757_gb300.vt import _lib as lib

    one = C.c_void_p(16)
    pool = vt.vt_track_pool(one, one, one, one, one, 100)
    job = vt.vt_carry_job(pool, one, one, None)
    jobs = (vt.vt_carry_job * 1)(job)
    assert lib.vt_tracks_carry(jobs, 0, C.c_float(8.0), None) == vt.VT_OK  # nothing to do
    assert lib.vt_tracks_carry(jobs, -1, C.c_float(8.0), None) == vt.VT_ERR_ARG
    assert lib.vt_tracks_carry(jobs, 1, C.c_float(0.0), None) == vt.VT_ERR_ARG  # min_dist must be > 0
    assert lib.vt_tracks_carry(jobs, 1, C.c_float(float("nan")), None) == vt.VT_ERR_ARG
    assert lib.vt_tracks_carry(jobs, 193, C.c_float(8.0), None) == vt.VT_ERR_ARG  # more jobs than one launch holds
    for bad_cap in (0, vt.VT_POOL_MAX + 1):
        bad = (vt.vt_carry_job * 1)(vt.vt_carry_job(vt.vt_track_pool(one, one, one, one, one, bad_cap), one, one,
                                                    None))
        assert lib.vt_tracks_carry(bad, 1, C.c_float(8.0), None) == vt.VT_ERR_ARG
    nop = (vt.vt_carry_job * 1)(vt.vt_carry_job(pool, None, one, None))
    assert lib.vt_tracks_carry(nop, 1, C.c_float(8.0), None) == vt.VT_ERR_ARG  # no tracked positions
    sj = (vt.vt_spawn_job * 1)(vt.vt_spawn_job(pool, None, one, None))
    assert lib.vt_tracks_spawn(sj, 1, None) == vt.VT_ERR_ARG  # no corners
    prm = vt.GfttParams().c()
    gj = (vt.vt_gftt_job * 1)()
    assert lib.vt_gftt_detect_many(None, gj, 1, C.byref(prm), None) == vt.VT_ERR_ARG
