"""The C-ABI library builds, loads, exports every entry point its header
declares, and validates arguments on the host (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def _declared():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(drt_\w+)\s*\(", text, re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2401_11882_gb300 import _lib
    return _lib.load()


def test_header_declares_entry_points():
    names = _declared()
    assert {"drt_forward", "drt_vjp", "drt_loss", "drt_num_candidates"} <= names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_binding_covers_every_declared_symbol():
    from paper_2401_11882_gb300 import _lib
    assert _declared() <= set(_lib.SIGNATURES), sorted(_declared() - set(_lib.SIGNATURES))


def test_binding_constants_match_the_header():
    """The binding's copies of the header's #define values (tile flags, limits)."""
    from paper_2401_11882_gb300 import _lib
    text = "".join(open(h).read() for h in HEADERS)
    defs = {m.group(1): int(m.group(2))
            for m in re.finditer(r"^#define\s+DRT_(\w+)\s+(\d+)\b", text, re.M)}
    for name in ("TILE_CULL_INVALID", "TILE_SINGLE_RX", "TILE_EXIT_BLOCKED", "MAX_ORDER",
                 "MAX_WALLS"):
        assert defs[name] == getattr(_lib, name), name
    flags = [v for k, v in defs.items() if k.startswith("TILE_")]
    assert all(f & (f - 1) == 0 for f in flags) and len(set(flags)) == len(flags)


def test_num_candidates_host_only(lib):
    out = ctypes.c_int64()
    assert lib.drt_num_candidates(64, 2, ctypes.byref(out)) == 0 and out.value == 4097
    assert lib.drt_num_candidates(128, 2, ctypes.byref(out)) == 0 and out.value == 16385
    assert lib.drt_num_candidates(0, 1, ctypes.byref(out)) == 1
    assert lib.drt_num_candidates(5, 4, ctypes.byref(out)) == 2      # K above the maximum
    assert lib.drt_num_candidates(5, 1, None) == 1


def test_status_strings(lib):
    assert lib.drt_status_string(0) == b"ok"
    assert lib.drt_status_string(5) == b"workspace too small"


def _scene(**kw):
    from paper_2401_11882_gb300 import _lib
    d = dict(walls=16, n_walls=4, rx=64, n_rx=3, tx=128, max_order=1, alpha=10.0, smoothing=1,
             refl_coef=0.5)
    d.update(kw)
    return _lib.Scene(**d)


@pytest.mark.parametrize("field,value,status", [
    ("n_walls", 0, 1), ("n_walls", 70000, 2), ("max_order", 4, 2), ("max_order", -1, 1),
    ("alpha", -1.0, 1), ("alpha", float("nan"), 1), ("smoothing", 7, 1), ("walls", 0, 1),
    ("walls", 8, 1), ("rx", 4, 1), ("n_rx", -2, 1), ("refl_coef", float("inf"), 1)])
def test_forward_rejects_bad_scene_before_any_launch(lib, field, value, status):
    # Rejected on the host: no CUDA call is made, so this runs without a GPU.
    sc = _scene(**{field: value})
    out = ctypes.c_size_t()
    assert lib.drt_forward_workspace_size(ctypes.byref(sc), None, ctypes.byref(out)) == status
    assert lib.drt_forward(ctypes.byref(sc), None, ctypes.c_void_p(256), None, 0, None) == status
    assert lib.drt_vjp(ctypes.byref(sc), None, ctypes.c_void_p(256), ctypes.c_void_p(256), None,
                       None, 0, None) == status
    assert len(lib.drt_last_error()) > 0


def test_loss_rejects_bad_args(lib):
    p = ctypes.c_void_p(256)
    assert lib.drt_loss(None, 4, p, p, None) == 1
    assert lib.drt_loss(p, 0, p, p, None) == 1
    assert lib.drt_loss_backward(None, None, 4, p, None) == 1


@pytest.mark.parametrize("wavelength,eps_r,refl,field_ptr", [
    (0.0, 5.0, 0.5, 256), (-1.0, 5.0, 0.5, 256), (float("nan"), 5.0, 0.5, 256),
    (float("inf"), 5.0, 0.5, 256), (0.1, 0.5, 0.5, 256), (0.1, -2.0, 0.5, 256),
    (0.1, float("inf"), 0.5, 256), (0.1, 0.0, -0.5, 256), (0.1, 5.0, 0.5, 0),
    (0.1, 5.0, 0.5, 260)])
def test_field_rejects_bad_args_before_any_launch(lib, wavelength, eps_r, refl, field_ptr):
    # Rejected on the host (wavelength, permittivity, coefficient, field pointer).
    sc = _scene(refl_coef=refl)
    p = ctypes.c_void_p(256)
    st = lib.drt_field(ctypes.byref(sc), None, ctypes.c_float(wavelength), ctypes.c_float(eps_r),
                       ctypes.c_void_p(field_ptr), None, p, 1 << 20, None)
    assert st == 1 and len(lib.drt_last_error()) > 0


def test_field_rejects_bad_scene_before_any_launch(lib):
    sc = _scene(n_walls=0)
    out = ctypes.c_size_t()
    assert lib.drt_field_workspace_size(ctypes.byref(sc), None, ctypes.byref(out)) == 1
    assert lib.drt_field(ctypes.byref(sc), None, ctypes.c_float(0.1), ctypes.c_float(5.0),
                         ctypes.c_void_p(256), None, None, 0, None) == 1


@pytest.mark.parametrize("wavelength,eps_r,field_ptr,gp_ptr,gtx_ptr,gw_ptr", [
    (0.0, 5.0, 256, 256, 256, None), (0.1, 0.5, 256, 256, 256, None),
    (0.1, float("nan"), 256, 256, 256, None), (0.1, 5.0, 0, 256, 256, None),
    (0.1, 5.0, 260, 256, 256, None), (0.1, 5.0, 256, 0, 256, None),
    (0.1, 5.0, 256, 256, 0, None), (0.1, 5.0, 256, 256, 256, 264)])
def test_field_vjp_rejects_bad_args_before_any_launch(lib, wavelength, eps_r, field_ptr, gp_ptr,
                                                      gtx_ptr, gw_ptr):
    sc = _scene()
    st = lib.drt_field_vjp(ctypes.byref(sc), None, ctypes.c_float(wavelength),
                           ctypes.c_float(eps_r), ctypes.c_void_p(field_ptr),
                           ctypes.c_void_p(gp_ptr), ctypes.c_void_p(gtx_ptr),
                           None if gw_ptr is None else ctypes.c_void_p(gw_ptr),
                           ctypes.c_void_p(256), 1 << 20, None)
    assert st == 1 and len(lib.drt_last_error()) > 0


def _scene3(**kw):
    from paper_2401_11882_gb300 import _lib
    d = dict(tris=16, n_tris=4, rx=64, n_rx=3, tx=128, max_order=1, alpha=10.0, smoothing=1,
             refl_coef=0.5)
    d.update(kw)
    return _lib.Scene3(**d)


@pytest.mark.parametrize("field,value,status", [
    ("n_tris", 0, 1), ("n_tris", 5000, 2), ("max_order", 4, 2), ("alpha", -1.0, 1),
    ("smoothing", 7, 1), ("tris", 0, 1), ("tris", 2, 1), ("rx", 6, 1), ("n_rx", -1, 1),
    ("refl_coef", float("nan"), 1)])
def test_forward3_rejects_bad_scene_before_any_launch(lib, field, value, status):
    sc = _scene3(**{field: value})
    out = ctypes.c_size_t()
    assert lib.drt3_forward_workspace_size(ctypes.byref(sc), None, ctypes.byref(out)) == status
    assert lib.drt3_forward(ctypes.byref(sc), None, ctypes.c_void_p(256), None, 0, None) == status
    assert len(lib.drt_last_error()) > 0


def test_vjp3_tx_rejects_bad_args_before_any_launch(lib):
    p = ctypes.c_void_p(256)
    sc = _scene3()
    assert lib.drt3_vjp_tx(ctypes.byref(sc), None, p, None, p, 1 << 20, None) == 1
    assert lib.drt3_vjp_tx(ctypes.byref(sc), None, None, p, p, 1 << 20, None) == 1
    bad = _scene3(n_tris=0)
    out = ctypes.c_size_t()
    assert lib.drt3_vjp_tx_workspace_size(ctypes.byref(bad), None, ctypes.byref(out)) == 1


@pytest.mark.parametrize("field,value,status", [
    ("n_walls", 0, 1), ("n_walls", 70000, 2), ("max_order", 4, 2), ("alpha", -1.0, 1),
    ("smoothing", 7, 1), ("walls", 0, 1), ("tx", 0, 1), ("rx", 0, 1), ("n_rx", 0, 1),
    ("refl_coef", float("nan"), 1)])
def test_objective_host_rejects_bad_scene_before_any_copy(lib, field, value, status):
    # host arrays need no alignment (walls = 8 is accepted below); everything else as
    # for drt_forward, checked on the host before any CUDA call
    sc = _scene(walls=8, **{field: value}) if field != "walls" else _scene(walls=value)
    out = ctypes.c_size_t()
    p = ctypes.c_void_p(256)
    assert lib.drt_objective_host_workspace_size(ctypes.byref(sc), None,
                                                 ctypes.byref(out)) == status
    assert lib.drt_objective_host(ctypes.byref(sc), None, p, None, None, p, None, p, 1 << 20,
                                  None) == status
    assert len(lib.drt_last_error()) > 0


def test_objective_host_requires_loss_and_grad_tx(lib):
    sc = _scene(walls=8)
    p = ctypes.c_void_p(256)
    assert lib.drt_objective_host(ctypes.byref(sc), None, None, None, None, p, None, p, 1 << 20,
                                  None) == 1
    assert lib.drt_objective_host(ctypes.byref(sc), None, p, None, None, None, None, p, 1 << 20,
                                  None) == 1
    assert lib.drt_objective_host(None, None, p, None, None, p, None, p, 1 << 20, None) == 1


def test_forward_wall_limits_on_the_host(lib):
    # drt_forward takes up to DRT_MAX_WALLS_STREAMED walls, the other calls DRT_MAX_WALLS;
    # more than 2^31 - 1 candidates is refused everywhere (all before any CUDA call)
    out = ctypes.c_size_t()
    sc = _scene(n_walls=70000)
    assert lib.drt_forward_workspace_size(ctypes.byref(sc), None, ctypes.byref(out)) == 2
    assert b"n_walls" in lib.drt_last_error()
    sc = _scene(n_walls=2000, max_order=3)
    assert lib.drt_forward_workspace_size(ctypes.byref(sc), None, ctypes.byref(out)) == 2
    assert b"candidates" in lib.drt_last_error()
    p = ctypes.c_void_p(256)
    sc = _scene(n_walls=2000, max_order=1)
    assert lib.drt_vjp(ctypes.byref(sc), None, p, p, None, p, 1 << 20, None) == 2


def test_mlp_path_switch_host_only(lib):
    # 0 = mma.sync, 1 = fused tcgen05 inference + mma.sync training (default), 2 = tcgen05
    assert lib.drt_mlp_set_tensor_core_path(3) == 1
    assert lib.drt_mlp_set_tensor_core_path(-1) == 1
    for mode in (0, 2, 1):
        assert lib.drt_mlp_set_tensor_core_path(mode) == 0


def test_batch_plan_dimension_checks(lib):
    # host-only: the plan is built from host copies; nothing is enqueued
    from paper_2401_11882_gb300 import _lib
    off = (ctypes.c_int32 * 2)(0, 20)
    roff = (ctypes.c_int32 * 2)(0, 40)
    order = (ctypes.c_int32 * 1)(1)
    plan = ctypes.c_void_p()
    b = _lib.Batch(256, 256, 256, 256, 256, ctypes.addressof(off), ctypes.addressof(roff),
                   ctypes.addressof(order), 1, 2, 1, 0.5, 5)
    assert lib.drt_batch_plan_create(ctypes.byref(b), None, ctypes.byref(plan)) == 1
    assert b"dim" in lib.drt_last_error()
    # 3D arrays need 4-byte alignment only (2D walls need 16)
    b3 = _lib.Batch(260, 256, 260, 256, 256, ctypes.addressof(off), ctypes.addressof(roff),
                    ctypes.addressof(order), 1, 2, 1, 0.5, 3)
    assert lib.drt_batch_plan_create(ctypes.byref(b3), None, ctypes.byref(plan)) == 0
    n = ctypes.c_size_t()
    assert lib.drt_batch_workspace_size(plan, ctypes.byref(n)) == 0 and n.value > 0
    assert lib.drt_batch_plan_destroy(plan) == 0
    b2 = _lib.Batch(260, 256, 260, 256, 256, ctypes.addressof(off), ctypes.addressof(roff),
                    ctypes.addressof(order), 1, 2, 1, 0.5, 2)
    assert lib.drt_batch_plan_create(ctypes.byref(b2), None, ctypes.byref(plan)) == 1


def test_saved_visibilities_size_host_only(lib):
    out = ctypes.c_int64()
    sc = _scene(n_walls=4, n_rx=3, max_order=1, smoothing=0)    # sigmoid
    assert lib.drt_saved_vis_size(ctypes.byref(sc), ctypes.byref(out)) == 0
    assert out.value == (1 + 4) * 2 * 3                        # N_K (K + 1) R
    sc = _scene(n_walls=4, n_rx=3, max_order=1, smoothing=1)    # hard sigmoid: not kept
    assert lib.drt_saved_vis_size(ctypes.byref(sc), ctypes.byref(out)) == 2
    assert b"sigmoid" in lib.drt_last_error()
    p = ctypes.c_void_p(256)
    assert lib.drt_forward_save(ctypes.byref(sc), None, p, p, p, 1 << 20, None) == 2
    assert lib.drt_vjp_saved(ctypes.byref(sc), None, p, p, p, None, p, 1 << 20, None) == 2
    # the coherent field's pair: also refused for the hard sigmoid, and for a NULL
    # buffer with the sigmoid, before anything is enqueued
    f = ctypes.c_float
    assert lib.drt_field_save(ctypes.byref(sc), None, f(0.02), f(5.0), p, p, p, p, 1 << 20,
                              None) == 2
    assert lib.drt_field_vjp_saved(ctypes.byref(sc), None, f(0.02), f(5.0), p, p, p, p, None,
                                   p, 1 << 20, None) == 2
    sg = _scene(n_walls=4, n_rx=3, max_order=1, smoothing=0)
    assert lib.drt_field_save(ctypes.byref(sg), None, f(0.02), f(5.0), p, p, None, p, 1 << 20,
                              None) == 1
    assert lib.drt_field_vjp_saved(ctypes.byref(sg), None, f(0.02), f(5.0), p, p, None, p,
                                   None, p, 1 << 20, None) == 1
