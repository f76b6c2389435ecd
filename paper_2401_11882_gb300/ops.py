"""PyTorch-facing calls of the library: argument marshalling over the C ABI.

Every step of the computation runs in the CUDA kernels of libdrt.so; this
module only checks tensors, provides workspace memory from PyTorch's
allocator, passes raw device pointers and the current CUDA stream, and wraps
the forward / adjoint pair as a ``torch.autograd.Function``.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import _lib


@dataclass(frozen=True)
class TileConfig:
    """Work decomposition of the path kernels (0 = library default)."""

    warps_per_cta: int = 0
    cands_per_unit: int = 0
    ctas_per_sm: int = 0
    cull_invalid: bool = False
    single_rx: bool = False   # (hard) sigmoid forward: one receiver per lane instead of two
    exit_blocked: bool = False   # hard sigmoid forward: leave the wall loop of blocked warps

    def as_c(self) -> _lib.Tile:
        flags = ((_lib.TILE_CULL_INVALID if self.cull_invalid else 0)
                 | (_lib.TILE_SINGLE_RX if self.single_rx else 0)
                 | (_lib.TILE_EXIT_BLOCKED if self.exit_blocked else 0))
        return _lib.Tile(self.warps_per_cta, self.cands_per_unit, self.ctas_per_sm, flags)


def _stream_ptr(device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _ptr(t: torch.Tensor) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


def _as_f32(t: torch.Tensor, shape_last: int | None, name: str, align: int) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    t = t.detach()
    if t.dtype != torch.float32:
        raise TypeError(f"{name} must be float32, got {t.dtype}")
    if shape_last is not None and (t.dim() != 2 or t.shape[1] != shape_last):
        raise ValueError(f"{name} must have shape [n, {shape_last}]")
    if not t.is_contiguous() or t.data_ptr() % align:
        t = t.contiguous().clone()
    return t


def _workspace(device: torch.device, nbytes: int) -> torch.Tensor:
    """Scratch memory from PyTorch's stream-aware caching allocator."""
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def make_scene(walls: torch.Tensor, tx: torch.Tensor, rx: torch.Tensor, max_order: int,
               alpha: float, smoothing: str, refl_coef: float = 0.5):
    """Validate tensors and build the C scene descriptor (keeps tensors alive)."""
    walls = _as_f32(walls, 4, "walls", 16)
    rx = _as_f32(rx, 2, "rx", 8)
    tx = _as_f32(tx.reshape(1, 2), 2, "tx", 4)
    if walls.device != rx.device or walls.device != tx.device:
        raise ValueError("walls, tx and rx must be on the same device")
    if smoothing not in _lib.SMOOTHING:
        raise ValueError(f"unknown smoothing {smoothing!r}")
    sc = _lib.Scene(walls.data_ptr(), walls.shape[0], rx.data_ptr(), rx.shape[0], tx.data_ptr(),
                    int(max_order), float(alpha), _lib.SMOOTHING[smoothing], float(refl_coef))
    return sc, (walls, tx, rx)


def num_candidates(n_walls: int, max_order: int) -> int:
    out = ctypes.c_int64()
    _lib.call("drt_num_candidates", n_walls, max_order, ctypes.byref(out))
    return out.value


def forward(walls, tx, rx, max_order: int, alpha: float, smoothing: str = "hard_sigmoid",
            refl_coef: float = 0.5, tile: TileConfig | None = None,
            out: torch.Tensor | None = None) -> torch.Tensor:
    """Received power per receiver (float32 [R]) on the current stream.

    ``tile``: a TileConfig, None (library defaults) or "auto" (autotuned, cached)."""
    if isinstance(tile, str):
        if tile != "auto":
            raise ValueError("tile must be a TileConfig, None or 'auto'")
        from . import autotune
        tile = autotune.tune_forward(walls, tx, rx, max_order, alpha, smoothing, refl_coef)
    sc, keep = make_scene(walls, tx, rx, max_order, alpha, smoothing, refl_coef)
    dev = keep[0].device
    tl = tile.as_c() if tile else None
    tlp = ctypes.byref(tl) if tl is not None else None
    nbytes = ctypes.c_size_t()
    _lib.call("drt_forward_workspace_size", ctypes.byref(sc), tlp, ctypes.byref(nbytes))
    ws = _workspace(dev, nbytes.value)
    power = out if out is not None else torch.empty(sc.n_rx, dtype=torch.float32, device=dev)
    _lib.call("drt_forward", ctypes.byref(sc), tlp, _ptr(power), _ptr(ws),
              ctypes.c_size_t(ws.numel()), _stream_ptr(dev))
    return power


def saved_vis_floats(walls, tx, rx, max_order: int, alpha: float,
                     smoothing: str = "sigmoid") -> int:
    """Floats of the leg visibilities forward_save keeps (N_K (K + 1) R); raises when
    they are not kept for this scene (not the sigmoid, or more than 1024 walls)."""
    sc, _ = make_scene(walls, tx, rx, max_order, alpha, smoothing)
    n = ctypes.c_int64()
    _lib.call("drt_saved_vis_size", ctypes.byref(sc), ctypes.byref(n))
    return int(n.value)


def forward_save(walls, tx, rx, max_order: int, alpha: float, smoothing: str = "sigmoid",
                 refl_coef: float = 0.5, tile: TileConfig | None = None):
    """(power [R], saved): the forward that also keeps every path's leg visibilities
    (float32 [N_K (K + 1) R]) for ``vjp(..., saved=saved)``, which then skips the
    adjoint's first wall sweep (drt_forward_save; sigmoid)."""
    sc, keep = make_scene(walls, tx, rx, max_order, alpha, smoothing, refl_coef)
    dev = keep[0].device
    n = ctypes.c_int64()
    _lib.call("drt_saved_vis_size", ctypes.byref(sc), ctypes.byref(n))
    saved = torch.empty(max(int(n.value), 1), dtype=torch.float32, device=dev)
    tl = tile.as_c() if tile else None
    tlp = ctypes.byref(tl) if tl is not None else None
    nbytes = ctypes.c_size_t()
    _lib.call("drt_forward_workspace_size", ctypes.byref(sc), tlp, ctypes.byref(nbytes))
    ws = _workspace(dev, nbytes.value)
    power = torch.empty(sc.n_rx, dtype=torch.float32, device=dev)
    _lib.call("drt_forward_save", ctypes.byref(sc), tlp, _ptr(power), _ptr(saved), _ptr(ws),
              ctypes.c_size_t(ws.numel()), _stream_ptr(dev))
    return power, saved


def _finder_forward(name: str, walls, tx, rx, max_order, alpha, smoothing, n_iter, check_eps,
                    refl_coef, tile) -> torch.Tensor:
    sc, keep = make_scene(walls, tx, rx, max_order, alpha, smoothing, refl_coef)
    dev = keep[0].device
    tl = tile.as_c() if tile else None
    tlp = ctypes.byref(tl) if tl is not None else None
    nbytes = ctypes.c_size_t()
    _lib.call(f"drt_forward_{name}_workspace_size", ctypes.byref(sc), tlp, ctypes.byref(nbytes))
    ws = _workspace(dev, nbytes.value)
    power = torch.empty(sc.n_rx, dtype=torch.float32, device=dev)
    _lib.call(f"drt_forward_{name}", ctypes.byref(sc), tlp, int(n_iter),
              ctypes.c_float(check_eps), _ptr(power), _ptr(ws), ctypes.c_size_t(ws.numel()),
              _stream_ptr(dev))
    return power


def _finder_paths(name: str, walls, tx, rx, max_order, alpha, smoothing, n_iter, check_eps,
                  refl_coef) -> torch.Tensor:
    sc, keep = make_scene(walls, tx, rx, max_order, alpha, smoothing, refl_coef)
    dev = keep[0].device
    n = num_candidates(sc.n_walls, int(max_order))
    out = torch.empty(sc.n_rx, n, int(max_order) + 2, dtype=torch.float32, device=dev)
    _lib.call(f"drt_{name}_paths", ctypes.byref(sc), int(n_iter), ctypes.c_float(check_eps),
              _ptr(out), _stream_ptr(dev))
    return out


def forward_mpt(walls, tx, rx, max_order: int, alpha: float, smoothing: str = "hard_sigmoid",
                n_iter: int = 10, check_eps: float = 0.05, refl_coef: float = 0.5,
                tile: TileConfig | None = None) -> torch.Tensor:
    """Received power per receiver (float32 [R]) with the reflection points found by
    ``n_iter`` Min-Path-Tracing steps and the smoothed convergence check
    s(check_eps - C) (drt_forward_mpt, Sec. V-B)."""
    return _finder_forward("mpt", walls, tx, rx, max_order, alpha, smoothing, n_iter,
                           check_eps, refl_coef, tile)


def mpt_paths(walls, tx, rx, max_order: int, alpha: float, smoothing: str = "hard_sigmoid",
              n_iter: int = 10, check_eps: float = 0.05, refl_coef: float = 0.5) -> torch.Tensor:
    """Path finder record per (receiver, candidate): float32 [R, N_K, K + 2] holding
    tau_1..tau_K (NaN past the path's order or for a degenerate path), the MPT cost
    C and the check kappa (drt_mpt_paths)."""
    return _finder_paths("mpt", walls, tx, rx, max_order, alpha, smoothing, n_iter, check_eps,
                         refl_coef)


def forward_fpt(walls, tx, rx, max_order: int, alpha: float, smoothing: str = "hard_sigmoid",
                n_iter: int = 10, check_eps: float = 0.05, refl_coef: float = 0.5,
                tile: TileConfig | None = None) -> torch.Tensor:
    """forward_mpt with Fermat path tracing (Newton steps on the path length) as the
    finder and the same MPT convergence check (drt_forward_fpt)."""
    return _finder_forward("fpt", walls, tx, rx, max_order, alpha, smoothing, n_iter,
                           check_eps, refl_coef, tile)


def fpt_paths(walls, tx, rx, max_order: int, alpha: float, smoothing: str = "hard_sigmoid",
              n_iter: int = 10, check_eps: float = 0.05, refl_coef: float = 0.5) -> torch.Tensor:
    """mpt_paths with Fermat path tracing as the finder (drt_fpt_paths)."""
    return _finder_paths("fpt", walls, tx, rx, max_order, alpha, smoothing, n_iter, check_eps,
                         refl_coef)


def _field(walls, tx, rx, max_order, alpha, smoothing, wavelength, eps_r, refl_coef, tile,
           save):
    sc, keep = make_scene(walls, tx, rx, max_order, alpha, smoothing, refl_coef)
    dev = keep[0].device
    tl = tile.as_c() if tile else None
    tlp = ctypes.byref(tl) if tl is not None else None
    nbytes = ctypes.c_size_t()
    _lib.call("drt_field_workspace_size", ctypes.byref(sc), tlp, ctypes.byref(nbytes))
    ws = _workspace(dev, nbytes.value)
    E = torch.empty(sc.n_rx, 2, dtype=torch.float32, device=dev)
    power = torch.empty(sc.n_rx, dtype=torch.float32, device=dev)
    if not save:
        _lib.call("drt_field", ctypes.byref(sc), tlp, ctypes.c_float(wavelength),
                  ctypes.c_float(eps_r), _ptr(E), _ptr(power), _ptr(ws),
                  ctypes.c_size_t(ws.numel()), _stream_ptr(dev))
        return E, power
    n = ctypes.c_int64()
    _lib.call("drt_saved_vis_size", ctypes.byref(sc), ctypes.byref(n))
    saved = torch.empty(max(int(n.value), 1), dtype=torch.float32, device=dev)
    _lib.call("drt_field_save", ctypes.byref(sc), tlp, ctypes.c_float(wavelength),
              ctypes.c_float(eps_r), _ptr(E), _ptr(power), _ptr(saved), _ptr(ws),
              ctypes.c_size_t(ws.numel()), _stream_ptr(dev))
    return E, power, saved


def field(walls, tx, rx, max_order: int, alpha: float, smoothing: str, wavelength: float,
          eps_r: float, refl_coef: float = 0.5, tile: TileConfig | None = None):
    """Coherent field and power per receiver on the current stream:
    (field float32 [R, 2] = (re, im), power float32 [R] = |field|^2).

    Eq. 7 as a sum of complex path fields prod_j C_j V vis exp(-2 pi i L / wavelength) / L,
    C_j the Fresnel TE coefficient of relative permittivity ``eps_r`` (>= 1) at
    each reflection, or -sqrt(refl_coef) when ``eps_r`` is 0 (drt_field)."""
    return _field(walls, tx, rx, max_order, alpha, smoothing, wavelength, eps_r, refl_coef,
                  tile, False)


def field_save(walls, tx, rx, max_order: int, alpha: float, smoothing: str, wavelength: float,
               eps_r: float, refl_coef: float = 0.5, tile: TileConfig | None = None):
    """(field, power, saved): ``field`` that also keeps every path's leg visibilities
    (the sigmoid; forward_save's layout and values) for ``field_vjp(..., saved=saved)``."""
    return _field(walls, tx, rx, max_order, alpha, smoothing, wavelength, eps_r, refl_coef,
                  tile, True)


def field_vjp(walls, tx, rx, max_order: int, alpha: float, smoothing: str, wavelength: float,
              eps_r: float, field_values: torch.Tensor, grad_power: torch.Tensor,
              refl_coef: float = 0.5, wall_grad: bool = True, tile: TileConfig | None = None,
              saved: torch.Tensor | None = None):
    """(grad_tx [2], grad_walls [W, 4] or None) = grad_power^T d|E|^2 / d(tx, walls), with
    ``field_values`` the [R, 2] field that ``field`` returned for the same arguments.
    ``saved``: the visibilities of ``field_save`` or ``forward_save`` on the same scene
    (drt_field_vjp_saved), or None."""
    sc, keep = make_scene(walls, tx, rx, max_order, alpha, smoothing, refl_coef)
    dev = keep[0].device
    gp = _as_f32(grad_power.reshape(-1, 1), 1, "grad_power", 4)
    E = _as_f32(field_values, 2, "field", 8)
    if gp.shape[0] != sc.n_rx or E.shape[0] != sc.n_rx:
        raise ValueError("grad_power and field must have one entry per receiver")
    tl = tile.as_c() if tile else None
    tlp = ctypes.byref(tl) if tl is not None else None
    nbytes = ctypes.c_size_t()
    _lib.call("drt_field_vjp_workspace_size", ctypes.byref(sc), tlp, ctypes.byref(nbytes))
    ws = _workspace(dev, nbytes.value)
    gtx = torch.empty(2, dtype=torch.float32, device=dev)
    gw = torch.empty(sc.n_walls, 4, dtype=torch.float32, device=dev) if wall_grad else None
    if saved is None:
        _lib.call("drt_field_vjp", ctypes.byref(sc), tlp, ctypes.c_float(wavelength),
                  ctypes.c_float(eps_r), _ptr(E), _ptr(gp), _ptr(gtx),
                  None if gw is None else _ptr(gw), _ptr(ws), ctypes.c_size_t(ws.numel()),
                  _stream_ptr(dev))
    else:
        sv = _as_f32(saved.reshape(-1, 1), 1, "saved", 4)
        _lib.call("drt_field_vjp_saved", ctypes.byref(sc), tlp, ctypes.c_float(wavelength),
                  ctypes.c_float(eps_r), _ptr(E), _ptr(gp), _ptr(sv), _ptr(gtx),
                  None if gw is None else _ptr(gw), _ptr(ws), ctypes.c_size_t(ws.numel()),
                  _stream_ptr(dev))
    return gtx, gw


def _scene3(tris, tx, rx, max_order, alpha, smoothing, refl_coef):
    tris = _as_f32(tris, 9, "tris", 4)
    rx = _as_f32(rx, 3, "rx", 4)
    tx = _as_f32(tx.reshape(1, 3), 3, "tx", 4)
    if tris.device != rx.device or tris.device != tx.device:
        raise ValueError("tris, tx and rx must be on the same device")
    if smoothing not in _lib.SMOOTHING:
        raise ValueError(f"unknown smoothing {smoothing!r}")
    sc = _lib.Scene3(tris.data_ptr(), tris.shape[0], rx.data_ptr(), rx.shape[0], tx.data_ptr(),
                     int(max_order), float(alpha), _lib.SMOOTHING[smoothing], float(refl_coef))
    return sc, (tris, tx, rx)


def forward3(tris, tx, rx, max_order: int, alpha: float, smoothing: str = "hard_sigmoid",
             refl_coef: float = 0.5, tile: TileConfig | None = None) -> torch.Tensor:
    """Received power per receiver of a 3D scene of triangle walls (float32 [R]) on the
    current stream: tris [W, 9] (corners A, B, C), tx [3], rx [R, 3] (drt3_forward)."""
    sc, keep = _scene3(tris, tx, rx, max_order, alpha, smoothing, refl_coef)
    dev = keep[0].device
    tl = tile.as_c() if tile else None
    tlp = ctypes.byref(tl) if tl is not None else None
    nbytes = ctypes.c_size_t()
    _lib.call("drt3_forward_workspace_size", ctypes.byref(sc), tlp, ctypes.byref(nbytes))
    ws = _workspace(dev, nbytes.value)
    power = torch.empty(sc.n_rx, dtype=torch.float32, device=dev)
    _lib.call("drt3_forward", ctypes.byref(sc), tlp, _ptr(power), _ptr(ws),
              ctypes.c_size_t(ws.numel()), _stream_ptr(dev))
    return power


def vjp3_tx(tris, tx, rx, max_order: int, alpha: float, smoothing: str,
            grad_power: torch.Tensor, refl_coef: float = 0.5,
            tile: TileConfig | None = None) -> torch.Tensor:
    """grad_power^T dP / dTX [3] of a 3D scene (drt3_vjp_tx)."""
    sc, keep = _scene3(tris, tx, rx, max_order, alpha, smoothing, refl_coef)
    dev = keep[0].device
    gp = _as_f32(grad_power.reshape(-1, 1), 1, "grad_power", 4)
    if gp.shape[0] != sc.n_rx:
        raise ValueError("grad_power must have one entry per receiver")
    tl = tile.as_c() if tile else None
    tlp = ctypes.byref(tl) if tl is not None else None
    nbytes = ctypes.c_size_t()
    _lib.call("drt3_vjp_tx_workspace_size", ctypes.byref(sc), tlp, ctypes.byref(nbytes))
    ws = _workspace(dev, nbytes.value)
    gtx = torch.empty(3, dtype=torch.float32, device=dev)
    _lib.call("drt3_vjp_tx", ctypes.byref(sc), tlp, _ptr(gp), _ptr(gtx), _ptr(ws),
              ctypes.c_size_t(ws.numel()), _stream_ptr(dev))
    return gtx


def vjp3(tris, tx, rx, max_order: int, alpha: float, smoothing: str,
         grad_power: torch.Tensor, refl_coef: float = 0.5, tri_grad: bool = True,
         tile: TileConfig | None = None):
    """(grad_tx [3], grad_tris [W, 9] or None) = grad_power^T dP / d(tx, tris) of a 3D
    scene (drt3_vjp)."""
    sc, keep = _scene3(tris, tx, rx, max_order, alpha, smoothing, refl_coef)
    dev = keep[0].device
    gp = _as_f32(grad_power.reshape(-1, 1), 1, "grad_power", 4)
    if gp.shape[0] != sc.n_rx:
        raise ValueError("grad_power must have one entry per receiver")
    tl = tile.as_c() if tile else None
    tlp = ctypes.byref(tl) if tl is not None else None
    nbytes = ctypes.c_size_t()
    _lib.call("drt3_vjp_workspace_size", ctypes.byref(sc), tlp, ctypes.byref(nbytes))
    ws = _workspace(dev, nbytes.value)
    gtx = torch.empty(3, dtype=torch.float32, device=dev)
    gtr = torch.empty(sc.n_tris, 9, dtype=torch.float32, device=dev) if tri_grad else None
    _lib.call("drt3_vjp", ctypes.byref(sc), tlp, _ptr(gp), _ptr(gtx),
              None if gtr is None else _ptr(gtr), _ptr(ws), ctypes.c_size_t(ws.numel()),
              _stream_ptr(dev))
    return gtx, gtr


class Power3Function(torch.autograd.Function):
    """3D received power, differentiable in the transmitter and the triangles
    (drt3_vjp backward)."""

    @staticmethod
    def forward(ctx, tris, tx, rx, max_order, alpha, smoothing, refl_coef, tile):
        ctx.save_for_backward(tris, tx, rx)
        ctx.args = (max_order, alpha, smoothing, refl_coef, tile)
        return forward3(tris, tx, rx, max_order, alpha, smoothing, refl_coef, tile)

    @staticmethod
    def backward(ctx, grad_power):
        tris, tx, rx = ctx.saved_tensors
        max_order, alpha, smoothing, refl_coef, tile = ctx.args
        need_t, need_tx = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if not (need_t or need_tx):
            return (None,) * 8
        gtx, gtr = vjp3(tris, tx, rx, max_order, alpha, smoothing, grad_power.contiguous(),
                        refl_coef, tri_grad=need_t, tile=tile)
        return (gtr.reshape(tris.shape) if need_t else None,
                gtx.reshape(tx.shape) if need_tx else None, None, None, None, None, None, None)


def power3(tris, tx, rx, max_order: int, alpha: float, smoothing: str = "hard_sigmoid",
           refl_coef: float = 0.5, tile: TileConfig | None = None) -> torch.Tensor:
    """3D received power per receiver, differentiable in ``tris`` and ``tx``."""
    return Power3Function.apply(tris, tx, rx, max_order, alpha, smoothing, refl_coef, tile)


def tune_forward_timings(walls, tx, rx, max_order: int, alpha: float, smoothing: str,
                         candidates, refl_coef: float = 0.5, reps: int = 3):
    """Times drt_forward with each TileConfig of ``candidates`` in the library
    (drt_tune_forward: CUDA events on the current stream) and returns
    (fastest TileConfig, [ms per launch for each candidate])."""
    sc, keep = make_scene(walls, tx, rx, max_order, alpha, smoothing, refl_coef)
    dev = keep[0].device
    cands = list(candidates)
    arr = (_lib.Tile * len(cands))(*[c.as_c() for c in cands])
    need = 0
    for c in arr:
        nbytes = ctypes.c_size_t()
        _lib.call("drt_forward_workspace_size", ctypes.byref(sc), ctypes.byref(c),
                  ctypes.byref(nbytes))
        need = max(need, nbytes.value)
    ws = _workspace(dev, need)
    power = torch.empty(sc.n_rx, dtype=torch.float32, device=dev)
    best = _lib.Tile()
    ms = (ctypes.c_float * len(cands))()
    _lib.call("drt_tune_forward", ctypes.byref(sc), arr, len(cands), int(reps), _ptr(power),
              _ptr(ws), ctypes.c_size_t(ws.numel()), ctypes.byref(best), ms, _stream_ptr(dev))
    key = (best.warps_per_cta, best.cands_per_unit, best.ctas_per_sm, best.flags)
    i = next(i for i, c in enumerate(arr)
             if (c.warps_per_cta, c.cands_per_unit, c.ctas_per_sm, c.flags) == key)
    return cands[i], list(ms)


def min_loss(power: torch.Tensor):
    """(loss, argmin): loss = -min_r power[r] (float32 [1]), argmin int32 [1]."""
    power = _as_f32(power.reshape(-1, 1), 1, "power", 4)
    dev = power.device
    loss = torch.empty(1, dtype=torch.float32, device=dev)
    arg = torch.empty(1, dtype=torch.int32, device=dev)
    _lib.call("drt_loss", _ptr(power), power.shape[0], _ptr(loss), _ptr(arg), _stream_ptr(dev))
    return loss, arg


def min_loss_backward(argmin: torch.Tensor, grad_loss: torch.Tensor | None, n_rx: int) -> torch.Tensor:
    dev = argmin.device
    g = torch.empty(n_rx, dtype=torch.float32, device=dev)
    gl = None if grad_loss is None else _as_f32(grad_loss.reshape(1, 1), 1, "grad_loss", 4)
    _lib.call("drt_loss_backward", _ptr(argmin), None if gl is None else _ptr(gl), n_rx, _ptr(g),
              _stream_ptr(dev))
    return g


def vjp(walls, tx, rx, max_order: int, alpha: float, smoothing: str, grad_power: torch.Tensor,
        refl_coef: float = 0.5, wall_grad: bool = True, tile: TileConfig | None = None,
        saved: torch.Tensor | None = None):
    """(grad_tx [2], grad_walls [W, 4] or None) = grad_power^T d power / d (tx, walls).
    ``saved``: the leg visibilities of a ``forward_save`` on the same scene (sigmoid),
    read instead of the adjoint's first wall sweep (drt_vjp_saved)."""
    sc, keep = make_scene(walls, tx, rx, max_order, alpha, smoothing, refl_coef)
    dev = keep[0].device
    gp = _as_f32(grad_power.reshape(-1, 1), 1, "grad_power", 4)
    if gp.shape[0] != sc.n_rx:
        raise ValueError("grad_power must have one entry per receiver")
    tl = tile.as_c() if tile else None
    tlp = ctypes.byref(tl) if tl is not None else None
    nbytes = ctypes.c_size_t()
    _lib.call("drt_vjp_workspace_size", ctypes.byref(sc), tlp, ctypes.byref(nbytes))
    ws = _workspace(dev, nbytes.value)
    gtx = torch.empty(2, dtype=torch.float32, device=dev)
    gw = torch.empty(sc.n_walls, 4, dtype=torch.float32, device=dev) if wall_grad else None
    if saved is not None:
        if not (saved.is_cuda and saved.dtype == torch.float32 and saved.is_contiguous()):
            raise TypeError("saved must be the float32 CUDA tensor forward_save returned")
        _lib.call("drt_vjp_saved", ctypes.byref(sc), tlp, _ptr(gp), _ptr(saved), _ptr(gtx),
                  None if gw is None else _ptr(gw), _ptr(ws), ctypes.c_size_t(ws.numel()),
                  _stream_ptr(dev))
    else:
        _lib.call("drt_vjp", ctypes.byref(sc), tlp, _ptr(gp), _ptr(gtx),
                  None if gw is None else _ptr(gw), _ptr(ws), ctypes.c_size_t(ws.numel()),
                  _stream_ptr(dev))
    return gtx, gw


def min_loss_vjp(walls, tx, rx, max_order: int, alpha: float, smoothing: str,
                 argmin: torch.Tensor, grad_loss: torch.Tensor | None = None,
                 refl_coef: float = 0.5, wall_grad: bool = True,
                 tile: TileConfig | None = None):
    """Gradient of loss = -power[argmin] w.r.t. (tx, walls), times grad_loss (default 1)."""
    sc, keep = make_scene(walls, tx, rx, max_order, alpha, smoothing, refl_coef)
    dev = keep[0].device
    if argmin.dtype != torch.int32 or not argmin.is_cuda:
        raise TypeError("argmin must be an int32 CUDA tensor")
    gl = None if grad_loss is None else _as_f32(grad_loss.reshape(1, 1), 1, "grad_loss", 4)
    tl = tile.as_c() if tile else None
    tlp = ctypes.byref(tl) if tl is not None else None
    nbytes = ctypes.c_size_t()
    _lib.call("drt_vjp_workspace_size", ctypes.byref(sc), tlp, ctypes.byref(nbytes))
    ws = _workspace(dev, nbytes.value)
    gtx = torch.empty(2, dtype=torch.float32, device=dev)
    gw = torch.empty(sc.n_walls, 4, dtype=torch.float32, device=dev) if wall_grad else None
    _lib.call("drt_min_loss_vjp", ctypes.byref(sc), tlp, _ptr(argmin.contiguous()),
              None if gl is None else _ptr(gl), _ptr(gtx), None if gw is None else _ptr(gw),
              _ptr(ws), ctypes.c_size_t(ws.numel()), _stream_ptr(dev))
    return gtx, gw


class ObjectiveFunction(torch.autograd.Function):
    """loss = -min_r P_r(walls, tx), with the one-receiver min-loss adjoint as backward."""

    @staticmethod
    def forward(ctx, walls, tx, rx, max_order, alpha, smoothing, refl_coef, tile):
        P = forward(walls, tx, rx, max_order, alpha, smoothing, refl_coef, tile)
        loss_v, arg = min_loss(P)
        ctx.save_for_backward(walls, tx, rx, arg)
        ctx.args = (max_order, alpha, smoothing, refl_coef, tile)
        return loss_v.reshape(())

    @staticmethod
    def backward(ctx, grad_loss):
        walls, tx, rx, arg = ctx.saved_tensors
        max_order, alpha, smoothing, refl_coef, tile = ctx.args
        need_w, need_tx = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if not (need_w or need_tx):
            return (None,) * 8
        gtx, gw = min_loss_vjp(walls, tx, rx, max_order, alpha, smoothing, arg,
                               grad_loss.reshape(1).float().contiguous(), refl_coef,
                               wall_grad=need_w, tile=tile)
        return (gw if need_w else None, gtx.reshape(tx.shape) if need_tx else None,
                None, None, None, None, None, None)


# Largest leg-visibility buffer (bytes) PowerFunction keeps for its backward
# (sigmoid; override with DRT_SAVED_VIS_MAX_BYTES, 0 to always recompute).
SAVED_VIS_MAX_BYTES = 4 << 30


def _saved_vis_limit() -> int:
    import os
    v = os.environ.get("DRT_SAVED_VIS_MAX_BYTES")
    return int(v) if v is not None else SAVED_VIS_MAX_BYTES


class PowerFunction(torch.autograd.Function):
    """power = P(walls, tx) with the hand-written adjoint as backward.

    The backward recomputes the path geometry; for the sigmoid the forward also keeps
    every path's leg visibilities (up to ``SAVED_VIS_MAX_BYTES``), so that the backward
    skips its first wall sweep."""

    @staticmethod
    def forward(ctx, walls, tx, rx, max_order, alpha, smoothing, refl_coef, tile):
        ctx.args = (max_order, alpha, smoothing, refl_coef, tile)
        saved = None
        if (smoothing == "sigmoid" and walls.shape[0] <= 1024 and rx.shape[0] > 0 and
                (ctx.needs_input_grad[0] or ctx.needs_input_grad[1])):
            n = saved_vis_floats(walls, tx, rx, max_order, alpha, smoothing)
            if 4 * n <= _saved_vis_limit():
                power, saved = forward_save(walls, tx, rx, max_order, alpha, smoothing,
                                            refl_coef, tile)
        if saved is None:
            power = forward(walls, tx, rx, max_order, alpha, smoothing, refl_coef, tile)
            ctx.save_for_backward(walls, tx, rx)
        else:
            ctx.save_for_backward(walls, tx, rx, saved)
        return power

    @staticmethod
    def backward(ctx, grad_power):
        walls, tx, rx, *rest = ctx.saved_tensors
        saved = rest[0] if rest else None
        max_order, alpha, smoothing, refl_coef, tile = ctx.args
        need_w, need_tx = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if not (need_w or need_tx):
            return (None,) * 8
        gtx, gw = vjp(walls, tx, rx, max_order, alpha, smoothing, grad_power.contiguous(),
                      refl_coef, wall_grad=need_w, tile=tile, saved=saved)
        return (gw if need_w else None, gtx.reshape(tx.shape) if need_tx else None,
                None, None, None, None, None, None)


class MinLossFunction(torch.autograd.Function):
    """loss = -min_r power[r] (Eq. 8 objective, Sec. III loss)."""

    @staticmethod
    def forward(ctx, power):
        loss, arg = min_loss(power)
        ctx.save_for_backward(arg)
        ctx.n = power.shape[0]
        return loss.reshape(())

    @staticmethod
    def backward(ctx, grad_loss):
        (arg,) = ctx.saved_tensors
        return min_loss_backward(arg, grad_loss.reshape(1).float().contiguous(), ctx.n)


class FieldPowerFunction(torch.autograd.Function):
    """|E|^2 of the coherent field, with drt_field_vjp as backward (the field E is
    saved; the geometry is recomputed; for the sigmoid the leg visibilities are kept
    as in PowerFunction)."""

    @staticmethod
    def forward(ctx, walls, tx, rx, max_order, alpha, smoothing, wavelength, eps_r, refl_coef,
                tile):
        saved = None
        if (smoothing == "sigmoid" and walls.shape[0] <= 1024 and rx.shape[0] > 0 and
                (ctx.needs_input_grad[0] or ctx.needs_input_grad[1])):
            n = saved_vis_floats(walls, tx, rx, max_order, alpha, smoothing)
            if 4 * n <= _saved_vis_limit():
                E, P, saved = field_save(walls, tx, rx, max_order, alpha, smoothing,
                                         wavelength, eps_r, refl_coef, tile)
        if saved is None:
            E, P = field(walls, tx, rx, max_order, alpha, smoothing, wavelength, eps_r,
                         refl_coef, tile)
            ctx.save_for_backward(walls, tx, rx, E)
        else:
            ctx.save_for_backward(walls, tx, rx, E, saved)
        ctx.args = (max_order, alpha, smoothing, wavelength, eps_r, refl_coef, tile)
        return P

    @staticmethod
    def backward(ctx, grad_power):
        walls, tx, rx, E, *rest = ctx.saved_tensors
        saved = rest[0] if rest else None
        max_order, alpha, smoothing, wavelength, eps_r, refl_coef, tile = ctx.args
        need_w, need_tx = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if not (need_w or need_tx):
            return (None,) * 10
        gtx, gw = field_vjp(walls, tx, rx, max_order, alpha, smoothing, wavelength, eps_r, E,
                            grad_power.contiguous(), refl_coef, wall_grad=need_w, tile=tile,
                            saved=saved)
        return (gw if need_w else None, gtx.reshape(tx.shape) if need_tx else None,
                None, None, None, None, None, None, None, None)


def field_power(walls, tx, rx, max_order: int, alpha: float, smoothing: str, wavelength: float,
                eps_r: float, refl_coef: float = 0.5, tile: TileConfig | None = None):
    """Differentiable (in walls and tx) coherent power |E_r|^2 per receiver."""
    return FieldPowerFunction.apply(walls, tx, rx, max_order, alpha, smoothing, wavelength, eps_r,
                                    refl_coef, tile)


def power(walls, tx, rx, max_order: int, alpha: float, smoothing: str = "hard_sigmoid",
          refl_coef: float = 0.5, tile: TileConfig | None = None) -> torch.Tensor:
    """Differentiable (in walls and tx) received power per receiver."""
    return PowerFunction.apply(walls, tx, rx, max_order, alpha, smoothing, refl_coef, tile)


def loss(power_values: torch.Tensor) -> torch.Tensor:
    """Differentiable loss -min_r power[r]."""
    return MinLossFunction.apply(power_values)


def objective(walls, tx, rx, max_order, alpha, smoothing="hard_sigmoid", refl_coef=0.5,
              tile=None):
    """loss(power(...)) = -min_r P_r as one differentiable call (min-loss adjoint backward)."""
    return ObjectiveFunction.apply(walls, tx, rx, max_order, alpha, smoothing, refl_coef, tile)


def _host_f32(a, cols: int, name: str) -> torch.Tensor:
    t = torch.as_tensor(a)
    if t.is_cuda:
        raise TypeError(f"{name} must be a host array")
    t = t.detach().to(torch.float32).reshape(-1, cols)
    return t.contiguous()


def objective_host(walls, tx, rx, max_order, alpha, smoothing="hard_sigmoid", refl_coef=0.5,
                   device="cuda", grad_walls=False, tile=None):
    """End-to-end call from host arrays (drt_objective_host): the library copies the
    inputs to the device, runs power, loss and its gradient, and copies
    (loss, power, grad_tx[, grad_walls]) back into host tensors.  Pinned host inputs
    keep the copies asynchronous; the call returns after the stream has finished."""
    dev = torch.device(device)
    w = _host_f32(walls, 4, "walls")
    t = _host_f32(tx, 2, "tx")
    r = _host_f32(rx, 2, "rx")
    if smoothing not in _lib.SMOOTHING:
        raise ValueError(f"unknown smoothing {smoothing!r}")
    sc = _lib.Scene(w.data_ptr(), w.shape[0], r.data_ptr(), r.shape[0], t.data_ptr(),
                    int(max_order), float(alpha), _lib.SMOOTHING[smoothing], float(refl_coef))
    tl = tile.as_c() if tile else None
    tlp = ctypes.byref(tl) if tl is not None else None
    nbytes = ctypes.c_size_t()
    _lib.call("drt_objective_host_workspace_size", ctypes.byref(sc), tlp, ctypes.byref(nbytes))
    ws = _workspace(dev, nbytes.value)
    pin = w.is_pinned()
    loss_h = torch.empty(1, dtype=torch.float32, pin_memory=pin)
    arg_h = torch.empty(1, dtype=torch.int32, pin_memory=pin)
    p_h = torch.empty(r.shape[0], dtype=torch.float32, pin_memory=pin)
    gtx_h = torch.empty(2, dtype=torch.float32, pin_memory=pin)
    gw_h = torch.empty(w.shape[0], 4, dtype=torch.float32, pin_memory=pin) if grad_walls else None
    _lib.call("drt_objective_host", ctypes.byref(sc), tlp, _ptr(loss_h), _ptr(arg_h), _ptr(p_h),
              _ptr(gtx_h), None if gw_h is None else _ptr(gw_h), _ptr(ws),
              ctypes.c_size_t(ws.numel()), _stream_ptr(dev))
    torch.cuda.current_stream(dev).synchronize()
    out = [loss_h, p_h, gtx_h]
    if grad_walls:
        out.append(gw_h)
    return tuple(out)
