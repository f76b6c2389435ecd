"""Batched gradient descent on the transmitter position over many scenes.

Marshalling over the batched C ABI (drt_batch_*): the scenes of a
``scenes.SceneBatch`` and the descent state live in device tensors owned by
this object; one descent step (forward, min loss, adjoint of the argmin
receiver, Adam, clamp) runs entirely in the library's kernels and is replayed
as a CUDA graph.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from .ops import TileConfig


class BatchedDescent:
    """Adam on the TX of every (scene, start) problem of a batch.

    ``batch`` is a ``scenes.SceneBatch`` (2D walls) or a ``scenes.SceneBatch3``
    (triangle walls, 3D receivers and TX; Sec. VI).
    ``alpha`` is a float or a per-step schedule (the last value repeats);
    ``box`` = (lo_x, lo_y, hi_x, hi_y) clamps the TX after every step, with
    (lo_x, lo_y, lo_z, hi_x, hi_y, hi_z) for a 3D batch (default the unit cube);
    the learning rate of step i is ``lr * lr_decay**i``;
    ``history`` rows of per-step losses are kept on the device.
    """

    def __init__(self, batch, lr=1e-2, betas=(0.9, 0.999), eps=1e-8, alpha=100.0,
                 box=None, history=0, device="cuda",
                 tile: TileConfig | None = None, tx0=None, lr_decay: float = 1.0):
        self.device = torch.device(device)
        dev = self.device
        self.batch = batch
        self.dim = 3 if hasattr(batch, "tris") else 2
        d = self.dim
        if box is None:
            box = (0.0,) * d + (1.0,) * d
        if len(box) != 2 * d:
            raise ValueError(f"box must have {2 * d} values")
        lo, hi = list(box[:d]) + [0.0] * (3 - d), list(box[d:]) + [0.0] * (3 - d)
        self.S, self.T = batch.n_scenes, batch.tx0.shape[1]
        self.P = self.S * self.T
        self._wall_off_h = np.ascontiguousarray(batch.wall_off, np.int32)
        self._rx_off_h = np.ascontiguousarray(batch.rx_off, np.int32)
        self._order_h = np.ascontiguousarray(batch.max_order, np.int32)
        self.walls = torch.tensor(batch.tris if d == 3 else batch.walls, device=dev)
        self.rx = torch.tensor(batch.rx, device=dev)
        self.wall_off = torch.tensor(self._wall_off_h, device=dev)
        self.rx_off = torch.tensor(self._rx_off_h, device=dev)
        self.order = torch.tensor(self._order_h, device=dev)
        start = batch.tx0 if tx0 is None else tx0
        self.tx = torch.tensor(np.asarray(start, np.float32).reshape(self.P, d), device=dev)
        self.m = torch.zeros(self.P, d, device=dev)
        self.v = torch.zeros(self.P, d, device=dev)
        self.step = torch.zeros(1, dtype=torch.int32, device=dev)
        self.loss = torch.zeros(self.P, device=dev)
        self.history = torch.full((history, self.P), float("nan"), device=dev) if history else None
        sched = np.atleast_1d(np.asarray(alpha, np.float32))
        self.alpha = torch.tensor(sched, device=dev)
        self._desc = _lib.Batch(self.walls.data_ptr(), self.wall_off.data_ptr(), self.rx.data_ptr(),
                                self.rx_off.data_ptr(), self.order.data_ptr(),
                                self._wall_off_h.ctypes.data, self._rx_off_h.ctypes.data,
                                self._order_h.ctypes.data, self.S, self.T,
                                _lib.SMOOTHING[batch.smoothing], float(batch.refl_coef), d)
        self._tile = tile.as_c() if tile else None
        plan = ctypes.c_void_p()
        _lib.call("drt_batch_plan_create", ctypes.byref(self._desc),
                  ctypes.byref(self._tile) if self._tile is not None else None, ctypes.byref(plan))
        self._plan = plan
        nbytes = ctypes.c_size_t()
        _lib.call("drt_batch_workspace_size", self._plan, ctypes.byref(nbytes))
        self.workspace = torch.empty(max(nbytes.value, 256), dtype=torch.uint8, device=dev)
        self._state = _lib.DescentState(
            self.tx.data_ptr(), self.m.data_ptr(), self.v.data_ptr(), self.step.data_ptr(),
            self.loss.data_ptr(), self.history.data_ptr() if self.history is not None else None,
            history, self.alpha.data_ptr(), len(sched), float(lr), float(betas[0]),
            float(betas[1]), float(eps), float(lo[0]), float(lo[1]), float(hi[0]),
            float(hi[1]), float(lr_decay), float(lo[2]), float(hi[2]))
        _lib.call("drt_batch_bind", self._plan, ctypes.byref(self._state),
                  ctypes.c_void_p(self.workspace.data_ptr()), ctypes.c_size_t(self.workspace.numel()),
                  ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream))

    def run(self, n_steps: int, use_graph: bool = True) -> None:
        """Enqueue n_steps descent steps on the current stream."""
        _lib.call("drt_batch_run", self._plan, int(n_steps), 1 if use_graph else 0,
                  ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream))

    def evaluate(self) -> torch.Tensor:
        """Loss of every problem at its current TX (no update); returns self.loss."""
        _lib.call("drt_batch_evaluate", self._plan,
                  ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream))
        return self.loss

    def info(self) -> dict:
        out = (ctypes.c_int64 * 8)()
        _lib.call("drt_batch_plan_info", self._plan, out)
        keys = ["problems", "forward_units", "adjoint_units", "forward_ctas", "adjoint_ctas",
                "max_walls", "receiver_problems", "threads"]
        return dict(zip(keys, list(out)))

    def state_dict(self) -> dict:
        torch.cuda.synchronize(self.device)
        return {"tx": self.tx.cpu().numpy().copy(), "m": self.m.cpu().numpy().copy(),
                "v": self.v.cpu().numpy().copy(), "step": int(self.step.item())}

    def load_state_dict(self, st: dict) -> None:
        """Restore a saved state in place (the bound buffers keep their addresses)."""
        self.tx.copy_(torch.as_tensor(st["tx"]).to(self.device))
        self.m.copy_(torch.as_tensor(st["m"]).to(self.device))
        self.v.copy_(torch.as_tensor(st["v"]).to(self.device))
        self.step.fill_(int(st["step"]))

    def save(self, path: str) -> None:
        st = self.state_dict()
        np.savez(path, tx=st["tx"], m=st["m"], v=st["v"], step=np.int64(st["step"]))

    def load(self, path: str) -> None:
        d = np.load(path)
        self.load_state_dict({"tx": d["tx"], "m": d["m"], "v": d["v"], "step": int(d["step"])})

    def close(self) -> None:
        if getattr(self, "_plan", None):
            _lib.load().drt_batch_plan_destroy(self._plan)
            self._plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def geometric_alpha(start: float, stop: float, n: int) -> np.ndarray:
    """alpha_i = start (stop/start)^(i/(n-1)), i = 0..n-1 (the schedule of Sec. VII, Fig. 5)."""
    i = np.arange(n, dtype=np.float64)
    return (start * (stop / start) ** (i / max(n - 1, 1))).astype(np.float32)
