"""Learned surrogate of the objective over the transmitter position, and the
surrogate-seeded multi-start search that uses it.

* ``SurrogateMLP``: the BF16 tensor-core MLP of libdrt (drt_mlp_*): forward,
  loss gradient and Adam, all in the library's kernels; FP32 master weights.
* ``sample_objective``: the exact objective F(tx) = min_r P_r(tx) at many TX
  positions, by the batched forward (one scene, one problem per sample).
* ``SurrogateSearch``: sample -> train -> propose starts at the surrogate's
  best separated minima -> refine them with the exact batched descent; the
  surrogate's prediction is checked against the exact loss at the proposals,
  and plain random multi-start is the fallback when it is off.
"""
from __future__ import annotations

import ctypes
import time
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib
from .ops import TileConfig

N_FREQ = 32
WIDTH = 256
LAYERS = 4


def _ptr(t: torch.Tensor):
    return ctypes.c_void_p(t.data_ptr())


def _stream(dev):
    return ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


def init_params(seed: int = 0) -> np.ndarray:
    """He-style uniform weights, zero biases (flat float32, library layout)."""
    rng = np.random.default_rng(seed)
    parts = []
    for l in range(LAYERS):
        k = 2 * N_FREQ if l == 0 else WIDTH
        lim = np.sqrt(6.0 / k)
        parts += [rng.uniform(-lim, lim, WIDTH * k), np.zeros(WIDTH)]
    parts += [rng.uniform(-np.sqrt(3.0 / WIDTH), np.sqrt(3.0 / WIDTH), WIDTH), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)


class SurrogateMLP:
    """x in [0,1]^2 -> scalar.  Fourier features with frequencies ~ N(0, sigma^2)."""

    def __init__(self, device="cuda", seed: int = 0, sigma: float = 4.0, batch: int = 4096):
        self.device = torch.device(device)
        if batch % 64:
            raise ValueError("batch must be a multiple of 64")
        self.batch = batch
        n = ctypes.c_int64()
        sb = ctypes.c_size_t()
        wb = ctypes.c_size_t()
        _lib.call("drt_mlp_sizes", batch, ctypes.byref(n), ctypes.byref(sb), ctypes.byref(wb))
        self.n_params = n.value
        rng = np.random.default_rng(seed + 1)
        self.freqs = torch.tensor(rng.normal(0.0, sigma, (N_FREQ, 2)).astype(np.float32),
                                  device=self.device)
        self.params = torch.tensor(init_params(seed), device=self.device)
        assert self.params.numel() == self.n_params
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step = torch.zeros(1, dtype=torch.int32, device=self.device)
        self.shadow = torch.empty(sb.value, dtype=torch.uint8, device=self.device)
        self.workspace = torch.empty(wb.value, dtype=torch.uint8, device=self.device)
        self.grad = torch.zeros_like(self.params)
        self.loss = torch.zeros(1, device=self.device)
        self.sync_shadow()

    def sync_shadow(self):
        _lib.call("drt_mlp_shadow", _ptr(self.params), _ptr(self.shadow), _stream(self.device))

    def set_params(self, theta):
        self.params.copy_(torch.as_tensor(np.asarray(theta, np.float32)).to(self.device))
        self.sync_shadow()

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        """Predictions for x [N, 2] (float32, any N), in chunks of the batch size."""
        x = x.to(self.device, torch.float32).contiguous()
        N = x.shape[0]
        out = torch.empty(N, device=self.device)
        pad = torch.zeros(self.batch, 2, device=self.device)
        ybuf = torch.empty(self.batch, device=self.device)
        for s in range(0, N, self.batch):
            n = min(self.batch, N - s)
            if n == self.batch:
                xb, yb = x[s:s + n], out[s:s + n]
            else:
                pad[:n] = x[s:s + n]
                xb, yb = pad, ybuf
            _lib.call("drt_mlp_forward", _ptr(self.params), _ptr(self.shadow), _ptr(self.freqs),
                      _ptr(xb), self.batch, _ptr(yb), _ptr(self.workspace),
                      ctypes.c_size_t(self.workspace.numel()), _stream(self.device))
            if n < self.batch:
                out[s:s + n] = ybuf[:n]
        return out

    def loss_grad(self, x: torch.Tensor, t: torch.Tensor):
        """(loss [1], grad [n_params]) of the mean squared error on one batch."""
        if x.shape[0] != self.batch:
            raise ValueError("loss_grad takes exactly one batch")
        _lib.call("drt_mlp_loss_grad", _ptr(self.params), _ptr(self.shadow), _ptr(self.freqs),
                  _ptr(x), _ptr(t), self.batch, _ptr(self.loss), _ptr(self.grad),
                  _ptr(self.workspace), ctypes.c_size_t(self.workspace.numel()),
                  _stream(self.device))
        return self.loss, self.grad

    def adam(self, lr=1e-3, betas=(0.9, 0.999), eps=1e-8):
        _lib.call("drt_mlp_adam", _ptr(self.params), _ptr(self.m), _ptr(self.v), _ptr(self.grad),
                  _ptr(self.step), float(lr), float(betas[0]), float(betas[1]), float(eps),
                  _ptr(self.shadow), _stream(self.device))

    def fit(self, x: np.ndarray, t: np.ndarray, epochs: int = 20, lr: float = 1e-3,
            seed: int = 0, lr_final: float | None = None) -> list[float]:
        """Adam on mini-batches of a host dataset, reshuffled on the host every epoch;
        returns the mean loss per epoch.  Cosine decay to lr_final when given."""
        rng = np.random.default_rng(seed)
        n = (x.shape[0] // self.batch) * self.batch
        xd = torch.empty(n, 2, device=self.device)
        td = torch.empty(n, device=self.device)
        hist = []
        total = epochs * (n // self.batch)
        it = 0
        for ep in range(epochs):
            perm = rng.permutation(x.shape[0])[:n]
            xd.copy_(torch.from_numpy(np.ascontiguousarray(x[perm], np.float32)))
            td.copy_(torch.from_numpy(np.ascontiguousarray(t[perm], np.float32)))
            acc = torch.zeros(1, device=self.device)
            for b in range(0, n, self.batch):
                cur = lr
                if lr_final is not None:
                    cur = lr_final + 0.5 * (lr - lr_final) * (1 + np.cos(np.pi * it / max(total, 1)))
                loss, _ = self.loss_grad(xd[b:b + self.batch], td[b:b + self.batch])
                acc += loss
                self.adam(cur)
                it += 1
            hist.append(float(acc) / (n // self.batch))
        return hist


def sample_objective(scene, tx: np.ndarray, device="cuda", cull: bool = True,
                     chunk: int = 1 << 18) -> np.ndarray:
    """F(tx_i) = min_r P_r(tx_i) for every row of tx [N, 2] (exact, batched forward).

    F does not depend on the order of the receivers, so they are passed in
    Z-order: the receivers of one warp are then near each other, and the exact
    invalid-path skip (a path whose validity is 0 for every receiver of the
    warp) applies far more often.  One warp per CTA: a work unit (one sample, 64
    receivers) is then never split between warps that wait for each other."""
    from . import scenes
    from .batched import BatchedDescent
    out = np.empty(tx.shape[0], np.float32)
    tile = TileConfig(warps_per_cta=1, cull_invalid=cull and scene.smoothing != "sigmoid")
    rx = np.ascontiguousarray(scene.rx[scenes.spatial_order(scene.rx)])
    for s in range(0, tx.shape[0], chunk):
        part = np.asarray(tx[s:s + chunk], np.float32)
        b = scenes.SceneBatch(scene.walls, np.array([0, scene.n_walls], np.int32), rx,
                              np.array([0, scene.n_rx], np.int32),
                              np.array([scene.max_order], np.int32), part[None], scene.alpha,
                              scene.smoothing, scene.refl_coef)
        bd = BatchedDescent(b, device=device, tile=tile, alpha=scene.alpha)
        out[s:s + part.shape[0]] = (-bd.evaluate()).cpu().numpy()
        bd.close()
    return out


def target_of(F: np.ndarray) -> np.ndarray:
    """Monotone (decreasing) transform of the objective: lower is better."""
    return -np.log(np.maximum(F, 0.0) + 1e-12)


def separated_minima(points: np.ndarray, values: np.ndarray, k: int, min_sep: float,
                     max_scan: int = 50000) -> np.ndarray:
    """Up to k points of lowest value, greedily keeping those at least min_sep apart
    (scanning at most max_scan candidates in order of value)."""
    order = np.argsort(values, kind="stable")[:max_scan]
    chosen = np.empty((0, 2), np.float64)
    idx = []
    for i in order:
        p = points[i]
        if chosen.shape[0] == 0 or np.min(np.hypot(*(chosen - p).T)) >= min_sep:
            idx.append(i)
            chosen = np.vstack([chosen, p])
            if len(idx) == k:
                break
    return points[np.array(idx, dtype=np.int64)]


def grid_local_minima(values: np.ndarray) -> np.ndarray:
    """Mask of the points of a 2D grid not above any of their 8 neighbours."""
    pad = np.pad(values, 1, mode="edge")
    h, w = values.shape
    mask = np.ones_like(values, dtype=bool)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            if dy or dx:
                mask &= values <= pad[1 + dy:1 + dy + h, 1 + dx:1 + dx + w]
    return mask


@dataclass
class SearchResult:
    best_loss: float
    best_tx: np.ndarray
    steps: int
    seconds: float
    reached: bool
    used_surrogate: bool
    history: list


class SurrogateSearch:
    """Surrogate-seeded multi-start descent on one scene."""

    def __init__(self, scene, device="cuda", seed: int = 0, batch: int = 4096):
        self.scene = scene
        self.device = torch.device(device)
        self.model = SurrogateMLP(device, seed=seed, batch=batch)
        self.t_mean = 0.0
        self.t_std = 1.0
        self.timings = {}

    def generate(self, n_samples: int, seed: int = 0):
        t0 = time.perf_counter()
        rng = np.random.default_rng(seed)
        x = rng.uniform(0.0, 1.0, (n_samples, 2)).astype(np.float32)
        F = sample_objective(self.scene, x, self.device)
        torch.cuda.synchronize(self.device)
        self.timings["generate_s"] = time.perf_counter() - t0
        return x, F

    def train(self, x, F, epochs=20, lr=2e-3, lr_final=1e-4, seed=0):
        t0 = time.perf_counter()
        t = target_of(F)
        self.t_mean, self.t_std = float(t.mean()), float(t.std() + 1e-12)
        hist = self.model.fit(x, (t - self.t_mean) / self.t_std, epochs, lr, seed, lr_final)
        torch.cuda.synchronize(self.device)
        self.timings["train_s"] = time.perf_counter() - t0
        return hist

    def predict_F(self, x: np.ndarray) -> np.ndarray:
        y = self.model.forward(torch.from_numpy(np.asarray(x, np.float32))).cpu().numpy()
        return np.exp(-(y * self.t_std + self.t_mean))

    def propose(self, k: int = 64, grid: int = 512, min_sep: float = 0.03) -> np.ndarray:
        c = (np.arange(grid) + 0.5) / grid
        gx, gy = np.meshgrid(c, c, indexing="xy")
        pts = np.stack([gx.ravel(), gy.ravel()], 1).astype(np.float32)
        y = self.model.forward(torch.from_numpy(pts)).cpu().numpy()
        # local minima of the surrogate first, then the best remaining separated points
        m = grid_local_minima(y.reshape(grid, grid)).ravel()
        props = separated_minima(pts[m], y[m], k, min_sep)
        if props.shape[0] < k:
            extra = separated_minima(pts, y, 4 * k, min_sep)
            keep = [p for p in extra
                    if props.shape[0] == 0 or np.min(np.hypot(*(props - p).T)) >= min_sep]
            props = np.concatenate([props, np.asarray(keep, np.float32).reshape(-1, 2)])[:k]
        return props.astype(np.float32)


def descend(scene, starts: np.ndarray, n_steps: int, target_loss: float | None = None,
            rel_tol: float = 1e-3, lr: float = 1e-2, device="cuda", check_every: int = 5,
            lr_decay: float = 1.0, box=(0.005, 0.005, 0.995, 0.995)):
    """Exact batched Adam from the given starts; stops once the best loss is within
    rel_tol of target_loss (checked every check_every steps).  Returns SearchResult-like
    (best_loss, best_tx, steps, seconds, reached, history).

    As in sample_objective, the receivers go in Z-order and the forward skips, per
    warp, the obstruction loop of paths whose validity is exactly 0 (the loss, a
    min over receivers, and its gradient are unchanged)."""
    from . import scenes
    from .batched import BatchedDescent
    rx = np.ascontiguousarray(scene.rx[scenes.spatial_order(scene.rx)])
    b = scenes.SceneBatch(scene.walls, np.array([0, scene.n_walls], np.int32), rx,
                          np.array([0, scene.n_rx], np.int32), np.array([scene.max_order], np.int32),
                          np.asarray(starts, np.float32)[None], scene.alpha, scene.smoothing,
                          scene.refl_coef)
    dev = torch.device(device)
    bd = BatchedDescent(b, lr=lr, device=dev, alpha=scene.alpha, lr_decay=lr_decay, box=box,
                        tile=TileConfig(cull_invalid=True))
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    steps, hist, reached = 0, [], False
    best_loss, best_tx = np.inf, None
    while steps < n_steps:
        n = min(check_every, n_steps - steps)
        bd.run(n)
        steps += n
        loss = bd.evaluate().cpu().numpy()
        i = int(np.argmin(loss))
        if loss[i] < best_loss:
            best_loss, best_tx = float(loss[i]), bd.tx[i].cpu().numpy().copy()
        hist.append((steps, time.perf_counter() - t0, best_loss))
        if target_loss is not None and best_loss <= target_loss + rel_tol * abs(target_loss):
            reached = True
            break
    seconds = time.perf_counter() - t0
    bd.close()
    return best_loss, best_tx, steps, seconds, reached, hist
