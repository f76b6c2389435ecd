"""Time-to-optimum study: surrogate-seeded vs plain multi-start descent.

For one scene (64 walls, 256 random receivers, K <= 2, alpha = 100), with
the surrogate trained on exact samples of the objective F(tx) = min_r P_r:

* reference optimum L*: the 16 best separated samples refined by a long
  exact descent (decaying learning rate); L* is the best loss (-F) found;
* seeded: the surrogate proposes `n_starts` separated minima on a grid, the
  exact batched descent refines them; the surrogate's predictions at the
  proposals are checked against the exact objective there, and when the best
  proposal is worse than the samples' 90th percentile the search falls back to
  plain multi-start;
* plain: `n_starts` uniform random starts, same descent.

Both searches stop once their best loss is within `rel_tol` of L*; wall-clock
time on the GPU counts surrogate inference and proposal selection for the
seeded search.  Data generation and training are reported separately, with
the number of problems after which the surrogate pays for itself.

    python -m paper_2401_11882_gb300.experiments --seeds 0 1 2 --samples 1048576

The annealing study (Sec. VII, convergence success with and without smoothing):

    python -m paper_2401_11882_gb300.experiments --study annealing --scenes 256
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import scenes
from .surrogate import SurrogateSearch, descend, sample_objective, separated_minima


def reference_optimum(scene, x, F, n_top=16, steps=1500, lr=1e-2, lr_decay=0.995,
                      device="cuda"):
    """(L*, tx*): the best of the best separated samples refined by a long descent,
    or the best sample itself if no refinement beats it."""
    starts = separated_minima(x, -F, n_top, 0.03)
    best, tx, steps_done, secs, _, _ = descend(scene, starts, steps, None, lr=lr,
                                               lr_decay=lr_decay, device=device, check_every=50)
    i = int(np.argmax(F))
    if -float(F[i]) < best:
        return -float(F[i]), np.asarray(x[i], np.float32)
    return best, tx


def time_to_optimum(scene_seed=0, n_samples=1 << 20, epochs=20, n_starts=64, max_steps=1000,
                    lr=1e-2, lr_decay=0.99, rel_tol=1e-3, device="cuda", seed=0) -> dict:
    sc = scenes.surrogate_scene(seed=scene_seed)
    search = SurrogateSearch(sc, device=device, seed=seed, batch=8192)
    x, F = search.generate(n_samples, seed=seed)
    train_hist = search.train(x, F, epochs=epochs)
    L_star, tx_star = reference_optimum(sc, x, F, device=device)

    # seeded search (inference + proposals + exact refinement, fallback when off)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    props = search.propose(k=n_starts)
    F_pred = search.predict_F(props)
    F_exact = sample_objective(sc, props, device)
    t_prop = time.perf_counter() - t0
    off = F_exact.max() < np.quantile(F, 0.90)
    if off:
        props = np.random.default_rng(seed + 7).uniform(0.02, 0.98, (n_starts, 2)).astype(np.float32)
    s_best, s_tx, s_steps, s_secs, s_ok, s_hist = descend(sc, props, max_steps, L_star, rel_tol,
                                                          lr=lr, lr_decay=lr_decay, device=device,
                                                          check_every=10)
    seeded_s = t_prop + s_secs

    starts = np.random.default_rng(seed + 1).uniform(0.02, 0.98, (n_starts, 2)).astype(np.float32)
    p_best, p_tx, p_steps, p_secs, p_ok, p_hist = descend(sc, starts, max_steps, L_star, rel_tol,
                                                          lr=lr, lr_decay=lr_decay, device=device,
                                                          check_every=10)
    setup = search.timings["generate_s"] + search.timings["train_s"]
    gain = p_secs - seeded_s
    rel_err = float(np.median(np.abs(np.log(F_pred + 1e-12) - np.log(F_exact + 1e-12))))
    return {
        "scene_seed": scene_seed, "samples": n_samples, "epochs": epochs,
        "final_train_mse": train_hist[-1], "L_star": L_star, "tx_star": tx_star.tolist(),
        "seeded": {"seconds": seeded_s, "proposal_seconds": t_prop, "steps": s_steps,
                   "reached": bool(s_ok), "best_loss": s_best, "fallback": bool(off),
                   "gap": (s_best - L_star) / abs(L_star)},
        "plain": {"seconds": p_secs, "steps": p_steps, "reached": bool(p_ok), "best_loss": p_best,
                  "gap": (p_best - L_star) / abs(L_star)},
        "surrogate_log_error_median": rel_err,
        "generate_seconds": search.timings["generate_s"], "train_seconds": search.timings["train_s"],
        "break_even_problems": (setup / gain) if gain > 0 else None,
    }


def _los_batch(rng, n_scenes, n_rx, n_walls, n_starts, smoothing, grid_tx=None):
    """Square + n_walls random segments (lengths 0.1-0.4), n_rx receivers, K = 0."""
    walls, rxs, w_off, r_off, txs = [], [], [0], [0], []
    for _ in range(n_scenes):
        w = np.concatenate([scenes.unit_square_walls(),
                            scenes.random_segments(rng, n_walls, (0.1, 0.4))])
        r = scenes.rx_uniform(rng, n_rx)
        t = scenes.rx_uniform(rng, n_starts, 0.05, 0.95)
        walls.append(w); rxs.append(r); txs.append(t if grid_tx is None else grid_tx)
        w_off.append(w_off[-1] + w.shape[0]); r_off.append(r_off[-1] + n_rx)
    return scenes.SceneBatch(np.concatenate(walls), np.asarray(w_off, np.int32), np.concatenate(rxs),
                             np.asarray(r_off, np.int32), np.zeros(n_scenes, np.int32),
                             np.stack(txs).astype(np.float32), 1.0, smoothing)


def annealing_study(n_scenes=256, rx_counts=(2, 3, 4), n_starts=4, n_walls=5, steps=100,
                    lr=2e-2, lr_decay=0.96, grid=128, tols=(1e-2, 5e-2), seed=0,
                    device="cuda") -> dict:
    """Sec. VII: TX placement by gradient descent on -min_r P_r (LOS only), with the
    smoothing annealed as alpha_i = 100^(i/(steps-1)) (sigmoid) against no smoothing
    (unit step); Adam with a learning rate decaying by lr_decay per step, so that a
    run settles instead of circling the (non-smooth) max-min optimum.  A run
    converges when the unsmoothed objective at its final TX is within tol
    (relative) of the best value seen for that scene (a grid x grid scan and every
    final point)."""
    from .batched import BatchedDescent, geometric_alpha
    out = {}
    sched = geometric_alpha(1.0, 100.0, steps)
    c = (np.arange(grid) + 0.5) / grid
    gx, gy = np.meshgrid(c, c, indexing="xy")
    grid_tx = np.stack([gx.ravel(), gy.ravel()], 1).astype(np.float32)
    for n_rx in rx_counts:
        rng = np.random.default_rng(seed + n_rx)
        smooth = _los_batch(rng, n_scenes, n_rx, n_walls, n_starts, "sigmoid")
        step = scenes.SceneBatch(smooth.walls, smooth.wall_off, smooth.rx, smooth.rx_off,
                                 smooth.max_order, smooth.tx0, 1.0, "step")
        # best unsmoothed objective per scene over the grid
        scan = scenes.SceneBatch(smooth.walls, smooth.wall_off, smooth.rx, smooth.rx_off,
                                 smooth.max_order,
                                 np.broadcast_to(grid_tx, (n_scenes,) + grid_tx.shape).copy(),
                                 1.0, "step")
        bd = BatchedDescent(scan, device=device, alpha=1.0)
        F_grid = (-bd.evaluate()).cpu().numpy().reshape(n_scenes, -1).max(axis=1)
        bd.close()
        finals = {}
        for name, b, alpha in (("smoothed", smooth, sched), ("unsmoothed", step, 1.0)):
            bd = BatchedDescent(b, lr=lr, alpha=alpha, device=device, lr_decay=lr_decay)
            bd.run(steps)
            tx = bd.tx.cpu().numpy().reshape(n_scenes, n_starts, 2)
            bd.close()
            ev = scenes.SceneBatch(b.walls, b.wall_off, b.rx, b.rx_off, b.max_order, tx, 1.0, "step")
            e = BatchedDescent(ev, device=device, alpha=1.0)
            finals[name] = (-e.evaluate()).cpu().numpy().reshape(n_scenes, n_starts)
            e.close()
        best = np.maximum(F_grid[:, None], np.maximum(finals["smoothed"].max(1, keepdims=True),
                                                      finals["unsmoothed"].max(1, keepdims=True)))
        res = {"runs": int(n_scenes * n_starts)}
        for tol in tols:
            ok = {k: v >= (1.0 - tol) * best for k, v in finals.items()}
            n_ok_unsmoothed = int(ok["unsmoothed"].sum())
            res[f"tol_{tol:g}"] = {
                "success_smoothed": float(ok["smoothed"].mean()),
                "success_unsmoothed": float(ok["unsmoothed"].mean()),
                "ratio": float(ok["smoothed"].mean() / max(ok["unsmoothed"].mean(), 1e-12)),
                "retained": (float((ok["smoothed"] & ok["unsmoothed"]).sum() / n_ok_unsmoothed)
                             if n_ok_unsmoothed else None),
            }
        out[f"{n_rx}_rx"] = res
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--seeds", type=int, nargs="+", default=[0])
    ap.add_argument("--samples", type=int, default=1 << 20)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--starts", type=int, default=64)
    ap.add_argument("--study", choices=["surrogate", "annealing"], default="surrogate")
    ap.add_argument("--scenes", type=int, default=256)
    args = ap.parse_args()
    if args.study == "annealing":
        print(json.dumps(annealing_study(n_scenes=args.scenes)), flush=True)
        return
    rows = []
    for s in args.seeds:
        r = time_to_optimum(s, args.samples, args.epochs, args.starts)
        rows.append(r)
        print(json.dumps(r), flush=True)
    summary = {
        "seeds": len(rows),
        "seeded_reached": sum(r["seeded"]["reached"] for r in rows),
        "plain_reached": sum(r["plain"]["reached"] for r in rows),
        "seeded_median_seconds_when_reached": float(np.median([r["seeded"]["seconds"] for r in rows if r["seeded"]["reached"]])) if any(r["seeded"]["reached"] for r in rows) else None,
        "plain_median_seconds_when_reached": float(np.median([r["plain"]["seconds"] for r in rows if r["plain"]["reached"]])) if any(r["plain"]["reached"] for r in rows) else None,
        "seeded_median_gap": float(np.median([r["seeded"]["gap"] for r in rows])),
        "plain_median_gap": float(np.median([r["plain"]["gap"] for r in rows])),
    }
    print(json.dumps({"summary": summary}), flush=True)


if __name__ == "__main__":
    main()
