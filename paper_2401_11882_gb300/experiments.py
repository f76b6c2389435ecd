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

The batched-descent study (4096 uneven scenes x 4 starts: full-batch step time;
200 Adam steps on the first 256 scenes):

    python -m paper_2401_11882_gb300.experiments --study batch

The batch tiles (the autotuner's choice on the first 64 scenes, then full-batch
steps with the default tile, the tuned tile, and the tuned tile with the exact
invalid-path skip):

    python -m paper_2401_11882_gb300.experiments --study batch_tiles --timed-steps 1
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
                    lr=1e-2, lr_decay=0.99, rel_tol=1e-3, device="cuda", seed=0,
                    ref_samples=None) -> dict:
    """One scene: the surrogate trained on n_samples exact samples proposes n_starts
    starts for the exact descent, against n_starts uniform starts.  The reference
    optimum L* comes from the same samples, or from ref_samples others (a larger,
    independent set) when given, so that a small surrogate training set does not
    also weaken the reference."""
    sc = scenes.surrogate_scene(seed=scene_seed)
    search = SurrogateSearch(sc, device=device, seed=seed, batch=8192)
    x, F = search.generate(n_samples, seed=seed)
    setup = search.timings["generate_s"]
    train_hist = search.train(x, F, epochs=epochs)
    setup += search.timings["train_s"]
    if ref_samples and ref_samples > n_samples:
        xr, Fr = search.generate(ref_samples, seed=seed + 1000)
        L_star, tx_star = reference_optimum(sc, xr, Fr, device=device)
    else:
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
    gain = p_secs - seeded_s
    rel_err = float(np.median(np.abs(np.log(F_pred + 1e-12) - np.log(F_exact + 1e-12))))
    return {
        "scene_seed": scene_seed, "samples": n_samples, "epochs": epochs,
        "final_train_mse": train_hist[-1], "L_star": L_star, "tx_star": tx_star.tolist(),
        "seeded": {"seconds": seeded_s, "proposal_seconds": t_prop, "steps": s_steps,
                   "reached": bool(s_ok), "best_loss": s_best, "fallback": bool(off),
                   "gap": (s_best - L_star) / abs(L_star),
                   "seconds_with_surrogate_setup": seeded_s + setup},
        "plain": {"seconds": p_secs, "steps": p_steps, "reached": bool(p_ok), "best_loss": p_best,
                  "gap": (p_best - L_star) / abs(L_star)},
        "surrogate_log_error_median": rel_err,
        "generate_seconds": setup - search.timings["train_s"],
        "train_seconds": search.timings["train_s"], "reference_samples": ref_samples or n_samples,
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


def batch_study(n_scenes=4096, timed_steps=3, conv_scenes=256, conv_steps=200, seed=0,
                device="cuda", smoothing="hard_sigmoid") -> dict:
    """Batched descent on the 4096-scene batch (W 8-256, R 64-4096, K 0-2, 4 starts,
    alpha = 100, hard sigmoid, Adam lr 1e-2): (1) time of full-batch steps after one
    warm-up step; (2) 200 steps on the first conv_scenes scenes, with the loss
    trajectory and the final TX of every problem (the batched losses themselves are
    checked against the oracle by the GPU tests)."""
    from . import workload
    full = scenes.scene_batch(n_scenes, seed, smoothing=smoothing)
    dev = torch.device(device)
    T = full.tx0.shape[1]

    def fwd_flops(b):
        return sum(T * workload.forward_work(int(b.wall_off[i + 1] - b.wall_off[i]),
                                             int(b.max_order[i]),
                                             int(b.rx_off[i + 1] - b.rx_off[i]))["flops"]
                   for i in range(b.n_scenes))

    out = {"batch": {"scenes": n_scenes, "starts": T,
                     "evaluations_per_step": sum(
                         T * int(full.rx_off[i + 1] - full.rx_off[i]) *
                         int(workload.num_candidates(int(full.wall_off[i + 1] - full.wall_off[i]),
                                                     int(full.max_order[i])))
                         for i in range(n_scenes))}}
    if timed_steps > 0:
        out["full_batch"] = _time_full_batch(full, timed_steps, fwd_flops(full),
                                             out["batch"]["evaluations_per_step"], dev)
    if conv_steps > 0:
        out["convergence"] = _convergence_run(full, conv_scenes, conv_steps, dev)
    return out


def _time_full_batch(full, timed_steps, fl, evals, dev, tile=None):
    from .batched import BatchedDescent
    bd = BatchedDescent(full, device=dev, tile=tile)
    bd.run(1)
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    bd.run(timed_steps)
    b.record()
    torch.cuda.synchronize(dev)
    s_step = a.elapsed_time(b) / 1e3 / timed_steps
    res = {"timed_steps": timed_steps, "s_per_step": s_step, "steps_per_s": 1.0 / s_step,
           "forward_flop_per_step_convention": fl, "tflops_by_convention": fl / s_step / 1e12,
           "evals_per_s": evals / s_step, "info": bd.info()}
    bd.close()
    return res


def batch_tile_study(n_scenes=4096, tune_scenes=64, timed_steps=1, seed=0, device="cuda",
                     smoothing="hard_sigmoid") -> dict:
    """The batch autotuner on the 4096-scene batch: autotune.tune_batch times every
    candidate tile (warps per CTA x CTAs per SM) on the first tune_scenes scenes; the
    full batch is then timed with the library's default tile, with the tuned tile,
    with the tuned tile plus the exact invalid-path skip (DRT_TILE_CULL_INVALID:
    warps whose paths all have hard-sigmoid validity exactly 0 skip the obstruction
    loop; the losses are unchanged bit for bit, but the step no longer does the
    literal work the FLOP convention counts, so its rate is reported apart), and
    with the exact blocked-warp exit (DRT_TILE_EXIT_BLOCKED: a warp whose paths all
    have a leg of visibility exactly 0 leaves the wall loop), alone and with the
    skip, reported apart for the same reason."""
    from dataclasses import asdict, replace
    from . import autotune, workload
    full = scenes.scene_batch(n_scenes, seed, smoothing=smoothing)
    dev = torch.device(device)
    T = full.tx0.shape[1]
    fl = sum(T * workload.forward_work(int(full.wall_off[i + 1] - full.wall_off[i]),
                                       int(full.max_order[i]),
                                       int(full.rx_off[i + 1] - full.rx_off[i]))["flops"]
             for i in range(full.n_scenes))
    evals = sum(T * int(full.rx_off[i + 1] - full.rx_off[i]) *
                int(workload.num_candidates(int(full.wall_off[i + 1] - full.wall_off[i]),
                                            int(full.max_order[i])))
                for i in range(n_scenes))
    best, timings = autotune.tune_batch(full, n_scenes=tune_scenes, steps=1, return_timings=True)
    out = {"tuned_on_first_scenes": tune_scenes,
           "candidates_ms_per_step": [[asdict(c), ms] for c, ms in timings],
           "best": asdict(best)}
    out["default_tile"] = _time_full_batch(full, timed_steps, fl, evals, dev)
    out["tuned_tile"] = _time_full_batch(full, timed_steps, fl, evals, dev, tile=best)
    skip = _time_full_batch(full, timed_steps, fl, evals, dev,
                            tile=replace(best, cull_invalid=True))
    skip.pop("tflops_by_convention")   # the skipped paths are not computed
    out["tuned_tile_exact_skip"] = skip
    for key, t in (("tuned_tile_blocked_exit", replace(best, exit_blocked=True)),
                   ("tuned_tile_exact_skip_blocked_exit",
                    replace(best, cull_invalid=True, exit_blocked=True))):
        r = _time_full_batch(full, timed_steps, fl, evals, dev, tile=t)
        r.pop("tflops_by_convention")
        out[key] = r
    return out


def _convergence_run(full, n, conv_steps, dev):
    """conv_steps Adam steps on the first n scenes.  A problem whose minimum power is
    exactly 0 (a receiver in full hard-sigmoid shadow) has loss 0 and gradient 0:
    the statistics of improvement are taken over the problems with a non-zero loss."""
    from .batched import BatchedDescent
    T = full.tx0.shape[1]
    sub = scenes.SceneBatch(full.walls[:full.wall_off[n]], full.wall_off[:n + 1],
                            full.rx[:full.rx_off[n]], full.rx_off[:n + 1], full.max_order[:n],
                            full.tx0[:n], full.alpha, full.smoothing, full.refl_coef)
    bd = BatchedDescent(sub, history=conv_steps, device=dev)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    bd.run(conv_steps)
    torch.cuda.synchronize(dev)
    secs = time.perf_counter() - t0
    hist = bd.history.cpu().numpy()            # [steps][P], loss before each step's update
    final = bd.evaluate().cpu().numpy().copy()  # loss at the final TX
    tx = bd.tx.cpu().numpy().reshape(n, T, 2)
    bd.close()
    first = hist[0]
    marks = sorted({0, conv_steps // 4 - 1, conv_steps // 2 - 1, 3 * conv_steps // 4 - 1,
                    conv_steps - 1} - {-1})
    rows = {str(i): float(np.mean(hist[i])) for i in marks}
    rows["final"] = float(np.mean(final))
    best_start = final.reshape(n, T).min(axis=1)
    live = first < 0
    rel = (first[live] - final[live]) / np.abs(first[live])
    return {
        "scenes": n, "problems": int(n * T), "steps": conv_steps, "seconds": secs,
        "s_per_step": secs / conv_steps,
        "mean_loss_by_step": rows,
        "problems_with_nonzero_initial_loss": int(live.sum()),
        "problems_with_nonzero_final_loss": int((final < 0).sum()),
        "fraction_improved_of_nonzero": float(np.mean(final[live] < first[live])) if live.any() else None,
        "median_relative_improvement_of_nonzero": float(np.median(rel)) if live.any() else None,
        "mean_best_of_starts_loss": float(np.mean(best_start)),
        "last_10_steps_mean_abs_change": float(np.mean(np.abs(np.diff(hist[-10:], axis=0)))),
        "final_tx_first_8_problems": tx.reshape(-1, 2)[:8].tolist(),
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--seeds", type=int, nargs="+", default=[0])
    ap.add_argument("--samples", type=int, default=1 << 20)
    ap.add_argument("--ref-samples", type=int, default=0,
                    help="time to optimum: samples for the reference optimum (0: the training set)")
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--starts", type=int, default=64)
    ap.add_argument("--study", choices=["surrogate", "annealing", "batch", "batch_tiles"],
                    default="surrogate")
    ap.add_argument("--scenes", type=int, default=256)
    ap.add_argument("--timed-steps", type=int, default=3, help="batch study: full-batch steps timed")
    ap.add_argument("--conv-steps", type=int, default=200, help="batch study: convergence steps")
    ap.add_argument("--smoothing", default="hard_sigmoid", choices=["hard_sigmoid", "sigmoid"],
                    help="batch study: smoothing of the descent")
    args = ap.parse_args()
    if args.study == "annealing":
        print(json.dumps(annealing_study(n_scenes=args.scenes)), flush=True)
        return
    if args.study == "batch_tiles":
        print(json.dumps(batch_tile_study(timed_steps=args.timed_steps)), flush=True)
        return
    if args.study == "batch":
        print(json.dumps(batch_study(timed_steps=args.timed_steps, conv_scenes=args.scenes,
                                     smoothing=args.smoothing,
                                     conv_steps=args.conv_steps)), flush=True)
        return
    rows = []
    for s in args.seeds:
        r = time_to_optimum(s, args.samples, args.epochs, args.starts,
                            ref_samples=args.ref_samples)
        rows.append(r)
        print(json.dumps(r), flush=True)
    summary = {
        "seeds": len(rows),
        "seeded_reached": sum(r["seeded"]["reached"] for r in rows),
        "plain_reached": sum(r["plain"]["reached"] for r in rows),
        "seeded_median_seconds_when_reached": float(np.median([r["seeded"]["seconds"] for r in rows if r["seeded"]["reached"]])) if any(r["seeded"]["reached"] for r in rows) else None,
        "plain_median_seconds_when_reached": float(np.median([r["plain"]["seconds"] for r in rows if r["plain"]["reached"]])) if any(r["plain"]["reached"] for r in rows) else None,
        "seeded_median_gap": float(np.median([r["seeded"]["gap"] for r in rows])),
        "seeded_median_seconds_with_setup_when_reached": float(np.median([r["seeded"]["seconds_with_surrogate_setup"] for r in rows if r["seeded"]["reached"]])) if any(r["seeded"]["reached"] for r in rows) else None,
        "scenes_reached_by_seeded_with_setup_before_plain": sum(
            r["seeded"]["reached"] and (not r["plain"]["reached"] or
                                         r["seeded"]["seconds_with_surrogate_setup"] < r["plain"]["seconds"])
            for r in rows),
        "plain_median_gap": float(np.median([r["plain"]["gap"] for r in rows])),
    }
    print(json.dumps({"summary": summary}), flush=True)


if __name__ == "__main__":
    main()
