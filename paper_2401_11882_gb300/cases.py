"""Runs one named workload a few times and prints its CUDA-event timings, so that
a profiler can capture a chosen launch of it (e.g. ``ncu --clock-control none -k
regex:vjp_kernel -s 2 -c 1 python -m paper_2401_11882_gb300.cases vjp --rx-grid 32``;
without ``--clock-control none`` ncu locks the GPU's clocks).

    forward   drt.forward on the scene
    vjp       drt.vjp with dense g = 1/R (gradient w.r.t. the TX and every wall;
              --saved: the sigmoid adjoint reading drt.forward_save's visibilities)
    field     drt.field (coherent field, Fresnel TE, --eps-r, --wavelength)
    field_vjp drt.field_vjp with dense g = 1/R (after one drt.field)
    forward_mpt drt.forward_mpt (the iterative path finder, --n-iter steps, --check-eps)
    forward_fpt drt.forward_fpt (the same with Fermat path tracing)
    forward3  drt.forward3 on the 3D room (``scenes.room3d``, --rx-grid receivers a side)
    vjp3      drt.vjp3 (transmitter and triangle gradients; --tx-only: drt.vjp3_tx) on
              the same room, dense g = 1/R
    mlp       the surrogate MLP's inference on --batch random points

Scenes: ``gradient`` (128 random segments, K <= 2, the dense-adjoint workload),
``large`` (square + 60 segments, K <= 2, the benchmark workload) and ``clutter``
(square + --segments random segments, K <= --order; more than 1020 segments
exceed what shared memory holds), each on an n x n receiver grid.
"""
from __future__ import annotations

import argparse
import json

import torch

from . import ops, scenes


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("op", choices=["forward", "vjp", "mlp", "field", "field_vjp", "forward3",
                                   "vjp3", "forward_mpt", "forward_fpt"])
    ap.add_argument("--batch", type=int, default=65536)
    ap.add_argument("--scene", choices=["gradient", "large", "clutter"], default="gradient")
    ap.add_argument("--segments", type=int, default=4092)
    ap.add_argument("--order", type=int, default=1)
    ap.add_argument("--n-iter", type=int, default=10)
    ap.add_argument("--check-eps", type=float, default=0.05)
    ap.add_argument("--smoothing", default="sigmoid", choices=["hard_sigmoid", "sigmoid", "step"])
    ap.add_argument("--alpha", type=float, default=100.0)
    ap.add_argument("--rx-grid", type=int, default=32)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--wavelength", type=float, default=0.02)
    ap.add_argument("--eps-r", type=float, default=5.0)
    ap.add_argument("--single-rx", action="store_true", help="one receiver per lane")
    ap.add_argument("--tx-only", action="store_true", help="vjp3: transmitter gradient only")
    ap.add_argument("--saved", action="store_true",
                    help="vjp: read the forward's saved visibilities (sigmoid)")
    args = ap.parse_args()
    dev = torch.device("cuda:0")
    if args.op == "mlp":
        from .surrogate import SurrogateMLP
        m = SurrogateMLP(dev, batch=args.batch)
        xm = torch.rand(args.batch, 2, device=dev)
        for _ in range(2):
            m.forward(xm)
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(args.reps):
            m.forward(xm)
        b.record()
        torch.cuda.synchronize(dev)
        print(json.dumps({"op": "mlp", "batch": args.batch, "ms": a.elapsed_time(b) / args.reps}))
        return 0
    if args.op in ("forward3", "vjp3"):
        sc3 = scenes.room3d(args.rx_grid, args.alpha, args.smoothing)
        w3, t3, r3 = (torch.tensor(x, device=dev) for x in (sc3.tris, sc3.tx, sc3.rx))
        g3 = torch.full((sc3.n_rx,), 1.0 / sc3.n_rx, device=dev)

        def run3():
            if args.op == "vjp3" and args.tx_only:
                return ops.vjp3_tx(w3, t3, r3, sc3.max_order, args.alpha, args.smoothing, g3)
            if args.op == "vjp3":
                return ops.vjp3(w3, t3, r3, sc3.max_order, args.alpha, args.smoothing, g3)
            return ops.forward3(w3, t3, r3, sc3.max_order, args.alpha, args.smoothing)

        for _ in range(2):
            run3()
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(args.reps):
            run3()
        b.record()
        torch.cuda.synchronize(dev)
        ms = a.elapsed_time(b) / args.reps
        n = sc3.n_rx * ops.num_candidates(sc3.n_tris, sc3.max_order)
        print(json.dumps({"op": args.op, "scene": "room3d", "smoothing": args.smoothing,
                          "alpha": args.alpha, "n_tris": sc3.n_tris, "n_rx": sc3.n_rx, "ms": ms,
                          "evals_per_s": n / (ms / 1e3)}))
        return 0
    if args.scene == "clutter":
        sc = scenes.clutter_scene(args.segments, 1, seed=1, alpha=args.alpha,
                                  smoothing=args.smoothing, max_order=args.order)
    else:
        sc = (scenes.gradient_scene if args.scene == "gradient" else scenes.large_scene)(
            alpha=args.alpha, smoothing=args.smoothing)
    rx = scenes.rx_grid(args.rx_grid)
    w, t, r = (torch.tensor(x, device=dev) for x in (sc.walls, sc.tx, rx))
    g = torch.full((r.shape[0],), 1.0 / r.shape[0], device=dev)
    E = None
    saved = None
    if args.op == "vjp" and args.saved:
        tile0 = ops.TileConfig(single_rx=True) if args.single_rx else None
        _, saved = ops.forward_save(w, t, r, sc.max_order, args.alpha, args.smoothing,
                                    tile=tile0)
    if args.op == "field_vjp":
        E, _ = ops.field(w, t, r, sc.max_order, args.alpha, args.smoothing, args.wavelength,
                         args.eps_r)

    def run():
        tile = ops.TileConfig(single_rx=True) if args.single_rx else None
        if args.op == "forward":
            return ops.forward(w, t, r, sc.max_order, args.alpha, args.smoothing, tile=tile)
        if args.op in ("forward_mpt", "forward_fpt"):
            fn = ops.forward_mpt if args.op == "forward_mpt" else ops.forward_fpt
            return fn(w, t, r, sc.max_order, args.alpha, args.smoothing, args.n_iter,
                      args.check_eps, tile=tile)
        if args.op == "field":
            return ops.field(w, t, r, sc.max_order, args.alpha, args.smoothing, args.wavelength,
                             args.eps_r, tile=tile)
        if args.op == "field_vjp":
            return ops.field_vjp(w, t, r, sc.max_order, args.alpha, args.smoothing,
                                 args.wavelength, args.eps_r, E, g)
        return ops.vjp(w, t, r, sc.max_order, args.alpha, args.smoothing, g, tile=tile,
                       saved=saved)

    for _ in range(2):
        run()
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.reps):
        out = run()
    b.record()
    torch.cuda.synchronize(dev)
    res = {"op": args.op, "scene": args.scene, "smoothing": args.smoothing, "alpha": args.alpha,
           "single_rx": args.single_rx, "saved": saved is not None,
           "n_rx": int(r.shape[0]), "ms": a.elapsed_time(b) / args.reps,
           "evals_per_s": int(r.shape[0]) * ops.num_candidates(sc.walls.shape[0], sc.max_order)
           / (a.elapsed_time(b) / args.reps / 1e3)}
    if args.op in ("vjp", "field_vjp"):
        res["grad_tx"] = out[0].tolist()
    print(json.dumps(res), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
