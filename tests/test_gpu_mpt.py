"""The iterative path finders on the GPU (drt_forward_mpt, drt_mpt_paths and their
Fermat counterparts drt_forward_fpt, drt_fpt_paths; Sec. V-B,
"Continuous Path Finding": Min-Path-Tracing steps with the smoothed convergence
check) against the FP64 oracle's finder, path by path and per receiver."""
import numpy as np
import pytest

from parity import assert_power_close, fp32_sensitivity
from oracle import mpt
from paper_2401_11882_gb300 import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N_ITER, EPS = 10, 0.05


@pytest.fixture(scope="module")
def drt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_11882_gb300 as m
    return m


def _t(sc):
    dev = torch.device("cuda:0")
    return (torch.tensor(sc.walls, device=dev), torch.tensor(sc.tx, device=dev),
            torch.tensor(sc.rx, device=dev))


FINDERS = ["mpt", "fpt"]


def _gpu_paths(drt, sc, n_iter=N_ITER, eps=EPS, finder="mpt"):
    w, t, r = _t(sc)
    out = getattr(drt, f"{finder}_paths")(w, t, r, sc.max_order, sc.alpha, sc.smoothing, n_iter,
                                          eps,
                        sc.refl_coef)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def _gpu_power(drt, sc, n_iter=N_ITER, eps=EPS, tile=None, finder="mpt"):
    w, t, r = _t(sc)
    P = getattr(drt, f"forward_{finder}")(w, t, r, sc.max_order, sc.alpha, sc.smoothing, n_iter,
                                          eps,
                        sc.refl_coef, tile=tile)
    torch.cuda.synchronize()
    return P.cpu().numpy()


def _compare_paths(oracle_mod, sc, gpu, what, finder="mpt"):
    """Per (receiver, candidate): converged paths (oracle C < 1e-10) at the same points
    (FP32 rounding of a unit-scale point: 1e-4 is generous) with C ~ 0 and the same
    kappa; the degenerate paths and the non-converged paths' C agree except for a
    few (at most 2% together) whose FP32 and FP64 iterations took different
    backtracking decisions or ended on different sides of the short-leg limit."""
    K = sc.max_order
    n_conv = n_far = n_all = 0
    for r, rx in enumerate(sc.rx):
        ref = getattr(oracle_mod, f"{finder}_paths")(sc.walls, sc.tx, rx, K, sc.alpha,
                                                     sc.smoothing, N_ITER, EPS, sc.refl_coef)
        g = gpu[r]
        refl = ref["order"] > 0
        deg = ref["degenerate"].astype(bool)
        gdeg = np.isnan(g[:, 0]) & refl
        # a path that creeps into a corner ends with one leg near the 1e-3 limit; the
        # two precisions may land on either side of it (counted with the far paths)
        n_flip = int(np.sum(gdeg != (deg & refl)))
        n_far += n_flip
        n_all += n_flip
        for c in np.nonzero(~deg & ~gdeg)[0]:
            k = int(ref["order"][c])
            n_all += 1
            Cg, kg = g[c, K], g[c, K + 1]
            assert np.all(np.isnan(g[c, k:K])), what
            if ref["cost"][c] < 1e-10:
                # converged: the same points; FP32 leaves C at its rounding floor, which
                # near a short leg (a reflection point next to TX or RX) is ~1e-7
                n_conv += 1
                np.testing.assert_allclose(g[c, :k], ref["tau"][c][:k], atol=1e-4, err_msg=what)
                assert Cg < 1e-6, (what, c, Cg)
                assert kg == pytest.approx(ref["kappa"][c], abs=1e-4), (what, c)
            elif abs(Cg - ref["cost"][c]) > 1e-3 * ref["cost"][c] + 1e-6:
                n_far += 1
    assert n_far <= 0.02 * n_all, (what, n_far, n_all)
    return n_conv, n_all


CASES = [
    # (seed, W, R, K, alpha, smoothing): ragged 32-receiver tiles, every order
    (0, 5, 33, 0, 50.0, "hard_sigmoid"),
    (1, 6, 37, 1, 30.0, "sigmoid"),
    (2, 8, 45, 2, 100.0, "hard_sigmoid"),
    (3, 7, 33, 2, 20.0, "sigmoid"),
    (4, 5, 31, 3, 60.0, "hard_sigmoid"),
    (5, 9, 40, 2, 1.0, "step"),
    (6, 10, 64, 2, 300.0, "sigmoid"),
]


@pytest.mark.parametrize("finder", FINDERS)
@pytest.mark.parametrize("seed,W,R,K,alpha,smoothing", CASES)
def test_paths_match_the_oracle(drt, oracle_mod, seed, W, R, K, alpha, smoothing, finder):
    rng = np.random.default_rng(seed)
    sc = scenes.random_small_scene(rng, W, R, K, alpha, smoothing, boundary=(seed % 2 == 0))
    n_conv, n_all = _compare_paths(oracle_mod, sc, _gpu_paths(drt, sc, finder=finder),
                                   f"{finder} seed {seed}", finder)
    assert n_all > 0 and (K == 0 or n_conv > 0)


def _gpu_path_points(sc, seq, tau):
    """TX and the reflection points at tau along the walls of a GPU path record."""
    walls = sc.walls.astype(np.float64)
    pts = [sc.tx.astype(np.float64)]
    for w, t in zip(seq, tau):
        a, b = walls[w, :2], walls[w, 2:]
        pts.append(a + t * (b - a) / np.linalg.norm(b - a))
    return pts


def _path_agreement(oracle_mod, sc, gpu, finder="mpt"):
    return _path_agreement_n(oracle_mod, sc, gpu, N_ITER, finder)


def _path_agreement_n(oracle_mod, sc, gpu, n_iter, finder="mpt"):
    """Per receiver: (agree, slack).  agree is True when every path's record agrees
    with the oracle's where it matters for the power: the same check factor (kappa,
    0 for a degenerate path) within 1e-3 relative (or 1e-6 absolute), and where
    kappa exceeds 1e-3 on either side, the same points within 1e-4.  A finder
    iteration that FP32 and FP64 steer differently (a path creeping into a corner,
    or another ill-conditioned, non-converged one) changes a receiver's power by
    that path's share, which no input-rounding sensitivity of the oracle measures;
    a path whose kappa stays below 1e-3 adds less than 1e-3 of its unobstructed
    power whatever its points are.  slack is the sum, over the paths that disagree,
    of the oracle's path power and the GPU path's largest possible power (kappa
    Gamma^k / L^2)."""
    K = sc.max_order
    ok = np.ones(sc.n_rx, bool)
    slack = np.zeros(sc.n_rx)
    for r, rx in enumerate(sc.rx):
        ref = getattr(oracle_mod, f"{finder}_paths")(sc.walls, sc.tx, rx, K, sc.alpha,
                                                     sc.smoothing, n_iter, EPS, sc.refl_coef)
        g = gpu[r]
        refl = ref["order"] > 0
        gdeg = np.isnan(g[:, 0]) & refl
        deg = ref["degenerate"].astype(bool)
        kg = np.where(gdeg, 0.0, g[:, K + 1])
        kr = np.where(deg, 0.0, ref["kappa"])
        kmax = np.maximum(kg, kr)
        bad = np.abs(kg - kr) > 1e-3 * kmax + 1e-6
        for c in np.nonzero((kmax > 1e-3) & ~gdeg & ~deg & refl)[0]:
            k = int(ref["order"][c])
            bad[c] |= np.max(np.abs(g[c, :k] - ref["tau"][c][:k])) > 1e-4
        ok[r] = not bad.any()
        for c in np.nonzero(bad)[0]:
            k = int(ref["order"][c])
            slack[r] += ref["power"][c]
            if not gdeg[c] and kg[c] > 0:
                # the GPU path adds at most kappa Gamma^k / L^2 (validity, visibility <= 1)
                pts = _gpu_path_points(sc, [int(w) for w in ref["seq"][c][:k]], g[c, :k])
                pts.append(rx.astype(np.float64))
                L = sum(np.linalg.norm(q - p) for p, q in zip(pts[:-1], pts[1:]))
                slack[r] += kg[c] * sc.refl_coef ** k / L ** 2
    return ok, slack


@pytest.mark.parametrize("finder", FINDERS)
@pytest.mark.parametrize("seed,W,R,K,alpha,smoothing", CASES)
def test_power_matches_the_oracle(drt, oracle_mod, seed, W, R, K, alpha, smoothing, finder):
    """Receivers whose path records all agree with the oracle's are held to the
    power bound (1e-4 relative, or the FP32 input sensitivity); the others (at most
    a quarter: corners of the boundary square make K = 3 paths creep into them) to
    that bound plus the powers of the paths that the two precisions steered apart."""
    rng = np.random.default_rng(seed)
    sc = scenes.random_small_scene(rng, W, R, K, alpha, smoothing, boundary=(seed % 2 == 0))
    power_fn = getattr(oracle_mod, f"power_{finder}")
    ref = power_fn(sc.walls, sc.tx, sc.rx, K, alpha, smoothing, N_ITER, EPS, sc.refl_coef)
    sens = fp32_sensitivity(lambda w, t, r: power_fn(w, t, r, K, alpha, smoothing, N_ITER, EPS),
                            sc.walls, sc.tx, sc.rx)
    agree, slack = _path_agreement(oracle_mod, sc, _gpu_paths(drt, sc, finder=finder), finder)
    assert agree.mean() >= 0.75, agree.mean()
    P = _gpu_power(drt, sc, finder=finder)
    assert_power_close(P[agree], ref[agree], sens=sens[agree], min_strict=0.95)
    err = np.abs(P.astype(np.float64) - ref)
    tol = np.maximum(1e-4 * np.abs(ref), 2.0 * sens) + slack
    assert np.all(err[~agree] <= tol[~agree]), (err[~agree], tol[~agree])


@pytest.mark.parametrize("finder,rate", [("mpt", 0.98), ("fpt", 0.95)])
def test_converged_points_are_the_image_method_points(drt, oracle_mod, finder, rate):
    """On every valid path (the image-method point lies on its wall with both
    neighbours on one side) that the finder converges on, the GPU's points are the
    image-method points within 1e-4; MPT converges on 98% of them, Fermat path
    tracing (which runs into corners more often) on 95%."""
    sc = scenes.clutter_scene(16, 6, seed=3, alpha=100.0, smoothing="hard_sigmoid", max_order=2)
    gpu = _gpu_paths(drt, sc, n_iter=12, finder=finder)
    walls = sc.walls.astype(np.float64)
    tx = sc.tx.astype(np.float64)
    n_valid = n_conv = 0
    for r, rx in enumerate(sc.rx.astype(np.float64)):
        im = oracle_mod.paths(walls, tx, rx, 2, 100.0, "step")
        for c in range(1, len(im["order"])):
            k = int(im["order"][c])
            if im["degenerate"][c]:
                continue
            seq = tuple(int(w) for w in im["seq"][c][:k])
            tau_im = mpt.tau_of(walls, seq, im["verts"][c][1:k + 1])
            lens = np.hypot(walls[list(seq), 2] - walls[list(seq), 0],
                            walls[list(seq), 3] - walls[list(seq), 1])
            if (mpt.cost(walls, seq, tau_im, tx, rx) < 1e-20 and
                    np.all((tau_im > 0) & (tau_im < lens))):
                n_valid += 1
                if not np.isnan(gpu[r, c, 0]) and gpu[r, c, 2] < 1e-9:   # converged, not degenerate
                    n_conv += 1
                    np.testing.assert_allclose(gpu[r, c, :k], tau_im, atol=1e-4)
    assert n_valid > 100 and n_conv >= rate * n_valid


@pytest.mark.parametrize("finder", FINDERS)
def test_square_room_closed_form_on_gpu(drt, finder):
    sc = scenes.Scene(scenes.unit_square_walls(), np.array([0.31, 0.42], np.float32),
                      np.array([[0.7, 0.66], [0.15, 0.8], [0.55, 0.2]], np.float32),
                      max_order=1, alpha=1e4, smoothing="hard_sigmoid")
    tx = sc.tx.astype(np.float64)
    images = [np.array([tx[0], -tx[1]]), np.array([2 - tx[0], tx[1]]),
              np.array([tx[0], 2 - tx[1]]), np.array([-tx[0], tx[1]])]
    rx = sc.rx.astype(np.float64)
    ref = [1 / np.sum((r - tx) ** 2) + 0.5 * sum(1 / np.sum((I - r) ** 2) for I in images)
           for r in rx]
    np.testing.assert_allclose(_gpu_power(drt, sc, finder=finder), ref, rtol=2e-6)


def test_large_scene_sampled(drt, oracle_mod):
    # the benchmark scene (64 walls, K <= 2, 4097 sequences) on 16 sampled receivers
    sc = scenes.large_scene(alpha=100.0, smoothing="hard_sigmoid")
    idx = np.random.default_rng(5).choice(sc.n_rx, 16, replace=False)
    sub = sc.replace(rx=sc.rx[idx])
    ref = oracle_mod.power_mpt(sub.walls, sub.tx, sub.rx, 2, 100.0, "hard_sigmoid", N_ITER, EPS)
    sens = fp32_sensitivity(lambda w, t, r: oracle_mod.power_mpt(w, t, r, 2, 100.0,
                                                                  "hard_sigmoid", N_ITER, EPS),
                            sub.walls, sub.tx, sub.rx)
    assert_power_close(_gpu_power(drt, sub), ref, sens=sens, min_strict=0.9)


@pytest.mark.parametrize("finder", FINDERS)
def test_tile_shapes_and_determinism(drt, oracle_mod, finder):
    rng = np.random.default_rng(8)
    sc = scenes.random_small_scene(rng, 9, 70, 2, 80.0, "sigmoid", boundary=True)
    a = _gpu_power(drt, sc, finder=finder)
    np.testing.assert_array_equal(a, _gpu_power(drt, sc, finder=finder))
    b = _gpu_power(drt, sc, tile=drt.TileConfig(warps_per_cta=2, cands_per_unit=7),
                   finder=finder)
    np.testing.assert_allclose(a, b, rtol=1e-6)


def test_rejects_bad_arguments(drt):
    from paper_2401_11882_gb300._lib import DrtError
    sc = scenes.tiny_scene()
    w, t, r = _t(sc)
    with pytest.raises(DrtError):
        drt.forward_mpt(w, t, r, 1, 100.0, "hard_sigmoid", n_iter=65)
    with pytest.raises(DrtError):
        drt.forward_mpt(w, t, r, 1, 100.0, "hard_sigmoid", check_eps=float("nan"))
    with pytest.raises(DrtError):
        drt.mpt_paths(w, t, r, 1, 100.0, "hard_sigmoid", n_iter=-1)
    with pytest.raises(DrtError):
        drt.forward_fpt(w, t, r, 1, 100.0, "hard_sigmoid", n_iter=65)
    with pytest.raises(DrtError):
        drt.fpt_paths(w, t, r, 1, 100.0, "hard_sigmoid", check_eps=float("inf"))
    empty = sc.replace(rx=np.zeros((0, 2), np.float32))
    assert _gpu_power(drt, empty).shape == (0,)


@pytest.mark.parametrize("n_iter", [0, 1, 64])
def test_iteration_count_edges(drt, oracle_mod, n_iter):
    """No step (the points stay at the walls' midpoints), one step, and the largest
    count DRT_MPT_MAX_ITER: converged paths and the power as in the oracle."""
    rng = np.random.default_rng(30 + n_iter)
    sc = scenes.random_small_scene(rng, 6, 40, 2, 50.0, "hard_sigmoid", boundary=True)
    w, t, r = _t(sc)
    gpu = drt.mpt_paths(w, t, r, 2, 50.0, "hard_sigmoid", n_iter, EPS, sc.refl_coef)
    torch.cuda.synchronize()
    gpu = gpu.cpu().numpy().astype(np.float64)
    walls = sc.walls.astype(np.float64)
    lens = np.hypot(walls[:, 2] - walls[:, 0], walls[:, 3] - walls[:, 1])
    for rr, rx in enumerate(sc.rx[:8]):
        ref = oracle_mod.mpt_paths(sc.walls, sc.tx, rx, 2, 50.0, "hard_sigmoid", n_iter, EPS,
                                   sc.refl_coef)
        for c in np.nonzero((ref["order"] > 0) & ~ref["degenerate"].astype(bool))[0]:
            k = int(ref["order"][c])
            if n_iter == 0:   # the start: every point at its wall's midpoint
                seq = [int(x) for x in ref["seq"][c][:k]]
                np.testing.assert_allclose(ref["tau"][c][:k], 0.5 * lens[seq], rtol=1e-12)
                if not np.isnan(gpu[rr, c, 0]):
                    np.testing.assert_allclose(gpu[rr, c, :k], 0.5 * lens[seq], rtol=1e-6)
            elif ref["cost"][c] < 1e-10 and not np.isnan(gpu[rr, c, 0]):
                np.testing.assert_allclose(gpu[rr, c, :k], ref["tau"][c][:k], atol=1e-4)
    P = drt.forward_mpt(w, t, r, 2, 50.0, "hard_sigmoid", n_iter, EPS, sc.refl_coef)
    ref = oracle_mod.power_mpt(sc.walls, sc.tx, sc.rx, 2, 50.0, "hard_sigmoid", n_iter, EPS,
                               sc.refl_coef)
    agree, slack = _path_agreement_n(oracle_mod, sc, gpu, n_iter)
    err = np.abs(P.cpu().numpy().astype(np.float64) - ref)
    sens = fp32_sensitivity(lambda a, b, c: oracle_mod.power_mpt(a, b, c, 2, 50.0, "hard_sigmoid",
                                                                  n_iter, EPS), sc.walls, sc.tx,
                            sc.rx)
    tol = np.maximum(1e-4 * np.abs(ref), 2.0 * sens) + slack
    assert agree.mean() >= 0.75 and np.all(err <= tol)


def test_fermat_separating_line_on_gpu(drt, oracle_mod):
    """Where the mirror's line separates TX and RX, Fermat path tracing ends at the
    straight crossing (C = 4 (i . n)^2, rejected by the check); the GPU's record
    matches the closed form."""
    walls = np.array([[0.0, 0.0, 1.0, 0.0]], np.float32)
    tx = np.array([0.2, 0.4], np.float32)
    rx = np.array([[0.8, -0.3]], np.float32)
    sc = scenes.Scene(walls, tx, rx, max_order=1, alpha=100.0, smoothing="hard_sigmoid")
    g = _gpu_paths(drt, sc, finder="fpt")[0]
    x_c = 0.2 + 0.6 * 0.4 / 0.7
    i_dir = np.array([0.6, -0.7]) / np.hypot(0.6, 0.7)
    assert g[1, 0] == pytest.approx(x_c, abs=1e-5)
    assert g[1, 1] == pytest.approx(4.0 * i_dir[1] ** 2, rel=1e-4)
    assert g[1, 2] == 0.0
