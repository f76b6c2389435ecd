"""Hand-written adjoint (drt_vjp) against the FP64 oracle's exact derivatives and
against central finite differences."""
import numpy as np
import pytest

from parity import assert_grad_close
from paper_2401_11882_gb300 import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def drt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_11882_gb300 as m
    return m


def _tensors(sc):
    dev = torch.device("cuda:0")
    return (torch.tensor(sc.walls, device=dev), torch.tensor(sc.tx, device=dev),
            torch.tensor(sc.rx, device=dev))


def _vjp(drt, sc, g, wall_grad=True, tile=None):
    w, t, r = _tensors(sc)
    gtx, gw = drt.vjp(w, t, r, sc.max_order, sc.alpha, sc.smoothing,
                      torch.tensor(g, dtype=torch.float32, device=w.device), sc.refl_coef,
                      wall_grad=wall_grad, tile=tile)
    torch.cuda.synchronize()
    return gtx.cpu().numpy(), (gw.cpu().numpy() if gw is not None else None)


def _oracle_grad(oracle_mod, sc, g, params="all"):
    return oracle_mod.gradient(sc.walls, sc.tx, sc.rx, sc.max_order, sc.alpha, sc.smoothing, g,
                               params, sc.refl_coef)


CASES = [
    (0, 6, 45, 1, 20.0, "sigmoid"),
    (1, 8, 40, 2, 10.0, "sigmoid"),
    (2, 8, 33, 2, 40.0, "hard_sigmoid"),
    (3, 5, 70, 0, 30.0, "hard_sigmoid"),
    (4, 7, 40, 2, 1.0, "step"),
    (5, 5, 36, 3, 15.0, "sigmoid"),
    (6, 10, 64, 2, 100.0, "hard_sigmoid"),
    (7, 9, 50, 2, 100.0, "sigmoid"),
    (8, 6, 40, 2, 0.0, "sigmoid"),
]


@pytest.mark.parametrize("seed,W,R,K,alpha,smoothing", CASES)
def test_dense_vjp_all_parameters(drt, oracle_mod, seed, W, R, K, alpha, smoothing):
    rng = np.random.default_rng(seed)
    sc = scenes.random_small_scene(rng, W, R, K, alpha, smoothing, boundary=(seed % 2 == 1))
    g = rng.normal(size=sc.n_rx)
    gtx, gw = _vjp(drt, sc, g)
    ref = _oracle_grad(oracle_mod, sc, g.astype(np.float32).astype(np.float64))
    assert_grad_close(gtx, ref[:2], "grad_tx")
    assert_grad_close(gw.ravel(), ref[2:], "grad_walls")


@pytest.mark.parametrize("smoothing", ["hard_sigmoid", "sigmoid", "step"])
def test_tiny_scene_loss_gradient(drt, oracle_mod, smoothing):
    sc = scenes.tiny_scene(alpha=100.0, smoothing=smoothing)
    w, t, r = _tensors(sc)
    w.requires_grad_(True)
    t.requires_grad_(True)
    L = drt.objective(w, t, r, sc.max_order, sc.alpha, sc.smoothing)
    L.backward()
    P = oracle_mod.power(sc.walls, sc.tx, sc.rx, sc.max_order, sc.alpha, sc.smoothing)
    _, am = oracle_mod.loss(P)
    g = np.zeros(sc.n_rx)
    g[am] = -1.0
    ref = _oracle_grad(oracle_mod, sc, g)
    assert_grad_close(t.grad.cpu().numpy(), ref[:2], "grad_tx")
    assert_grad_close(w.grad.cpu().numpy().ravel(), ref[2:], "grad_walls")


def test_against_central_differences(drt, oracle_mod):
    # h = 1e-4 central differences of the FP64 forward, smooth case.
    rng = np.random.default_rng(21)
    sc = scenes.random_small_scene(rng, 6, 30, 2, 10.0, "sigmoid", boundary=True)
    g = rng.normal(size=sc.n_rx)
    gtx, gw = _vjp(drt, sc, g)
    h = 1e-4
    walls = sc.walls.astype(np.float64)
    tx = sc.tx.astype(np.float64)
    fd = []
    for p in range(2 + walls.size):
        dt, dw = np.zeros(2), np.zeros(walls.size)
        if p < 2:
            dt[p] = h
        else:
            dw[p - 2] = h
        Pp = oracle_mod.power(walls + dw.reshape(walls.shape), tx + dt, sc.rx, 2, 10.0, "sigmoid")
        Pm = oracle_mod.power(walls - dw.reshape(walls.shape), tx - dt, sc.rx, 2, 10.0, "sigmoid")
        fd.append(g @ (Pp - Pm) / (2 * h))
    fd = np.array(fd)
    assert_grad_close(np.concatenate([gtx, gw.ravel()]), fd, "adjoint vs central FD")


@pytest.mark.parametrize("smoothing", ["hard_sigmoid", "sigmoid"])
def test_gradient_scene_sampled(drt, oracle_mod, smoothing):
    # 128 random walls, 128 x 128 receivers, K <= 2 (16385 sequences): the VJP is linear in g,
    # so g = indicator of 8 sampled receivers is checked against the oracle's derivative of
    # their summed power, for the TX and 10 sampled wall coordinates.
    sc = scenes.gradient_scene(alpha=100.0, smoothing=smoothing)
    rng = np.random.default_rng(0)
    idx = rng.choice(sc.n_rx, 8, replace=False)
    g = np.zeros(sc.n_rx)
    g[idx] = 1.0
    gtx, gw = _vjp(drt, sc, g)
    coords = rng.choice(4 * sc.n_walls, 10, replace=False)
    sub = sc.replace(rx=sc.rx[idx])
    ref = _oracle_grad(oracle_mod, sub, np.ones(8), [0, 1] + [2 + int(c) for c in coords])
    assert_grad_close(gtx, ref[:2], "grad_tx")
    got = gw.ravel()[coords]
    # per-coordinate: each sampled wall coordinate against its exact derivative
    np.testing.assert_allclose(got, ref[2:], rtol=1e-3,
                               atol=1e-3 * 1e-3 * max(np.abs(ref[2:]).max(), np.abs(ref[:2]).max()))


def test_tx_only_matches_full(drt):
    rng = np.random.default_rng(5)
    sc = scenes.random_small_scene(rng, 9, 50, 2, 50.0, "hard_sigmoid", boundary=True)
    g = rng.normal(size=sc.n_rx)
    a, _ = _vjp(drt, sc, g, wall_grad=False)
    b, _ = _vjp(drt, sc, g, wall_grad=True)
    np.testing.assert_allclose(a, b, rtol=1e-6, atol=1e-6 * np.abs(b).max())


def test_sparse_g_skips_but_matches(drt, oracle_mod):
    rng = np.random.default_rng(6)
    sc = scenes.random_small_scene(rng, 8, 100, 2, 30.0, "sigmoid", boundary=True)
    g = np.zeros(sc.n_rx)
    g[57] = 2.0
    gtx, gw = _vjp(drt, sc, g)
    ref = _oracle_grad(oracle_mod, sc, g)
    assert_grad_close(gtx, ref[:2], "grad_tx")
    assert_grad_close(gw.ravel(), ref[2:], "grad_walls")


def test_autograd_matches_direct_vjp(drt):
    rng = np.random.default_rng(7)
    sc = scenes.random_small_scene(rng, 7, 40, 2, 25.0, "sigmoid", boundary=True)
    w, t, r = _tensors(sc)
    w.requires_grad_(True)
    t.requires_grad_(True)
    P = drt.power(w, t, r, sc.max_order, sc.alpha, sc.smoothing)
    gvec = torch.randn_like(P)
    (P * gvec).sum().backward()
    gtx, gw = _vjp(drt, sc, gvec.cpu().numpy())
    # wall gradients are summed with shared-memory atomics, whose order varies
    np.testing.assert_allclose(t.grad.cpu().numpy(), gtx, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(w.grad.cpu().numpy(), gw, rtol=2e-5, atol=1e-6 * np.abs(gw).max())


def test_vjp_deterministic_tx(drt):
    sc = scenes.clutter_scene(12, 8, seed=1, max_order=2, alpha=50.0)
    g = np.random.default_rng(0).normal(size=sc.n_rx)
    a, _ = _vjp(drt, sc, g, wall_grad=False)
    b, _ = _vjp(drt, sc, g, wall_grad=False)
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("smoothing", ["hard_sigmoid", "sigmoid"])
def test_work_stealing_keeps_the_tx_gradient_bitwise(drt, smoothing):
    """Warps take their units from a counter, so which warp handles which unit
    changes from run to run; the TX gradient is added per unit in unit order and
    must not change, with and without the wall gradient (the gradient scene: 128
    walls, 128 x 128 receivers, 16,385 sequences, uneven units after the exact
    zero-gradient skip)."""
    sc = scenes.gradient_scene(alpha=100.0, smoothing=smoothing)
    g = np.random.default_rng(3).normal(size=sc.n_rx)
    for wall_grad in (True, False):
        runs = [_vjp(drt, sc, g, wall_grad=wall_grad) for _ in range(3)]
        for gtx, gw in runs[1:]:
            np.testing.assert_array_equal(gtx, runs[0][0])
            if wall_grad:
                np.testing.assert_allclose(gw, runs[0][1], rtol=1e-4,
                                           atol=1e-5 * np.abs(runs[0][1]).max())


@pytest.mark.parametrize("seed,W,R,K,alpha,smoothing", CASES)
def test_min_loss_vjp_matches_oracle(drt, oracle_mod, seed, W, R, K, alpha, smoothing):
    # loss = -P[argmin]: the one-receiver kernel (lanes = candidates) against the oracle
    rng = np.random.default_rng(100 + seed)
    sc = scenes.random_small_scene(rng, W, R, K, alpha, smoothing, boundary=(seed % 2 == 0))
    w, t, r = _tensors(sc)
    P = drt.forward(w, t, r, sc.max_order, sc.alpha, sc.smoothing)
    loss, am = drt.min_loss(P)
    gl = torch.tensor([0.75], device=w.device)
    gtx, gw = drt.min_loss_vjp(w, t, r, sc.max_order, sc.alpha, sc.smoothing, am, gl)
    torch.cuda.synchronize()
    g = np.zeros(sc.n_rx)
    g[int(am)] = -0.75
    ref = _oracle_grad(oracle_mod, sc, g)
    assert_grad_close(gtx.cpu().numpy(), ref[:2], "grad_tx")
    assert_grad_close(gw.cpu().numpy().ravel(), ref[2:], "grad_walls")
    # and the receiver-tile kernel with the same one-hot weight
    gtx2, gw2 = _vjp(drt, sc, g)
    np.testing.assert_allclose(gtx.cpu().numpy(), gtx2, rtol=1e-5, atol=1e-6 * np.abs(gtx2).max())


def test_min_loss_vjp_large_scene(drt, oracle_mod):
    # the benchmark step's gradient: 64 walls, 256 x 256 receivers, K <= 2, alpha = 100
    sc = scenes.large_scene(alpha=100.0, smoothing="hard_sigmoid")
    w, t, r = _tensors(sc)
    P = drt.forward(w, t, r, 2, 100.0, "hard_sigmoid")
    loss, am = drt.min_loss(P)
    gtx, gw = drt.min_loss_vjp(w, t, r, 2, 100.0, "hard_sigmoid", am)
    torch.cuda.synchronize()
    i = int(am)
    Pref = oracle_mod.power(sc.walls, sc.tx, sc.rx[i:i + 1], 2, 100.0, "hard_sigmoid")
    assert float(loss) == pytest.approx(-Pref[0], rel=1e-4)
    coords = np.random.default_rng(1).choice(4 * sc.n_walls, 12, replace=False)
    sub = sc.replace(rx=sc.rx[i:i + 1])
    ref = _oracle_grad(oracle_mod, sub, np.array([-1.0]), [0, 1] + [2 + int(c) for c in coords])
    assert_grad_close(gtx.cpu().numpy(), ref[:2], "grad_tx")
    got = gw.cpu().numpy().ravel()[coords]
    np.testing.assert_allclose(got, ref[2:], rtol=1e-3,
                               atol=1e-6 * max(np.abs(ref).max(), 1e-30))


PAIR_CASES = [
    # (seed, W, R, K, alpha): receiver counts around the 64-receiver tile of the
    # sigmoid adjoint's two-receivers-per-lane kernel (a lone receiver, half tiles,
    # ragged tails), every order, alpha from 0 to 1000
    (40, 5, 1, 0, 30.0),
    (41, 8, 33, 1, 20.0),
    (42, 9, 63, 2, 100.0),
    (43, 9, 64, 2, 10.0),
    (44, 10, 65, 2, 300.0),
    (45, 6, 130, 3, 40.0),
    (46, 12, 97, 2, 0.0),
    (47, 14, 80, 2, 1000.0),
]


@pytest.mark.parametrize("wall_grad", [True, False])
@pytest.mark.parametrize("seed,W,R,K,alpha", PAIR_CASES)
def test_sigmoid_two_receivers_per_lane(drt, oracle_mod, seed, W, R, K, alpha, wall_grad):
    # the paired adjoint against the one-receiver-per-lane kernel (same per-path
    # arithmetic up to rounding; the receivers' sums are grouped differently) and
    # against the oracle's exact gradient
    rng = np.random.default_rng(seed)
    sc = scenes.random_small_scene(rng, W, R, K, alpha, "sigmoid", boundary=(seed % 2 == 0))
    g = rng.normal(size=sc.n_rx)
    gtx, gw = _vjp(drt, sc, g, wall_grad=wall_grad)
    gtx1, gw1 = _vjp(drt, sc, g, wall_grad=wall_grad, tile=drt.TileConfig(single_rx=True))
    scale = np.linalg.norm(gtx1)
    assert np.linalg.norm(gtx - gtx1) <= 1e-5 * scale + 1e-30, (gtx, gtx1)
    ref = _oracle_grad(oracle_mod, sc, g.astype(np.float32).astype(np.float64))
    assert_grad_close(gtx, ref[:2], "grad_tx")
    if wall_grad:
        assert np.linalg.norm(gw - gw1) <= 1e-5 * np.linalg.norm(gw1) + 1e-30
        assert_grad_close(gw.ravel(), ref[2:], "grad_walls")
    else:
        assert gw is None


def test_sigmoid_pair_adjoint_on_gradient_scene(drt):
    # the benchmark's dense adjoint (128 walls, 16384 receivers, 16385 sequences): both
    # kernels agree on every gradient component
    sc = scenes.gradient_scene(alpha=100.0, smoothing="sigmoid")
    g = np.full(sc.n_rx, 1.0 / sc.n_rx)
    gtx, gw = _vjp(drt, sc, g)
    gtx1, gw1 = _vjp(drt, sc, g, tile=drt.TileConfig(single_rx=True))
    assert np.linalg.norm(gtx - gtx1) <= 1e-5 * np.linalg.norm(gtx1)
    assert np.linalg.norm(gw - gw1) <= 1e-5 * np.linalg.norm(gw1)
    assert np.all(np.abs(gw - gw1) <= 1e-4 * np.abs(gw1) + 1e-6 * np.abs(gw1).max())


SAVED_CASES = [   # sigmoid: (seed, W, R, K, alpha)
    (60, 6, 45, 1, 20.0),
    (61, 8, 70, 2, 50.0),
    (62, 5, 33, 3, 15.0),
    (63, 9, 64, 2, 100.0),
]


@pytest.mark.parametrize("seed,W,R,K,alpha", SAVED_CASES)
@pytest.mark.parametrize("single_rx", [False, True])
def test_saved_visibilities(drt, oracle_mod, seed, W, R, K, alpha, single_rx):
    """drt_forward_save: the power of drt_forward bit for bit, and every path's leg
    visibilities as the oracle computes them; drt_vjp_saved: drt_vjp's gradient (the
    first wall sweep replaced by the saved values) and the oracle's."""
    rng = np.random.default_rng(seed)
    sc = scenes.random_small_scene(rng, W, R, K, alpha, "sigmoid", boundary=(seed % 2 == 0))
    w, t, r = _tensors(sc)
    tile = drt.TileConfig(single_rx=True) if single_rx else None
    P, saved = drt.forward_save(w, t, r, K, alpha, "sigmoid", sc.refl_coef, tile=tile)
    P_plain = drt.forward(w, t, r, K, alpha, "sigmoid", sc.refl_coef, tile=tile)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(P.cpu().numpy(), P_plain.cpu().numpy())
    sv = saved.cpu().numpy().astype(np.float64).reshape(-1, K + 1, sc.n_rx)
    n_checked = 0
    for ri in range(0, sc.n_rx, 7):
        ref = oracle_mod.paths(sc.walls, sc.tx, sc.rx[ri], K, alpha, "sigmoid", sc.refl_coef)
        ok = (ref["validity"] > 0) & ~ref["degenerate"].astype(bool)
        for c in np.nonzero(ok)[0]:
            k = int(ref["order"][c])
            got, want = sv[c, :k + 1, ri], ref["vis"][c, :k + 1]
            # a factor s(alpha z) moves by alpha (1 - s) dz relative for an FP32 error dz
            # in a smoothed distance of the backtraced vertices (~1e-6 after two
            # reflections): 2e-3 covers alpha <= 100
            np.testing.assert_allclose(got, want, rtol=2e-3, atol=1e-6)
            n_checked += k + 1
    assert n_checked > 50
    g = torch.tensor(rng.normal(size=sc.n_rx), dtype=torch.float32, device=w.device)
    gtx_s, gw_s = drt.vjp(w, t, r, K, alpha, "sigmoid", g, sc.refl_coef, tile=tile, saved=saved)
    gtx, gw = drt.vjp(w, t, r, K, alpha, "sigmoid", g, sc.refl_coef, tile=tile)
    torch.cuda.synchronize()
    assert_grad_close(gtx_s.cpu().numpy(), gtx.cpu().numpy(), "saved vs recomputed TX gradient")
    assert_grad_close(gw_s.cpu().numpy().ravel(), gw.cpu().numpy().ravel(),
                      "saved vs recomputed wall gradient")
    ref = _oracle_grad(oracle_mod, sc, g.cpu().numpy().astype(np.float64))
    assert_grad_close(np.concatenate([gtx_s.cpu().numpy(), gw_s.cpu().numpy().ravel()]), ref,
                      "saved-visibility gradient vs oracle")
    # the TX-only adjoint reads them too
    gtx_only, _ = drt.vjp(w, t, r, K, alpha, "sigmoid", g, sc.refl_coef, wall_grad=False,
                          tile=tile, saved=saved)
    torch.cuda.synchronize()
    assert_grad_close(gtx_only.cpu().numpy(), gtx.cpu().numpy(), "TX-only with saved values")


def test_power_autograd_keeps_the_visibilities_for_the_sigmoid(drt, oracle_mod, monkeypatch):
    from paper_2401_11882_gb300 import ops
    rng = np.random.default_rng(64)
    sc = scenes.random_small_scene(rng, 7, 50, 2, 40.0, "sigmoid", boundary=True)
    dev = torch.device("cuda:0")
    g = torch.tensor(rng.normal(size=sc.n_rx), dtype=torch.float32, device=dev)
    grads = {}
    calls = []
    real = ops.forward_save
    monkeypatch.setattr(ops, "forward_save", lambda *a, **k: calls.append(1) or real(*a, **k))
    for limit in (None, "0"):
        if limit is not None:
            monkeypatch.setenv("DRT_SAVED_VIS_MAX_BYTES", limit)
        w = torch.tensor(sc.walls, device=dev, requires_grad=True)
        t = torch.tensor(sc.tx, device=dev, requires_grad=True)
        r = torch.tensor(sc.rx, device=dev)
        P = drt.power(w, t, r, 2, 40.0, "sigmoid")
        (P * g).sum().backward()
        grads[limit] = (t.grad.cpu().numpy(), w.grad.cpu().numpy())
    assert len(calls) == 1                 # kept the first time, recomputed with limit 0
    assert_grad_close(grads[None][0], grads["0"][0], "autograd TX gradient, saved vs not")
    assert_grad_close(grads[None][1].ravel(), grads["0"][1].ravel(),
                      "autograd wall gradient, saved vs not")


@pytest.mark.parametrize("single_rx", [False, True])
def test_saved_visibilities_with_degenerate_paths(drt, single_rx):
    """Receivers where a path has a zero-length leg (one on the transmitter, one on an
    axis-aligned wall's line, where the reflection point is the receiver itself): the
    forward saves no finite visibilities for those paths, and the adjoint that reads
    them still gives drt_vjp's finite gradient."""
    rng = np.random.default_rng(65)
    sc = scenes.random_small_scene(rng, 8, 40, 2, 60.0, "sigmoid", boundary=True)
    sc.walls[4] = np.array([0.2, 0.5, 0.8, 0.5], np.float32)
    sc.tx[:] = np.array([0.35, 0.25], np.float32)
    sc.rx[0] = sc.tx
    sc.rx[1] = np.array([0.5, 0.5], np.float32)
    sc.rx[33] = np.array([0.625, 0.5], np.float32)
    w, t, r = _tensors(sc)
    tile = drt.TileConfig(single_rx=True) if single_rx else None
    P, saved = drt.forward_save(w, t, r, 2, 60.0, "sigmoid", sc.refl_coef, tile=tile)
    assert torch.isfinite(P).all()
    g = torch.tensor(rng.normal(size=sc.n_rx), dtype=torch.float32, device=w.device)
    gtx_s, gw_s = drt.vjp(w, t, r, 2, 60.0, "sigmoid", g, sc.refl_coef, tile=tile, saved=saved)
    gtx, gw = drt.vjp(w, t, r, 2, 60.0, "sigmoid", g, sc.refl_coef, tile=tile)
    torch.cuda.synchronize()
    for a in (gtx_s, gw_s, gtx, gw):
        assert torch.isfinite(a).all()
    assert_grad_close(gtx_s.cpu().numpy(), gtx.cpu().numpy(), "TX gradient, degenerate paths")
    assert_grad_close(gw_s.cpu().numpy().ravel(), gw.cpu().numpy().ravel(),
                      "wall gradient, degenerate paths")


def test_saved_visibilities_full_gradient_scene(drt):
    """The 128-wall, 128 x 128-receiver scene at K <= 2 (16,385 sequences, 3.2 GB of
    saved visibilities; 19 path legs are degenerate there): the adjoint reading them
    equals the recomputing adjoint within 1e-5 of the largest component."""
    g = scenes.gradient_scene()
    w, t, r = _tensors(g)
    gp = torch.full((g.n_rx,), 1.0 / g.n_rx, device=w.device)
    _, saved = drt.forward_save(w, t, r, 2, 100.0, "sigmoid")
    a = drt.vjp(w, t, r, 2, 100.0, "sigmoid", gp, saved=saved)
    del saved
    b = drt.vjp(w, t, r, 2, 100.0, "sigmoid", gp)
    torch.cuda.synchronize()
    for x, y in zip(a, b):
        assert torch.isfinite(x).all()
        assert float((x - y).abs().max()) <= 1e-5 * float(y.abs().max())
