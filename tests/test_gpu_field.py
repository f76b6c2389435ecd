"""CUDA coherent field (drt_field: Eq. 7 as a sum of complex path fields) against the
FP64 oracle.

Bound per receiver (derived from the FP32 arithmetic): each path field may carry
the forward's relative tolerance 1e-4 on its magnitude, and its phase the FP32
error of the path length, a few units of 2^-24 of L, magnified by 2 pi L / lambda:

    |E_gpu - E_ref| <= mag * (1e-4 + 2 pi (lmax / lambda) * 16 * 2^-24)

with mag the oracle's sum of path-field magnitudes and lmax its longest
contributing path.  Where the field is ill-conditioned in FP32 (large alpha:
two FP32 roundings of the inputs move the oracle's own FP64 field further), at
least 99% of receivers meet that bound and all meet 4x the field's measured
sensitivity.  The power |E|^2 follows: |dP| <= 2 |E| |dE| + |dE|^2.
"""
import numpy as np
import pytest

from paper_2401_11882_gb300 import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

AMP_RTOL = 1e-4
LEN_ULPS = 16 * 2.0 ** -24


@pytest.fixture(scope="module")
def drt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_11882_gb300 as m
    return m


def _gpu(drt, walls, tx, rx, K, alpha, smoothing, lam, eps, refl=0.5, tile=None):
    dev = torch.device("cuda:0")
    w = torch.tensor(np.asarray(walls, np.float32), device=dev)
    t = torch.tensor(np.asarray(tx, np.float32), device=dev)
    r = torch.tensor(np.asarray(rx, np.float32), device=dev)
    E, P = drt.field(w, t, r, K, alpha, smoothing, lam, eps, refl, tile=tile)
    torch.cuda.synchronize()
    E = E.cpu().numpy().astype(np.float64)
    return E[:, 0] + 1j * E[:, 1], P.cpu().numpy().astype(np.float64)


def _sensitivity(oracle_mod, walls, tx, rx, K, alpha, smoothing, lam, eps, refl=0.5, seed=0):
    rng = np.random.default_rng(seed)
    walls, tx, rx = (np.asarray(a, np.float64) for a in (walls, tx, rx))
    base = oracle_mod.field(walls, tx, rx, K, alpha, smoothing, lam, eps, refl)
    out = np.zeros(base.shape)

    def jit(a):
        return a + rng.uniform(-2.0 ** -23, 2.0 ** -23, a.shape) * np.maximum(np.abs(a), 1.0)

    for _ in range(4):
        out = np.maximum(out, np.abs(oracle_mod.field(jit(walls), jit(tx), jit(rx), K, alpha,
                                                      smoothing, lam, eps, refl) - base))
    return out


def _check(oracle_mod, E, P, walls, tx, rx, K, alpha, smoothing, lam, eps, refl=0.5,
           min_strict=1.0):
    ref, mag, lmax = oracle_mod.field(np.asarray(walls, np.float64), np.asarray(tx, np.float64),
                                      np.asarray(rx, np.float64), K, alpha, smoothing, lam, eps,
                                      refl, scales=True)
    bound = mag * (AMP_RTOL + 2 * np.pi * (lmax / lam) * LEN_ULPS) + 1e-30
    err = np.abs(E - ref)
    strict = err <= bound
    if strict.mean() < 1.0:
        sens = _sensitivity(oracle_mod, walls, tx, rx, K, alpha, smoothing, lam, eps, refl)
        wide = np.maximum(bound, 4 * sens)
        bad = np.nonzero(err > wide)[0]
        assert bad.size == 0, (bad[:5], err[bad[:5]], wide[bad[:5]], ref[bad[:5]])
        assert strict.mean() >= min_strict, strict.mean()
    dP = 2 * np.abs(ref) * np.maximum(bound, err) + np.maximum(bound, err) ** 2
    assert np.all(np.abs(P - np.abs(ref) ** 2) <= 1.01 * dP + 1e-6 * np.abs(ref) ** 2 + 1e-30)
    return ref


@pytest.mark.parametrize("smoothing", ["hard_sigmoid", "sigmoid", "step"])
@pytest.mark.parametrize("eps", [0.0, 5.0])
def test_tiny_scene(drt, oracle_mod, smoothing, eps):
    sc = scenes.tiny_scene(alpha=100.0, smoothing=smoothing)
    E, P = _gpu(drt, sc.walls, sc.tx, sc.rx, sc.max_order, sc.alpha, smoothing, 0.05, eps)
    _check(oracle_mod, E, P, sc.walls, sc.tx, sc.rx, sc.max_order, sc.alpha, smoothing, 0.05, eps)


CASES = [
    # (seed, W, R, K, alpha, smoothing, wavelength, eps_r): ragged 32-receiver tiles
    (0, 5, 77, 0, 50.0, "hard_sigmoid", 0.013, 4.0),
    (1, 9, 100, 1, 30.0, "sigmoid", 0.1, 0.0),
    (2, 12, 33, 2, 100.0, "hard_sigmoid", 0.02, 15.0),
    (3, 12, 65, 2, 20.0, "sigmoid", 0.05, 2.5),
    (4, 10, 40, 2, 1.0, "step", 0.01, 81.0),
    (5, 6, 31, 3, 40.0, "hard_sigmoid", 0.07, 0.0),
    (6, 6, 45, 3, 15.0, "sigmoid", 0.03, 6.0),
    (7, 16, 50, 2, 3e4, "hard_sigmoid", 0.04, 3.0),
]


@pytest.mark.parametrize("seed,W,R,K,alpha,smoothing,lam,eps", CASES)
def test_random_scenes(drt, oracle_mod, seed, W, R, K, alpha, smoothing, lam, eps):
    rng = np.random.default_rng(seed)
    sc = scenes.random_small_scene(rng, W, R, K, alpha, smoothing, boundary=(seed % 2 == 0))
    E, P = _gpu(drt, sc.walls, sc.tx, sc.rx, K, alpha, smoothing, lam, eps)
    _check(oracle_mod, E, P, sc.walls, sc.tx, sc.rx, K, alpha, smoothing, lam, eps,
           min_strict=0.99)


def test_benchmark_scene_sampled_receivers(drt, oracle_mod):
    # the 64-wall scene on its full 256 x 256 receiver grid, in the launch configuration
    # the benchmark times; 96 receivers sampled for the oracle
    sc = scenes.large_scene(alpha=100.0, smoothing="hard_sigmoid")
    lam, eps = 0.02, 5.0
    E, P = _gpu(drt, sc.walls, sc.tx, sc.rx, sc.max_order, sc.alpha, sc.smoothing, lam, eps)
    idx = np.random.default_rng(5).choice(sc.rx.shape[0], 96, replace=False)
    _check(oracle_mod, E[idx], P[idx], sc.walls, sc.tx, sc.rx[idx], sc.max_order, sc.alpha,
           sc.smoothing, lam, eps, min_strict=0.99)
    assert np.all(np.isfinite(E)) and np.all(P >= 0)


def test_unit_permittivity_leaves_the_line_of_sight(drt):
    # eps_r = 1: every reflection coefficient is 0, so K = 2 gives exactly the K = 0 field
    rng = np.random.default_rng(12)
    sc = scenes.random_small_scene(rng, 10, 70, 2, 60.0, "hard_sigmoid", boundary=True)
    E2, P2 = _gpu(drt, sc.walls, sc.tx, sc.rx, 2, 60.0, "hard_sigmoid", 0.03, 1.0)
    E0, P0 = _gpu(drt, sc.walls, sc.tx, sc.rx, 0, 60.0, "hard_sigmoid", 0.03, 1.0)
    np.testing.assert_array_equal(E2, E0)
    np.testing.assert_array_equal(P2, P0)


def test_tile_shapes_agree_up_to_sum_order(drt, oracle_mod):
    rng = np.random.default_rng(13)
    sc = scenes.random_small_scene(rng, 10, 90, 2, 60.0, "sigmoid", boundary=True)
    base, _ = _gpu(drt, sc.walls, sc.tx, sc.rx, 2, 60.0, "sigmoid", 0.05, 4.0)
    for kw in (dict(warps_per_cta=1, cands_per_unit=1), dict(warps_per_cta=8, cands_per_unit=1000)):
        E, P = _gpu(drt, sc.walls, sc.tx, sc.rx, 2, 60.0, "sigmoid", 0.05, 4.0,
                    tile=drt.TileConfig(**kw))
        _check(oracle_mod, E, P, sc.walls, sc.tx, sc.rx, 2, 60.0, "sigmoid", 0.05, 4.0)
        assert np.max(np.abs(E - base)) <= 1e-5 * np.max(np.abs(base))


def test_empty_receiver_set(drt):
    sc = scenes.tiny_scene(alpha=100.0, smoothing="hard_sigmoid")
    E, P = _gpu(drt, sc.walls, sc.tx, np.zeros((0, 2), np.float32), 1, 100.0, "hard_sigmoid",
                0.05, 5.0)
    assert E.shape == (0,) and P.shape == (0,)


@pytest.mark.parametrize("smoothing,alpha", [("hard_sigmoid", 100.0), ("sigmoid", 40.0),
                                             ("hard_sigmoid", 1e4)])
def test_two_receivers_per_lane_equal_one_bit_for_bit(drt, smoothing, alpha):
    # same chunking, same per-path arithmetic: the packed obstruction loop gives the
    # same visibilities, so the fields agree exactly (R = 101 leaves a ragged 64-tile)
    rng = np.random.default_rng(21)
    sc = scenes.random_small_scene(rng, 14, 101, 2, alpha, smoothing, boundary=True)
    for K in (0, 1, 2):
        Ep, Pp = _gpu(drt, sc.walls, sc.tx, sc.rx, K, alpha, smoothing, 0.03, 5.0)
        Es, Ps = _gpu(drt, sc.walls, sc.tx, sc.rx, K, alpha, smoothing, 0.03, 5.0,
                      tile=drt.TileConfig(single_rx=True))
        np.testing.assert_array_equal(Ep, Es)
        np.testing.assert_array_equal(Pp, Ps)


# --------------------------------------------------------------------------- adjoint
# Gradient bar for the coherent power: norm-wise 1e-3 relative (as for the power's
# gradient); per element 1e-3 |ref| + 1e-4 max|ref|: a component is a sum of path
# terms whose phases differ, so a small component is a near-cancellation of large
# terms of both signs, and FP32 rounding of those terms sets its absolute error.
FGRAD_FLOOR = 1e-4


def _assert_field_grad_close(gpu, ref, what):
    gpu = np.asarray(gpu, np.float64).ravel()
    ref = np.asarray(ref, np.float64).ravel()
    assert np.linalg.norm(gpu - ref) <= 1e-3 * np.linalg.norm(ref), (what, gpu, ref)
    tol = 1e-3 * np.abs(ref) + FGRAD_FLOOR * np.abs(ref).max()
    bad = np.nonzero(np.abs(gpu - ref) > tol)[0]
    assert bad.size == 0, (what, bad[:5], gpu[bad[:5]], ref[bad[:5]])


def _field_vjp(drt, walls, tx, rx, K, alpha, smoothing, lam, eps, g, wall_grad=True):
    dev = torch.device("cuda:0")
    w = torch.tensor(np.asarray(walls, np.float32), device=dev)
    t = torch.tensor(np.asarray(tx, np.float32), device=dev)
    r = torch.tensor(np.asarray(rx, np.float32), device=dev)
    E, _ = drt.field(w, t, r, K, alpha, smoothing, lam, eps)
    gp = torch.tensor(np.asarray(g, np.float32), device=dev)
    gtx, gw = drt.field_vjp(w, t, r, K, alpha, smoothing, lam, eps, E, gp, wall_grad=wall_grad)
    torch.cuda.synchronize()
    return gtx.cpu().numpy(), (gw.cpu().numpy() if gw is not None else None)


FVJP_CASES = [
    # (seed, W, R, K, alpha, smoothing, wavelength, eps_r)
    (0, 6, 45, 1, 20.0, "sigmoid", 0.05, 4.0),
    (1, 8, 40, 2, 10.0, "sigmoid", 0.08, 0.0),
    (2, 8, 33, 2, 40.0, "hard_sigmoid", 0.05, 6.0),
    (3, 5, 70, 0, 30.0, "hard_sigmoid", 0.03, 0.0),
    (4, 7, 40, 2, 1.0, "step", 0.05, 3.0),
    (5, 5, 36, 3, 15.0, "sigmoid", 0.1, 2.0),
    (6, 9, 50, 2, 100.0, "hard_sigmoid", 0.02, 15.0),
]


@pytest.mark.parametrize("seed,W,R,K,alpha,smoothing,lam,eps", FVJP_CASES)
def test_field_vjp_all_parameters(drt, oracle_mod, seed, W, R, K, alpha, smoothing, lam, eps):
    rng = np.random.default_rng(seed)
    sc = scenes.random_small_scene(rng, W, R, K, alpha, smoothing, boundary=(seed % 2 == 1))
    g = rng.normal(size=sc.n_rx)
    gtx, gw = _field_vjp(drt, sc.walls, sc.tx, sc.rx, K, alpha, smoothing, lam, eps, g)
    ref = oracle_mod.field_gradient(sc.walls, sc.tx, sc.rx, K, alpha, smoothing, lam, eps,
                                    g.astype(np.float32).astype(np.float64), "all", 0.5)
    _assert_field_grad_close(gtx, ref[:2], "grad_tx")
    _assert_field_grad_close(gw.ravel(), ref[2:], "grad_walls")


def test_field_vjp_tx_only_matches_full(drt):
    rng = np.random.default_rng(31)
    sc = scenes.random_small_scene(rng, 8, 60, 2, 50.0, "sigmoid", boundary=True)
    g = rng.normal(size=sc.n_rx)
    a, _ = _field_vjp(drt, sc.walls, sc.tx, sc.rx, 2, 50.0, "sigmoid", 0.04, 5.0, g, False)
    b, _ = _field_vjp(drt, sc.walls, sc.tx, sc.rx, 2, 50.0, "sigmoid", 0.04, 5.0, g, True)
    np.testing.assert_allclose(a, b, rtol=1e-6, atol=1e-6 * np.abs(b).max())


def test_field_power_autograd(drt, oracle_mod):
    rng = np.random.default_rng(32)
    sc = scenes.random_small_scene(rng, 7, 50, 2, 30.0, "hard_sigmoid", boundary=True)
    dev = torch.device("cuda:0")
    w = torch.tensor(sc.walls, device=dev, requires_grad=True)
    t = torch.tensor(sc.tx, device=dev, requires_grad=True)
    r = torch.tensor(sc.rx, device=dev)
    P = drt.field_power(w, t, r, 2, 30.0, "hard_sigmoid", 0.05, 4.0)
    g = torch.tensor(rng.normal(size=sc.n_rx).astype(np.float32), device=dev)
    (P * g).sum().backward()
    ref = oracle_mod.field_gradient(sc.walls, sc.tx, sc.rx, 2, 30.0, "hard_sigmoid", 0.05, 4.0,
                                    g.cpu().numpy().astype(np.float64), "all", 0.5)
    _assert_field_grad_close(t.grad.cpu().numpy(), ref[:2], "grad_tx")
    _assert_field_grad_close(w.grad.cpu().numpy().ravel(), ref[2:], "grad_walls")


def test_field_vjp_benchmark_scene_sampled(drt, oracle_mod):
    # full 256 x 256 launch with g on 12 sampled receivers; TX and 8 wall coordinates
    sc = scenes.large_scene(alpha=100.0, smoothing="hard_sigmoid")
    lam, eps = 0.02, 5.0
    rng = np.random.default_rng(33)
    idx = rng.choice(sc.n_rx, 12, replace=False)
    g = np.zeros(sc.n_rx)
    g[idx] = rng.normal(size=12)
    gtx, gw = _field_vjp(drt, sc.walls, sc.tx, sc.rx, 2, 100.0, "hard_sigmoid", lam, eps, g)
    params = [0, 1] + [2 + 4 * w + c for w in (4, 20, 40) for c in (0, 3)] + [2 + 4 * 63, 2 + 4 * 63 + 1]
    ref = oracle_mod.field_gradient(sc.walls, sc.tx, sc.rx[idx], 2, 100.0, "hard_sigmoid", lam,
                                    eps, g[idx], params, 0.5)
    got = np.concatenate([gtx, gw.ravel()])[params]
    _assert_field_grad_close(got, ref, "sampled gradient")


def test_field_vjp_work_stealing_keeps_the_tx_gradient_bitwise(drt):
    """The coherent-field adjoint takes its units from a counter; its TX gradient is
    added per unit in unit order and does not change between runs."""
    sc = scenes.gradient_scene(alpha=100.0, smoothing="hard_sigmoid")
    g = np.random.default_rng(5).normal(size=sc.n_rx)
    runs = [_field_vjp(drt, sc.walls, sc.tx, sc.rx, 2, 100.0, "hard_sigmoid", 0.02, 5.0, g)
            for _ in range(3)]
    for r in runs[1:]:
        np.testing.assert_array_equal(r[0], runs[0][0])


@pytest.mark.parametrize("single_rx", [False, True])
@pytest.mark.parametrize("seed,W,R,K,alpha,lam,eps", [(40, 6, 45, 1, 20.0, 0.05, 4.0),
                                                      (41, 8, 70, 2, 50.0, 0.03, 0.0),
                                                      (42, 5, 33, 3, 15.0, 0.1, 2.0)])
def test_field_saved_visibilities(drt, oracle_mod, single_rx, seed, W, R, K, alpha, lam, eps):
    """drt_field_save: drt_field's field and power bit for bit, and drt_forward_save's
    visibilities bit for bit (the same obstruction loops); drt_field_vjp_saved:
    drt_field_vjp's gradient within FP32 rounding, and the oracle's."""
    rng = np.random.default_rng(seed)
    sc = scenes.random_small_scene(rng, W, R, K, alpha, "sigmoid", boundary=(seed % 2 == 0))
    dev = torch.device("cuda:0")
    w, t, r = (torch.tensor(x, device=dev) for x in (sc.walls, sc.tx, sc.rx))
    tile = drt.TileConfig(single_rx=True) if single_rx else None
    E, P, sv = drt.field_save(w, t, r, K, alpha, "sigmoid", lam, eps, tile=tile)
    E0, P0 = drt.field(w, t, r, K, alpha, "sigmoid", lam, eps, tile=tile)
    _, sv_power = drt.forward_save(w, t, r, K, alpha, "sigmoid", tile=tile)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(E.cpu().numpy(), E0.cpu().numpy())
    np.testing.assert_array_equal(P.cpu().numpy(), P0.cpu().numpy())
    # compare the written slots only (a path's legs beyond its order are not written)
    order = np.array([0] + [k for k in range(1, K + 1)
                            for _ in range(W * (W - 1) ** (k - 1))])
    written = (np.arange(K + 1)[None, :] <= order[:, None])
    a = sv.cpu().numpy().reshape(-1, K + 1, sc.n_rx)[written]
    b = sv_power.cpu().numpy().reshape(-1, K + 1, sc.n_rx)[written]
    np.testing.assert_array_equal(a, b)
    g = rng.normal(size=sc.n_rx)
    gp = torch.tensor(g.astype(np.float32), device=dev)
    gtx_s, gw_s = drt.field_vjp(w, t, r, K, alpha, "sigmoid", lam, eps, E, gp, saved=sv)
    gtx, gw = drt.field_vjp(w, t, r, K, alpha, "sigmoid", lam, eps, E, gp)
    torch.cuda.synchronize()
    both = lambda x, y: np.concatenate([x.cpu().numpy(), y.cpu().numpy().ravel()])
    got, plain = both(gtx_s, gw_s), both(gtx, gw)
    np.testing.assert_allclose(got, plain, rtol=1e-4, atol=1e-5 * np.abs(plain).max())
    ref = oracle_mod.field_gradient(sc.walls, sc.tx, sc.rx, K, alpha, "sigmoid", lam, eps,
                                    g.astype(np.float32).astype(np.float64), "all", 0.5)
    _assert_field_grad_close(got, ref, "saved-visibility field gradient vs oracle")


def test_field_power_autograd_keeps_the_visibilities(drt, oracle_mod, monkeypatch):
    from paper_2401_11882_gb300 import ops
    rng = np.random.default_rng(43)
    sc = scenes.random_small_scene(rng, 7, 50, 2, 30.0, "sigmoid", boundary=True)
    dev = torch.device("cuda:0")
    calls = []
    real = ops.field_save
    monkeypatch.setattr(ops, "field_save", lambda *a, **k: calls.append(1) or real(*a, **k))
    w = torch.tensor(sc.walls, device=dev, requires_grad=True)
    t = torch.tensor(sc.tx, device=dev, requires_grad=True)
    r = torch.tensor(sc.rx, device=dev)
    P = drt.field_power(w, t, r, 2, 30.0, "sigmoid", 0.05, 4.0)
    g = torch.tensor(rng.normal(size=sc.n_rx).astype(np.float32), device=dev)
    (P * g).sum().backward()
    assert len(calls) == 1
    ref = oracle_mod.field_gradient(sc.walls, sc.tx, sc.rx, 2, 30.0, "sigmoid", 0.05, 4.0,
                                    g.cpu().numpy().astype(np.float64), "all", 0.5)
    _assert_field_grad_close(t.grad.cpu().numpy(), ref[:2], "grad_tx")
    _assert_field_grad_close(w.grad.cpu().numpy().ravel(), ref[2:], "grad_walls")


def test_field_saved_visibilities_full_gradient_scene(drt):
    """128 walls, 128 x 128 receivers, K <= 2 (3.2 GB of visibilities, degenerate legs
    among them): the adjoint reading them equals the recomputing one within 1e-5 of
    the largest component."""
    g = scenes.gradient_scene(alpha=100.0, smoothing="sigmoid")
    dev = torch.device("cuda:0")
    w, t, r = (torch.tensor(x, device=dev) for x in (g.walls, g.tx, g.rx))
    gp = torch.full((g.n_rx,), 1.0 / g.n_rx, device=dev)
    E, _, sv = drt.field_save(w, t, r, 2, 100.0, "sigmoid", 0.02, 5.0)
    a = drt.field_vjp(w, t, r, 2, 100.0, "sigmoid", 0.02, 5.0, E, gp, saved=sv)
    del sv
    b = drt.field_vjp(w, t, r, 2, 100.0, "sigmoid", 0.02, 5.0, E, gp)
    torch.cuda.synchronize()
    for x, y in zip(a, b):
        assert torch.isfinite(x).all()
        assert float((x - y).abs().max()) <= 1e-5 * float(y.abs().max())
