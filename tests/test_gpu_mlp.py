"""Surrogate MLP kernels (BF16 tensor cores, FP32 accumulate) against the FP64
MLP oracle with the same BF16 rounding points; training and the search pipeline."""
import numpy as np
import pytest

from oracle import mlp_oracle as M
from paper_2401_11882_gb300 import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sur():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_11882_gb300 import surrogate
    return surrogate


def _model(sur, seed=0, batch=128):
    m = sur.SurrogateMLP("cuda", seed=seed, batch=batch)
    return m


def test_layout_matches_oracle(sur):
    m = _model(sur)
    assert m.n_params == M.n_params()
    np.testing.assert_array_equal(sur.init_params(3), sur.init_params(3))


def test_forward_matches_oracle(sur):
    m = _model(sur, 1, batch=128)
    rng = np.random.default_rng(0)
    theta = (M.init_params(4) + rng.normal(0, 0.01, M.n_params())).astype(np.float32)
    m.set_params(theta)
    x = rng.uniform(0, 1, (300, 2)).astype(np.float32)
    y = m.forward(torch.from_numpy(x)).cpu().numpy()
    ref, _ = M.forward(theta.astype(np.float64), m.freqs.cpu().numpy(), x, emulate_bf16=True)
    np.testing.assert_allclose(y, ref, rtol=2e-3, atol=2e-3 * np.abs(ref).max())
    ref64, _ = M.forward(theta.astype(np.float64), m.freqs.cpu().numpy(), x, emulate_bf16=False)
    np.testing.assert_allclose(y, ref64, rtol=5e-2, atol=5e-2 * np.abs(ref64).max())


def test_loss_gradient_matches_oracle(sur):
    m = _model(sur, 2, batch=192)
    rng = np.random.default_rng(1)
    theta = M.init_params(5).astype(np.float32)
    m.set_params(theta)
    x = rng.uniform(0, 1, (192, 2)).astype(np.float32)
    t = rng.normal(size=192).astype(np.float32)
    loss, grad = m.loss_grad(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    lref, gref = M.loss_grad(theta.astype(np.float64), m.freqs.cpu().numpy(), x, t, emulate_bf16=True)
    assert float(loss) == pytest.approx(lref, rel=2e-3)
    g = grad.cpu().numpy()
    assert np.linalg.norm(g - gref) <= 1e-2 * np.linalg.norm(gref)
    # per block: each layer's weight gradient
    L = 0
    for l in range(4):
        k = 64 if l == 0 else 256
        blk = slice(L, L + 256 * k)
        assert np.linalg.norm(g[blk] - gref[blk]) <= 2e-2 * np.linalg.norm(gref[blk])
        L += 256 * k + 256


def test_adam_step_and_shadow(sur):
    m = _model(sur, 3, batch=64)
    rng = np.random.default_rng(2)
    p0 = m.params.cpu().numpy().copy()
    g = rng.normal(size=p0.size).astype(np.float32)
    m.grad.copy_(torch.from_numpy(g))
    m.adam(lr=1e-2)
    m.grad.copy_(torch.from_numpy(g * 0.5))
    m.adam(lr=1e-2)
    p = p0.copy().astype(np.float64)
    mm = np.zeros_like(p)
    vv = np.zeros_like(p)
    for t, gg in enumerate([g, 0.5 * g], 1):
        mm = 0.9 * mm + 0.1 * gg
        vv = 0.999 * vv + 0.001 * gg * gg
        p = p - 1e-2 * (mm / (1 - 0.9 ** t)) / (np.sqrt(vv / (1 - 0.999 ** t)) + 1e-8)
    np.testing.assert_allclose(m.params.cpu().numpy(), p, rtol=1e-5, atol=1e-6)
    assert int(m.step.item()) == 2
    # the shadow holds bf16 copies of the weights (W1 block and its transpose)
    sh = m.shadow.view(torch.bfloat16).float().cpu().numpy()
    W1 = m.params.cpu().numpy()[:256 * 64].reshape(256, 64)
    np.testing.assert_array_equal(sh[:256 * 64].reshape(256, 64), M.bf16(W1))
    np.testing.assert_array_equal(sh[256 * 64:2 * 256 * 64].reshape(64, 256), M.bf16(W1).T)
    # ... and, after w5, every W again in 256 x 32 K-chunks laid out for the tensor
    # cores: element (n, k) of a chunk at byte ((n//8)*4 + k//8)*128 + (n%8)*16 + (k%8)*2
    p_all = m.params.cpu().numpy()
    ks = [64, 256, 256, 256]
    off_w, off_s = 0, sum(2 * 256 * k for k in ks) + 256
    n = np.arange(256)[:, None]
    for k_l in ks:
        W = p_all[off_w:off_w + 256 * k_l].reshape(256, k_l)
        for q in range(k_l // 32):
            k = np.arange(32)[None, :]
            idx = ((n // 8) * 4 + k // 8) * 64 + (n % 8) * 8 + (k % 8)
            chunk = sh[off_s + q * 256 * 32: off_s + (q + 1) * 256 * 32]
            np.testing.assert_array_equal(chunk[idx], M.bf16(W[:, q * 32:(q + 1) * 32]))
        off_w += 256 * k_l + 256
        off_s += 256 * k_l


def test_fit_learns_a_smooth_function(sur):
    m = _model(sur, 4, batch=512)
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, (8192, 2)).astype(np.float32)
    t = (np.sin(3 * x[:, 0]) + np.cos(2 * x[:, 1])).astype(np.float32)
    hist = m.fit(x, t, epochs=15, lr=2e-3, lr_final=1e-4)
    assert hist[-1] < 0.05 * hist[0]
    xt = rng.uniform(0, 1, (1000, 2)).astype(np.float32)
    y = m.forward(torch.from_numpy(xt)).cpu().numpy()
    tt = np.sin(3 * xt[:, 0]) + np.cos(2 * xt[:, 1])
    assert np.sqrt(np.mean((y - tt) ** 2)) < 0.1


def test_sample_objective_matches_single_scene_and_oracle(sur, oracle_mod):
    import paper_2401_11882_gb300 as drt
    sc = scenes.clutter_scene(10, 6, seed=5, max_order=2, alpha=80.0)
    rng = np.random.default_rng(4)
    tx = rng.uniform(0.05, 0.95, (40, 2)).astype(np.float32)
    F = sur.sample_objective(sc, tx, chunk=16)
    dev = torch.device("cuda:0")
    w, r = torch.tensor(sc.walls, device=dev), torch.tensor(sc.rx, device=dev)
    for i in (0, 7, 23, 39):
        P = drt.forward(w, torch.tensor(tx[i], device=dev), r, 2, 80.0, sc.smoothing)
        assert F[i] == pytest.approx(float(P.min()), rel=1e-5)
        Pref = oracle_mod.power(sc.walls, tx[i], sc.rx, 2, 80.0, sc.smoothing)
        assert F[i] == pytest.approx(Pref.min(), rel=1e-4, abs=1e-10 * Pref.max())


def test_sample_objective_receiver_order_does_not_change_F(sur):
    # the sampler passes the receivers in Z-order; F = min over receivers is the
    # same bit for bit as with the original order and the same tile
    from paper_2401_11882_gb300.batched import BatchedDescent
    from paper_2401_11882_gb300.ops import TileConfig
    rng = np.random.default_rng(5)
    sc = scenes.clutter_scene(16, 1, seed=8, max_order=2, alpha=100.0,
                              rx=rng.uniform(0.05, 0.95, (200, 2)).astype(np.float32))
    tx = rng.uniform(0.05, 0.95, (300, 2)).astype(np.float32)
    F = sur.sample_objective(sc, tx)
    b = scenes.SceneBatch(sc.walls, np.array([0, sc.n_walls], np.int32), sc.rx,
                          np.array([0, sc.n_rx], np.int32), np.array([2], np.int32), tx[None],
                          sc.alpha, sc.smoothing, sc.refl_coef)
    bd = BatchedDescent(b, tile=TileConfig(warps_per_cta=1, cull_invalid=True), alpha=sc.alpha)
    F0 = (-bd.evaluate()).cpu().numpy()
    bd.close()
    np.testing.assert_array_equal(F, F0)


def test_surrogate_proposals_beat_random_points(sur):
    sc = scenes.clutter_scene(12, 4, seed=6, max_order=1, alpha=50.0)
    search = sur.SurrogateSearch(sc, batch=512, seed=1)
    x, F = search.generate(16384, seed=1)
    search.train(x, F, epochs=12)
    props = search.propose(k=16, grid=128, min_sep=0.05)
    Fp = sur.sample_objective(sc, props)
    rng = np.random.default_rng(9)
    Fr = sur.sample_objective(sc, rng.uniform(0, 1, (256, 2)).astype(np.float32))
    assert np.median(Fp) > np.median(Fr)
    assert Fp.max() >= np.quantile(F, 0.95)
