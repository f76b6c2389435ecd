"""Batched descent (drt_batch_*) against the single-scene calls and the oracle,
scene by scene; graph replay, determinism and checkpoint/resume."""
import numpy as np
import pytest

from parity import assert_grad_close, assert_power_close
from paper_2401_11882_gb300 import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def drt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_11882_gb300 as m
    return m


def _small_batch(seed=0, n=6, smoothing="hard_sigmoid", alpha=100.0):
    # uneven: W 5..24 (4 boundary walls + random), R 33..100 (ragged tiles), K in {0, 1, 2}
    return scenes.scene_batch(n, seed, walls_range=(5, 24), rx_range=(33, 100), orders=(0, 1, 2),
                              n_tx=3, alpha=alpha, smoothing=smoothing)


def _reference_steps(drt, batch, n_steps, lr=1e-2, b1=0.9, b2=0.999, eps=1e-8, alpha=100.0):
    """Single-scene forward + min loss + min-loss adjoint per problem, Adam in float32 numpy."""
    dev = torch.device("cuda:0")
    S, T = batch.n_scenes, batch.tx0.shape[1]
    tx = batch.tx0.reshape(S * T, 2).astype(np.float32).copy()
    m = np.zeros_like(tx)
    v = np.zeros_like(tx)
    losses = []
    for step in range(n_steps):
        L = np.zeros(S * T, np.float32)
        G = np.zeros_like(tx)
        for s in range(S):
            sc = batch.scene(s)
            w = torch.tensor(sc.walls, device=dev)
            r = torch.tensor(sc.rx, device=dev)
            for t in range(T):
                p = s * T + t
                txp = torch.tensor(tx[p], device=dev)
                P = drt.forward(w, txp, r, sc.max_order, alpha, batch.smoothing)
                loss, am = drt.min_loss(P)
                gtx, _ = drt.min_loss_vjp(w, txp, r, sc.max_order, alpha, batch.smoothing, am,
                                          wall_grad=False)
                L[p] = float(loss)
                G[p] = gtx.cpu().numpy()
        losses.append(L)
        t1 = step + 1
        m = (np.float32(b1) * m + np.float32(1 - b1) * G).astype(np.float32)
        v = (np.float32(b2) * v + np.float32(1 - b2) * G * G).astype(np.float32)
        mh = m / np.float32(1 - b1 ** t1)
        vh = v / np.float32(1 - b2 ** t1)
        tx = np.clip(tx - np.float32(lr) * mh / (np.sqrt(vh) + np.float32(eps)), 0.0, 1.0).astype(np.float32)
    return tx, m, v, losses


def test_one_step_matches_single_scene_calls(drt, oracle_mod):
    from paper_2401_11882_gb300.batched import BatchedDescent
    batch = _small_batch(0)
    bd = BatchedDescent(batch, history=4)
    bd.run(1)
    torch.cuda.synchronize()
    tx_ref, m_ref, v_ref, losses = _reference_steps(drt, batch, 1)
    loss = bd.history[0].cpu().numpy()
    assert_power_close(-loss, -losses[0], "batched loss vs single-scene loss")
    g_batched = bd.m.cpu().numpy() / 0.1          # m_1 = (1 - beta1) g
    g_single = m_ref / 0.1
    assert_grad_close(g_batched.ravel(), g_single.ravel(), "batched TX gradient vs single-scene")
    np.testing.assert_allclose(bd.tx.cpu().numpy(), tx_ref, atol=2e-6)
    # and against the oracle for a few problems
    T = batch.tx0.shape[1]
    for p in (0, 4, 10, 17):
        s, t = divmod(p, T)
        sc = batch.scene(s, t)
        Pref = oracle_mod.power(sc.walls, sc.tx, sc.rx, sc.max_order, 100.0, batch.smoothing)
        lref, am = oracle_mod.loss(Pref)
        assert abs(loss[p] - lref) <= 1e-4 * abs(lref) + 1e-10 * np.abs(Pref).max()
        g = np.zeros(sc.n_rx)
        g[am] = -1.0
        gref = oracle_mod.gradient(sc.walls, sc.tx, sc.rx, sc.max_order, 100.0, batch.smoothing,
                                   g, "tx")
        assert_grad_close(g_batched[p], gref, f"problem {p} vs oracle")
    bd.close()


@pytest.mark.parametrize("smoothing", ["sigmoid", "hard_sigmoid"])
def test_three_steps_match_reference_loop(drt, smoothing):
    from paper_2401_11882_gb300.batched import BatchedDescent
    batch = _small_batch(1, n=4, smoothing=smoothing, alpha=30.0)
    bd = BatchedDescent(batch, alpha=30.0, history=3)
    bd.run(3)
    torch.cuda.synchronize()
    tx_ref, m_ref, v_ref, losses = _reference_steps(drt, batch, 3, alpha=30.0)
    np.testing.assert_allclose(bd.tx.cpu().numpy(), tx_ref, atol=5e-6)
    hist = bd.history.cpu().numpy()
    for i in range(3):
        assert_power_close(-hist[i], -losses[i], f"loss of step {i}")
    bd.close()


def test_graph_and_direct_launch_agree_and_are_deterministic(drt):
    from paper_2401_11882_gb300.batched import BatchedDescent
    batch = _small_batch(2)
    a = BatchedDescent(batch, history=5)
    a.run(5, use_graph=True)
    b = BatchedDescent(batch, history=5)
    b.run(5, use_graph=False)
    c = BatchedDescent(batch, history=5)
    c.run(5, use_graph=True)
    torch.cuda.synchronize()
    for x, y in ((a, b), (a, c)):
        np.testing.assert_array_equal(x.tx.cpu().numpy(), y.tx.cpu().numpy())
        np.testing.assert_array_equal(x.history.cpu().numpy(), y.history.cpu().numpy())
    for o in (a, b, c):
        o.close()


@pytest.mark.parametrize("smoothing,alpha", [("hard_sigmoid", 100.0), ("sigmoid", 60.0),
                                             ("hard_sigmoid", 2e4)])
def test_two_receivers_per_lane_match_one_per_lane_bitwise(drt, smoothing, alpha):
    # the batched forward's 64-receiver tiles (packed loop; above alpha = 1e4 two
    # masked single-receiver calls) against 32-receiver tiles: same operations per
    # receiver, same candidate blocks per warp, same sum order
    from paper_2401_11882_gb300.batched import BatchedDescent
    batch = _small_batch(4, n=7, smoothing=smoothing, alpha=alpha)
    a = BatchedDescent(batch, history=4, alpha=alpha)
    b = BatchedDescent(batch, history=4, alpha=alpha, tile=drt.TileConfig(single_rx=True))
    assert a.info()["forward_units"] < b.info()["forward_units"]
    a.run(4)
    b.run(4)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(a.history.cpu().numpy(), b.history.cpu().numpy())
    np.testing.assert_array_equal(a.tx.cpu().numpy(), b.tx.cpu().numpy())
    a.close()
    b.close()


def test_checkpoint_resume_is_bitwise(drt, tmp_path):
    from paper_2401_11882_gb300.batched import BatchedDescent
    batch = _small_batch(3)
    straight = BatchedDescent(batch)
    straight.run(6)
    first = BatchedDescent(batch)
    first.run(3)
    path = str(tmp_path / "state.npz")
    first.save(path)
    first.close()
    second = BatchedDescent(batch)
    second.load(path)
    second.run(3)
    a, b = straight.state_dict(), second.state_dict()
    assert a["step"] == b["step"] == 6
    for k in ("tx", "m", "v"):
        np.testing.assert_array_equal(a[k], b[k])
    straight.close()
    second.close()


def test_alpha_schedule_is_applied_per_step(drt):
    from paper_2401_11882_gb300.batched import BatchedDescent, geometric_alpha
    batch = _small_batch(4, n=3, smoothing="sigmoid")
    sched = geometric_alpha(1.0, 100.0, 4)
    bd = BatchedDescent(batch, alpha=sched, history=4, lr=0.0)   # lr 0: the TX never moves
    bd.run(4)
    torch.cuda.synchronize()
    hist = bd.history.cpu().numpy()
    dev = torch.device("cuda:0")
    T = batch.tx0.shape[1]
    for i, a in enumerate(sched):
        for p in range(batch.n_scenes * T):
            s, t = divmod(p, T)
            sc = batch.scene(s, t)
            P = drt.forward(torch.tensor(sc.walls, device=dev), torch.tensor(sc.tx, device=dev),
                            torch.tensor(sc.rx, device=dev), sc.max_order, float(a), "sigmoid")
            l, _ = drt.min_loss(P)
            assert hist[i, p] == pytest.approx(float(l), rel=1e-5, abs=1e-12)
    bd.close()


def test_tx_stays_in_box(drt):
    from paper_2401_11882_gb300.batched import BatchedDescent
    batch = _small_batch(5)
    bd = BatchedDescent(batch, lr=0.2, box=(0.1, 0.2, 0.8, 0.9))
    bd.run(10)
    tx = bd.state_dict()["tx"]
    assert tx[:, 0].min() >= 0.1 and tx[:, 0].max() <= 0.8
    assert tx[:, 1].min() >= 0.2 and tx[:, 1].max() <= 0.9
    bd.close()


def test_autotuned_tile_runs_the_same_descent(drt):
    """autotune.tune_batch times every batch candidate (warps per CTA x CTAs per SM)
    on the device and returns the fastest; the tile moves work between CTAs but not
    the candidates' order within a receiver's sum, so the descent is the same bit for
    bit as with the library's default tile."""
    from paper_2401_11882_gb300 import autotune
    from paper_2401_11882_gb300.batched import BatchedDescent
    batch = _small_batch(5, n=8)
    best, timings = autotune.tune_batch(batch, steps=2, return_timings=True)
    assert best in autotune.BATCH_CANDIDATES
    assert len(timings) == len(autotune.BATCH_CANDIDATES)
    assert all(ms > 0 for _, ms in timings)
    assert dict(timings)[best] == min(ms for _, ms in timings)
    a = BatchedDescent(batch, history=3)
    b = BatchedDescent(batch, history=3, tile=best)
    a.run(3)
    b.run(3)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(a.history.cpu().numpy(), b.history.cpu().numpy())
    np.testing.assert_array_equal(a.tx.cpu().numpy(), b.tx.cpu().numpy())
    a.close()
    b.close()


def test_exact_skip_gives_the_same_descent(drt):
    # DRT_TILE_CULL_INVALID skips the obstruction loop of paths whose hard-sigmoid
    # validity is exactly 0 in every lane of the warp: such a path adds exactly 0
    from paper_2401_11882_gb300.batched import BatchedDescent
    batch = _small_batch(6, n=8)
    a = BatchedDescent(batch, history=3)
    b = BatchedDescent(batch, history=3, tile=drt.TileConfig(cull_invalid=True))
    a.run(3)
    b.run(3)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(a.history.cpu().numpy(), b.history.cpu().numpy())
    np.testing.assert_array_equal(a.tx.cpu().numpy(), b.tx.cpu().numpy())
    a.close()
    b.close()


@pytest.mark.parametrize("alpha", [100.0, 1000.0])
def test_blocked_warp_exit_gives_the_same_descent(drt, alpha):
    # DRT_TILE_EXIT_BLOCKED: a warp whose 64 paths all have a leg of hard-sigmoid
    # visibility exactly 0 leaves the wall loop; those powers are 0 either way.
    # W up to 60, so that the exit's check (every 8 walls) runs
    from paper_2401_11882_gb300.batched import BatchedDescent
    batch = scenes.scene_batch(8, 7, walls_range=(9, 60), rx_range=(33, 150), orders=(0, 1, 2),
                               n_tx=3, alpha=alpha, smoothing="hard_sigmoid")
    runs = []
    for tile in (None, drt.TileConfig(exit_blocked=True),
                 drt.TileConfig(cull_invalid=True), drt.TileConfig(cull_invalid=True,
                                                                   exit_blocked=True)):
        d = BatchedDescent(batch, history=3, tile=tile, alpha=alpha)
        d.run(3)
        torch.cuda.synchronize()
        runs.append((d.history.cpu().numpy(), d.tx.cpu().numpy()))
        d.close()
    for h, tx in runs[1:]:
        np.testing.assert_array_equal(runs[0][0], h)
        np.testing.assert_array_equal(runs[0][1], tx)
