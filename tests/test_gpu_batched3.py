"""Batched descent on 3D scenes (drt_batch_* with dim = 3; Sec. VI with Sec. VII's
antenna placement): one step against the single-scene 3D calls and the FP64
oracle, several steps against a reference loop, graph replay and determinism."""
import numpy as np
import pytest

from parity import assert_grad_close, assert_power_close
from paper_2401_11882_gb300 import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

BOX = (0.02, 0.02, 0.02, 0.98, 0.98, 0.98)


@pytest.fixture(scope="module")
def drt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_11882_gb300 as m
    return m


def _small_batch3(seed=0, n=5, smoothing="hard_sigmoid", alpha=100.0):
    # uneven: 2..6 segments (2 (n + 4) + 4 = 16..24 triangles), 33..90 receivers
    # (ragged 32-receiver tiles), K in {0, 1, 2}, 3 starts
    return scenes.scene_batch3(n, seed, segments_range=(2, 6), rx_range=(33, 90),
                               orders=(0, 1, 2), n_tx=3, alpha=alpha, smoothing=smoothing)


def _reference_steps(drt, batch, n_steps, lr=1e-2, b1=0.9, b2=0.999, eps=1e-8, alpha=100.0):
    """Single-scene forward3 + min loss + drt3_vjp_tx with the argmin's one-hot weight per
    problem, Adam in float32 numpy with the same clamp."""
    dev = torch.device("cuda:0")
    S, T = batch.n_scenes, batch.tx0.shape[1]
    tx = batch.tx0.reshape(S * T, 3).astype(np.float32).copy()
    m = np.zeros_like(tx)
    v = np.zeros_like(tx)
    lo, hi = np.array(BOX[:3], np.float32), np.array(BOX[3:], np.float32)
    losses = []
    for step in range(n_steps):
        L = np.zeros(S * T, np.float32)
        G = np.zeros_like(tx)
        for s in range(S):
            sc = batch.scene(s)
            w = torch.tensor(sc.tris, device=dev)
            r = torch.tensor(sc.rx, device=dev)
            for t in range(T):
                p = s * T + t
                txp = torch.tensor(tx[p], device=dev)
                P = drt.forward3(w, txp, r, sc.max_order, alpha, batch.smoothing)
                loss, am = drt.min_loss(P)
                g = torch.zeros(sc.n_rx, device=dev)
                g[int(am)] = -1.0
                gtx = drt.vjp3_tx(w, txp, r, sc.max_order, alpha, batch.smoothing, g)
                L[p] = float(loss)
                G[p] = gtx.cpu().numpy()
        losses.append(L)
        t1 = step + 1
        m = (np.float32(b1) * m + np.float32(1 - b1) * G).astype(np.float32)
        v = (np.float32(b2) * v + np.float32(1 - b2) * G * G).astype(np.float32)
        mh = m / np.float32(1 - b1 ** t1)
        vh = v / np.float32(1 - b2 ** t1)
        tx = np.clip(tx - np.float32(lr) * mh / (np.sqrt(vh) + np.float32(eps)), lo, hi)
        tx = tx.astype(np.float32)
    return tx, m, v, losses


def test_one_step_matches_single_scene_calls_and_the_oracle(drt, oracle_mod):
    from paper_2401_11882_gb300.batched import BatchedDescent
    batch = _small_batch3(0)
    bd = BatchedDescent(batch, history=2, box=BOX)
    assert bd.dim == 3
    bd.run(1)
    torch.cuda.synchronize()
    tx_ref, m_ref, v_ref, losses = _reference_steps(drt, batch, 1)
    loss = bd.history[0].cpu().numpy()
    assert_power_close(-loss, -losses[0], "batched 3D loss vs single-scene loss")
    g_batched = bd.m.cpu().numpy() / 0.1          # m_1 = (1 - beta1) g
    assert_grad_close(g_batched.ravel(), (m_ref / 0.1).ravel(),
                      "batched 3D TX gradient vs single-scene")
    np.testing.assert_allclose(bd.tx.cpu().numpy(), tx_ref, atol=2e-6)
    T = batch.tx0.shape[1]
    n_checked = 0
    for p in range(0, batch.n_scenes * T, 2):
        s, t = divmod(p, T)
        sc = batch.scene(s, t)
        Pref = oracle_mod.power3(sc.tris, sc.tx, sc.rx, sc.max_order, 100.0, batch.smoothing)
        lref, am = oracle_mod.loss(Pref)
        assert abs(loss[p] - lref) <= 1e-4 * abs(lref) + 1e-10 * np.abs(Pref).max()
        if lref == 0.0:
            continue   # a receiver in full shadow: no gradient to compare
        g = np.zeros(sc.n_rx)
        g[am] = -1.0
        gref = oracle_mod.gradient3_tx(sc.tris, sc.tx, sc.rx, sc.max_order, 100.0,
                                       batch.smoothing, g)
        assert_grad_close(g_batched[p], gref, f"problem {p} vs oracle")
        n_checked += 1
    assert n_checked >= 2
    bd.close()


@pytest.mark.parametrize("smoothing", ["sigmoid", "hard_sigmoid"])
def test_three_steps_match_reference_loop(drt, smoothing):
    from paper_2401_11882_gb300.batched import BatchedDescent
    batch = _small_batch3(1, n=3, smoothing=smoothing, alpha=30.0)
    bd = BatchedDescent(batch, alpha=30.0, history=3, box=BOX)
    bd.run(3)
    torch.cuda.synchronize()
    tx_ref, m_ref, v_ref, losses = _reference_steps(drt, batch, 3, alpha=30.0)
    np.testing.assert_allclose(bd.tx.cpu().numpy(), tx_ref, atol=5e-6)
    hist = bd.history.cpu().numpy()
    for i in range(3):
        assert_power_close(-hist[i], -losses[i], f"3D loss of step {i}")
    bd.close()


def test_graph_and_direct_launch_agree_and_evaluate_does_not_step(drt):
    from paper_2401_11882_gb300.batched import BatchedDescent
    batch = _small_batch3(2, n=4, smoothing="sigmoid", alpha=50.0)
    a = BatchedDescent(batch, history=4, alpha=50.0, box=BOX)
    b = BatchedDescent(batch, history=4, alpha=50.0, box=BOX)
    a.run(4, use_graph=True)
    b.run(4, use_graph=False)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(a.tx.cpu().numpy(), b.tx.cpu().numpy())
    np.testing.assert_array_equal(a.history.cpu().numpy(), b.history.cpu().numpy())
    tx_before = a.tx.cpu().numpy().copy()
    step_before = int(a.step.item())
    loss = a.evaluate().cpu().numpy().copy()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(a.tx.cpu().numpy(), tx_before)
    assert int(a.step.item()) == step_before
    # the evaluated loss is the loss at the current TX: the next step records it
    a.run(1)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(a.loss.cpu().numpy(), loss)
    for o in (a, b):
        o.close()


def test_tx_stays_in_the_box(drt):
    from paper_2401_11882_gb300.batched import BatchedDescent
    batch = _small_batch3(3, n=3)
    box = (0.1, 0.2, 0.3, 0.8, 0.9, 0.7)
    bd = BatchedDescent(batch, lr=0.2, box=box)
    bd.run(5)
    torch.cuda.synchronize()
    tx = bd.tx.cpu().numpy()
    assert np.all(tx >= np.array(box[:3], np.float32)) and np.all(tx <= np.array(box[3:], np.float32))
    bd.close()
