"""drt_objective_host: the objective of Sec. III end to end from host arrays to
host arrays (input copies, power, loss -min P of Eq. 8, its gradient, output
copies), against the device-pointer calls it chains and against the FP64 oracle."""
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


def _device_chain(drt, sc, dev):
    w, t, r = (torch.tensor(a, device=dev) for a in (sc.walls, sc.tx, sc.rx))
    P = drt.forward(w, t, r, sc.max_order, sc.alpha, sc.smoothing, sc.refl_coef)
    L, am = drt.min_loss(P)
    gtx, gw = drt.min_loss_vjp(w, t, r, sc.max_order, sc.alpha, sc.smoothing, am, None,
                               sc.refl_coef)
    torch.cuda.synchronize(dev)
    return L.cpu().numpy(), P.cpu().numpy(), gtx.cpu().numpy(), gw.cpu().numpy()


CASES = [
    ("tiny", None),
    ("random", (3, 14, 70, 2, 60.0, "hard_sigmoid")),
    ("random", (4, 9, 33, 1, 25.0, "sigmoid")),
]


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("kind,args", CASES)
def test_matches_device_chain_and_oracle(drt, oracle_mod, kind, args, pinned):
    dev = torch.device("cuda:0")
    if kind == "tiny":
        sc = scenes.tiny_scene(alpha=100.0, smoothing="hard_sigmoid")
    else:
        seed, W, R, K, alpha, sm = args
        sc = scenes.random_small_scene(np.random.default_rng(seed), W, R, K, alpha, sm,
                                       boundary=True)
    hw, ht, hr = (torch.tensor(a) for a in (sc.walls, sc.tx, sc.rx))
    if pinned:
        hw, ht, hr = hw.pin_memory(), ht.pin_memory(), hr.pin_memory()
    L, P, gtx, gw = drt.objective_host(hw, ht, hr, sc.max_order, sc.alpha, sc.smoothing,
                                       sc.refl_coef, device=dev, grad_walls=True)
    assert not any(o.is_cuda for o in (L, P, gtx, gw))
    # the same kernels with the same tiles as the device-pointer chain: identical bits
    # (the wall gradient's per-CTA atomics only fix it to summation order)
    Ld, Pd, gtxd, gwd = _device_chain(drt, sc, dev)
    np.testing.assert_array_equal(P.numpy(), Pd)
    np.testing.assert_array_equal(L.numpy(), Ld)
    np.testing.assert_array_equal(gtx.numpy(), gtxd)
    np.testing.assert_allclose(gw.numpy(), gwd, rtol=1e-5, atol=1e-6 * np.abs(gwd).max())
    # and the oracle
    ref = oracle_mod.power(sc.walls, sc.tx, sc.rx, sc.max_order, sc.alpha, sc.smoothing,
                           sc.refl_coef)
    assert_power_close(P.numpy(), ref)
    L_ref, am = oracle_mod.loss(ref)
    assert float(L[0]) == pytest.approx(L_ref, rel=1e-4)
    g = np.zeros(sc.n_rx)
    g[am] = -1.0
    gtx_ref = oracle_mod.gradient(sc.walls, sc.tx, sc.rx, sc.max_order, sc.alpha, sc.smoothing,
                                  g, "tx", sc.refl_coef)
    assert_grad_close(gtx.numpy(), gtx_ref, "objective_host grad_tx")


def test_optional_outputs_can_be_skipped(drt):
    import ctypes
    from paper_2401_11882_gb300 import _lib, ops
    dev = torch.device("cuda:0")
    sc = scenes.tiny_scene()
    hw, ht, hr = (torch.tensor(a) for a in (sc.walls, sc.tx, sc.rx))
    desc = _lib.Scene(hw.data_ptr(), sc.n_walls, hr.data_ptr(), sc.n_rx, ht.data_ptr(),
                      sc.max_order, sc.alpha, _lib.SMOOTHING[sc.smoothing], sc.refl_coef)
    n = ctypes.c_size_t()
    _lib.call("drt_objective_host_workspace_size", ctypes.byref(desc), None, ctypes.byref(n))
    ws = torch.empty(n.value, dtype=torch.uint8, device=dev)
    loss = torch.full((1,), float("nan"))
    gtx = torch.full((2,), float("nan"))
    _lib.call("drt_objective_host", ctypes.byref(desc), None, ctypes.c_void_p(loss.data_ptr()),
              None, None, ctypes.c_void_p(gtx.data_ptr()), None, ctypes.c_void_p(ws.data_ptr()),
              ctypes.c_size_t(ws.numel()), ops._stream_ptr(dev))
    torch.cuda.synchronize(dev)
    L, _, g = drt.objective_host(hw, ht, hr, sc.max_order, sc.alpha, sc.smoothing,
                                 sc.refl_coef, device=dev)
    assert float(loss[0]) == float(L[0]) and np.array_equal(gtx.numpy(), g.numpy())
    # a workspace one byte short is refused before anything is enqueued
    with pytest.raises(_lib.DrtError) as ei:
        _lib.call("drt_objective_host", ctypes.byref(desc), None,
                  ctypes.c_void_p(loss.data_ptr()), None, None, ctypes.c_void_p(gtx.data_ptr()),
                  None, ctypes.c_void_p(ws.data_ptr()), ctypes.c_size_t(n.value - 1),
                  ops._stream_ptr(dev))
    assert ei.value.status == 5
