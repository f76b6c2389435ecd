"""drt_forward_noalloc: the forward pass for callers that cannot allocate device
memory (plugins handed only their output buffers, applications with a fixed
device-memory plan).  It must give drt_forward's result, within the tolerance
the other parity tests use, on consecutive calls that share its static scratch
array.  The file name makes pytest collect it last."""
import ctypes

import numpy as np
import pytest

from parity import assert_power_close
from paper_2401_11882_gb300 import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_11882_gb300 import _lib
    return _lib.load()


def _noalloc(lib, sc, dev):
    """Call drt_forward_noalloc through the C ABI; the test owns inputs and output."""
    from paper_2401_11882_gb300 import _lib
    w = torch.tensor(sc.walls, device=dev)
    t = torch.tensor(sc.tx, device=dev)
    r = torch.tensor(sc.rx, device=dev)
    out = torch.full((sc.n_rx,), float("nan"), device=dev)
    desc = _lib.Scene(w.data_ptr(), sc.n_walls, r.data_ptr(), sc.n_rx, t.data_ptr(),
                      sc.max_order, sc.alpha, _lib.SMOOTHING[sc.smoothing], sc.refl_coef)
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    st = lib.drt_forward_noalloc(ctypes.byref(desc), ctypes.c_void_p(out.data_ptr()), stream)
    assert st == 0, lib.drt_last_error().decode()
    torch.cuda.synchronize(dev)
    return out.cpu().numpy()


def _existing(sc, dev):
    import paper_2401_11882_gb300 as drt
    P = drt.forward(torch.tensor(sc.walls, device=dev), torch.tensor(sc.tx, device=dev),
                    torch.tensor(sc.rx, device=dev), sc.max_order, sc.alpha, sc.smoothing,
                    sc.refl_coef)
    torch.cuda.synchronize(dev)
    return P.cpu().numpy()


def test_matches_drt_forward_on_two_calls_in_a_row(lib):
    dev = torch.device("cuda:0")
    first = scenes.large_scene(alpha=100.0, smoothing="hard_sigmoid")
    second = scenes.clutter_scene(20, 40, seed=3, alpha=30.0, smoothing="sigmoid", max_order=2)
    a1 = _noalloc(lib, first, dev)
    a2 = _noalloc(lib, second, dev)     # reuses the scratch the first call left behind
    assert np.all(np.isfinite(a1)) and np.all(np.isfinite(a2))
    assert_power_close(a1, _existing(first, dev), "noalloc vs drt_forward, first call")
    assert_power_close(a2, _existing(second, dev), "noalloc vs drt_forward, second call")
    a3 = _noalloc(lib, first, dev)
    np.testing.assert_array_equal(a3, a1)


def test_rejects_receiver_counts_beyond_the_scratch(lib):
    from paper_2401_11882_gb300 import _lib
    cap = (8 << 20) // 4
    desc = _lib.Scene(256, 4, 256, cap + 1, 256, 1, 10.0, 1, 0.5)
    st = lib.drt_forward_noalloc(ctypes.byref(desc), ctypes.c_void_p(256), None)
    assert st == 2                       # DRT_ERR_UNSUPPORTED, nothing enqueued
    assert b"scratch" in lib.drt_last_error()


def test_accepts_the_largest_receiver_count(lib):
    """n_rx exactly at capacity: one candidate chunk must hold every candidate,
    and the result still matches drt_forward."""
    dev = torch.device("cuda:0")
    cap = (8 << 20) // 4
    base = scenes.clutter_scene(4, 8, seed=5, alpha=100.0, smoothing="hard_sigmoid",
                                max_order=2)
    rng = np.random.default_rng(11)
    # receivers above y = 0.3, well clear of the transmitter at (0.5, 0.2)
    rx = np.stack([rng.uniform(0.05, 0.95, cap), rng.uniform(0.3, 0.95, cap)], 1)
    sc = base.replace(rx=rx.astype(np.float32))
    got = _noalloc(lib, sc, dev)
    assert got.shape == (cap,) and np.all(np.isfinite(got))
    ref = _existing(sc, dev)
    assert_power_close(got, ref, "noalloc at n_rx = capacity")


def test_rejects_an_oversized_wall_count_before_counting_candidates(lib):
    """A wall count beyond the largest the forward takes is refused by the scene
    check, before the candidate count (which would not fit in 64 bits) is formed."""
    from paper_2401_11882_gb300 import _lib
    desc = _lib.Scene(256, 2**31 - 1, 256, 16, 256, 3, 10.0, 1, 0.5)
    st = lib.drt_forward_noalloc(ctypes.byref(desc), ctypes.c_void_p(256), None)
    assert st == 2                       # DRT_ERR_UNSUPPORTED, nothing enqueued
    assert b"n_walls" in lib.drt_last_error()


def test_more_walls_than_shared_memory_holds(lib):
    """Above 1024 walls the forward stages the wall records in its workspace: here
    the static array holds them beside the partial sums."""
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(2)
    rx = rng.uniform(0.05, 0.95, (300, 2)).astype(np.float32)
    sc = scenes.clutter_scene(2044, 1, seed=4, alpha=100.0, smoothing="hard_sigmoid",
                              max_order=1, rx=rx)
    assert sc.n_walls == 2048
    got = _noalloc(lib, sc, dev)
    assert np.all(np.isfinite(got))
    assert_power_close(got, _existing(sc, dev), "noalloc vs drt_forward, 2048 walls")
