"""The CUDA path where a wall all but blocks a leg (the sigmoid at large alpha): a
line-of-sight path blocked by one wall (2D) or one triangle (3D), so that the
received power is a factor 1 - X1 X2 (or 1 - X in) far below the rounding of 1.
The kernels form that factor from sums of non-negative terms; the oracle does the
same and is pinned to 60-digit evaluations of the definition on such scenes."""
import numpy as np
import pytest

from parity import assert_grad_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# the oracle pins' scenes with their symmetry broken (end points at different
# distances from the wall's line and plane), so that no derivative vanishes by
# symmetry and is left to rounding
WALLS = np.array([[0.5, -0.5, 0.5, 0.6]], np.float32)
TX2, RX2 = np.array([0.2, 0.0], np.float32), np.array([[0.85, 0.02]], np.float32)
TRIS = np.array([[0.5, -1.0, -1.0, 0.5, 1.2, -1.0, 0.5, 0.0, 1.1]], np.float32)
TX3, RX3 = np.array([0.2, 0.05, 0.02], np.float32), np.array([[0.85, 0.0, 0.0]], np.float32)


@pytest.fixture(scope="module")
def drt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_11882_gb300 as m
    return m


def _t(a):
    return torch.tensor(a, device=torch.device("cuda:0"))


@pytest.mark.parametrize("alpha", [100.0, 150.0, 200.0])
@pytest.mark.parametrize("single_rx", [False, True])
def test_2d_blocked_line_of_sight(drt, oracle_mod, alpha, single_rx):
    tile = drt.TileConfig(single_rx=True) if single_rx else None
    P = drt.forward(_t(WALLS), _t(TX2), _t(RX2), 0, alpha, "sigmoid", tile=tile)
    torch.cuda.synchronize()
    ref = oracle_mod.power(WALLS, TX2, RX2, 0, alpha, "sigmoid")
    assert ref[0] > 0.0
    np.testing.assert_allclose(P.cpu().numpy(), ref, rtol=1e-4, atol=0.0)


@pytest.mark.parametrize("alpha", [100.0, 150.0])
def test_2d_blocked_line_of_sight_gradient(drt, oracle_mod, alpha):
    g = np.ones(1)
    gtx, gw = drt.vjp(_t(WALLS), _t(TX2), _t(RX2), 0, alpha, "sigmoid",
                      _t(g.astype(np.float32)))
    torch.cuda.synchronize()
    ref = oracle_mod.gradient(WALLS, TX2, RX2, 0, alpha, "sigmoid", g)
    assert_grad_close(np.concatenate([gtx.cpu().numpy(), gw.cpu().numpy().ravel()]), ref,
                      "blocked line-of-sight gradient")


@pytest.mark.parametrize("alpha", [100.0, 150.0, 200.0])
def test_3d_blocked_line_of_sight(drt, oracle_mod, alpha):
    P = drt.forward3(_t(TRIS), _t(TX3), _t(RX3), 0, alpha, "sigmoid")
    torch.cuda.synchronize()
    ref = oracle_mod.power3(TRIS, TX3, RX3, 0, alpha, "sigmoid")
    assert ref[0] > 0.0
    np.testing.assert_allclose(P.cpu().numpy(), ref, rtol=1e-4, atol=0.0)


@pytest.mark.parametrize("alpha", [100.0, 150.0])
def test_3d_blocked_line_of_sight_gradient(drt, oracle_mod, alpha):
    g = np.ones(1)
    gtx, gtr = drt.vjp3(_t(TRIS), _t(TX3), _t(RX3), 0, alpha, "sigmoid",
                        _t(g.astype(np.float32)))
    torch.cuda.synchronize()
    ref_tx, ref_tr = oracle_mod.gradient3(TRIS, TX3, RX3, 0, alpha, "sigmoid", g)
    assert_grad_close(gtx.cpu().numpy(), ref_tx, "3D blocked line-of-sight grad_tx")
    assert_grad_close(gtr.cpu().numpy().ravel(), ref_tr.ravel(),
                      "3D blocked line-of-sight grad_tris")


def test_2d_gradient_scene_deep_shadow_sigmoid_at_alpha_1000(drt, oracle_mod):
    """128 random segments, 128 x 128 receivers, K <= 2, sigmoid at alpha = 1000: the 12
    lowest powers above 1e-30 (the receivers the loss cares about; below FP32's normal
    range, from 1.2e-38, a power has no relative accuracy left and many receivers
    here sit at 1e-45) against the oracle to 1e-4 relative (or twice their FP32
    input sensitivity), no max-power floor."""
    from parity import fp32_sensitivity
    from paper_2401_11882_gb300 import scenes
    sc = scenes.gradient_scene(alpha=1000.0, smoothing="sigmoid")
    P = drt.forward(_t(sc.walls), _t(sc.tx), _t(sc.rx), 2, 1000.0, "sigmoid")
    torch.cuda.synchronize()
    P = P.cpu().numpy()
    pos = np.nonzero(P > 1e-30)[0]
    idx = pos[np.argsort(P[pos])[:12]]
    ref = oracle_mod.power(sc.walls, sc.tx, sc.rx[idx], 2, 1000.0, "sigmoid")
    sens = fp32_sensitivity(lambda w, t, r: oracle_mod.power(w, t, r, 2, 1000.0, "sigmoid"),
                            sc.walls, sc.tx, sc.rx[idx])
    tol = np.maximum(1e-4 * np.abs(ref), 2.0 * sens)
    err = np.abs(P[idx].astype(np.float64) - ref)
    assert np.all(err <= tol), (idx[err > tol], P[idx][err > tol], ref[err > tol])
