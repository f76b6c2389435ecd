"""FP64 CPU oracle of the smoothed 2D image-method objective.

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only users.  The product path never
imports this package.  It shares no code with the CUDA library.

The arithmetic lives in ``drt_oracle.cpp`` (plain C++, FP64, OpenMP over
receivers); this module compiles it on demand with g++ and wraps it with
ctypes.  Inputs are promoted from the FP32 scene arrays to float64 exactly.

Functions and the passages they follow:

* ``smooth``            Eq. 1 (step), Eq. 4 (sigmoid), Eqs. 5-6 (hard sigmoid), Eq. 3 (scaling)
* ``power``             Sec. V (candidate list, image method, continuous validity), Eq. 7 (sum over paths)
* ``loss``              Eq. 8 (min over receivers) and Sec. III (loss = -objective)
* ``power_jvp``         exact forward-mode derivative of ``power`` (Sec. III: gradient of the loss)
* ``power_cstep``       complex-step derivative of ``power`` (independent derivative mechanism)
* ``gradient``          sum_r g_r dP_r/dtheta, assembled from ``power_jvp``
* ``paths``             per-candidate vertices, validity, visibility, length and power for one receiver
* ``candidates``        the candidate table of Sec. V (no wall twice in a row)
* ``field``           Eq. 7 read as a coherent sum of path fields (Fresnel TE reflection)
* ``field_jvp``, ``field_gradient``  its exact forward-mode derivative, and the gradient of
                        sum_r g_r |E_r|^2
* ``power3``          Sec. VI's 3D extension for triangle walls (same steps, planes for lines)
* ``power3_jvp``, ``gradient3_tx``, ``gradient3``  its exact forward-mode derivative; the TX
                        gradient; the gradient w.r.t. the TX and every triangle corner
* ``mpt.cost``          Sec. V-B: the Min-Path-Tracing cost that the iterative path
                        finders' convergence check compares with zero (``oracle/mpt.py``)
* ``power_mpt``, ``mpt_paths``  Sec. V-B, "Continuous Path Finding": reflection points found
                        iteratively (Min-Path-Tracing: Gauss-Newton on the reflection law from the
                        walls' midpoints) with the smoothed convergence check s(eps - C)
* ``power_fpt``, ``fpt_paths``  the same with Fermat path tracing (Newton on the total path
                        length) as the finder, and the same MPT check

Readings of the paper that the oracle fixes (the paper leaves them open):
incoherent scalar power p = Gamma^k V / L^2 with Gamma = 0.5; smoothing
arguments are Euclidean signed distances; a leg is not tested against the
walls its own end points lie on; ties of the min go to the lowest index.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "drt_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_KIND = {"sigmoid": 0, "hard_sigmoid": 1, "step": 2}
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so (g++ -O2, no fast-math, no FMA contraction, OpenMP) if it is
    missing or stale."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    # -ffp-contract=off: every a * b + c is a rounded product and a rounded sum on
    # every host (gcc fuses them into one FMA by default on Arm), so the oracle's
    # results do not depend on the machine it is built on
    cmd = ["g++", "-O2", "-ffp-contract=off", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-o",
           tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        # DRT_ORACLE_LIB points the wrapper at another build of drt_oracle.cpp
        # (the mutation tests load deliberately broken copies this way).
        lib = ctypes.CDLL(os.environ.get("DRT_ORACLE_LIB") or build())
        d, i, ll = ctypes.c_double, ctypes.c_int, ctypes.c_longlong
        p = ctypes.c_void_p
        lib.drt_oracle_num_candidates.restype = ll
        lib.drt_oracle_num_candidates.argtypes = [i, i]
        lib.drt_oracle_candidates.argtypes = [i, i, p, p]
        lib.drt_oracle_smooth.argtypes = [d, d, i, p, p]
        lib.drt_oracle_power.argtypes = [p, i, p, p, i, i, d, i, d, i, p]
        lib.drt_oracle_power_jvp.argtypes = [p, i, p, p, i, i, d, i, d, p, p, i, p, p]
        lib.drt_oracle_power_cstep.argtypes = [p, i, p, p, i, i, d, i, d, p, p, d, i, p]
        lib.drt_oracle_paths.argtypes = [p, i, p, p, i, d, i, d, p, p, p, p, p, p]
        lib.drt_oracle_field.argtypes = [p, i, p, p, i, i, d, i, d, d, d, i, p, p, p]
        lib.drt_oracle_field_jvp.argtypes = [p, i, p, p, i, i, d, i, d, d, d, p, p, i, p, p]
        lib.drt_oracle_power3.argtypes = [p, i, p, p, i, i, d, i, d, i, p]
        lib.drt_oracle_power3_jvp.argtypes = [p, i, p, p, i, i, d, i, d, p, p, i, p, p]
        lib.drt_oracle_power_finder.argtypes = [p, i, p, p, i, i, d, i, d, i, i, d, i, p]
        lib.drt_oracle_finder_paths.argtypes = [p, i, p, p, i, d, i, d, i, i, d, p, p, p, p, p]
        _lib = lib
        return lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _kind(smoothing) -> int:
    return _KIND[smoothing] if isinstance(smoothing, str) else int(smoothing)


def _threads(threads):
    return int(threads) if threads else (os.cpu_count() or 1)


def num_candidates(n_walls: int, max_order: int) -> int:
    return int(_load().drt_oracle_num_candidates(n_walls, max_order))


def candidates(n_walls: int, max_order: int):
    """(seq [N, K] with -1 padding, order [N]) in table order."""
    n = num_candidates(n_walls, max_order)
    seq = np.zeros((n, max(max_order, 1)), dtype=np.int32)
    order = np.zeros(n, dtype=np.int32)
    _load().drt_oracle_candidates(n_walls, max_order, _ptr(seq), _ptr(order))
    return seq[:, :max_order], order


def smooth(x: float, alpha: float, smoothing) -> tuple[float, float]:
    """(s(x; alpha), ds/dx)."""
    s, ds = ctypes.c_double(), ctypes.c_double()
    _load().drt_oracle_smooth(float(x), float(alpha), _kind(smoothing), ctypes.byref(s),
                              ctypes.byref(ds))
    return s.value, ds.value


def _scene_args(walls, tx, rx):
    walls, tx, rx = _f64(walls).reshape(-1, 4), _f64(tx).reshape(2), _f64(rx).reshape(-1, 2)
    return walls, tx, rx


def power(walls, tx, rx, max_order: int, alpha: float, smoothing, refl_coef: float = 0.5,
          threads=None) -> np.ndarray:
    """Received power P_r (float64 [R])."""
    walls, tx, rx = _scene_args(walls, tx, rx)
    out = np.zeros(rx.shape[0], dtype=np.float64)
    rc = _load().drt_oracle_power(_ptr(walls), walls.shape[0], _ptr(tx), _ptr(rx), rx.shape[0],
                                  int(max_order), float(alpha), _kind(smoothing),
                                  float(refl_coef), _threads(threads), _ptr(out))
    if rc:
        raise ValueError("oracle rejected the arguments")
    return out


def power_jvp(walls, tx, rx, max_order, alpha, smoothing, dwalls, dtx, refl_coef=0.5,
              threads=None):
    """(P, dP) with dP the derivative of P along (dwalls, dtx)."""
    walls, tx, rx = _scene_args(walls, tx, rx)
    dwalls, dtx = _f64(dwalls).reshape(walls.shape), _f64(dtx).reshape(2)
    P = np.zeros(rx.shape[0]); dP = np.zeros(rx.shape[0])
    rc = _load().drt_oracle_power_jvp(_ptr(walls), walls.shape[0], _ptr(tx), _ptr(rx),
                                      rx.shape[0], int(max_order), float(alpha),
                                      _kind(smoothing), float(refl_coef), _ptr(dwalls),
                                      _ptr(dtx), _threads(threads), _ptr(P), _ptr(dP))
    if rc:
        raise ValueError("oracle rejected the arguments")
    return P, dP


def power_cstep(walls, tx, rx, max_order, alpha, smoothing, dwalls, dtx, h=1e-30,
                refl_coef=0.5, threads=None):
    """Complex-step derivative of P along (dwalls, dtx)."""
    walls, tx, rx = _scene_args(walls, tx, rx)
    dwalls, dtx = _f64(dwalls).reshape(walls.shape), _f64(dtx).reshape(2)
    dP = np.zeros(rx.shape[0])
    rc = _load().drt_oracle_power_cstep(_ptr(walls), walls.shape[0], _ptr(tx), _ptr(rx),
                                        rx.shape[0], int(max_order), float(alpha),
                                        _kind(smoothing), float(refl_coef), _ptr(dwalls),
                                        _ptr(dtx), float(h), _threads(threads), _ptr(dP))
    if rc:
        raise ValueError("oracle rejected the arguments")
    return dP


def gradient(walls, tx, rx, max_order, alpha, smoothing, g, params="all", refl_coef=0.5,
             threads=None):
    """sum_r g_r dP_r/dtheta for the requested parameters.

    ``params``: "tx" (2 values), "all" (tx then the W x 4 wall coordinates), or
    a list of flat indices into [tx (2), walls (4W)].  Each parameter costs one
    forward-mode pass over the receivers with g_r != 0.
    """
    walls, tx, rx = _scene_args(walls, tx, rx)
    g = _f64(g).reshape(-1)
    nz = np.nonzero(g)[0]
    rx_nz, g_nz = rx[nz], g[nz]
    W = walls.shape[0]
    if isinstance(params, str):
        idx = list(range(2)) if params == "tx" else list(range(2 + 4 * W))
    else:
        idx = list(params)
    out = np.zeros(len(idx))
    for n, p in enumerate(idx):
        dtx = np.zeros(2); dw = np.zeros(4 * W)
        if p < 2:
            dtx[p] = 1.0
        else:
            dw[p - 2] = 1.0
        if rx_nz.shape[0] == 0:
            continue
        _, dP = power_jvp(walls, tx, rx_nz, max_order, alpha, smoothing, dw, dtx, refl_coef,
                          threads)
        out[n] = float(np.dot(g_nz, dP))
    return out


def field(walls, tx, rx, max_order: int, alpha: float, smoothing, wavelength: float,
          eps_r: float, refl_coef: float = 0.5, threads=None, scales: bool = False):
    """Coherent field E_r (complex128 [R]): Eq. 7's sum of path fields, each
    prod_j C_j V vis exp(-2 pi i L / wavelength) / L with C_j the Fresnel TE
    coefficient of relative permittivity ``eps_r`` at reflection j, or the
    constant -sqrt(refl_coef) when ``eps_r`` is 0.  |E_r|^2 is the coherent power.

    With ``scales``: (E, mag, lmax), mag_r the sum of the path fields' magnitudes
    and lmax_r the longest length among the paths with a non-zero field."""
    walls, tx, rx = _scene_args(walls, tx, rx)
    R = rx.shape[0]
    out = np.zeros(2 * R, dtype=np.float64)
    mag = np.zeros(R)
    lmax = np.zeros(R)
    rc = _load().drt_oracle_field(_ptr(walls), walls.shape[0], _ptr(tx), _ptr(rx), R,
                                  int(max_order), float(alpha), _kind(smoothing),
                                  float(refl_coef), float(wavelength), float(eps_r),
                                  _threads(threads), _ptr(out), _ptr(mag), _ptr(lmax))
    if rc:
        raise ValueError("oracle rejected the arguments")
    E = out[0::2] + 1j * out[1::2]
    return (E, mag, lmax) if scales else E


def field_jvp(walls, tx, rx, max_order, alpha, smoothing, wavelength, eps_r, dwalls, dtx,
              refl_coef=0.5, threads=None):
    """(E, dE) complex128 [R]: the coherent field and its derivative along (dwalls, dtx)."""
    walls, tx, rx = _scene_args(walls, tx, rx)
    dwalls, dtx = _f64(dwalls).reshape(walls.shape), _f64(dtx).reshape(2)
    R = rx.shape[0]
    E = np.zeros(2 * R)
    dE = np.zeros(2 * R)
    rc = _load().drt_oracle_field_jvp(_ptr(walls), walls.shape[0], _ptr(tx), _ptr(rx), R,
                                      int(max_order), float(alpha), _kind(smoothing),
                                      float(refl_coef), float(wavelength), float(eps_r),
                                      _ptr(dwalls), _ptr(dtx), _threads(threads), _ptr(E),
                                      _ptr(dE))
    if rc:
        raise ValueError("oracle rejected the arguments")
    return E[0::2] + 1j * E[1::2], dE[0::2] + 1j * dE[1::2]


def field_gradient(walls, tx, rx, max_order, alpha, smoothing, wavelength, eps_r, g,
                   params="all", refl_coef=0.5, threads=None):
    """sum_r g_r d|E_r|^2 / dtheta (= sum_r g_r 2 Re(conj(E_r) dE_r)); ``params`` as
    for ``gradient``."""
    walls, tx, rx = _scene_args(walls, tx, rx)
    g = _f64(g).reshape(-1)
    nz = np.nonzero(g)[0]
    rx_nz, g_nz = rx[nz], g[nz]
    W = walls.shape[0]
    if isinstance(params, str):
        idx = list(range(2)) if params == "tx" else list(range(2 + 4 * W))
    else:
        idx = list(params)
    out = np.zeros(len(idx))
    for n, p in enumerate(idx):
        dtx = np.zeros(2); dw = np.zeros(4 * W)
        if p < 2:
            dtx[p] = 1.0
        else:
            dw[p - 2] = 1.0
        if rx_nz.shape[0] == 0:
            continue
        E, dE = field_jvp(walls, tx, rx_nz, max_order, alpha, smoothing, wavelength, eps_r, dw,
                          dtx, refl_coef, threads)
        out[n] = float(np.dot(g_nz, 2.0 * (E.real * dE.real + E.imag * dE.imag)))
    return out


def power3(tris, tx, rx, max_order: int, alpha: float, smoothing, refl_coef: float = 0.5,
           threads=None) -> np.ndarray:
    """Received power of a 3D scene of triangle walls (float64 [R]): tris [W, 9]
    (corners A, B, C), tx [3], rx [R, 3]; the reading of the method for triangles
    stated in drt_oracle.cpp (plane distances, in-plane edge distances)."""
    tris = _f64(tris).reshape(-1, 9)
    tx = _f64(tx).reshape(3)
    rx = _f64(rx).reshape(-1, 3)
    out = np.zeros(rx.shape[0])
    rc = _load().drt_oracle_power3(_ptr(tris), tris.shape[0], _ptr(tx), _ptr(rx), rx.shape[0],
                                   int(max_order), float(alpha), _kind(smoothing),
                                   float(refl_coef), _threads(threads), _ptr(out))
    if rc:
        raise ValueError("oracle rejected the arguments")
    return out


def power3_jvp(tris, tx, rx, max_order, alpha, smoothing, dtris, dtx, refl_coef=0.5,
               threads=None):
    """(P, dP): the 3D power and its exact derivative along (dtris [W, 9], dtx [3])."""
    tris = _f64(tris).reshape(-1, 9)
    tx = _f64(tx).reshape(3)
    rx = _f64(rx).reshape(-1, 3)
    dtris, dtx = _f64(dtris).reshape(tris.shape), _f64(dtx).reshape(3)
    P = np.zeros(rx.shape[0]); dP = np.zeros(rx.shape[0])
    rc = _load().drt_oracle_power3_jvp(_ptr(tris), tris.shape[0], _ptr(tx), _ptr(rx),
                                       rx.shape[0], int(max_order), float(alpha),
                                       _kind(smoothing), float(refl_coef), _ptr(dtris),
                                       _ptr(dtx), _threads(threads), _ptr(P), _ptr(dP))
    if rc:
        raise ValueError("oracle rejected the arguments")
    return P, dP


def gradient3_tx(tris, tx, rx, max_order, alpha, smoothing, g, refl_coef=0.5, threads=None):
    """sum_r g_r dP_r / d(TX) [3] of a 3D scene."""
    tris = _f64(tris).reshape(-1, 9)
    rx = _f64(rx).reshape(-1, 3)
    g = _f64(g).reshape(-1)
    nz = np.nonzero(g)[0]
    out = np.zeros(3)
    if nz.size == 0:
        return out
    for a in range(3):
        dtx = np.zeros(3)
        dtx[a] = 1.0
        _, dP = power3_jvp(tris, tx, rx[nz], max_order, alpha, smoothing, np.zeros_like(tris),
                           dtx, refl_coef, threads)
        out[a] = float(np.dot(g[nz], dP))
    return out


def gradient3(tris, tx, rx, max_order, alpha, smoothing, g, refl_coef=0.5, threads=None):
    """(sum_r g_r dP_r / dTX [3], sum_r g_r dP_r / dtris [W, 9]) of a 3D scene, one
    forward-mode pass per parameter over the receivers with g_r != 0."""
    tris = _f64(tris).reshape(-1, 9)
    rx = _f64(rx).reshape(-1, 3)
    g = _f64(g).reshape(-1)
    nz = np.nonzero(g)[0]
    gtx, gtris = np.zeros(3), np.zeros(tris.shape)
    if nz.size == 0:
        return gtx, gtris
    for a in range(3 + tris.size):
        dtx, dtr = np.zeros(3), np.zeros(tris.size)
        if a < 3:
            dtx[a] = 1.0
        else:
            dtr[a - 3] = 1.0
        _, dP = power3_jvp(tris, tx, rx[nz], max_order, alpha, smoothing, dtr.reshape(tris.shape),
                           dtx, refl_coef, threads)
        v = float(np.dot(g[nz], dP))
        if a < 3:
            gtx[a] = v
        else:
            gtris.flat[a - 3] = v
    return gtx, gtris


def loss(P) -> tuple[float, int]:
    """(L, argmin): L = -min_r P_r (Eq. 8, Sec. III); ties go to the lowest index."""
    P = np.asarray(P, dtype=np.float64)
    i = int(np.argmin(P))          # numpy returns the first minimum
    return -float(P[i]), i


def paths(walls, tx, rx1, max_order, alpha, smoothing, refl_coef=0.5) -> dict:
    """Per-candidate detail for one receiver ``rx1`` ([2])."""
    walls, tx, rx1 = _scene_args(walls, tx, rx1)
    W, K = walls.shape[0], int(max_order)
    n = num_candidates(W, K)
    deg = np.zeros(n, np.int32)
    verts = np.zeros((n, K + 2, 2)); val = np.zeros(n); vis = np.zeros((n, K + 1))
    length = np.zeros(n); pw = np.zeros(n)
    rc = _load().drt_oracle_paths(_ptr(walls), W, _ptr(tx), _ptr(rx1), K, float(alpha),
                                  _kind(smoothing), float(refl_coef), _ptr(deg), _ptr(verts),
                                  _ptr(val), _ptr(vis), _ptr(length), _ptr(pw))
    if rc:
        raise ValueError("oracle rejected the arguments")
    seq, order = candidates(W, K)
    return dict(seq=seq, order=order, degenerate=deg, verts=verts, validity=val, vis=vis,
                length=length, power=pw)




_FINDERS = {"mpt": 0, "fpt": 1}


def _power_finder(finder, walls, tx, rx, max_order, alpha, smoothing, n_iter, eps, refl_coef,
                  threads):
    walls, tx, rx = _scene_args(walls, tx, rx)
    out = np.zeros(rx.shape[0])
    rc = _load().drt_oracle_power_finder(_ptr(walls), walls.shape[0], _ptr(tx), _ptr(rx),
                                         rx.shape[0], int(max_order), float(alpha),
                                         _kind(smoothing), float(refl_coef), _FINDERS[finder],
                                         int(n_iter), float(eps), _threads(threads), _ptr(out))
    if rc:
        raise ValueError("oracle rejected the arguments")
    return out


def _finder_paths(finder, walls, tx, rx1, max_order, alpha, smoothing, n_iter, eps, refl_coef):
    walls, tx, rx1 = _scene_args(walls, tx, rx1)
    W, K = walls.shape[0], int(max_order)
    n = num_candidates(W, K)
    tau = np.zeros((n, max(K, 1)))
    cost = np.zeros(n); kappa = np.zeros(n); pw = np.zeros(n)
    deg = np.zeros(n, np.int32)
    rc = _load().drt_oracle_finder_paths(_ptr(walls), W, _ptr(tx), _ptr(rx1), K, float(alpha),
                                         _kind(smoothing), float(refl_coef), _FINDERS[finder],
                                         int(n_iter), float(eps), _ptr(tau), _ptr(cost),
                                         _ptr(kappa), _ptr(pw), _ptr(deg))
    if rc:
        raise ValueError("oracle rejected the arguments")
    seq, order = candidates(W, K)
    return dict(seq=seq, order=order, tau=tau[:, :K], cost=cost, kappa=kappa, power=pw,
                degenerate=deg)


def power_mpt(walls, tx, rx, max_order, alpha, smoothing, n_iter=10, eps=0.05, refl_coef=0.5,
              threads=None) -> np.ndarray:
    """Received power (float64 [R]) with the reflection points found by ``n_iter``
    Min-Path-Tracing steps from the walls' midpoints (Sec. V-B) and each path's
    validity taken as its on-segment tests times the convergence check
    s(eps - C), C the MPT cost (drt_oracle.cpp, path finder)."""
    return _power_finder("mpt", walls, tx, rx, max_order, alpha, smoothing, n_iter, eps,
                         refl_coef, threads)


def mpt_paths(walls, tx, rx1, max_order, alpha, smoothing, n_iter=10, eps=0.05,
              refl_coef=0.5) -> dict:
    """Per candidate of one receiver ``rx1``: the MPT finder's along-wall coordinates
    ``tau`` [n, K] (NaN past the path's order), the MPT ``cost`` and the convergence
    check ``kappa`` at the final points, the path ``power`` and a ``degenerate``
    flag, with the candidate table's ``seq`` and ``order``."""
    return _finder_paths("mpt", walls, tx, rx1, max_order, alpha, smoothing, n_iter, eps,
                         refl_coef)


def power_fpt(walls, tx, rx, max_order, alpha, smoothing, n_iter=10, eps=0.05, refl_coef=0.5,
              threads=None) -> np.ndarray:
    """power_mpt with Fermat path tracing as the finder: ``n_iter`` Newton steps on the
    total path length from the walls' midpoints (Sec. V-B), the same MPT check."""
    return _power_finder("fpt", walls, tx, rx, max_order, alpha, smoothing, n_iter, eps,
                         refl_coef, threads)


def fpt_paths(walls, tx, rx1, max_order, alpha, smoothing, n_iter=10, eps=0.05,
              refl_coef=0.5) -> dict:
    """mpt_paths with Fermat path tracing as the finder (``cost`` is still the MPT cost
    at the final points)."""
    return _finder_paths("fpt", walls, tx, rx1, max_order, alpha, smoothing, n_iter, eps,
                         refl_coef)
