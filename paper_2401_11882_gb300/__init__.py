"""GB300-native smoothed, differentiable 2D image-method ray tracing.

Public calls (PyTorch tensors on a CUDA device, float32):

* ``power(walls, tx, rx, max_order, alpha, smoothing)``: received power per
  receiver, differentiable in ``walls`` and ``tx`` (hand-written adjoint).
* ``loss(power)``: -min over receivers; ``objective(...)`` = loss(power(...)).
* ``forward``, ``vjp``, ``min_loss``: the raw C-ABI calls.
* ``field(...)``: the coherent reading of Eq. 7 (complex path fields, Fresnel
  reflection), field and power per receiver; ``field_power(...)`` is its power
  |E|^2, differentiable in ``walls`` and ``tx``; ``field_vjp`` the raw adjoint.
* ``forward_save`` / ``field_save`` (sigmoid): the forward that also keeps every
  path's leg visibilities, which ``vjp`` / ``field_vjp`` read with ``saved=``.
* ``forward3(tris, tx, rx, ...)``: the 3D extension (triangle walls), power per receiver;
  ``power3`` differentiable in ``tris`` and ``tx``; ``vjp3`` its raw adjoint (``vjp3_tx``
  for the transmitter only).
* ``forward_mpt(...)``: power with the reflection points found iteratively
  (Min-Path-Tracing) and the smoothed convergence check; ``mpt_paths`` its per-path
  record; ``forward_fpt`` / ``fpt_paths`` the same with Fermat path tracing.
* ``objective_host(...)``: the objective end to end from host arrays.

The compiled CUDA library is loaded lazily, on the first call that needs it,
so that the seeded scene generators (``scenes``) import without a GPU.
"""
from .ops import (TileConfig, field, field_power, field_save, field_vjp, forward, forward3,
                  forward_fpt, forward_mpt, forward_save, fpt_paths, loss, min_loss,
                  min_loss_backward, min_loss_vjp, mpt_paths, num_candidates, objective,
                  objective_host, power, power3, vjp, vjp3, vjp3_tx)

__all__ = ["TileConfig", "field", "field_power", "field_save", "field_vjp", "forward",
           "forward3", "forward_fpt", "forward_mpt", "forward_save", "fpt_paths", "loss",
           "min_loss", "min_loss_backward", "min_loss_vjp", "mpt_paths", "num_candidates",
           "objective", "objective_host", "power", "power3", "vjp", "vjp3", "vjp3_tx"]
