"""Work accounting for the path kernels (independent of the implementation).

Units:
* one evaluation = one (receiver, path candidate) pair;
* one leg x wall test = one smoothed obstruction test.

Frozen counting convention (FMA counts as 2 FLOP), per evaluation of order k
in a scene of W walls: 40 FLOP per leg x wall test ((k + 1) legs, each tested
against every wall but the walls its end points lie on: (k + 1) W - 2k tests),
40 FLOP per reflection (backtrace and validity), 20 FLOP per path (power and
sum).  The adjoint is counted as twice the forward.
"""
from __future__ import annotations


def candidates_per_order(n_walls: int, max_order: int) -> list[int]:
    out, level = [1], 1
    for k in range(1, max_order + 1):
        level = n_walls if k == 1 else level * (n_walls - 1)
        out.append(level)
    return out


def num_candidates(n_walls: int, max_order: int) -> int:
    return sum(candidates_per_order(n_walls, max_order))


def tests_per_eval(order: int, n_walls: int) -> int:
    return (order + 1) * n_walls - 2 * order


def flops_per_eval(order: int, n_walls: int) -> int:
    return 40 * tests_per_eval(order, n_walls) + 40 * order + 20


def forward_work(n_walls: int, max_order: int, n_rx: int) -> dict:
    """Evaluations, leg x wall tests and FLOP of one forward pass."""
    per = candidates_per_order(n_walls, max_order)
    evals = n_rx * sum(per)
    tests = n_rx * sum(c * tests_per_eval(k, n_walls) for k, c in enumerate(per))
    flops = n_rx * sum(c * flops_per_eval(k, n_walls) for k, c in enumerate(per))
    return dict(evals=evals, tests=tests, flops=flops)


def fp32_peak_tflops(n_sms: int, sm_mhz: float) -> float:
    """FP32 CUDA-core peak: SMs x 128 FP32 lanes x 2 FLOP (FMA) x clock."""
    return n_sms * 128 * 2 * sm_mhz * 1e6 / 1e12
