"""The candidate odometer used by the kernels (decode the first candidate of a
chunk, then step), transcribed here and checked against the oracle's candidate
table; the CUDA version is exercised by the GPU tests with chunk sizes that
cross every order boundary."""
import pytest


def decode(c, W, K):
    if c == 0:
        return 0, []
    c -= 1
    block, stride, k = W, 1, 1
    while k < K and c >= block:
        c -= block
        block *= W - 1
        stride *= W - 1
        k += 1
    prev = c // stride
    w = [prev]
    rem = c - prev * stride
    for _ in range(1, k):
        stride //= W - 1
        d = rem // stride
        rem -= d * stride
        prev = d if d < prev else d + 1
        w.append(prev)
    return k, w


def step(k, w, W):
    w = list(w)
    jstar = -1
    for j in range(k - 1, -1, -1):
        v = w[j] + 1
        if j > 0 and v == w[j - 1]:
            v += 1
        if v < W:
            w[j] = v
            jstar = j
            break
    if jstar < 0:
        return k + 1, [i & 1 for i in range(k + 1)]
    for i in range(jstar + 1, k):
        w[i] = 1 if w[i - 1] == 0 else 0
    return k, w


@pytest.mark.parametrize("W,K", [(2, 3), (3, 2), (5, 3), (9, 2), (1, 1)])
def test_decode_and_step_enumerate_the_table(oracle_mod, W, K):
    seq, order = oracle_mod.candidates(W, K)
    table = [(int(o), [int(x) for x in row[:o]]) for row, o in zip(seq, order)]
    assert [decode(c, W, K) for c in range(len(table))] == table
    for chunk in (1, 3, 7, 64):
        for c0 in range(0, len(table), chunk):
            k, w = decode(c0, W, K)
            got = [(k, w)]
            for _ in range(1, min(chunk, len(table) - c0)):
                k, w = step(k, w, W)
                got.append((k, w))
            assert got == table[c0:c0 + len(got)]
