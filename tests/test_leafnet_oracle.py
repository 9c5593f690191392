"""Pins of the leaf network's FP64 reference (oracle/leafnet.py) against closed forms and
brute force: BF16 rounding cases worked by hand, GELU identities and printed values of the
normal CDF, and a dense layer against an explicit triple loop."""
import math

import numpy as np
import pytest

from oracle import leafnet as ln


def test_bf16_rounding_cases():
    # near 1, BF16 steps by 2^-7 (7 stored significand bits)
    cases = {1.0: 1.0, 0.5: 0.5, -3.0: -3.0,
             1 + 2 ** -8: 1.0,                      # halfway, ties to the even (1.0)
             1 + 3 * 2 ** -8: 1 + 2 ** -6,          # halfway between 1+2^-7 and 1+2^-6: even is 1+2^-6
             1 + 2 ** -8 + 2 ** -20: 1 + 2 ** -7,   # just above halfway rounds up
             1 + 2 ** -8 - 2 ** -20: 1.0,           # just below rounds down
             -(1 + 3 * 2 ** -8): -(1 + 2 ** -6)}
    for x, want in cases.items():
        assert float(ln.bf16_round(np.float32(x))) == want, x


def test_bf16_rounding_is_nearest_representable():
    x = np.random.default_rng(1).standard_normal(10000).astype(np.float32) * 1e3
    r = ln.bf16_round(x)
    assert np.all((r.view(np.uint32) & 0xFFFF) == 0)
    # the two BF16 neighbours of x bracket it; the chosen one is the nearer
    down = (x.view(np.uint32) & 0xFFFF0000).view(np.float32)
    up = ((x.view(np.uint32) & 0xFFFF0000) + 0x10000).view(np.float32)
    d = np.minimum(np.abs(x.astype(np.float64) - down), np.abs(x.astype(np.float64) - up))
    assert np.all(np.abs(x.astype(np.float64) - r) <= d + 0.0)
    assert np.array_equal(ln.bf16_from_bits(ln.bf16_bits(x)), r)


def test_gelu_closed_forms():
    assert ln.gelu(0.0) == 0.0
    # Phi(1) and Phi(-1) of the standard normal distribution
    assert ln.gelu(1.0) == pytest.approx(0.8413447460685429, abs=1e-15)
    assert ln.gelu(-1.0) == pytest.approx(-0.15865525393145707, abs=1e-15)
    x = np.linspace(-6, 6, 101)
    # Phi(x) + Phi(-x) = 1  =>  gelu(x) - gelu(-x) = x
    assert np.allclose(ln.gelu(x) - ln.gelu(-x), x, atol=1e-14)
    assert ln.gelu(40.0) == pytest.approx(40.0) and abs(ln.gelu(-40.0)) < 1e-300


def test_dense_layer_against_a_triple_loop():
    rng = np.random.default_rng(2)
    x, w, b = rng.standard_normal((3, 5)), rng.standard_normal((4, 5)), rng.standard_normal(4)
    want = np.zeros((3, 4))
    for m in range(3):
        for n in range(4):
            s = b[n]
            for k in range(5):
                s += x[m, k] * w[n, k]
            want[m, n] = 0.5 * s * (1 + math.erf(s / math.sqrt(2)))
    assert np.allclose(ln.dense(x, w, b, act=True), want, atol=1e-13)


def test_forward_rounds_hidden_activations():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, 8))
    l1 = (rng.standard_normal((4, 8)), rng.standard_normal(4))
    l2 = (rng.standard_normal((3, 4)), rng.standard_normal(3))
    h = ln.bf16_round(ln.gelu(ln.bf16_round(x).astype(np.float64) @ ln.bf16_round(l1[0]).T.astype(np.float64) + l1[1]))
    want = h.astype(np.float64) @ ln.bf16_round(l2[0]).T.astype(np.float64) + l2[1]
    assert np.allclose(ln.forward(x, [l1, l2]), want, atol=1e-12)
