"""FP64 reference of the depth-limit leaf network's arithmetic.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU legs
may use this module; the product path may not.

The leaf network (Section 3, depth-limited solving: a network maps both players' normalised
reach and the public state to counterfactual values at a depth-limit leaf; the paper's
Stage 5, Section 4.3, evaluates it on the GPU) is a stack of dense layers y = act(x W^T + b)
with BF16 operands and FP32 accumulation on the GPU.  Here each layer is computed in FP64
from the same BF16-rounded operands (a library matmul is the contraction step), and
activations passed from one layer to the next are rounded to BF16 exactly as the GPU stores
them.
"""
from __future__ import annotations

import math

import numpy as np


def bf16_round(x) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even), returned as float32.  BF16 keeps the
    top 16 bits of the FP32 encoding: add 0x7fff plus the lowest kept bit, then truncate."""
    f = np.array(x, dtype=np.float32)
    u = f.reshape(-1).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).reshape(f.shape)


def bf16_bits(x) -> np.ndarray:
    """The 16-bit encodings of bf16_round(x) (uint16)."""
    return (bf16_round(x).view(np.uint32) >> 16).astype(np.uint16)


def bf16_from_bits(b) -> np.ndarray:
    return (np.asarray(b, dtype=np.uint32) << 16).view(np.float32)


_erf = np.vectorize(math.erf, otypes=[np.float64])


def gelu(x) -> np.ndarray:
    """GELU(x) = x Phi(x) = 0.5 x (1 + erf(x / sqrt 2)), in FP64."""
    x = np.asarray(x, dtype=np.float64)
    return 0.5 * x * (1.0 + _erf(x / math.sqrt(2.0)))


def dense(x, w, b=None, act: bool = False) -> np.ndarray:
    """act(x w^T + b) in FP64: x [M][K] and w [N][K] are taken exactly as given (the caller
    passes BF16-rounded values), b [N] or None."""
    y = np.asarray(x, dtype=np.float64) @ np.asarray(w, dtype=np.float64).T
    if b is not None:
        y = y + np.asarray(b, dtype=np.float64)[None, :]
    return gelu(y) if act else y


def abs_terms(x, w) -> np.ndarray:
    """sum_k |x_mk w_nk|: the scale an FP32 accumulation error of a dense layer is relative to."""
    return np.abs(np.asarray(x, dtype=np.float64)) @ np.abs(np.asarray(w, dtype=np.float64)).T


def forward(x, layers) -> np.ndarray:
    """The network: layers = [(w, b), ...] with GELU after every layer but the last; the
    input and every hidden activation are rounded to BF16 as the GPU stores them."""
    h = bf16_round(x)
    for k, (w, b) in enumerate(layers):
        last = k == len(layers) - 1
        y = dense(h, bf16_round(w), b, act=not last)
        h = y if last else bf16_round(y)
    return h


SLOTS = 1326
IN_FEATURES = 2 * SLOTS + 52 + 2
IN_PADDED = 2752


def pair_slot(a: int, b: int) -> int:
    """Slot of the two-card hand {a, b}: b (b - 1) / 2 + a for a < b (all 1326 pairs)."""
    a, b = min(a, b), max(a, b)
    return b * (b - 1) // 2 + a


def leaf_input(reach, hands, board, r: int, feat) -> np.ndarray:
    """FP64 network input at a leaf for river card r: reach[p] is player p's reach per hand
    (hands [n][2]), normalised to sum 1 over the live hands -- those holding neither r nor a
    card of the leaf's board (uniform over them if that sum is 0) -- and placed at each
    hand's slot; then a one-hot of board + r; then the two pot / stack features; zero
    padding to IN_PADDED."""
    x = np.zeros(IN_PADDED, np.float64)
    dead = set(int(c) for c in board) | {int(r)}
    live = np.array([not ({int(a), int(b)} & dead) for a, b in hands])
    slots = np.array([pair_slot(int(a), int(b)) for a, b in hands])
    for p in range(2):
        q = np.where(live, np.asarray(reach[p], dtype=np.float64), 0.0)
        s = q.sum()
        v = q / s if s > 0 else live / live.sum()
        x[p * SLOTS + slots[live]] = v[live]
    for c in list(board) + [r]:
        x[2 * SLOTS + int(c)] = 1.0
    x[2 * SLOTS + 52] = feat[0]
    x[2 * SLOTS + 53] = feat[1]
    return x


def leaf_features(pot: float, behind: float):
    """pot / (pot + 2 behind) and behind / (pot + 2 behind) at a leaf."""
    return pot / (pot + 2 * behind), behind / (pot + 2 * behind)
