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


# ---------------------------------------------------------------- depth-limit leaves in the oracle

def _turn(n_hands=12, seed=5, **kw):
    from paper_2605_19928_gb300 import synth
    kw.setdefault("bet_sizes", (1.0, synth.ALL_IN))
    kw.setdefault("max_raises", 1)
    return synth.turn_subgame(n_hands=n_hands, seed=seed, range_seed=seed + 1, **kw)


def test_leaves_replace_the_river_chance_nodes_with_chips_behind(oracle_mod):
    exact = _turn()
    limited = _turn()
    limited.depth_limit = 1
    oe, ol = oracle_mod.Oracle(exact, threads=1), oracle_mod.Oracle(limited, threads=1)
    ne, nl = oe.nodes(), ol.nodes()
    chance_with_chips = [n for n in ne if n["type"] == oracle_mod.T_CHANCE and max(n["contrib"]) < exact.pot / 2 + exact.stack]
    leaves = [n for n in nl if n["type"] == oracle_mod.T_LEAF]
    assert len(leaves) == len(chance_with_chips) > 0
    assert sorted(n["contrib"] for n in leaves) == sorted(n["contrib"] for n in chance_with_chips)
    # all-in run-outs stay exact: the limited tree keeps those chance nodes and their showdowns
    allin = sum(1 for n in ne if n["type"] == oracle_mod.T_CHANCE) - len(chance_with_chips)
    assert sum(1 for n in nl if n["type"] == oracle_mod.T_CHANCE) == allin


def test_constant_leaf_values_give_that_share_of_the_pot(oracle_mod):
    spec = _turn(max_raises=0)  # check / check: the turn ends at one leaf
    spec.depth_limit = 1
    o = oracle_mod.Oracle(spec, threads=1)
    leaves = [k for k, n in enumerate(o.nodes()) if n["type"] == oracle_mod.T_LEAF]
    assert len(leaves) == 1
    y = np.zeros((48, 2, spec.n_hands))
    y[:, 0, :], y[:, 1, :] = 0.25, -0.1
    o.set_leaf_values(leaves[0], y)
    o.load_profile("current")
    v = o.profile_value()
    assert v[0] == pytest.approx(0.25 * spec.pot, rel=1e-12)
    assert v[1] == pytest.approx(-0.1 * spec.pot, rel=1e-12)


def test_leaf_values_depend_on_the_cards_left(oracle_mod):
    """Values that depend on the river card only: a hand's leaf value is pot / 44 times the
    sum over the river cards neither hand holds, weighted by the opponent reach."""
    spec = _turn(n_hands=9, max_raises=0)
    spec.depth_limit = 1
    o = oracle_mod.Oracle(spec, threads=1)
    leaf = [k for k, n in enumerate(o.nodes()) if n["type"] == oracle_mod.T_LEAF][0]
    live = [c for c in range(52) if c not in set(int(b) for b in spec.board)]
    f = np.linspace(-1.0, 1.0, 48)
    y = np.zeros((48, 2, spec.n_hands))
    y[:, 0, :] = f[:, None]
    o.set_leaf_values(leaf, y)
    o.values_current(0)
    got = o.cfv(0, leaf)
    r = spec.ranges.astype(np.float64)
    r = r / r.sum(axis=1, keepdims=True)
    hands = [set(int(c) for c in h) for h in spec.hands]
    Z = sum(r[0, a] * r[1, b] for a in range(9) for b in range(9) if not hands[a] & hands[b])
    for h in range(9):
        want = 0.0
        for o_ in range(9):
            if hands[h] & hands[o_]:
                continue
            u = sum(f[k] for k, c in enumerate(live) if c not in hands[h] | hands[o_]) * spec.pot / 44
            want += r[1, o_] / Z * u
        assert got[h] == pytest.approx(want, rel=1e-12, abs=1e-15)


def _flop(n_hands=10, seed=4, **kw):
    from paper_2605_19928_gb300 import synth
    kw.setdefault("bet_sizes", (1.0, synth.ALL_IN))
    kw.setdefault("max_raises", 1)
    return synth.flop_subgame(n_hands=n_hands, seed=seed, range_seed=seed + 1, **kw)


def test_flop_leaves_sit_where_the_river_card_is_to_come(oracle_mod):
    """On the flop the depth limit ends the tree after the turn betting: the turn-card chance
    nodes stay, the river-card chance nodes with chips behind become leaves."""
    exact, limited = _flop(), _flop()
    limited.depth_limit = 1
    oe, ol = oracle_mod.Oracle(exact, threads=1), oracle_mod.Oracle(limited, threads=1)
    ne, nl = oe.nodes(), ol.nodes()
    cap = exact.pot / 2 + exact.stack
    chance = [n for n in ne if n["type"] == oracle_mod.T_CHANCE]
    river_with_chips = [n for n in chance if n["n_board"] == 4 and max(n["contrib"]) < cap]
    leaves = [n for n in nl if n["type"] == oracle_mod.T_LEAF]
    assert len(leaves) == len(river_with_chips) > 0
    assert all(n["n_board"] == 4 for n in leaves)
    turn_chance = [n for n in nl if n["type"] == oracle_mod.T_CHANCE and n["n_board"] == 3]
    assert len(turn_chance) == sum(1 for n in chance if n["n_board"] == 3) > 0
    assert all(n["n_actions"] == 49 for n in turn_chance)


def test_flop_constant_leaf_values_give_that_share_of_the_pot(oracle_mod):
    spec = _flop(max_raises=0)  # check / check on the flop and on each turn: 49 leaves
    spec.depth_limit = 1
    o = oracle_mod.Oracle(spec, threads=1)
    leaves = [k for k, n in enumerate(o.nodes()) if n["type"] == oracle_mod.T_LEAF]
    assert len(leaves) == 49
    y = np.zeros((48, 2, spec.n_hands))
    y[:, 0, :], y[:, 1, :] = 0.25, -0.1
    for leaf in leaves:
        o.set_leaf_values(leaf, y)
    o.load_profile("current")
    v = o.profile_value()
    assert v[0] == pytest.approx(0.25 * spec.pot, rel=1e-12)
    assert v[1] == pytest.approx(-0.1 * spec.pot, rel=1e-12)


def test_flop_leaf_values_weigh_turn_and_river_cards(oracle_mod):
    """Check-down flop to the leaves below each turn card, with outputs that depend on the
    turn and river cards: player 0's value is the mean, over the deals, of the mean over
    the 45 turn cards neither hand holds of the mean over the 44 river cards left of pot x
    output -- the chance weights 1/45 and 1/44 of the two dealt cards."""
    spec = _flop(n_hands=8, max_raises=0)
    spec.depth_limit = 1
    o = oracle_mod.Oracle(spec, threads=1)
    nodes = o.nodes()
    board = set(int(b) for b in spec.board)
    f = np.sin(np.arange(52 * 52, dtype=np.float64)).reshape(52, 52)  # output for (turn, river)
    for k, n in enumerate(nodes):
        if n["type"] != oracle_mod.T_LEAF:
            continue
        t = n["deal"] if n["deal"] >= 0 else nodes[n["parent"]]["deal"]
        while t < 0:  # the turn card is dealt above the leaf
            n = nodes[n["parent"]]
            t = n["deal"]
        rivers = [c for c in range(52) if c not in board and c != t]
        y = np.zeros((48, 2, spec.n_hands))
        y[:, 0, :] = f[t, rivers][:, None]
        o.set_leaf_values(k, y)
    o.load_profile("current")
    got = o.profile_value()[0]
    r = spec.ranges.astype(np.float64)
    r = r / r.sum(axis=1, keepdims=True)
    hands = [set(int(c) for c in h) for h in spec.hands]
    Z, acc = 0.0, 0.0
    for a in range(spec.n_hands):
        for b in range(spec.n_hands):
            if hands[a] & hands[b]:
                continue
            w = r[0, a] * r[1, b]
            dead = board | hands[a] | hands[b]
            turns = [c for c in range(52) if c not in dead]
            u = 0.0
            for t in turns:
                rivers = [c for c in range(52) if c not in dead and c != t]
                u += np.mean([spec.pot * f[t, c] for c in rivers])
            Z += w
            acc += w * u / len(turns)
    assert len(turns) == 45 and len(rivers) == 44
    assert got == pytest.approx(acc / Z, rel=1e-12, abs=1e-13)


def test_leaf_input_row_layout():
    hands = np.array([[0, 1], [2, 5], [1, 7]])
    x = ln.leaf_input([np.array([1.0, 3.0, 0.0]), np.array([0.0, 0.0, 2.0])], hands, [10, 20, 30, 40], 5,
                      ln.leaf_features(100.0, 50.0))
    # river card 5 removes hand [2, 5]: player 0's reach renormalises over the others
    assert x[ln.pair_slot(0, 1)] == 1.0 and x[ln.pair_slot(2, 5)] == 0.0
    assert x[ln.SLOTS + ln.pair_slot(1, 7)] == 1.0
    assert ln.pair_slot(0, 1) == 0 and ln.pair_slot(50, 51) == 1325
    assert [k - 2 * ln.SLOTS for k in np.flatnonzero(x[2 * ln.SLOTS:2 * ln.SLOTS + 52]) + 2 * ln.SLOTS] == [5, 10, 20, 30, 40]
    assert x[2 * ln.SLOTS + 52] == pytest.approx(0.5) and x[2 * ln.SLOTS + 53] == pytest.approx(0.25)
    assert x.shape == (2752,) and not x[2 * ln.SLOTS + 54:].any()
