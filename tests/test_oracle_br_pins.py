"""Pins of the oracle's hold'em best response and own-reach walk (no GPU).

The best response (Section 5's exploitability metric) on hold'em trees carries two-card
blockers at the terminal sums and 1/K chance weights with blocked hands zeroed at the
public-card deals; the own reach at a node (Stage 1) feeds the leaf network's input rows.
Both are checked here against the independent rules engine of tests/bruteforce.py:

* by definition: the best response value as the largest expected utility over every pure
  strategy, on a river whose hands share cards;
* per infoset: the maximum at each of the player's infosets over the engine's own
  enumeration of opponent hands and public cards (chance probabilities from the live cards
  of each pair of hands), root and every node, on rivers, a turn and a flop;
* own reach: the engine's walk of every deal and history, at every node (decision, chance,
  terminal, depth-limit leaf) under the current and the average strategy.

A last test plants plausible mistakes in copies of the oracle's source and checks that
these pins catch each of them.
"""
import os
import re
import subprocess

import numpy as np
import pytest

import bruteforce as bf
from paper_2605_19928_gb300 import synth
from test_oracle_pins import bf_game, small_flop, small_river, small_turn

ORACLE_SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "cfr_oracle.c")


def blocker_river():
    """River with five hands chosen to share cards (so that two-card blockers decide which
    deals exist), one tie between hands that can meet, all-in as the only bet."""
    board = np.array([0, 13, 26, 39, 51], np.int32)
    a, b, c, d, e, f = 4, 17, 30, 43, 8, 21
    hands = np.array([(a, b), (c, d), (a, c), (b, d), (e, f)], np.uint8)
    strength = np.array([[7, 9, 3, 5, 7]], np.int32)
    ranges = np.array([[0.3, 0.1, 0.25, 0.15, 0.2], [0.05, 0.35, 0.2, 0.1, 0.3]], np.float32)
    return synth.GameSpec(game=synth.GAME_HOLDEM, name="blocker river", board=board, hands=hands, ranges=ranges,
                          strength=strength, pot=100.0, stack=200.0, bet_sizes=(synth.ALL_IN,), max_raises=1)


def node_histories(o, g):
    """Oracle node id -> the engine's history (decision, chance, fold, showdown and
    depth-limit leaf nodes); the node kinds must agree with the engine's state."""
    info = o.nodes()
    out = {}
    stack = [(0, ())]
    while stack:
        n, hist = stack.pop()
        out[n] = hist
        nd = info[n]
        st = g.state(hist)
        if nd["type"] == 0:
            acts = g.legal(hist)
            assert nd["n_actions"] == len(acts) and nd["player"] == st["to_act"]
            stack += [(kid, hist + (acts[k],)) for k, kid in enumerate(nd["kids"])]
        elif nd["type"] == 3:
            assert st["over"] and st["folded"] < 0
            stack += [(kid, hist + (("d", info[kid]["deal"]),)) for kid in nd["kids"]]
        elif nd["type"] == 4:  # depth-limit leaf: where the next card is to come
            assert st["over"] and st["folded"] < 0 and st["street"] < g.n_streets - 1
        elif nd["type"] == 1:
            assert st["folded"] == nd["player"]
        else:
            assert st["over"] and st["street"] == g.n_streets - 1
    return out


def profile_table(o, g, hmap, player):
    """The oracle's loaded profile at the player's decision nodes, keyed as the engine keys
    infosets (hands holding a card dealt on the path left out)."""
    table = {}
    for n, nd in enumerate(o.nodes()):
        if nd["type"] == 0 and nd["player"] == player:
            p = o.profile(n)
            for h in range(o.n_hands):
                if not holds_dealt_card(g, h, hmap[n]):
                    table[bf.infoset_key(player, h, hmap[n])] = list(p[:, h])
    return bf.Profile(table)


def holds_dealt_card(g, h, hist):
    return any(tok[0] == "d" and tok[1] in g.hands[h] for tok in hist)


def solved(oracle_mod, spec, iters=4, lib_path=None):
    o = oracle_mod.Oracle(spec, variant="dcfr", threads=2, lib_path=lib_path)
    o.iterate(iters)
    o.load_profile("average")
    return o


def br_errors(o, g, hmap):
    """Largest differences (root value, per-node values), each relative to the largest
    magnitude, between the oracle's best responses and the engine's per-infoset maximum."""
    worst_root, worst_node = 0.0, 0.0
    for i in (0, 1):
        br, root, allv = o.best_response(i, all_nodes=True)
        want_br, vals = bf.best_response(g, profile_table(o, g, hmap, 1 - i), i)
        worst_root = max(worst_root, abs(br - want_br) / max(abs(want_br), 1e-300))
        want = np.zeros_like(allv)
        for n, hist in hmap.items():
            for h in range(o.n_hands):
                want[n, h] = vals.get((h, hist), 0.0)
        scale = max(np.abs(want).max(), 1e-300)
        worst_node = max(worst_node, float(np.abs(allv - want).max() / scale))
        worst_node = max(worst_node, float(np.abs(root - want[0]).max() / scale))
    return worst_root, worst_node


def set_random_state(o, seed):
    """Random regrets (signs mixed) and average sums at every decision node."""
    rng = np.random.default_rng(seed)
    for n, nd in enumerate(o.nodes()):
        if nd["type"] == 0:
            A = nd["n_actions"]
            R = rng.normal(size=(A, o.n_hands)) * (rng.random((A, o.n_hands)) < 0.8)
            S = rng.random((A, o.n_hands)) * (rng.random((A, o.n_hands)) < 0.9)
            o.set_node_state(n, R, S)


def reach_errors(o, g, hmap):
    """Largest difference between the oracle's own reach at every node and the engine's
    walk, both players, current and average strategies (and that hands holding a card
    dealt on the path get 0)."""
    worst, checked = 0.0, 0
    for kind in ("current", "average"):
        o.load_profile(kind)
        for p in (0, 1):
            want = bf.reach_at_histories(g, profile_table(o, g, hmap, p), p)
            for n, hist in hmap.items():
                got = o.node_reach(kind, p, n)
                for h in range(o.n_hands):
                    if holds_dealt_card(g, h, hist):
                        worst = max(worst, abs(got[h]))
                    elif (h, hist) in want:
                        worst = max(worst, abs(got[h] - want[(h, hist)]))
                        checked += 1
    assert checked > 0
    return worst


# ---------------------------------------------------------------- best response

def test_best_response_equals_pure_strategy_enumeration(oracle_mod):
    """The definition: max over all 2^10 pure strategies of each player (5 hands x 2
    decision nodes) of the expected utility, against the average strategy of 4 DCFR
    iterations.  Two-card blockers decide which deals exist."""
    spec = blocker_river()
    o = solved(oracle_mod, spec)
    g = bf_game(spec)
    hmap = node_histories(o, g)
    assert len(g.deals()) < 25  # several pairs of hands share a card
    for i in (0, 1):
        prof = profile_table(o, g, hmap, 1 - i)
        want = bf.pure_best_response(g, prof, i)
        br, _ = o.best_response(i)
        assert br == pytest.approx(want, rel=1e-12, abs=1e-12)
        assert bf.best_response(g, prof, i)[0] == pytest.approx(want, rel=1e-12, abs=1e-12)
    e, b0, b1 = o.exploitability()
    assert e > 0


BR_CASES = {
    "blocker_river": blocker_river,
    "river8": small_river,
    "river8_r4": lambda: small_river(seed=11, max_raises=4, bet_sizes=(0.33, 0.75, 1.25, synth.ALL_IN)),
    "turn6": small_turn,
    "flop4": small_flop,
}


@pytest.mark.parametrize("case", list(BR_CASES))
def test_best_response_values_at_every_node(oracle_mod, case):
    """Root value and v*_i(node, h) at every node against the engine's per-infoset maximum
    (river blockers; turn: 1/44 per river card; flop: 1/45 then 1/44)."""
    spec = BR_CASES[case]()
    o = solved(oracle_mod, spec, iters=3)
    g = bf_game(spec)
    hmap = node_histories(o, g)
    root, node = br_errors(o, g, hmap)
    assert root <= 1e-12 and node <= 1e-12, (root, node)


# ---------------------------------------------------------------- own reach
# (the exact 4-hand flop's 31k nodes take the engine's per-deal walk over a minute, so the
# flop is checked in its depth-limited form: turn card by chance, turn betting, leaves)

def depth_limited(spec):
    spec.depth_limit = 1
    return spec


REACH_CASES = {
    "turn6": small_turn,
    "turn6_depth_limited": lambda: depth_limited(small_turn()),
    "flop4_depth_limited": lambda: depth_limited(small_flop()),
}


@pytest.mark.parametrize("case", list(REACH_CASES))
def test_node_reach_matches_the_engine(oracle_mod, case):
    """ocfr_node_reach at every node (the depth-limit leaves included) from random regrets
    and average sums, against the engine's walk of every deal and history."""
    spec = REACH_CASES[case]()
    o = oracle_mod.Oracle(spec, variant="dcfr", threads=1)
    g = bf_game(spec)
    hmap = node_histories(o, g)
    if spec.depth_limit:
        assert any(nd["type"] == 4 for nd in o.nodes())
    set_random_state(o, 7)
    assert reach_errors(o, g, hmap) <= 1e-15


# ---------------------------------------------------------------- planted mistakes

# (name, text in the oracle's source, replacement): each is a mistake a plausible
# implementation could make; the pins above must catch every one.
MUTATIONS = [
    ("chance weight 1/46 instead of 1/44",
     "double K = (double)(o->deck - nd->nboard - 2 * o->hsize);",
     "double K = (double)(o->deck - nd->nboard - 2 * o->hsize + 2);"),
    ("opponent hands holding the dealt card kept",
     "hand_has(o, h, o->nodes[kid].deal) ? 0.0 : q[(size_t)n * o->nh + h] / K",
     "q[(size_t)n * o->nh + h] / K"),
    ("two-card blockers dropped at the terminal sums",
     "if (cm[ho] && q[ho] != 0.0)",
     "if (q[ho] != 0.0)"),
    ("opponent's own action probabilities left out of its reach",
     "(nd->player == opp ? o->prof[(size_t)(nd->row + a) * o->nh + h] : 1.0)",
     "1.0"),
    ("own reach keeps hands holding a dealt card",
     "if (child->deal >= 0 && hand_has(o, h, child->deal)) out[h] = 0.0;",
     ""),
    ("own reach takes the opponent's action probabilities",
     "if (par->type == T_DEC && par->player == p)",
     "if (par->type == T_DEC && par->player != p)"),
]


def build_mutant(tmp_path, name, old, new):
    src = open(ORACLE_SRC).read()
    assert src.count(old) == 1, f"{name}: the oracle's source no longer has the text this mutation replaces"
    path = tmp_path / (re.sub(r"\W+", "_", name) + ".so")
    csrc = tmp_path / (path.stem + ".c")
    csrc.write_text(src.replace(old, new))
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared", "-pthread", "-o",
                           str(path), str(csrc), "-lm"])
    return str(path)


@pytest.mark.parametrize("mutation", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistakes_fail_the_pins(oracle_mod, tmp_path, mutation):
    name, old, new = mutation
    lib = build_mutant(tmp_path, name, old, new)
    caught = []
    for case in ("blocker_river", "turn6"):
        spec = BR_CASES[case]()
        o = solved(oracle_mod, spec, iters=3, lib_path=lib)
        g = bf_game(spec)
        root, node = br_errors(o, g, node_histories(o, g))
        caught.append(root > 1e-9 or node > 1e-9)
    spec = REACH_CASES["turn6_depth_limited"]()
    o = oracle_mod.Oracle(spec, variant="dcfr", threads=1, lib_path=lib)
    g = bf_game(spec)
    set_random_state(o, 7)
    caught.append(reach_errors(o, g, node_histories(o, g)) > 1e-9)
    assert any(caught), f"no pin caught the planted mistake: {name}"
