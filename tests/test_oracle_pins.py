"""Pins of the FP64 oracle against things other than itself (no GPU).

* closed form: Kuhn poker's game value -1/18 over the whole equilibrium family;
* brute force: best response by enumerating all 64 pure Kuhn strategies;
* definitions by enumeration: regrets (Section 3), counterfactual values (Eq. cfv), regret
  matching (Eq. rm) and the Stage 7 variant updates, computed by an independent
  history-based rules engine (tests/bruteforce.py) on Kuhn, Leduc and small hold'em
  river/turn subgames;
* counts: Leduc's 936 infosets; the paper's printed node/infoset/history counts;
* invariants: zero sum, exploitability >= 0 and falling towards 0.
"""
import os

import numpy as np
import pytest

import bruteforce as bf
from paper_2605_19928_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def bf_game(spec):
    if spec.game == synth.GAME_KUHN:
        return bf.Game(bf.KUHN, ranges=spec.ranges)
    if spec.game == synth.GAME_LEDUC:
        return bf.Game(bf.LEDUC, ranges=spec.ranges)
    return bf.Game(bf.HOLDEM, hands=spec.hands, ranges=spec.ranges, board=spec.board, strength=spec.strength,
                   pot=spec.pot, stack=spec.stack, sizes=spec.bet_sizes, max_raises=spec.max_raises)


def history_map(o, g):
    """Oracle node id -> brute-force history; asserts that the two trees agree."""
    om_types = {0: "dec", 1: "fold", 2: "show", 3: "chance"}
    info = o.nodes()
    out = {}

    def rec(n, hist):
        out[n] = hist
        nd = info[n]
        st = g.state(hist)
        assert tuple(nd["contrib"]) == pytest.approx(tuple(st["c"]), abs=1e-9), (n, hist)
        kind = om_types[nd["type"]]
        if kind == "dec":
            acts = g.legal(hist)
            assert nd["n_actions"] == len(acts), (n, hist, acts)
            assert nd["player"] == st["to_act"]
            for k, kid in enumerate(nd["kids"]):
                rec(kid, hist + (acts[k],))
        elif kind == "chance":
            assert st["over"] and st["folded"] < 0
            for kid in nd["kids"]:
                rec(kid, hist + (("d", info[kid]["deal"]),))
        elif kind == "fold":
            assert st["folded"] == nd["player"]
        else:
            assert st["over"] and st["folded"] < 0 and st["street"] == g.n_streets - 1

    rec(0, ())
    return out


def blocked(g, h, hist):
    cards = set(g.hands[h])
    return any(tok[0] == "d" and tok[1] in cards for tok in hist)


def compare_state(o, g, hmap, R, S, rtol=1e-10):
    info = o.nodes()
    scale_r = max((abs(x) for v in R.values() for x in v), default=1.0)
    scale_s = max((abs(x) for v in S.values() for x in v), default=1.0)
    n_checked = 0
    for n, nd in enumerate(info):
        if nd["type"] != 0:
            continue
        hist = hmap[n]
        oR, oS = o.regrets(n), o.avg_sums(n)
        for h in range(o.n_hands):
            key = bf.infoset_key(nd["player"], h, hist)
            if blocked(g, h, hist):
                assert np.all(oR[:, h] == 0) and np.all(oS[:, h] == 0)
                continue
            if key not in R:  # never reached (e.g. a hand that meets no opponent hand)
                assert np.all(oR[:, h] == 0)
                continue
            np.testing.assert_allclose(oR[:, h], R[key], rtol=rtol, atol=rtol * scale_r)
            np.testing.assert_allclose(oS[:, h], S.get(key, [0.0] * nd["n_actions"]), rtol=rtol,
                                       atol=rtol * scale_s)
            n_checked += 1
    return n_checked


def small_river(n_hands=8, seed=3, **kw):
    return synth.river_subgame(n_hands=n_hands, seed=seed, range_seed=seed + 1, **kw)


def small_turn(n_hands=6, seed=5):
    return synth.turn_subgame(n_hands=n_hands, seed=seed, range_seed=seed + 1, bet_sizes=(1.0, synth.ALL_IN),
                              max_raises=1)


def small_flop(n_hands=4, seed=3):
    """Flop subgame small enough to enumerate: all-in the only bet, one per street."""
    return synth.flop_subgame(n_hands=n_hands, seed=seed, range_seed=seed + 1, bet_sizes=(synth.ALL_IN,),
                              max_raises=1)


# ---------------------------------------------------------------- trees and counts

def test_kuhn_tree(oracle_mod):
    o = oracle_mod.Oracle(synth.kuhn(), variant="cfr", threads=1)
    assert o.n_nodes == 9
    history_map(o, bf_game(synth.kuhn()))
    dec = [n for n in o.nodes() if n["type"] == 0]
    assert len(dec) * 3 == 12  # Kuhn has 12 infosets


def test_leduc_tree_has_936_infosets(oracle_mod):
    spec = synth.leduc()
    o = oracle_mod.Oracle(spec, variant="cfr", threads=1)
    g = bf_game(spec)
    hmap = history_map(o, g)
    infosets = 0
    for n, nd in enumerate(o.nodes()):
        if nd["type"] == 0:
            infosets += sum(not blocked(g, h, hmap[n]) for h in range(6))
    assert infosets == 936
    assert o.n_nodes == 465


@pytest.mark.parametrize("make", [lambda: small_river(), lambda: small_river(max_raises=4),
                                  lambda: small_turn(), lambda: small_flop()])
def test_holdem_trees_agree_with_rules_engine(oracle_mod, make):
    spec = make()
    o = oracle_mod.Oracle(spec, threads=1)
    history_map(o, bf_game(spec))


def test_card_removal_counts(oracle_mod):
    # C(47,2) river, C(48,2) turn, C(49,2) flop hands; C(45,2) opponent hands per river hand.
    rng = np.random.default_rng(0)
    board = rng.choice(52, size=5, replace=False)
    assert len(synth.all_combos(board)) == 1081
    assert len(synth.all_combos(board[:4])) == 1128
    assert len(synth.all_combos(board[:3])) == 1176
    spec = synth.river_subgame()
    spec.ranges[:] = 1.0
    o = oracle_mod.Oracle(spec, threads=1)
    assert o.Z == pytest.approx(990.0 / 1081.0, rel=1e-10)  # 1e6-term FP64 sum


def test_paper_printed_counts():
    """Section 5 'Baselines' and Table 4: histories = nodes x 1176 x 1081 and
    infosets = nodes x 2 x 1176 on a flop board (own hand, one opponent hand that shares
    no card with it)."""
    vals = {}
    rows = []
    with open(os.path.join(GOLDEN, "paper_counts.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            if parts[0] == "table4":
                rows.append(tuple(int(x) for x in parts[1:]))
            else:
                vals[parts[0]] = int(parts[1])
    board = np.array([0, 17, 33])
    hands = synth.all_combos(board)
    n_h = len(hands)
    opp = sum(1 for h in hands if not (set(h) & set(hands[0])))
    assert (n_h, opp) == (1176, 1081)
    assert vals["default_nodes"] * n_h * opp == vals["default_histories"]
    assert vals["default_nodes"] * 2 * n_h == vals["default_infosets"]
    for _, _, nodes, infosets in rows:
        assert nodes * 2 * n_h == infosets


# ---------------------------------------------------------------- closed form and brute-force BR

def kuhn_equilibrium(o, a):
    """Load Kuhn's equilibrium with parameter a (tests/golden/kuhn_equilibrium.txt)."""
    o.load_profile("current")
    paths = o.paths()
    # node paths: () P0 first; (0,) P1 after check; (0, 1) P0 after check-bet; (1,) P1 after bet
    bet0 = [a, 0.0, 3 * a]
    call0 = [0.0, a + 1.0 / 3, 1.0]
    bet1 = [1.0 / 3, 0.0, 1.0]
    call1 = [0.0, 1.0 / 3, 1.0]
    o.set_profile_node(paths[()], [[1 - x for x in bet0], bet0])
    o.set_profile_node(paths[(0, 1)], [[1 - x for x in call0], call0])
    o.set_profile_node(paths[(0,)], [[1 - x for x in bet1], bet1])
    o.set_profile_node(paths[(1,)], [[1 - x for x in call1], call1])


def golden_kuhn_value():
    with open(os.path.join(GOLDEN, "kuhn_equilibrium.txt")) as f:
        for line in f:
            if line.startswith("game_value_player0"):
                return float(line.split()[1])


@pytest.mark.parametrize("a", [0.0, 1.0 / 6, 1.0 / 3])
def test_kuhn_equilibrium_value_is_minus_one_eighteenth(oracle_mod, a):
    o = oracle_mod.Oracle(synth.kuhn(), variant="cfr", threads=1)
    kuhn_equilibrium(o, a)
    v = o.profile_value()
    assert v[0] == pytest.approx(golden_kuhn_value(), abs=1e-14)
    assert v[0] + v[1] == pytest.approx(0.0, abs=1e-15)
    br0, _ = o.best_response(0)
    br1, _ = o.best_response(1)
    # an equilibrium cannot be exploited: each best response earns exactly the game value
    assert br0 == pytest.approx(-1.0 / 18, abs=1e-14)
    assert br1 == pytest.approx(1.0 / 18, abs=1e-14)


def oracle_profile_table(o, g, player):
    hmap = history_map(o, g)
    table = {}
    for n, nd in enumerate(o.nodes()):
        if nd["type"] == 0 and nd["player"] == player:
            p = o.profile(n)
            for h in range(o.n_hands):
                if not blocked(g, h, hmap[n]):
                    table[bf.infoset_key(player, h, hmap[n])] = list(p[:, h])
    return bf.Profile(table)


@pytest.mark.parametrize("variant", ["cfr", "dcfr"])
def test_kuhn_best_response_equals_pure_strategy_enumeration(oracle_mod, variant):
    spec = synth.kuhn()
    o = oracle_mod.Oracle(spec, variant=variant, threads=1)
    g = bf_game(spec)
    o.iterate(7)
    o.load_profile("average")
    for i in (0, 1):
        br, _ = o.best_response(i)
        want = bf.kuhn_best_response_bruteforce(oracle_profile_table(o, g, 1 - i), i)
        assert br == pytest.approx(want, abs=1e-13)
    e, b0, b1 = o.exploitability()
    assert e >= 0 and e == pytest.approx(0.5 * (b0 + b1))


# ---------------------------------------------------------------- definitions by enumeration

CASES = {
    "kuhn": synth.kuhn,
    "leduc": synth.leduc,
    "river8": small_river,
    "river8_r4": lambda: small_river(seed=11, max_raises=4, bet_sizes=(0.33, 0.75, 1.25, synth.ALL_IN)),
    "turn6": small_turn,
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("variant,alternating", [("cfr", True), ("cfr+", True), ("dcfr", True), ("dcfr", False),
                                               ("pcfr+", True), ("pcfr+", False)])
def test_two_iterations_match_definitions(oracle_mod, case, variant, alternating):
    spec = CASES[case]()
    if case in ("kuhn", "leduc"):
        # non-uniform ranges make the range weighting visible
        spec.ranges[:] = synth.random_ranges(spec.n_hands, 99)
    o = oracle_mod.Oracle(spec, variant=variant, alternating=alternating, threads=2)
    g = bf_game(spec)
    hmap = history_map(o, g)
    n_it = 3 if variant == "pcfr+" else 2  # the prediction first steers iteration 2
    o.iterate(n_it)
    R, S = bf.run_cfr(g, n_it, variant=variant, alternating=alternating)
    assert compare_state(o, g, hmap, R, S) > 0


def test_flop_two_iterations_match_definitions(oracle_mod):
    """Three streets: the turn and river cards dealt by chance (1/45 then 1/44 given both
    hands), showdown strengths by completed board."""
    spec = small_flop()
    o = oracle_mod.Oracle(spec, variant="dcfr", threads=2)
    g = bf_game(spec)
    hmap = history_map(o, g)
    o.iterate(2)
    R, S = bf.run_cfr(g, 2, variant="dcfr")
    assert compare_state(o, g, hmap, R, S) > 0


@pytest.mark.parametrize("case", ["leduc", "river8", "turn6"])
def test_counterfactual_values_match_definition(oracle_mod, case):
    spec = CASES[case]()
    o = oracle_mod.Oracle(spec, variant="dcfr", threads=2)
    g = bf_game(spec)
    hmap = history_map(o, g)
    o.iterate(1)
    R, _ = bf.run_cfr(g, 1, variant="dcfr")
    prof = bf.regret_matching(R)
    for i in (0, 1):
        o.values_current(i)
        _, val = bf.regrets_and_values(g, prof, i)
        for n, nd in enumerate(o.nodes()):
            if nd["type"] != 0 or nd["player"] != i:
                continue
            got = o.cfv(i, n)
            for h in range(o.n_hands):
                key = bf.infoset_key(i, h, hmap[n])
                want = val.get(key, 0.0)
                assert got[h] == pytest.approx(want, rel=1e-11, abs=1e-13)


def test_regret_matching_rule(oracle_mod):
    """Eq. (rm): positive part normalised, uniform when no regret is positive."""
    o = oracle_mod.Oracle(synth.leduc(), variant="cfr", threads=1)
    for n, nd in enumerate(o.nodes()):
        if nd["type"] == 0:
            assert np.allclose(o.strategy(n), 1.0 / nd["n_actions"])
    o.iterate(3)
    n_uniform = 0
    for n, nd in enumerate(o.nodes()):
        if nd["type"] != 0:
            continue
        R, s = o.regrets(n), o.strategy(n)
        pos = np.maximum(R, 0.0)
        tot = pos.sum(axis=0)
        for h in range(o.n_hands):
            if tot[h] > 0:
                np.testing.assert_allclose(s[:, h], pos[:, h] / tot[h], rtol=1e-15)
            else:
                n_uniform += 1
                np.testing.assert_allclose(s[:, h], 1.0 / nd["n_actions"])
    assert n_uniform > 0


# ---------------------------------------------------------------- invariants

@pytest.mark.parametrize("case", ["leduc", "river8", "turn6"])
def test_zero_sum(oracle_mod, case):
    spec = CASES[case]()
    o = oracle_mod.Oracle(spec, variant="dcfr", threads=2)
    o.iterate(3)
    for kind in ("current", "average"):
        o.load_profile(kind)
        v = o.profile_value()
        assert abs(v[0] + v[1]) <= 1e-12 * max(1.0, spec.pot)


def test_leduc_average_strategy_reaches_the_game_value(oracle_mod):
    """CFR+ on Leduc: the average profile's value for player 0 approaches the game value
    quoted in tests/golden/leduc_value.txt, within its exploitability plus the quote's
    rounding."""
    with open(os.path.join(GOLDEN, "leduc_value.txt")) as f:
        want = float([ln.split()[1] for ln in f if ln.startswith("game_value_player0")][0])
    o = oracle_mod.Oracle(synth.leduc(), variant="cfr+", threads=4)
    o.iterate(2000)
    o.load_profile("average")
    v = o.profile_value()
    e = o.exploitability()[0]
    assert e < 2e-4
    assert abs(v[0] - want) <= e + 5e-5
    assert v[0] + v[1] == pytest.approx(0.0, abs=1e-12)


def test_cfr_plus_regrets_never_negative(oracle_mod):
    o = oracle_mod.Oracle(synth.leduc(), variant="cfr+", threads=1)
    o.iterate(20)
    for n, nd in enumerate(o.nodes()):
        if nd["type"] == 0:
            assert (o.regrets(n) >= 0).all()


@pytest.mark.parametrize("variant", ["cfr", "cfr+", "dcfr", "pcfr+"])
def test_leduc_exploitability_falls_to_zero(oracle_mod, variant):
    o = oracle_mod.Oracle(synth.leduc(), variant=variant, threads=1)
    seen = []
    for n in (10, 90, 900):
        o.iterate(n)
        e, b0, b1 = o.exploitability()
        assert e >= -1e-15
        seen.append(e)
    assert seen[0] > seen[1] > seen[2]
    assert seen[2] < {"cfr": 0.02, "cfr+": 0.002, "dcfr": 0.002, "pcfr+": 0.002}[variant]


def test_thread_count_does_not_change_results(oracle_mod):
    spec = small_river(n_hands=40, seed=2)
    a = oracle_mod.Oracle(spec, threads=1)
    b = oracle_mod.Oracle(spec, threads=5)
    a.iterate(2)
    b.iterate(2)
    for n, nd in enumerate(a.nodes()):
        if nd["type"] == 0:
            assert np.array_equal(a.regrets(n), b.regrets(n))
            assert np.array_equal(a.avg_sums(n), b.avg_sums(n))


def test_rejects_invalid_hands(oracle_mod):
    spec = small_river()
    spec.hands[0, 0] = spec.board[0]
    with pytest.raises(ValueError):
        oracle_mod.Oracle(spec, threads=1)
