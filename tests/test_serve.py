"""Host logic of the served depth-limited solve (learned leaves judged against exact
continuation solves, Section 3): continuation specs, leaf boards, row order, the error
statistic, and the keep-or-fall-back decision with its handle bookkeeping.  No GPU: the
tree walk runs on a fake public tree and the decision on a fake C ABI."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2605_19928_gb300 import capi, serve, synth


def test_river_cards_follow_the_leaf_rows():
    board = [3, 17, 30, 44]
    cards = serve.river_cards(board)
    assert len(cards) == capi.LEAF_CARDS
    assert cards == sorted(cards) and not set(cards) & set(board)


def test_turn_continuation_is_the_river_subgame_below_the_card():
    spec = synth.ranked_turn_subgame(n_hands=150, seed=3, range_seed=4, depth_limit=1)
    rng = np.random.default_rng(0)
    reach = rng.random((2, spec.n_hands))
    r = serve.river_cards(spec.board)[11]
    cont = serve.continuation_spec(spec, spec.board, r, reach, pot=160.0, behind=320.0)
    full = sorted([int(c) for c in spec.board] + [r])
    assert cont.board.tolist() == full and cont.depth_limit == 0
    live = ~np.any(spec.hands == r, axis=1)
    assert cont.n_hands == int(live.sum())
    assert not np.isin(cont.hands, full).any()
    np.testing.assert_array_equal(cont.hands, spec.hands[live])
    # strengths from the rules of poker on the completed board, computed afresh
    np.testing.assert_array_equal(cont.strength[0], synth.rank_strength(full, cont.hands))
    for p in (0, 1):
        want = reach[p][live] / reach[p][live].sum()
        np.testing.assert_allclose(cont.ranges[p], want, rtol=1e-6)
    assert (cont.pot, cont.stack) == (160.0, 320.0)
    assert cont.bet_sizes == spec.bet_sizes and cont.max_raises == spec.max_raises


def test_flop_continuation_uses_the_turn_and_river_row():
    spec = synth.ranked_flop_subgame(n_hands=60, seed=5, range_seed=6, depth_limit=1)
    t = serve.river_cards(spec.board)[7]
    board = [int(c) for c in spec.board] + [t]
    r = serve.river_cards(board)[30]
    reach = np.ones((2, spec.n_hands))
    cont = serve.continuation_spec(spec, board, r, reach, pot=200.0, behind=50.0)
    full = sorted(board + [r])
    np.testing.assert_array_equal(cont.strength[0], synth.rank_strength(full, cont.hands))
    assert not np.isin(cont.hands, full).any()


def test_continuation_without_reach_is_skipped():
    spec = synth.ranked_turn_subgame(n_hands=80, seed=1, range_seed=2, depth_limit=1)
    reach = np.ones((2, spec.n_hands))
    r = serve.river_cards(spec.board)[0]
    reach[1][~np.any(spec.hands == r, axis=1)] = 0.0  # player 1 only holds hands with card r
    assert serve.continuation_spec(spec, spec.board, r, reach, 100.0, 100.0) is None


def test_strength_row_rejects_other_boards():
    spec = synth.ranked_turn_subgame(n_hands=40, seed=1, range_seed=2)
    with pytest.raises(ValueError):
        serve.strength_row(spec, list(spec.board))


def test_row_errors_by_hand():
    hands = np.array([[0, 1], [2, 5]], np.uint8)
    sl = [1 * 0 // 2 + 0, 5 * 4 // 2 + 2]  # slot b (b - 1) / 2 + a
    y_net = np.zeros(2 * serve.SLOTS + 36, np.float32)
    y_ex = np.zeros_like(y_net)
    mask = np.zeros_like(y_net)
    y_net[sl[0]], y_ex[sl[0]], mask[sl[0]] = 0.5, 0.25, 1.0             # player 0, hand 0
    y_net[sl[1]], y_ex[sl[1]], mask[sl[1]] = -1.0, -1.0, 1.0            # player 0, hand 1
    y_net[serve.SLOTS + sl[1]], y_ex[serve.SLOTS + sl[1]] = 3.0, 1.0    # player 1, hand 1: masked
    y_net[serve.SLOTS + sl[0]], y_ex[serve.SLOTS + sl[0]], mask[serve.SLOTS + sl[0]] = 0.0, 0.1, 1.0
    ranges = np.array([[0.75, 0.25], [0.4, 0.6]])
    tot, weighted, cnt = serve.row_errors(y_net, y_ex, mask, ranges, hands)
    assert cnt == 3
    assert tot == pytest.approx(0.25 + 0.0 + 0.1, rel=1e-6)
    assert weighted == pytest.approx(0.5 * (0.75 * 0.25 + 0.4 * 0.1), rel=1e-6)


def test_leaf_board_collects_the_dealt_cards(monkeypatch):
    # root decision 0 -> chance 1 -> (turn card 9) 2 -> decision 3 -> leaf 4
    nodes = {0: (capi.CFR_NODE_DECISION, -1, -1), 1: (capi.CFR_NODE_CHANCE, 0, -1),
             2: (capi.CFR_NODE_DECISION, 1, 9), 3: (capi.CFR_NODE_DECISION, 2, -1),
             4: (capi.CFR_NODE_LEAF, 3, -1)}

    def fake_info(tree, node, game=0):
        t, parent, deal = nodes[node]
        return {"type": t, "parent": parent, "deal": deal}

    monkeypatch.setattr(serve.capi, "cfr_node_info", fake_info)
    spec = synth.flop_subgame(n_hands=10, seed=2, range_seed=3)
    assert serve.leaf_board(None, 4, spec) == [int(c) for c in spec.board] + [9]
    assert serve.leaf_board(None, 1, spec) == [int(c) for c in spec.board]


def test_solve_depth_limited_wants_a_depth_limit():
    spec = synth.ranked_turn_subgame(n_hands=20, seed=1, range_seed=2, depth_limit=0)
    with pytest.raises(ValueError):
        serve.solve_depth_limited(spec, None, None, 10)


class FakeABI:
    """Records the handles the served solve creates and destroys (no GPU)."""

    def __init__(self, fail_iterate=False):
        self.live, self.created, self.fail_iterate = set(), [], fail_iterate

    def cfr_tree_create(self, spec, opts, stream=None):
        kind = "exact" if spec.depth_limit == 0 else ("mixed" if getattr(spec, "exact_leaves", ()) else "learned")
        h = (kind, len(self.created), tuple(getattr(spec, "exact_leaves", ())))
        self.created.append(h)
        self.live.add(h)
        return h

    def cfr_leaf_info(self, h):
        return [(0, 10 + k, 48 * k) for k in range(4)]  # four leaves

    def cfr_tree_destroy(self, h):
        self.live.discard(h)

    def cfr_iterate(self, h, n):
        if self.fail_iterate:
            raise RuntimeError("iterate failed")

    def noop(self, *a, **k):
        return None


def _fake(monkeypatch, error, rows=8, fail_iterate=False, leaf_errors=None):
    abi = FakeABI(fail_iterate)
    for name in ("cfr_tree_create", "cfr_tree_destroy", "cfr_iterate", "cfr_leaf_info"):
        monkeypatch.setattr(serve.capi, name, getattr(abi, name))
    for name in ("cfr_set_leaf_net", "cfr_exploitability", "cfr_sync"):
        monkeypatch.setattr(serve.capi, name, abi.noop)
    monkeypatch.setattr(serve.capi, "make_opts", lambda *a, **k: None)
    j = serve.Judgement(rows, 100, error, error, error, 0.1, 1.0,
                        leaf_errors=[error] * 4 if leaf_errors is None else list(leaf_errors))
    monkeypatch.setattr(serve, "judge_leaves", lambda *a, **k: j)
    return abi


def test_fallback_leaves_are_those_above_tolerance():
    assert serve.fallback_leaves([5e-4, 2e-3, None, 3e-3, 1e-3], 1e-3) == [1, 3]
    assert serve.fallback_leaves([None, None], 1e-3) == []


def test_served_solve_keeps_the_learned_form_within_tolerance(monkeypatch):
    spec = synth.ranked_turn_subgame(n_hands=20, seed=1, range_seed=2, depth_limit=1)
    for per_leaf in (4, 0):
        abi = _fake(monkeypatch, error=5e-4)
        s = serve.solve_depth_limited(spec, None, None, 10, tol=1e-3, per_leaf=per_leaf)
        assert s.form == "learned" and s.tree[0] == "learned" and abi.live == {s.tree}
        assert s.ms["exact"] == 0.0 and s.exact_leaves == ()


def test_served_solve_falls_back_per_leaf(monkeypatch):
    """Leaves above the tolerance become exact river subtrees in one handle beside the
    network leaves of the rest; every leaf failing means the full-depth subgame."""
    spec = synth.ranked_turn_subgame(n_hands=20, seed=1, range_seed=2, depth_limit=1)
    abi = _fake(monkeypatch, error=0.0, leaf_errors=[5e-4, 2e-3, None, 3e-3])
    s = serve.solve_depth_limited(spec, None, None, 10, tol=1e-3)
    assert s.form == "mixed" and s.tree == ("mixed", 1, (1, 3)) and s.exact_leaves == (1, 3)
    assert abi.live == {s.tree}
    abi = _fake(monkeypatch, error=0.0, leaf_errors=[2e-3] * 4)
    s = serve.solve_depth_limited(spec, None, None, 10, tol=1e-3)
    assert s.form == "exact" and s.tree[0] == "exact" and abi.live == {s.tree}
    assert spec.depth_limit == 1 and spec.exact_leaves == ()  # the caller's spec is left as it was


def test_served_solve_falls_back_above_tolerance_or_without_rows(monkeypatch):
    """Judged over all leaves together (per_leaf = 0): the whole subgame to full depth."""
    spec = synth.ranked_turn_subgame(n_hands=20, seed=1, range_seed=2, depth_limit=1)
    for error, rows in ((2e-3, 8), (0.0, 0)):  # too large; nothing could be judged
        abi = _fake(monkeypatch, error=error, rows=rows)
        s = serve.solve_depth_limited(spec, None, None, 10, tol=1e-3, per_leaf=0)
        assert s.form == "exact" and s.tree[0] == "exact"
        assert abi.live == {s.tree}  # the learned handle was released
        assert spec.depth_limit == 1  # the caller's spec is left as it was


def test_served_solve_releases_its_handle_on_errors(monkeypatch):
    spec = synth.ranked_turn_subgame(n_hands=20, seed=1, range_seed=2, depth_limit=1)
    abi = _fake(monkeypatch, error=0.0, fail_iterate=True)
    with pytest.raises(RuntimeError):
        serve.solve_depth_limited(spec, None, None, 10)
    assert abi.created and not abi.live


def test_judge_without_leaves_judges_nothing(monkeypatch):
    passes = []
    monkeypatch.setattr(serve.capi, "cfr_leaf_info", lambda tree: [])
    monkeypatch.setattr(serve.capi, "cfr_exploitability", lambda tree: passes.append(tree))
    spec = synth.ranked_turn_subgame(n_hands=20, seed=1, range_seed=2, depth_limit=1)
    j = serve.judge_leaves("handle", spec)
    assert (j.rows, j.candidates) == (0, 0)
    assert passes == ["handle"]  # the leaf reach comes from a fresh exploitability pass
    serve.judge_leaves("handle", spec, evaluated=True)
    assert passes == ["handle"]


def test_exact_targets_of_a_check_down_river(oracle_mod):
    """The judge's exact values per unit pot (leafnet_train.example, also the training
    target) on a river with no betting: hand h of player i is worth pot/2 x (W - L) / Z,
    W / L the opponent reach weaker / stronger than h sharing no card with it, so the
    target is (W - L) / (2 M) with M the opponent reach sharing no card with h."""
    from paper_2605_19928_gb300 import leafnet_train
    spec = synth.river_subgame(n_hands=40, seed=6, range_seed=7, max_raises=0)
    spec.strength = synth.rank_strength(spec.board, spec.hands)[None, :].astype(np.int32)  # ties
    o = oracle_mod.Oracle(spec, variant="dcfr", threads=1)
    v = []
    for i in (0, 1):
        o.values_current(i)
        v.append(o.cfv(i, 0))
    _, y, m = leafnet_train.example(spec, v)
    r = spec.ranges.astype(np.float64)
    r = r / r.sum(axis=1, keepdims=True)
    s = spec.strength[0]
    sl = leafnet_train.slot_of(spec.hands)
    for i in (0, 1):
        for h in range(spec.n_hands):
            dis = ~np.isin(spec.hands, spec.hands[h]).any(axis=1)
            q = r[1 - i] * dis
            W, L, M = q[s < s[h]].sum(), q[s > s[h]].sum(), q.sum()
            assert m[i * serve.SLOTS + sl[h]] == 1.0
            assert y[i * serve.SLOTS + sl[h]] == pytest.approx((W - L) / (2 * M), rel=1e-5, abs=1e-7)
