"""Input generators: the rank-based showdown evaluator against hand-worked poker cases, and
the generators' shapes."""
import numpy as np

from paper_2605_19928_gb300 import synth


def card(rank, suit):
    return 4 * rank + suit


def test_rank_strength_orders_categories():
    # board: A K Q of suit 0, 5 of suit 1, 4 of suit 2 (ranks 0..12 = deuce..ace)
    board = [card(12, 0), card(11, 0), card(10, 0), card(3, 1), card(2, 2)]
    hands = np.array([[card(9, 0), card(8, 0)],    # J T suited: straight flush to the ace
                      [card(9, 1), card(8, 2)],    # J T: straight to the ace
                      [card(12, 1), card(12, 2)],  # A A: three of a kind
                      [card(1, 0), card(0, 0)],    # 3 2 of suit 0: flush, A K Q 3 2
                      [card(3, 0), card(2, 0)],    # 5 4 of suit 0: flush, A K Q 5 4
                      [card(0, 1), card(1, 2)],    # 2 3: straight to the five (ace low)
                      [card(6, 1), card(7, 2)]])   # 8 9: ace high
    s = synth.rank_strength(board, hands)
    order = list(np.argsort(s))
    assert order == [6, 2, 5, 1, 3, 4, 0]


def test_rank_strength_ties_and_kickers():
    board = [card(12, 0), card(12, 1), card(7, 2), card(5, 3), card(2, 0)]
    hands = np.array([[card(11, 2), card(3, 1)],   # A A K: pair of aces, king kicker
                      [card(11, 3), card(4, 1)],   # same five cards (A A K 9 7): tie
                      [card(10, 2), card(3, 3)],   # A A Q
                      [card(7, 0), card(3, 2)]])   # two pair, aces and nines
    s = synth.rank_strength(board, hands)
    assert s[0] == s[1] and s[2] < s[0] < s[3]


def test_training_rivers_are_seeded_and_valid():
    a = synth.leaf_training_rivers(3, seed=4)
    b = synth.leaf_training_rivers(3, seed=4)
    for x, y in zip(a, b):
        assert np.array_equal(x.board, y.board) and np.array_equal(x.ranges, y.ranges)
        assert x.hands.shape == (1081, 2) and np.allclose(x.ranges.sum(axis=1), 1.0, atol=1e-5)
        assert 100.0 <= x.pot <= 900.0 and 50.0 <= x.stack <= 500.0
    t = synth.ranked_turn_subgame(n_hands=30, depth_limit=1)
    assert t.depth_limit == 1 and t.strength.shape == (52, 30)


def test_flop_strength_rows_depend_only_on_the_completed_board():
    g = synth.flop_subgame(n_hands=40, seed=2)
    assert g.board.shape == (3,) and g.hands.shape == (40, 2) and g.strength.shape == (52 * 52, 40)
    on = set(int(c) for c in g.board)
    live = [c for c in range(52) if c not in on]
    for t, r in [(live[0], live[5]), (live[10], live[3]), (live[20], live[44])]:
        assert np.array_equal(g.strength[t * 52 + r], g.strength[r * 52 + t])  # same five cards
    assert not g.strength[live[0] * 52 + live[0]].any()          # a card cannot come twice
    assert not g.strength[int(g.board[0]) * 52 + live[1]].any()  # nor a board card
    r = synth.ranked_flop_subgame(n_hands=25, seed=6)
    t, v = live[1], live[7]
    ok = ~np.any((r.hands == t) | (r.hands == v), axis=1)
    want = synth.rank_strength(np.concatenate([r.board, [t, v]]), r.hands[ok])
    # the same order as the evaluator on the completed board (dense ranks may differ by offset)
    assert np.array_equal(np.argsort(r.strength[t * 52 + v][ok], kind="stable"), np.argsort(want, kind="stable"))


def test_training_turns_are_seeded_and_valid():
    a = synth.leaf_training_turns(2, seed=3)
    b = synth.leaf_training_turns(2, seed=3)
    for x, y in zip(a, b):
        assert np.array_equal(x.board, y.board) and np.array_equal(x.ranges, y.ranges)
        assert x.board.shape == (4,) and x.hands.shape == (1128, 2) and x.strength.shape == (52, 1128)
        assert np.allclose(x.ranges.sum(axis=1), 1.0, atol=1e-5)
        assert 100.0 <= x.pot <= 400.0 and 100.0 <= x.stack <= 600.0
        assert x.bet_sizes[-1] == synth.ALL_IN and 2 <= x.max_raises <= 3


def test_batch_shape(oracle_mod):
    """The batched-serving workload: 1-4 pot-fraction sizes (one below 1 pot) plus all-in,
    stacks 100-1000 behind a pot of 100, 2-3 bets/raises, and trees of 21 to 315 public
    nodes (median 84), counted on the oracle's own trees."""
    specs = synth.batch_rivers(256)
    nodes = []
    for g in specs:
        assert g.pot == 100.0 and 100 <= g.stack <= 1000 and g.max_raises in (2, 3)
        sizes = [x for x in g.bet_sizes if x > 0]
        assert 1 <= len(sizes) <= 4 and min(sizes) < 1.0 and g.bet_sizes[-1] == synth.ALL_IN
        assert g.n_hands == 1081
        nodes.append(oracle_mod.Oracle(g, variant="dcfr", threads=1).n_nodes)
    assert (min(nodes), float(np.median(nodes)), max(nodes)) == (21, 84.0, 315)
