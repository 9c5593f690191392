"""Seeded synthetic subgames shaped like the paper's poker workloads.

The paper measures on heads-up no-limit hold'em subgames solved to the end of a betting
round (Section 5, "Game" and "Baselines") and compares convergence on a 93-node river
subgame (Section 5, "Convergence comparison").  Real boards, a hand evaluator and trained
networks are not available here, so these generators stand in for them with the same
shapes: 1081 (river), 1128 (turn) or 1176 (flop) two-card hands per player, integer
showdown strengths with ties, Dirichlet(1) ranges, and pot-fraction bet trees.

This module draws numbers only.  It holds none of the method's arithmetic: the CUDA path
and the CPU oracle both receive exactly the arrays produced here.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from itertools import combinations

import numpy as np

GAME_HOLDEM = 0
GAME_KUHN = 1
GAME_LEDUC = 2

DECK = 52
ALL_IN = -1.0  # a bet size <= 0 means "all-in"


def card(rank: int, suit: int) -> int:
    """Hold'em card id: 4 * rank + suit, rank 0..12 (deuce..ace), suit 0..3."""
    return 4 * rank + suit


@dataclass
class GameSpec:
    """One subgame: the public state, the private-hand list and both players' ranges."""

    game: int
    name: str
    board: np.ndarray                     # int32 [n_board] public cards (hold'em only)
    hands: np.ndarray                     # uint8 [n_hands, hand_size] private cards
    ranges: np.ndarray                    # float32 [2, n_hands], >= 0 (normalised by the solvers)
    strength: np.ndarray | None = None    # int32 [rows, n_hands]; 1 row (river), 52 (turn, by river
                                          # card) or 52 x 52 (flop, turn card x 52 + river card)
    pot: float = 0.0                      # chips in the pot; each player has put in pot / 2
    stack: float = 0.0                    # chips behind for each player
    bet_sizes: tuple = ()                 # pot fractions, ALL_IN for the all-in bet
    max_raises: int = 0                   # bets + raises allowed per street
    seeds: dict = field(default_factory=dict)
    depth_limit: int = 0                  # 1: the tree stops where the river card is to come (leaf network)
    exact_leaves: tuple = ()              # depth_limit 1: leaves (by index in the depth-limited tree's
                                          # breadth-first order) solved exactly instead

    @property
    def n_hands(self) -> int:
        return int(self.hands.shape[0])


def all_combos(board) -> np.ndarray:
    """Every two-card hand not blocked by the board, in lexicographic (c1 < c2) order."""
    dead = set(int(c) for c in board)
    live = [c for c in range(DECK) if c not in dead]
    return np.array(list(combinations(live, 2)), dtype=np.uint8)


def _dirichlet_ranges(rng: np.random.Generator, n: int) -> np.ndarray:
    # Dirichlet(1) = normalised Exp(1) draws, one vector per player.
    r = rng.exponential(1.0, size=(2, n))
    r /= r.sum(axis=1, keepdims=True)
    return r.astype(np.float32)


def river_subgame(n_hands: int | None = None, seed: int = 0, range_seed: int = 1,
                  pot: float = 100.0, stack: float = 400.0,
                  bet_sizes=(0.5, 1.0, ALL_IN), max_raises: int = 3) -> GameSpec:
    """River subgame: 5 seeded board cards, one uniform strength in [0, 2000) per combo.

    With ``n_hands`` set, a seeded subset of the 1081 combos is kept (same strengths as in
    the full game), which gives small cases for the oracle.
    """
    rng = np.random.default_rng(seed)
    board = np.sort(rng.choice(DECK, size=5, replace=False)).astype(np.int32)
    combos = all_combos(board)
    strength = rng.integers(0, 2000, size=combos.shape[0]).astype(np.int32)
    if n_hands is not None and n_hands < combos.shape[0]:
        keep = np.sort(np.random.default_rng(seed + 7919).choice(combos.shape[0], size=n_hands, replace=False))
        combos, strength = combos[keep], strength[keep]
    ranges = _dirichlet_ranges(np.random.default_rng(range_seed), combos.shape[0])
    return GameSpec(GAME_HOLDEM, "river", board, combos, ranges, strength[None, :].copy(), pot, stack,
                    tuple(float(x) for x in bet_sizes), max_raises,
                    {"board_strength": seed, "ranges": range_seed})


def turn_subgame(n_hands: int | None = None, seed: int = 0, range_seed: int = 1,
                 pot: float = 100.0, stack: float = 400.0,
                 bet_sizes=(0.5, 1.0, ALL_IN), max_raises: int = 3) -> GameSpec:
    """Turn subgame: 4 seeded board cards; the river card is dealt by chance.

    Strength row r holds every hand's showdown strength on the board completed by card r
    (rows of cards already on the board are unused and left at zero).
    """
    rng = np.random.default_rng(seed)
    board = np.sort(rng.choice(DECK, size=4, replace=False)).astype(np.int32)
    combos = all_combos(board)
    strength = rng.integers(0, 2000, size=(DECK, combos.shape[0])).astype(np.int32)
    strength[board, :] = 0
    if n_hands is not None and n_hands < combos.shape[0]:
        keep = np.sort(np.random.default_rng(seed + 7919).choice(combos.shape[0], size=n_hands, replace=False))
        combos, strength = combos[keep], strength[:, keep]
    ranges = _dirichlet_ranges(np.random.default_rng(range_seed), combos.shape[0])
    return GameSpec(GAME_HOLDEM, "turn", board, combos, ranges, np.ascontiguousarray(strength), pot, stack,
                    tuple(float(x) for x in bet_sizes), max_raises,
                    {"board_strength": seed, "ranges": range_seed})


def flop_subgame(n_hands: int | None = None, seed: int = 0, range_seed: int = 1,
                 pot: float = 100.0, stack: float = 150.0,
                 bet_sizes=(0.33, 0.75, 1.25, ALL_IN), max_raises: int = 4, depth_limit: int = 0) -> GameSpec:
    """Flop subgame: 3 seeded board cards; the turn and river cards are dealt by chance.

    Strength row t * 52 + r holds every hand's showdown strength on the board completed by
    turn t and river r, one uniform draw in [0, 2000) per hand and unordered pair {t, r}
    (rows of the pairs that meet the board or repeat a card are unused and left at zero).
    """
    rng = np.random.default_rng(seed)
    board = np.sort(rng.choice(DECK, size=3, replace=False)).astype(np.int32)
    combos = all_combos(board)
    strength = np.zeros((DECK * DECK, combos.shape[0]), np.int32)
    live = [c for c in range(DECK) if c not in set(int(b) for b in board)]
    for a, b in combinations(live, 2):
        s = rng.integers(0, 2000, size=combos.shape[0]).astype(np.int32)
        strength[a * DECK + b] = s
        strength[b * DECK + a] = s
    if n_hands is not None and n_hands < combos.shape[0]:
        keep = np.sort(np.random.default_rng(seed + 7919).choice(combos.shape[0], size=n_hands, replace=False))
        combos, strength = combos[keep], strength[:, keep]
    ranges = _dirichlet_ranges(np.random.default_rng(range_seed), combos.shape[0])
    return GameSpec(GAME_HOLDEM, "flop", board, combos, ranges, np.ascontiguousarray(strength), pot, stack,
                    tuple(float(x) for x in bet_sizes), max_raises,
                    {"board_strength": seed, "ranges": range_seed}, depth_limit)


def kuhn() -> GameSpec:
    """Kuhn poker: cards J, Q, K (ids 0, 1, 2), ante 1, one bet of 1, uniform deal."""
    hands = np.arange(3, dtype=np.uint8)[:, None]
    return GameSpec(GAME_KUHN, "kuhn", np.zeros(0, np.int32), hands, np.full((2, 3), 1.0 / 3, np.float32),
                    None, 2.0, 0.0, (), 1)


def leduc() -> GameSpec:
    """Leduc hold'em: J, Q, K in two suits (id = 2 * rank + suit), ante 1, bets 2 then 4."""
    hands = np.arange(6, dtype=np.uint8)[:, None]
    return GameSpec(GAME_LEDUC, "leduc", np.zeros(0, np.int32), hands, np.full((2, 6), 1.0 / 6, np.float32),
                    None, 2.0, 0.0, (), 2)


def random_ranges(n_hands: int, seed: int) -> np.ndarray:
    """Dirichlet(1) ranges for both players (used to perturb small games in tests)."""
    return _dirichlet_ranges(np.random.default_rng(seed), n_hands)


def batch_rivers(n: int = 256, seed: int = 0, n_hands: int | None = None) -> list[GameSpec]:
    """Uneven river subgames for batched serving: seeded boards, strengths and ranges (seeds
    1000 + k and 5000 + k), 1-4 pot-fraction bet sizes (at least one below 1 pot) plus
    all-in, stacks 100-1000 behind a pot of 100, and 2-3 bets/raises (2 when four sizes meet
    a stack above 400); the 256 subgames of seed 0 have 21 to 315 public nodes (median 84)."""
    rng = np.random.default_rng(10_000 + seed)
    menu = np.array([0.33, 0.5, 0.75, 1.0, 1.5, 2.0])
    out = []
    for k in range(n):
        n_sizes = int(rng.integers(1, 5))
        small = float(rng.choice(menu[:3]))  # one size below 1 pot stays distinct from all-in
        rest = rng.choice(menu[menu != small], size=n_sizes - 1, replace=False)
        sizes = tuple(sorted([small] + [float(x) for x in rest])) + (ALL_IN,)
        stack = float(rng.integers(100, 1001))
        max_raises = int(rng.integers(2, 4))
        if n_sizes == 4 and stack > 400:
            max_raises = 2
        g = river_subgame(n_hands=n_hands, seed=1000 + k, range_seed=5000 + k, pot=100.0, stack=stack,
                          bet_sizes=sizes, max_raises=max_raises)
        g.name = f"river_batch_{k}"
        out.append(g)
    return out


# ---------------------------------------------------------------- rank-based showdown strengths

def rank_strength(board, hands) -> np.ndarray:
    """Showdown strength of each two-card hand on a 5-card board, from the rules of poker:
    the category of the best five of the seven cards (high card, pair, two pair, three of a
    kind, straight, flush, full house, four of a kind, straight flush), then the ranks that
    break ties within it.  Deterministic in the cards, so a network can learn it; returned
    as dense int32 ranks (equal strength, equal rank)."""
    board = np.asarray(board, dtype=np.int64)
    hands = np.asarray(hands, dtype=np.int64)
    n = hands.shape[0]
    cards = np.concatenate([hands, np.broadcast_to(board, (n, 5))], axis=1)  # [n, 7]
    rank, suit = cards // 4, cards % 4
    cnt = np.zeros((n, 13), np.int64)
    np.add.at(cnt, (np.arange(n)[:, None], rank), 1)
    scnt = np.zeros((n, 4), np.int64)
    np.add.at(scnt, (np.arange(n)[:, None], suit), 1)

    def straight_top(present):  # present [n, 13] bool -> highest straight top rank or -1
        p = np.concatenate([present[:, 12:13], present], axis=1)  # ace plays low
        top = np.full(n, -1)
        for hi in range(4, 14):
            ok = p[:, hi - 4:hi + 1].all(axis=1)
            top = np.where(ok, hi - 1, top)
        return top

    st = straight_top(cnt > 0)
    fsuit = np.argmax(scnt, axis=1)
    flush = scnt.max(axis=1) >= 5
    fpres = np.zeros((n, 13), bool)
    for k in range(7):
        m = suit[:, k] == fsuit
        fpres[np.arange(n)[m], rank[m, k]] = True
    sft = np.where(flush, straight_top(fpres), -1)
    ranks = np.arange(13)[None, :]

    def best(mask):  # highest rank where mask holds, else -1
        return np.where(mask.any(axis=1), 12 - np.argmax(mask[:, ::-1], axis=1), -1)

    def top(mask, k):  # the k highest ranks where mask holds (-1 where fewer)
        out, m = [], mask.copy()
        for _ in range(k):
            r = best(m)
            out.append(r)
            m = m & (ranks != r[:, None])
        return out

    quad = best(cnt == 4)
    trip = best(cnt >= 3)
    pair1 = best((cnt >= 2) & (ranks != trip[:, None]))
    pair2 = best((cnt >= 2) & (ranks != pair1[:, None]) & (ranks != trip[:, None]))
    quads = quad >= 0
    full = (trip >= 0) & (pair1 >= 0)
    trips = (trip >= 0) & ~full
    twop = (trip < 0) & (pair2 >= 0)
    pair = (trip < 0) & (pair1 >= 0) & (pair2 < 0)
    cat = np.zeros(n, np.int64)
    cat = np.where(pair, 1, cat)
    cat = np.where(twop, 2, cat)
    cat = np.where(trips, 3, cat)
    cat = np.where(st >= 0, 4, cat)
    cat = np.where(flush, 5, cat)
    cat = np.where(full, 6, cat)
    cat = np.where(quads, 7, cat)
    cat = np.where(sft >= 0, 8, cat)
    # tie-break: the ranks of the five cards that play, most significant first
    seen = cnt >= 1
    sel = {0: top(cnt == 1, 5),
           1: [pair1] + top(cnt == 1, 3),
           2: [pair1, pair2, best(seen & (ranks != pair1[:, None]) & (ranks != pair2[:, None]))],
           3: [trip] + top(cnt == 1, 2),
           4: [st],
           6: [trip, pair1],
           7: [quad, best(seen & (ranks != quad[:, None]))],
           8: [sft]}
    fr = np.where(fpres, np.arange(13)[None, :], -1)
    fr = -np.sort(-fr, axis=1)[:, :5]
    sel[5] = [fr[:, k] for k in range(5)]
    tb = np.zeros(n, np.int64)
    for c, seq in sel.items():
        v = np.zeros(n, np.int64)
        for k in range(5):
            v = v * 16 + (np.maximum(seq[k], 0) if k < len(seq) else 0)
        tb = np.where(cat == c, v, tb)
    score = cat * (16 ** 5) + tb
    _, dense = np.unique(score, return_inverse=True)
    return dense.astype(np.int32)


def ranked_turn_subgame(n_hands: int | None = None, seed: int = 0, range_seed: int = 1, pot: float = 100.0,
                        stack: float = 400.0, bet_sizes=(0.5, 1.0, ALL_IN), max_raises: int = 3,
                        depth_limit: int = 0) -> GameSpec:
    """A turn subgame like turn_subgame, with showdown strengths from rank_strength on each
    completed board (rows of board cards are unused and zero)."""
    g = turn_subgame(n_hands=n_hands, seed=seed, range_seed=range_seed, pot=pot, stack=stack,
                     bet_sizes=bet_sizes, max_raises=max_raises)
    strength = np.zeros((DECK, g.n_hands), np.int32)
    for c in range(DECK):
        if c in set(int(b) for b in g.board):
            continue
        live = ~np.any(g.hands == c, axis=1)
        s = np.zeros(g.n_hands, np.int32)
        s[live] = rank_strength(np.concatenate([g.board, [c]]), g.hands[live])
        strength[c] = s
    g.strength = strength
    g.name = "turn_ranked"
    g.depth_limit = depth_limit
    return g


def ranked_flop_subgame(n_hands: int | None = None, seed: int = 0, range_seed: int = 1, pot: float = 100.0,
                        stack: float = 150.0, bet_sizes=(0.33, 0.75, 1.25, ALL_IN), max_raises: int = 4,
                        depth_limit: int = 0) -> GameSpec:
    """A flop subgame like flop_subgame, with showdown strengths from rank_strength on each
    completed board."""
    g = flop_subgame(n_hands=n_hands, seed=seed, range_seed=range_seed, pot=pot, stack=stack,
                     bet_sizes=bet_sizes, max_raises=max_raises)
    strength = np.zeros((DECK * DECK, g.n_hands), np.int32)
    live = [c for c in range(DECK) if c not in set(int(b) for b in g.board)]
    for a, b in combinations(live, 2):
        ok = ~np.any((g.hands == a) | (g.hands == b), axis=1)
        s = np.zeros(g.n_hands, np.int32)
        s[ok] = rank_strength(np.concatenate([g.board, [a, b]]), g.hands[ok])
        strength[a * DECK + b] = s
        strength[b * DECK + a] = s
    g.strength = strength
    g.name = "flop_ranked"
    g.depth_limit = depth_limit
    return g


def leaf_training_rivers(n: int, seed: int = 0, pot_range=(100.0, 900.0), behind_range=(50.0, 500.0),
                         bet_sizes=(0.5, 1.0, ALL_IN), max_raises: int = 3) -> list[GameSpec]:
    """River subgames for training the leaf network: seeded boards, rank_strength showdowns,
    pots and chips behind spanning those of turn leaves, and ranges shaped like those that
    reach a leaf after betting.  Each player's range is, with equal odds, Dirichlet(1);
    tilted towards strong or weak hands, exp(b z) with z the hand's strength percentile in
    [-1, 1] and b uniform in [-6, 6]; or polarised, exp(b |z|) with b in [0, 6] -- each
    times Dirichlet(1) noise and thinned by a random keep-probability."""
    rng = np.random.default_rng(20_000 + seed)
    out = []
    for k in range(n):
        board = np.sort(rng.choice(DECK, size=5, replace=False)).astype(np.int32)
        combos = all_combos(board)
        strength = rank_strength(board, combos)
        z = 2.0 * (np.argsort(np.argsort(strength, kind="stable"), kind="stable") / max(1, len(strength) - 1)) - 1.0
        ranges = rng.exponential(1.0, size=(2, combos.shape[0]))
        for p in range(2):
            kind = int(rng.integers(0, 3))
            if kind == 1:
                ranges[p] *= np.exp(rng.uniform(-6.0, 6.0) * z)
            elif kind == 2:
                ranges[p] *= np.exp(rng.uniform(0.0, 6.0) * np.abs(z))
        keep = rng.random((2, combos.shape[0])) < rng.uniform(0.3, 1.0, size=(2, 1))
        ranges = ranges * keep
        ranges[ranges.sum(axis=1) == 0] = 1.0
        ranges = (ranges / ranges.sum(axis=1, keepdims=True)).astype(np.float32)
        pot = float(rng.uniform(*pot_range))
        behind = float(rng.uniform(*behind_range))
        out.append(GameSpec(GAME_HOLDEM, f"leaf_river_{k}", board, combos, ranges, strength[None, :].copy(), pot,
                            behind, tuple(float(x) for x in bet_sizes), max_raises,
                            {"leaf_river": 20_000 + seed, "k": k}))
    return out


def leaf_training_turns(n: int, seed: int = 0) -> list[GameSpec]:
    """Exact turn subgames whose solutions give leaf-network examples at the river card
    (the states a depth-limited solve meets at its leaves): seeded 4-card boards with
    rank_strength showdowns on every river, Dirichlet(1) or strength-tilted ranges, pot
    100-400 with 100-600 behind, and a turn bet tree drawn from the sizes of the
    benchmark trees ({0.33, 0.5, 0.75, 1.0, 1.25} pot, 1-3 of them, plus all-in; 2-3
    bets/raises)."""
    rng = np.random.default_rng(40_000 + seed)
    menu = np.array([0.33, 0.5, 0.75, 1.0, 1.25])
    out = []
    for k in range(n):
        board = np.sort(rng.choice(DECK, size=4, replace=False)).astype(np.int32)
        combos = all_combos(board)
        strength = np.zeros((DECK, combos.shape[0]), np.int32)
        for c in range(DECK):
            if c in set(int(b) for b in board):
                continue
            live = ~np.any(combos == c, axis=1)
            strength[c, live] = rank_strength(np.concatenate([board, [c]]), combos[live])
        # tilt by the mean strength percentile over the river cards
        pct = np.zeros(combos.shape[0])
        for c in range(DECK):
            if c in set(int(b) for b in board):
                continue
            live = ~np.any(combos == c, axis=1)
            srt = np.argsort(np.argsort(strength[c, live], kind="stable"), kind="stable")
            pct[live] += srt / max(1, live.sum() - 1)
        z = 2.0 * pct / (DECK - 4) - 1.0
        ranges = rng.exponential(1.0, size=(2, combos.shape[0]))
        for p in range(2):
            if rng.random() < 0.5:
                ranges[p] *= np.exp(rng.uniform(-3.0, 3.0) * z)
        ranges = (ranges / ranges.sum(axis=1, keepdims=True)).astype(np.float32)
        n_sizes = int(rng.integers(1, 4))
        sizes = tuple(sorted(float(x) for x in rng.choice(menu, size=n_sizes, replace=False))) + (ALL_IN,)
        pot = float(rng.uniform(100.0, 400.0))
        behind = float(rng.uniform(100.0, 600.0))
        out.append(GameSpec(GAME_HOLDEM, f"leaf_turn_{k}", board, combos, ranges, strength, pot, behind, sizes,
                            int(rng.integers(2, 4)), {"leaf_turn": 40_000 + seed, "k": k}))
    return out
