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
    strength: np.ndarray | None = None    # int32 [rows, n_hands]; 1 row (river) or 52 (turn, by river card)
    pot: float = 0.0                      # chips in the pot; each player has put in pot / 2
    stack: float = 0.0                    # chips behind for each player
    bet_sizes: tuple = ()                 # pot fractions, ALL_IN for the all-in bet
    max_raises: int = 0                   # bets + raises allowed per street
    seeds: dict = field(default_factory=dict)
    depth_limit: int = 0                  # 1: the turn tree stops at the river card (leaf network)

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
    a stack above 400), which gives 27 to 357 public nodes per tree."""
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
