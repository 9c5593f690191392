"""Depth-limited solving with the learned leaf network, judged against exact solving of the
continuation, with a per-leaf fallback to exact solving.

Section 3 (depth-limited solving): at a depth limit the tree stops and a network supplies
the counterfactual values of the rest of the game from both players' ranges and the public
state.  Those values are only as good as the network, so a served solve checks them: after
the depth-limited solve, a seeded sample of leaf rows (a leaf and one river card) is taken
at the average strategy's reach, each row's continuation -- the river subgame below that
card, with the leaf's pot, chips behind, bet tree and the two players' reach as ranges --
is solved exactly (DCFR, all sampled rows in one batched handle), and the network's values
on the same rows are compared with the exact best-response values, per unit pot as the
network is trained.  Rows are sampled per leaf, and every leaf whose reach-weighted error is
above the tolerance is solved exactly in a new handle -- its position becomes the river-card
chance node with the exact river subtrees -- while the other leaves keep the network: the
fallback is per leaf, in one handle (the whole subgame to full depth when every leaf fails).

Host orchestration only: every solve, network evaluation and exploitability pass runs in
the library's kernels through the C ABI (capi); this module builds continuation specs from
the handle's public tree and compares result rows.
"""
from __future__ import annotations

import dataclasses
import time
from dataclasses import dataclass, field

import numpy as np

from paper_2605_19928_gb300 import capi, leafnet_train, synth

SLOTS = leafnet_train.SLOTS
# Default bar on the reach-weighted leaf value error, in units of the leaf's pot.  A leaf
# value off by e x pot moves the depth-limited solution's value by at most e x pot times
# the chance of reaching the leaf; at pot 100 and a 100-chip big blind, 1e-3 keeps that
# under 1 mbb/hand.
DEFAULT_TOL = 1e-3


@dataclass
class Judgement:
    """The network against exact continuation solves on sampled leaf rows."""
    rows: int                      # leaf rows judged
    candidates: int                # leaf rows reached by both players (the sampling pool)
    mean_abs_error: float          # mean |network - exact| per unit pot over live hands
    reach_weighted_error: float    # per row: sum over players and hands of the hand's
                                   # normalised reach x |error|, halved; mean over rows
    max_row_error: float           # largest per-row reach-weighted error
    continuation_exploitability_mbb: float  # median over the exact continuation solves
    ms: float                      # wall time of the judge (continuation solves included)
    samples: list = field(default_factory=list, repr=False)  # (network row, continuation spec)
    leaf_errors: list = field(default_factory=list)  # per leaf (cfr_leaf_info order): mean
                                                     # reach-weighted error of its judged rows,
                                                     # None where none was judged


@dataclass
class Served:
    tree: object                   # the handle of the chosen form (the caller destroys it)
    form: str                      # "learned", "mixed" (some leaves exact) or "exact"
    judgement: Judgement
    ms: dict                       # wall time per phase: learned, judge, exact
    exact_leaves: tuple = ()       # leaves solved exactly (cfr_leaf_info order of the learned form)


def leaf_board(tree, node: int, spec) -> list[int]:
    """The public cards at a node: the subgame's board plus the cards chance dealt on the
    path from the root."""
    cards = [int(c) for c in spec.board]
    while node > 0:
        info = capi.cfr_node_info(tree, node)
        parent = info["parent"]
        if capi.cfr_node_info(tree, parent)["type"] == capi.CFR_NODE_CHANCE:
            cards.append(int(info["deal"]))
        node = parent
    return cards


def river_cards(board) -> list[int]:
    """The river cards of a leaf in the order of its network rows (ascending, not on the
    board)."""
    dead = set(int(c) for c in board)
    return [c for c in range(synth.DECK) if c not in dead]


def strength_row(spec, board) -> np.ndarray:
    """The showdown strengths the subgame gives on the completed 5-card board: turn
    subgames index their table by the river card, flop subgames by turn x 52 + river."""
    extra = [int(c) for c in board[len(spec.board):]]
    n_board = len(spec.board)
    if n_board == 4 and len(extra) == 1:
        return spec.strength[extra[0]]
    if n_board == 3 and len(extra) == 2:
        return spec.strength[extra[0] * synth.DECK + extra[1]]
    raise ValueError("a leaf row completes a 3- or 4-card board to 5 cards")


def continuation_spec(spec, board, river: int, reach, pot: float, behind: float, name: str = "continuation"):
    """The river subgame below one leaf row: the hands of `spec` holding no card of the
    completed board, the two players' reach at the leaf as ranges (None if a player's live
    reach is zero), the subgame's showdown strengths on that board, the leaf's pot and
    chips behind, and the subgame's bet tree."""
    full = [int(c) for c in board] + [int(river)]
    hands = np.asarray(spec.hands)
    live = ~np.isin(hands, full).any(axis=1)
    r = np.stack([np.asarray(reach[p], np.float64)[live] for p in (0, 1)])
    if (r.sum(axis=1) <= 0.0).any():
        return None
    r = r / r.sum(axis=1, keepdims=True)
    strength = np.asarray(strength_row(spec, full))[live]
    return synth.GameSpec(synth.GAME_HOLDEM, name, np.array(sorted(full), np.int32),
                          np.ascontiguousarray(hands[live]), r.astype(np.float32),
                          strength[None, :].astype(np.int32), float(pot), float(behind),
                          tuple(spec.bet_sizes), int(spec.max_raises), dict(spec.seeds), 0)


def row_errors(y_net, y_exact, mask, ranges, hands) -> tuple[float, float, int]:
    """(sum |error|, reach-weighted error, live entries) of one leaf row: network and exact
    rows in the slot layout (player i's values at i x 1326 + slot), mask 1 where the exact
    value exists, ranges [2][n] the continuation's normalised ranges over `hands`."""
    sl = leafnet_train.slot_of(np.asarray(hands))
    tot, weighted, cnt = 0.0, 0.0, 0
    for i in (0, 1):
        idx = i * SLOTS + sl
        m = np.asarray(mask)[idx] > 0
        d = np.abs(np.asarray(y_net, np.float64)[idx] - np.asarray(y_exact, np.float64)[idx])
        tot += float(d[m].sum())
        cnt += int(m.sum())
        weighted += 0.5 * float((np.asarray(ranges[i], np.float64) * d * m).sum())
    return tot, weighted, cnt


def fallback_leaves(leaf_errors, tol: float) -> list[int]:
    """The leaves to solve exactly: those whose judged error is above `tol` (a leaf none of
    whose rows was reached by both players keeps the network)."""
    return [k for k, e in enumerate(leaf_errors) if e is not None and e > tol]


def judge_leaves(tree, spec, n_rows: int = 64, iters: int = 300, seed: int = 0, stream=None,
                 evaluated: bool = False, per_leaf: int = 0) -> Judgement:
    """Judge the network of a depth-limited handle at its average strategy: sample up to
    n_rows leaf rows reached by both players (per_leaf > 0: up to per_leaf rows of every
    leaf instead), solve their continuations exactly in one batched handle (`iters` DCFR
    iterations, FP32 values) and compare the network's values on the same rows.  The leaf
    reach comes from an exploitability pass, run here unless `evaluated` says that
    cfr_exploitability was the handle's last pass."""
    t0 = time.perf_counter()
    if not evaluated:
        capi.cfr_exploitability(tree)
    cap = spec.pot / 2.0 + spec.stack
    hands = np.asarray(spec.hands, np.int64)
    leaves, pool = [], []
    for _, node, row0 in capi.cfr_leaf_info(tree):
        info = capi.cfr_node_info(tree, node)
        board = leaf_board(tree, node, spec)
        reach = [capi.cfr_read_values(tree, capi.CFR_READ_AVG_REACH, node, player=p) for p in (0, 1)]
        leaves.append((board, reach, info["contrib"][0] + info["contrib"][1], cap - info["contrib"][0]))
        # a player's reach on the hands holding neither the board nor river card r:
        # total - (reach of hands holding r); the board's hands already have none
        live = []
        for p in (0, 1):
            by_card = np.zeros(synth.DECK)
            np.add.at(by_card, hands[:, 0], reach[p])
            np.add.at(by_card, hands[:, 1], reach[p])
            live.append(reach[p].sum() - by_card)
        for j, r in enumerate(river_cards(board)):
            if live[0][r] > 0.0 and live[1][r] > 0.0:
                pool.append((row0 + j, len(leaves) - 1, r))
    rng = np.random.default_rng(seed)
    if per_leaf > 0:  # up to per_leaf rows of each leaf
        pick = []
        for leaf in range(len(leaves)):
            mine = [k for k, e in enumerate(pool) if e[1] == leaf]
            pick += rng.choice(mine, size=min(per_leaf, len(mine)), replace=False).tolist() if mine else []
        pick.sort()
    else:
        pick = sorted(rng.choice(len(pool), size=min(n_rows, len(pool)), replace=False).tolist()) if pool else []
    chosen, leaf_of = [], []
    for k in pick:
        row, leaf, r = pool[k]
        board, reach, pot, behind = leaves[leaf]
        cont = continuation_spec(spec, board, r, reach, pot, behind, name=f"leaf_row{row}")
        if cont is not None:
            chosen.append((row, cont))
            leaf_of.append(leaf)
    if not chosen:
        return Judgement(0, len(pool), 0.0, 0.0, 0.0, 0.0, 1000.0 * (time.perf_counter() - t0),
                         leaf_errors=[None] * len(leaves))
    capi.cfr_eval_leaves(tree, average=True)
    y_net = [capi.cfr_read_leaf_rows(tree, 1, row, 1)[0] for row, _ in chosen]
    specs = [c for _, c in chosen]
    opts = capi.make_opts("dcfr", precision="single")
    ex = capi.cfr_batch_create(specs, opts, stream=stream)
    try:
        capi.cfr_iterate(ex, iters)
        expl, _ = capi.cfr_exploitability(ex, len(specs))
        v = [[capi.cfr_read_values(ex, capi.CFR_READ_BR_CFV, 0, player=i, game=g) for i in (0, 1)]
             for g in range(len(specs))]
    finally:
        capi.cfr_tree_destroy(ex)
    tot, cnt, per_row = 0.0, 0, []
    for g, cont in enumerate(specs):
        _, y, m = leafnet_train.example(cont, v[g])
        t, w, c = row_errors(y_net[g], y, m, cont.ranges, cont.hands)
        tot += t
        cnt += c
        per_row.append(w)
    leaf_errors = [None] * len(leaves)
    for leaf in range(len(leaves)):
        mine = [w for w, l in zip(per_row, leaf_of) if l == leaf]
        if mine:
            leaf_errors[leaf] = float(np.mean(mine))
    return Judgement(len(specs), len(pool), tot / max(cnt, 1), float(np.mean(per_row)), float(np.max(per_row)),
                     float(np.median(1000.0 * expl / 100.0)), 1000.0 * (time.perf_counter() - t0), chosen,
                     leaf_errors)


def solve_depth_limited(spec, weights, biases, iters: int, opts=None, tol: float = DEFAULT_TOL,
                        judge_rows: int = 64, judge_iters: int = 300, seed: int = 0, stream=None,
                        per_leaf: int = 4) -> Served:
    """Solve `spec` (depth_limit 1) with network leaves for `iters` iterations and judge the
    network on its own leaf rows.  per_leaf > 0: up to per_leaf rows of every leaf are
    judged, the leaves whose error is above `tol` (pot units) are solved exactly in a new
    handle beside the network leaves of the rest ("mixed"; the full-depth subgame when every
    leaf fails, "exact"), and the learned result is kept when none fails.  per_leaf = 0:
    judge_rows rows of all leaves together, and the full-depth subgame when their mean error
    is above `tol` or no row could be judged."""
    if spec.depth_limit != 1:
        raise ValueError("solve_depth_limited takes a depth-limited subgame (depth_limit 1)")
    opts = opts if opts is not None else capi.make_opts("dcfr")
    ms = {"learned": 0.0, "judge": 0.0, "exact": 0.0}
    t0 = time.perf_counter()
    tree = capi.cfr_tree_create(spec, opts, stream=stream)
    try:
        capi.cfr_set_leaf_net(tree, weights, biases)
        capi.cfr_iterate(tree, iters)
        capi.cfr_exploitability(tree)
        ms["learned"] = 1000.0 * (time.perf_counter() - t0)
        j = judge_leaves(tree, spec, judge_rows, judge_iters, seed, stream, evaluated=True, per_leaf=per_leaf)
        n_leaves = len(capi.cfr_leaf_info(tree))
    except BaseException:
        capi.cfr_tree_destroy(tree)
        raise
    ms["judge"] = j.ms
    if per_leaf > 0:
        exact = fallback_leaves(j.leaf_errors, tol)
        if not exact:
            return Served(tree, "learned", j, ms)
    elif j.rows > 0 and j.reach_weighted_error <= tol:
        return Served(tree, "learned", j, ms)
    else:
        exact = list(range(n_leaves))
    capi.cfr_tree_destroy(tree)
    t1 = time.perf_counter()
    whole = len(exact) == n_leaves
    sub = dataclasses.replace(spec, depth_limit=0) if whole else dataclasses.replace(spec, exact_leaves=tuple(exact))
    fallback = capi.cfr_tree_create(sub, opts, stream=stream)
    try:
        if not whole:
            capi.cfr_set_leaf_net(fallback, weights, biases)
        capi.cfr_iterate(fallback, iters)
        capi.cfr_sync(fallback)
    except BaseException:
        capi.cfr_tree_destroy(fallback)
        raise
    ms["exact"] = 1000.0 * (time.perf_counter() - t1)
    return Served(fallback, "exact" if whole else "mixed", j, ms, tuple(exact))
