"""The CUDA path's host-side construction (csrc/tree.cpp), on the CPU.

tree.cpp builds what the kernels are given: the public tree in level order, the depth-first
program and load tables of the stream schedule, the run-out reach sources, and the
showdown tables of the O(n) terminal evaluation (Section 4.3: strength-sorted order, tie
groups, per-card hand lists).  Here it is compiled with g++ beside a copying shim
(tests/host_probe.cpp) and checked against the oracle's independently built trees (node
by node, by action path) and against the definitions of the program, the loads, the
chunking and the tables, re-derived in Python."""
from __future__ import annotations

import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2605_19928_gb300 import capi, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2605_19928_gb300", "csrc")
DECISION, FOLD, SHOWDOWN, CHANCE, LEAF = 0, 1, 2, 3, 4
NO_CARD = 255
# load descriptors: array << 29 | element offset (R, S, reach, values, prediction M)
SHIFT, ARR_R, ARR_S, ARR_REACH, ARR_CFV, ARR_M = 29, 0, 1, 2, 3, 4


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    out = str(tmp_path_factory.mktemp("host_probe") / "libhostprobe.so")
    subprocess.run([gxx, "-O1", "-std=c++17", "-fPIC", "-shared", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                    os.path.join(ROOT, "tests", "host_probe.cpp"), os.path.join(CSRC, "tree.cpp"), "-o", out],
                   check=True, capture_output=True)
    lib = C.CDLL(out)
    lib.probe_create.restype = C.c_void_p
    lib.probe_create.argtypes = [C.c_void_p]
    lib.probe_destroy.argtypes = [C.c_void_p]
    lib.probe_error.restype = C.c_char_p
    for f in ("probe_sizes", "probe_nodes", "probe_program", "probe_tables"):
        getattr(lib, f).argtypes = None
    return lib


class Built:
    def __init__(self, lib, spec):
        self.lib = lib
        s, self._keep = capi.make_spec(spec)
        self.h = lib.probe_create(C.byref(s))
        assert self.h, lib.probe_error()
        sz = np.zeros(8, np.int32)
        lib.probe_sizes(C.c_void_p(self.h), sz.ctypes.data_as(C.c_void_p))
        (self.n_nodes, self.n_hands, self.hstride, self.n_rows, n_prog, self.depth, self.max_actions,
         self.ok) = (int(x) for x in sz)
        self.nodes = np.zeros((self.n_nodes, 8), np.int32)
        self.contrib = np.zeros((self.n_nodes, 2), np.float64)
        lib.probe_nodes(C.c_void_p(self.h), self.nodes.ctypes.data_as(C.c_void_p),
                        self.contrib.ctypes.data_as(C.c_void_p))
        self.prog = np.zeros(n_prog, np.int32)
        lib.probe_program(C.c_void_p(self.h), self.prog.ctypes.data_as(C.c_void_p))
        (self.parent, self.first, self.n_kids, self.type, self.player, self.deal, self.row,
         self.reach_src) = (self.nodes[:, k] for k in range(8))

    def kids(self, n):
        return list(range(self.first[n], self.first[n] + self.n_kids[n]))

    def tables(self, half, pred):
        cap = 1 << 20
        units = np.zeros(cap, np.uint32)
        meta = np.zeros(16, np.int32)
        chunks = np.zeros(cap, np.int32)
        n_ch = C.c_int32()
        n = self.lib.probe_tables(C.c_void_p(self.h), C.c_int(half), C.c_int(int(pred)),
                                  units.ctypes.data_as(C.c_void_p), C.c_int(cap), meta.ctypes.data_as(C.c_void_p),
                                  chunks.ctypes.data_as(C.c_void_p), C.c_int(cap), C.byref(n_ch))
        assert n <= cap and n_ch.value <= cap
        return units[:n], meta, chunks[:n_ch.value]

    def close(self):
        self.lib.probe_destroy(C.c_void_p(self.h))


def is_end(t):
    return t in (FOLD, SHOWDOWN, LEAF)


SPECS = {
    "kuhn": synth.kuhn,
    "leduc": synth.leduc,
    "river": lambda: synth.river_subgame(n_hands=12, seed=3, range_seed=4, bet_sizes=(0.33, 0.75, 1.25, synth.ALL_IN),
                                         max_raises=4),
    "turn": lambda: synth.turn_subgame(n_hands=10, seed=5, range_seed=6, bet_sizes=(1.0, synth.ALL_IN),
                                       max_raises=2),
    "turn_limited": lambda: _limited(synth.turn_subgame(n_hands=10, seed=5, range_seed=6,
                                                        bet_sizes=(0.5, synth.ALL_IN), max_raises=2)),
    "flop": lambda: synth.flop_subgame(n_hands=4, seed=3, range_seed=4, bet_sizes=(synth.ALL_IN,), max_raises=1),
    "flop_limited": lambda: _limited(synth.flop_subgame(n_hands=6, seed=7, range_seed=8, bet_sizes=(1.0, synth.ALL_IN),
                                                        max_raises=1)),
    # depth-limited with some leaves solved exactly (mixed network leaves and river subtrees)
    "turn_mixed": lambda: _limited(synth.turn_subgame(n_hands=10, seed=5, range_seed=6,
                                                      bet_sizes=(0.5, synth.ALL_IN), max_raises=2), exact=(1, 3)),
    "flop_mixed": lambda: _limited(synth.flop_subgame(n_hands=6, seed=7, range_seed=8, bet_sizes=(1.0, synth.ALL_IN),
                                                      max_raises=1), exact=(0, 17, 60)),
}


def _limited(spec, exact=()):
    spec.depth_limit = 1
    spec.exact_leaves = tuple(exact)
    return spec


@pytest.mark.parametrize("case", list(SPECS))
def test_public_tree_matches_the_oracle(probe, oracle_mod, case):
    spec = SPECS[case]()
    t = Built(probe, spec)
    o = oracle_mod.Oracle(spec, variant="dcfr", threads=1)
    try:
        assert t.n_nodes == o.n_nodes
        info = o.nodes()
        # walk both trees by action path
        todo = [(0, 0)]
        seen = 0
        while todo:
            g, n = todo.pop()
            seen += 1
            oi = info[n]
            assert t.type[g] == oi["type"], (case, g)
            assert t.n_kids[g] == oi["n_actions"], (case, g)
            if t.type[g] in (DECISION, FOLD):
                assert t.player[g] == oi["player"], (case, g)
            assert tuple(t.contrib[g]) == pytest.approx(oi["contrib"], abs=1e-9), (case, g)
            deal = -1 if t.deal[g] == NO_CARD else int(t.deal[g])
            assert deal == oi["deal"], (case, g)
            kids = t.kids(g)
            assert all(t.parent[k] == g for k in kids)
            todo.extend(zip(kids, oi["kids"]))
        assert seen == t.n_nodes
        # level order: parents come before children, children consecutive
        assert t.parent[0] == -1 and np.all(t.parent[1:] < np.arange(1, t.n_nodes))
        # regret rows: each decision node's actions, player 0's rows first
        dec = np.flatnonzero(t.type == DECISION)
        rows = sorted((int(t.row[n]), int(t.n_kids[n]), int(t.player[n])) for n in dec)
        assert sum(r[1] for r in rows) == t.n_rows
        start = 0
        for r, a, _ in rows:
            assert r == start
            start += a
        players = [p for _, _, p in rows]
        assert players == sorted(players)
        if case.endswith("limited"):
            assert (t.type == LEAF).any()
    finally:
        t.close()


@pytest.mark.parametrize("case", ["leduc", "river", "turn", "flop", "flop_limited"])
def test_program_is_the_inner_nodes_in_preorder(probe, case):
    t = Built(probe, SPECS[case]())
    try:
        pre, todo = [], [0]
        while todo:
            n = todo.pop()
            if is_end(t.type[n]):
                continue
            pre.append(n)
            todo.extend(reversed(t.kids(n)))
        assert t.prog.tolist() == pre
        # the stacks the kernel keeps: top-down pops a node's reach and pushes its inner
        # children's; bottom-up pushes a node's value and pops its inner children's
        inner = [sum(not is_end(t.type[k]) for k in t.kids(n)) for n in pre]
        sp, most = 1, 1
        for c in inner:
            sp += c - 1
            most = max(most, sp)
        assert sp == 0
        sp = 0
        for c in reversed(inner):
            sp += 1 - c
            most = max(most, sp)
        assert sp == 1
        assert t.depth == most
        assert t.max_actions == max(int(t.n_kids[n]) for n in pre if t.type[n] == DECISION)
        # a chance node's children are all inner or all terminal
        for n in pre:
            if t.type[n] == CHANCE:
                assert len({is_end(t.type[k]) for k in t.kids(n)}) == 1
        assert t.ok == 1
    finally:
        t.close()


def expected_loads(t, n, p, backward, pred):
    """The loads of node n in one pass: bottom-up, the values of its terminal children in
    child order, then at p's decision nodes R (and M) and S of each action and p's reach;
    top-down, R (and M) of each action at p's decision nodes."""
    S = t.hstride
    out = []
    if backward:
        out += [ARR_CFV << SHIFT | k * S for k in t.kids(n) if is_end(t.type[k])]
    if t.type[n] == DECISION and t.player[n] == p:
        rows = range(t.row[n], t.row[n] + t.n_kids[n])
        out += [ARR_R << SHIFT | r * S for r in rows]
        if pred:
            out += [ARR_M << SHIFT | r * S for r in rows]
        if backward:
            out += [ARR_S << SHIFT | r * S for r in rows]
            out.append(ARR_REACH << SHIFT | n * S)
    return out


@pytest.mark.parametrize("case,pred", [("river", False), ("river", True), ("turn", False), ("flop", False),
                                       ("turn_limited", True)])
def test_load_tables_and_chunks_follow_the_definitions(probe, case, pred):
    t = Built(probe, SPECS[case]())
    try:
        N = len(t.prog)
        most = max(len(expected_loads(t, n, p, True, pred)) for n in t.prog for p in (0, 1))
        for half in (most, most + 5):
            units, meta, chunks = t.tables(half, pred)
            unit_off, unit_count, chunk_off, chunk_count = meta[0:4], meta[4:8], meta[8:12], meta[12:16]
            for q in range(4):
                p, backward = q & 1, q < 2
                order = list(reversed(t.prog)) if backward else list(t.prog)
                per_node = [expected_loads(t, n, p, backward, pred) for n in order]
                want = [u for loads in per_node for u in loads]
                got = units[unit_off[q]:unit_off[q] + unit_count[q]].tolist()
                assert got == want, (case, q)
                # chunks: (first node position, first unit) pairs, then (N, unit count)
                pairs = chunks[2 * chunk_off[q]:2 * (chunk_off[q] + chunk_count[q] + 1)].reshape(-1, 2)
                assert pairs[0].tolist() == [0, 0] and pairs[-1].tolist() == [N, unit_count[q]]
                starts = np.concatenate([[0], np.cumsum([len(x) for x in per_node])])
                for c in range(len(pairs) - 1):
                    k0, k1 = pairs[c, 0], pairs[c + 1, 0]
                    assert k0 < k1 and pairs[c, 1] == starts[k0]
                    assert starts[k1] - starts[k0] <= half  # one ring half holds the chunk
                    if c + 1 < len(pairs) - 1:  # greedy: the next node did not fit
                        assert starts[k1] - starts[k0] + len(per_node[k1]) > half
    finally:
        t.close()


@pytest.mark.parametrize("case", ["turn", "flop", "flop_limited"])
def test_run_out_reach_sources(probe, case):
    """A node's reach source is the top chance node of the all-in run-out it lies in (its
    reach up to zeroing the hands that hold a dealt card), the node itself elsewhere."""
    t = Built(probe, SPECS[case]())
    try:
        sub_has_action = np.zeros(t.n_nodes, bool)
        for n in range(t.n_nodes - 1, -1, -1):  # children come after their parent
            sub_has_action[n] = t.type[n] in (DECISION, LEAF) or any(sub_has_action[k] for k in t.kids(n))
        redirected = 0
        for n in range(t.n_nodes):
            s = t.reach_src[n]
            if s == n:
                continue
            redirected += 1
            assert t.type[n] in (CHANCE, SHOWDOWN, FOLD)
            assert t.type[s] == CHANCE and t.reach_src[s] == s
            assert not sub_has_action[s]  # nobody acts below the run-out's top
            assert t.parent[s] < 0 or t.type[t.parent[s]] != CHANCE
            a = t.parent[n]
            while a != s:  # only chance nodes between them
                assert t.type[a] == CHANCE
                a = t.parent[a]
        # every chance or showdown node below a chance node is redirected
        for n in range(1, t.n_nodes):
            if t.type[t.parent[n]] == CHANCE and t.type[n] in (CHANCE, SHOWDOWN):
                assert t.reach_src[n] != n
        if case != "turn":
            assert redirected > 0
    finally:
        t.close()


TABLE_SPECS = {
    "river": SPECS["river"],
    "river_ranked": lambda: _ranked_river(),
    "turn": SPECS["turn"],
    "turn_ranked": lambda: synth.ranked_turn_subgame(n_hands=40, seed=2, range_seed=3, bet_sizes=(1.0, synth.ALL_IN),
                                                     max_raises=1),
    "flop": SPECS["flop"],
}


def _ranked_river():
    g = synth.river_subgame(n_hands=60, seed=9, range_seed=10, bet_sizes=(synth.ALL_IN,), max_raises=1)
    g.strength = synth.rank_strength(g.board, g.hands)[None, :].astype(np.int32)  # many ties
    return g


@pytest.mark.parametrize("case", list(TABLE_SPECS))
def test_showdown_tables_follow_their_definitions(probe, case):
    """Per showdown board: perm sorts the hands by strength, [gs, ge) is each hand's tie
    group, clh / cloff list the hands holding each card in sorted order, and lo / hi give,
    per (hand, card), the first list entry at or after the tie group's start / end."""
    spec = TABLE_SPECS[case]()
    t = Built(probe, spec)
    try:
        meta = np.zeros(4, np.int32)
        probe.probe_game(C.c_void_p(t.h), meta.ctypes.data_as(C.c_void_p))
        _, deck, k, n_boards = (int(x) for x in meta)
        tt = np.zeros(10, np.int32)
        n = probe.probe_term_tables(C.c_void_p(t.h), tt.ctypes.data_as(C.c_void_p), None, C.c_int(0))
        tab = np.zeros(n, np.uint16)
        probe.probe_term_tables(C.c_void_p(t.h), tt.ctypes.data_as(C.c_void_p), tab.ctypes.data_as(C.c_void_p),
                                C.c_int(n))
        clh, cards, cloff, _, perm, gs, ge, lo, hi, L = (int(x) for x in tt)
        assert n == n_boards * L and L % 8 == 0
        boards = np.zeros(t.n_nodes, np.uint64)
        probe.probe_boards(C.c_void_p(t.h), boards.ctypes.data_as(C.c_void_p))
        H = spec.n_hands
        hands = spec.hands.astype(np.int64)
        base = set(int(c) for c in spec.board)
        checked = set()
        for nd in np.flatnonzero(t.type == SHOWDOWN):
            b = int(t.row[nd])
            if b in checked:
                continue
            checked.add(b)
            dealt = sorted(c for c in range(52) if (int(boards[nd]) >> c) & 1 and c not in base)
            if len(base) == 5:
                srow = spec.strength[0]
            elif len(base) == 4:
                srow = spec.strength[dealt[0]]
            else:
                srow = spec.strength[dealt[0] * 52 + dealt[1]]
            blk = tab[b * L:(b + 1) * L].astype(np.int64)
            P = blk[perm:perm + H]
            assert sorted(P.tolist()) == list(range(H))
            s_sorted = srow[P]
            assert np.all(np.diff(s_sorted) >= 0) or np.all(np.diff(s_sorted) <= 0)
            pos = np.empty(H, np.int64)
            pos[P] = np.arange(H)
            for h in range(H):
                group = np.flatnonzero(s_sorted == srow[h])
                assert (blk[gs + h], blk[ge + h]) == (group[0], group[-1] + 1), (case, b, h)
            for c in range(deck):
                lst = blk[clh + blk[cloff + c]:clh + blk[cloff + c + 1]]
                holders = [h for h in range(H) if c in hands[h]]
                assert sorted(lst.tolist()) == sorted(holders)
                assert np.all(np.diff(pos[lst]) > 0)  # rank-sorted order
            for h in range(H):
                for s in range(k):
                    c = int(hands[h, s])
                    lst_pos = pos[blk[clh + blk[cloff + c]:clh + blk[cloff + c + 1]]]
                    first_lo = blk[cloff + c] + int(np.searchsorted(lst_pos, blk[gs + h], side="left"))
                    first_hi = blk[cloff + c] + int(np.searchsorted(lst_pos, blk[ge + h], side="left"))
                    assert blk[lo + 2 * h + s] == first_lo and blk[hi + 2 * h + s] == first_hi, (case, b, h, s)
                c1 = int(blk[cards + h]) & 0xFF
                c2 = int(blk[cards + h]) >> 8
                assert (c1, c2) == (int(hands[h, 0]), int(hands[h, 1]))
            _check_sorted_prefix_sums(blk, clh, cloff, perm, gs, ge, lo, hi, H, hands, srow,
                                      np.sign(s_sorted[-1] - s_sorted[0]))
            if b == 0:
                _check_fold_inclusion_exclusion(blk, clh, cloff, H, hands, deck)
        assert len(checked) == n_boards or case.startswith("river")
    finally:
        t.close()


def _check_sorted_prefix_sums(blk, clh, cloff, perm, gs, ge, lo, hi, H, hands, srow, order):
    """Section 4.3, Stage 4 on these tables: with q the opponent reach, W(h) (mass of the
    opponent hands weaker than h sharing no card with it) is the prefix of q before h's tie
    group minus, for each of h's cards, the prefix of that card's list up to lo; L(h)
    (stronger) is the suffix after the group minus the card lists' suffixes from hi.
    Compared with a direct sum over the opponent hands."""
    rng = np.random.default_rng(H)
    q = rng.random(H) * (rng.random(H) < 0.8)
    P = np.concatenate([[0.0], np.cumsum(q[blk[perm:perm + H]])])
    T = P[-1]
    weaker_first = order >= 0  # sorted by increasing strength
    for h in range(H):
        pre, post = P[blk[gs + h]], T - P[blk[ge + h]]
        for s_ in range(2):
            c = int(hands[h, s_])
            lst = blk[clh + blk[cloff + c]:clh + blk[cloff + c + 1]]
            cp = np.concatenate([[0.0], np.cumsum(q[lst])])
            pre -= cp[blk[lo + 2 * h + s_] - blk[cloff + c]]
            post -= cp[-1] - cp[blk[hi + 2 * h + s_] - blk[cloff + c]]
        W, L = (pre, post) if weaker_first else (post, pre)
        disjoint = ~np.isin(hands, hands[h]).any(axis=1)
        W_ref = q[disjoint & (srow < srow[h])].sum()
        L_ref = q[disjoint & (srow > srow[h])].sum()
        assert W == pytest.approx(W_ref, abs=1e-12) and L == pytest.approx(L_ref, abs=1e-12), h


def _check_fold_inclusion_exclusion(blk, clh, cloff, H, hands, deck):
    """Section 4.3, Stages 2-3 on the card lists the fold nodes read: the opponent mass
    sharing no card with h is T - C(c1) - C(c2) + q(h), C(c) the mass of card c's list."""
    rng = np.random.default_rng(H + 1)
    q = rng.random(H)
    C_ = np.array([q[blk[clh + blk[cloff + c]:clh + blk[cloff + c + 1]]].sum() for c in range(deck)])
    for h in range(H):
        M = q.sum() - C_[hands[h, 0]] - C_[hands[h, 1]] + q[h]
        disjoint = ~np.isin(hands, hands[h]).any(axis=1)
        assert M == pytest.approx(q[disjoint].sum(), abs=1e-12), h


@pytest.mark.parametrize("case", list(SPECS) + ["river_full"])
def test_deal_normaliser_matches_the_oracle(probe, oracle_mod, case):
    """Z, the probability mass of the private deals (pairs of hands sharing no card), which
    scales every terminal value: the library's O(H) inclusion-exclusion against the
    oracle's sum over every pair."""
    spec = synth.river_subgame() if case == "river_full" else SPECS[case]()
    t = Built(probe, spec)
    try:
        probe.probe_Z.restype = C.c_double
        z = probe.probe_Z(C.c_void_p(t.h))
        o = oracle_mod.Oracle(spec, variant="dcfr", threads=1)
        assert z == pytest.approx(o.Z, rel=1e-13)
        if spec.game == synth.GAME_HOLDEM:  # and against a direct sum here
            r = spec.ranges.astype(np.float64)
            r = r / r.sum(axis=1, keepdims=True)
            h = spec.hands.astype(np.int64)
            clash = (h[:, None, :, None] == h[None, :, None, :]).any(axis=(2, 3))
            assert z == pytest.approx(float(r[0] @ (~clash * 1.0) @ r[1]), rel=1e-13)
    finally:
        t.close()


@pytest.mark.parametrize("case", ["leduc", "river", "turn", "flop", "flop_limited"])
def test_program_ops_encode_the_tree(probe, case):
    """The 16-byte program entries the stream kernel decodes: node and row offsets in
    elements (x hstride), and a code of type (2 bits), player (1), child count (6), dealt
    card (8) and the terminal-children mask (bit a: child a is a fold, showdown or leaf;
    chance nodes: bit 0 when all children are)."""
    t = Built(probe, SPECS[case]())
    try:
        ops = np.zeros((len(t.prog), 4), np.int32)
        probe.probe_program_ops(C.c_void_p(t.h), ops.ctypes.data_as(C.c_void_p))
        for (node_off, row_off, code, first_kid), n in zip(ops.tolist(), t.prog.tolist()):
            code &= 0xFFFFFFFF
            assert node_off == n * t.hstride and first_kid == t.first[n]
            assert code & 3 == t.type[n]
            assert (code >> 3) & 63 == t.n_kids[n]
            assert (code >> 9) & 0xFF == t.deal[n]
            ends = [is_end(t.type[k]) for k in t.kids(n)]
            if t.type[n] == DECISION:
                assert row_off == t.row[n] * t.hstride and (code >> 2) & 1 == t.player[n]
                assert code >> 17 == sum(1 << a for a, e in enumerate(ends) if e)
            else:
                assert row_off == 0 and code >> 17 == (1 if all(ends) else 0)
    finally:
        t.close()


@pytest.mark.parametrize("case", list(SPECS))
def test_terminal_payoffs_and_chance_weights(probe, case):
    """The per-node factor of the terminal values: a fold costs the folder its whole
    contribution, a showdown moves the loser's contribution (both equal there), a
    depth-limit leaf carries the pot times the chance of each river card; each is times
    the chance of the cards dealt on the way, 1 / (cards left given the board and both
    private hands) per chance node: 1/44 per river card below a turn, 1/45 per turn card
    below a flop, 1/4 per public card in Leduc."""
    spec = SPECS[case]()
    t = Built(probe, spec)
    try:
        pay = np.zeros(t.n_nodes)
        probe.probe_payoff(C.c_void_p(t.h), pay.ctypes.data_as(C.c_void_p))
        boards = np.zeros(t.n_nodes, np.uint64)
        probe.probe_boards(C.c_void_p(t.h), boards.ctypes.data_as(C.c_void_p))
        meta = np.zeros(4, np.int32)
        probe.probe_game(C.c_void_p(t.h), meta.ctypes.data_as(C.c_void_p))
        deck, k = int(meta[1]), int(meta[2])

        def left(n):  # cards chance can deal at node n, given its board and both hands
            return deck - bin(int(boards[n])).count("1") - 2 * k

        chance = np.ones(t.n_nodes)
        for n in range(1, t.n_nodes):
            par = t.parent[n]
            chance[n] = chance[par] / left(par) if t.type[par] == CHANCE else chance[par]
        for n in range(t.n_nodes):
            c0, c1 = t.contrib[n]
            if t.type[n] == FOLD:
                want = (c0, c1)[t.player[n]] * chance[n]
            elif t.type[n] == SHOWDOWN:
                assert c0 == c1
                want = c0 * chance[n]
            elif t.type[n] == LEAF:
                assert left(n) == 44
                want = (c0 + c1) * chance[n] / 44.0
            else:
                continue
            assert pay[n] == pytest.approx(want, rel=1e-15), (case, n)
        if case == "leduc":
            assert {left(n) for n in range(t.n_nodes) if t.type[n] == CHANCE} == {4}
        if case.startswith("flop"):
            assert {left(n) for n in range(t.n_nodes) if t.type[n] == CHANCE} >= {45}
    finally:
        t.close()


def _rejected(lib, spec):
    s, keep = capi.make_spec(spec)
    h = lib.probe_create(C.byref(s))
    if h:
        lib.probe_destroy(C.c_void_p(h))
        return None
    return lib.probe_error().decode()


def test_invalid_subgames_are_rejected(probe):
    """build_game's checks (what cfr_tree_create reports as CFR_EINVAL), on the CPU."""
    import copy

    def river(**kw):
        return synth.river_subgame(n_hands=12, seed=3, range_seed=4, **kw)

    assert _rejected(probe, river()) is None
    bad = river()
    bad.hands = bad.hands.copy()
    bad.hands[1] = bad.hands[0]
    assert "duplicate" in _rejected(probe, bad)
    bad = river()
    bad.hands = bad.hands.copy()
    bad.hands[0, 0] = bad.board[0]
    assert "board" in _rejected(probe, bad)
    bad = river()
    bad.ranges = bad.ranges.copy()
    bad.ranges[0, 3] = -1.0
    assert "non-negative" in _rejected(probe, bad)
    bad = river()
    bad.ranges = np.zeros_like(bad.ranges)
    assert "sums to zero" in _rejected(probe, bad)
    bad = river()
    bad.depth_limit = 1  # a river has no card to come
    assert "depth_limit" in _rejected(probe, bad)
    bad = synth.turn_subgame(n_hands=10, seed=5, range_seed=6)
    bad.strength = bad.strength[:1].copy()  # a turn needs one row per river card
    assert "strength" in _rejected(probe, bad)
    bad = copy.deepcopy(river())
    bad.pot = 0.0
    assert "pot" in _rejected(probe, bad)
    # every hand of player 0 blocks every hand of player 1: no deal is possible
    bad = river()
    keep = np.flatnonzero((bad.hands == bad.hands[0, 0]).any(axis=1))
    bad.hands = bad.hands[keep].copy()
    bad.strength = bad.strength[:, keep].copy()
    bad.ranges = np.ones((2, len(keep)), np.float32)
    assert "no pair of hands" in _rejected(probe, bad)


def test_exact_leaves_are_checked(probe):
    """exact_leaves: depth-limited subgames only, distinct indices naming leaves."""
    def turn(**kw):
        spec = synth.turn_subgame(n_hands=10, seed=5, range_seed=6, bet_sizes=(0.5, synth.ALL_IN), max_raises=2)
        for k, v in kw.items():
            setattr(spec, k, v)
        return spec

    assert _rejected(probe, turn(depth_limit=1, exact_leaves=(0, 4))) is None  # five leaf positions
    assert "exact_leaves" in _rejected(probe, turn(depth_limit=1, exact_leaves=(5,)))
    assert "exact_leaves" in _rejected(probe, turn(depth_limit=1, exact_leaves=(2, 2)))
    assert "exact_leaves" in _rejected(probe, turn(depth_limit=1, exact_leaves=(-1,)))
    assert "exact_leaves" in _rejected(probe, turn(depth_limit=0, exact_leaves=(0,)))


@pytest.mark.parametrize("case", ["turn", "flop", "turn_limited", "river", "leduc"])
def test_runout_plan_follows_its_definition(probe, case):
    """The all-in run-outs the tables evaluate (`runout_tables`): the tops are the chance
    nodes below a decision with only chance and showdown nodes beneath, every node below a
    top is inside, a top's table lists the boards (cards, board table) of its showdowns and
    tops that show down on the same boards share one, u is the showdowns' common payoff over
    Z rounded to FP32, tables of more than 127 boards hold 16-bit entries, and the pool holds
    each table's n_hands x hstride entries at 256-byte offsets."""
    spec = SPECS[case]()
    t = Built(probe, spec)
    try:
        N = t.n_nodes
        sizes, pool = np.zeros(4, np.int32), C.c_int64()
        probe.probe_runouts(C.c_void_p(t.h), sizes.ctypes.data_as(C.c_void_p), C.byref(pool), None, None, None,
                            None, None, None, None)
        n8, n16, nt, nb = (int(x) for x in sizes)
        top, inside = np.zeros(N, np.int8), np.zeros(N, np.int8)
        items, u = np.zeros((n8 + n16, 2), np.int32), np.zeros(n8 + n16, np.float32)
        tables, bcards, btab = np.zeros((nt, 4), np.int64), np.zeros(nb, np.uint64), np.zeros(nb, np.int32)
        probe.probe_runouts(C.c_void_p(t.h), sizes.ctypes.data_as(C.c_void_p), C.byref(pool),
                            top.ctypes.data_as(C.c_void_p), inside.ctypes.data_as(C.c_void_p),
                            items.ctypes.data_as(C.c_void_p), u.ctypes.data_as(C.c_void_p),
                            tables.ctypes.data_as(C.c_void_p), bcards.ctypes.data_as(C.c_void_p),
                            btab.ctypes.data_as(C.c_void_p))
        pay = np.zeros(N)
        probe.probe_payoff(C.c_void_p(t.h), pay.ctypes.data_as(C.c_void_p))
        boards = np.zeros(N, np.uint64)
        probe.probe_boards(C.c_void_p(t.h), boards.ctypes.data_as(C.c_void_p))
        probe.probe_Z.restype = C.c_double
        z = probe.probe_Z(C.c_void_p(t.h))

        def below(n):  # the nodes strictly below n
            out, stack = [], list(t.kids(n))
            while stack:
                m = stack.pop()
                out.append(m)
                stack.extend(t.kids(m))
            return out

        want_top = [n for n in range(1, N) if t.type[n] == CHANCE and t.type[t.parent[n]] != CHANCE
                    and all(t.type[m] in (CHANCE, SHOWDOWN) for m in below(n))]
        assert list(np.nonzero(top)[0]) == want_top
        want_inside = set()
        for n in want_top:
            want_inside |= set(below(n))
        assert set(np.nonzero(inside)[0].tolist()) == want_inside
        if case in ("turn", "flop"):
            assert want_top, "the all-in bets leave run-outs"
        if case in ("river", "leduc"):
            assert not want_top
        assert sorted(items[:, 0].tolist()) == want_top
        sig_of = {}
        for k, (n, tb) in enumerate(items.tolist()):
            shows = [m for m in below(n) if t.type[m] == SHOWDOWN]
            sig = sorted((int(boards[m]), int(t.row[m])) for m in shows)
            wide, nbd, b0, off = (int(x) for x in tables[tb])
            assert sorted(zip(bcards[b0:b0 + nbd].tolist(), btab[b0:b0 + nbd].tolist())) == sig
            assert wide == (nbd > 127) and (k >= n8) == bool(wide)
            assert len({pay[m] for m in shows}) == 1
            assert u[k] == np.float32(pay[shows[0]] * (1.0 / z))
            assert sig_of.setdefault(tuple(sig), tb) == tb
        assert len(sig_of) == nt
        offs = sorted((int(tables[k, 3]), int(tables[k, 0])) for k in range(nt))
        at = 0
        for off, wide in offs:
            assert off == at and off % 256 == 0
            at += (t.n_hands * t.hstride * (2 if wide else 1) + 255) // 256 * 256
        assert pool.value == at
    finally:
        t.close()


@pytest.mark.parametrize("case", ["turn", "flop"])
def test_runout_tables_reproduce_the_oracle_runout_values(probe, oracle_mod, case):
    """The table form of a run-out, restated in numpy from the host's plan and showdown
    tables: u sum_o E[h][o] q(o), E counting the boards (of the top's table) that share no card
    with h or o on which h's tie group ranks above o's less those on which it ranks below.
    Against the oracle's value at each top -- its sum over the run-out's boards -- under the
    strategies of two DCFR iterations, both players."""
    spec = SPECS[case]()
    t = Built(probe, spec)
    o = oracle_mod.Oracle(spec, variant="dcfr", threads=1)
    try:
        N, H = t.n_nodes, t.n_hands
        sizes, pool = np.zeros(4, np.int32), C.c_int64()
        probe.probe_runouts(C.c_void_p(t.h), sizes.ctypes.data_as(C.c_void_p), C.byref(pool), None, None, None,
                            None, None, None, None)
        n8, n16, nt, nb = (int(x) for x in sizes)
        top, inside = np.zeros(N, np.int8), np.zeros(N, np.int8)
        items, u = np.zeros((n8 + n16, 2), np.int32), np.zeros(n8 + n16, np.float32)
        tables, bcards, btab = np.zeros((nt, 4), np.int64), np.zeros(nb, np.uint64), np.zeros(nb, np.int32)
        probe.probe_runouts(C.c_void_p(t.h), sizes.ctypes.data_as(C.c_void_p), C.byref(pool),
                            top.ctypes.data_as(C.c_void_p), inside.ctypes.data_as(C.c_void_p),
                            items.ctypes.data_as(C.c_void_p), u.ctypes.data_as(C.c_void_p),
                            tables.ctypes.data_as(C.c_void_p), bcards.ctypes.data_as(C.c_void_p),
                            btab.ctypes.data_as(C.c_void_p))
        assert n8 + n16 > 0
        tt = np.zeros(10, np.int32)
        n = probe.probe_term_tables(C.c_void_p(t.h), tt.ctypes.data_as(C.c_void_p), None, C.c_int(0))
        tab = np.zeros(n, np.uint16)
        probe.probe_term_tables(C.c_void_p(t.h), tt.ctypes.data_as(C.c_void_p), tab.ctypes.data_as(C.c_void_p),
                                C.c_int(n))
        length, off_gs = int(tt[9]), int(tt[5])
        gs = np.stack([tab[b * length + off_gs: b * length + off_gs + H].astype(np.int64)
                       for b in range(n // length)])
        masks = np.array([(1 << int(a)) | (1 << int(c)) for a, c in spec.hands], dtype=np.uint64)
        # GPU node -> oracle node, walking both trees by child index
        info, g2o, todo = o.nodes(), {}, [(0, 0)]
        while todo:
            g, m = todo.pop()
            g2o[g] = m
            todo.extend(zip(t.kids(g), info[m]["kids"]))
        o.iterate(2)
        for i in (0, 1):
            o.values_current(i)
            for k, (node, tb) in enumerate(items.tolist()):
                wide, nbd, b0, _ = (int(x) for x in tables[tb])
                E = np.zeros((H, H))
                for b in range(b0, b0 + nbd):
                    r = gs[int(btab[b])]
                    ok = (masks & np.uint64(int(bcards[b]))) == 0
                    E += np.sign(r[:, None] - r[None, :]) * (ok[:, None] & ok[None, :])
                E *= (masks[:, None] & masks[None, :]) == 0
                assert np.abs(E).max() <= (32767 if wide else 127)
                q = o.node_reach("current", 1 - i, g2o[node])
                got = float(u[k]) * (E @ q)
                want = o.cfv(i, g2o[node])
                assert np.max(np.abs(got - want)) <= 1e-6 * np.max(np.abs(want)) + 1e-12, (case, i, node)
    finally:
        t.close()


def test_runout_plan_of_the_benchmarked_flop(probe):
    """The learned-leaf flop of the benchmark (1176 hands, pot 100, stacks 150, sizes 0.33,
    0.75, 1.25 pot and all-in): 10 flop all-ins run out turn and river (2352 boards, one 16-bit
    table) and 1,470 turn all-ins the river (48 boards, one 8-bit table per turn card: 49),
    71 MB of tables."""
    t = Built(probe, synth.ranked_flop_subgame(depth_limit=1))
    try:
        sizes, pool = np.zeros(4, np.int32), C.c_int64()
        probe.probe_runouts(C.c_void_p(t.h), sizes.ctypes.data_as(C.c_void_p), C.byref(pool), None, None, None,
                            None, None, None, None)
        n8, n16, nt, nb = (int(x) for x in sizes)
        assert (n8, n16, nt) == (1470, 10, 50)
        assert nb == 49 * 48 + 2352
        assert pool.value == 49 * t.n_hands * t.hstride + 2 * t.n_hands * t.hstride == 71_011_584
    finally:
        t.close()


def test_runout_table_entries_decode_exactly():
    """The run-out kernel turns a biased table entry x (uint8: E + 128, uint16: E + 32768)
    into E as FP32 by placing x in the mantissa of 2^23 and subtracting 2^23 + bias: exact
    for every entry (IEEE FP32, as numpy computes it)."""
    for bits, bias in ((8, 128), (16, 32768)):
        x = np.arange(1 << bits, dtype=np.uint32)
        as_float = (np.uint32(0x4B000000) | x).view(np.float32)
        e = as_float - np.float32(8388608.0 + bias)
        assert e.dtype == np.float32
        assert np.array_equal(e.astype(np.int64), x.astype(np.int64) - bias)
