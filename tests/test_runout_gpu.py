"""All-in run-outs evaluated by win-minus-loss tables (`runout_tables`): the value at a
run-out's top node is u E q in one step instead of the sum of its showdowns board by board.
Against the oracle from identical state (each player's update: R, S and the values at every
node the handle keeps, the run-out tops included), the best-response pass, and against the
board-by-board form of the same handle; plus the refusals."""
import numpy as np
import pytest

from gpu_helpers import close, forced_step, inject, node_map
from oracle import leafnet as ln
from paper_2605_19928_gb300 import capi, synth
from test_gpu_parity import flop, turn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2605_19928_gb300 import build as pbuild
    pbuild.build()
    capi.load()
    import torch
    assert torch.cuda.is_available()
    capi.use_torch_allocator()


CASES = {
    # one all-in bet: every call is a run-out of the river card (48 boards, 8-bit tables)
    "turn_allin": lambda: turn(24, seed=54, bet_sizes=(synth.ALL_IN,), max_raises=1),
    "turn_40": lambda: turn(40, seed=5, bet_sizes=(1.0, synth.ALL_IN), max_raises=2),
    # flop all-ins run out turn and river (2352 boards, 16-bit tables), turn all-ins the river
    "flop_12": lambda: flop(12, seed=5, bet_sizes=(synth.ALL_IN,), max_raises=1),
}


def opts(variant="dcfr", tables=True):
    return capi.make_opts(variant, precision="single", schedule="wide", runout_tables=tables)


def runouts(tree):
    """GPU node ids of the run-out tops and of the nodes below them."""
    n_nodes = capi.cfr_tree_info(tree)[0]
    info = [capi.cfr_node_info(tree, n) for n in range(n_nodes)]
    kids = {n: [] for n in range(n_nodes)}
    for n in range(1, n_nodes):
        kids[info[n]["parent"]].append(n)

    def below(n):
        out, stack = [], list(kids[n])
        while stack:
            m = stack.pop()
            out.append(m)
            stack.extend(kids[m])
        return out

    tops = [n for n in range(1, n_nodes) if info[n]["type"] == capi.CFR_NODE_CHANCE
            and info[info[n]["parent"]]["type"] != capi.CFR_NODE_CHANCE
            and all(info[m]["type"] in (capi.CFR_NODE_CHANCE, capi.CFR_NODE_SHOWDOWN) for m in below(n))]
    inside = set()
    for n in tops:
        inside |= set(below(n))
    return tops, inside


@pytest.mark.parametrize("variant", ["dcfr", "cfr+"])
@pytest.mark.parametrize("case", list(CASES))
def test_runout_tables_match_the_oracle_from_the_same_state(case, variant):
    from oracle.oracle import Oracle
    spec = CASES[case]()
    tree = capi.cfr_tree_create(spec, opts(variant))
    try:
        orc = Oracle(spec, variant=variant)
        mapping = node_map(tree, orc)
        g2o = {g: o for g, o, _ in mapping}
        tops, inside = runouts(tree)
        assert tops, "the case has run-outs"
        pot = spec.pot
        for t in range(1, 4):
            forced_step(tree, orc, mapping, t, skip=inside)
            for i in (0, 1):  # the value at each top: u E q against the oracle's sum over its boards
                for g in tops:
                    close(capi.cfr_read_values(tree, capi.CFR_READ_CFV, g, player=i), orc.cfv(i, g2o[g]),
                          floor=1e-8 * pot, what=f"top {g} player {i}")
        inject(tree, orc, mapping)
        expl_g, br_g = capi.cfr_exploitability(tree)
        e_o, b0, b1 = orc.exploitability()
        assert expl_g[0] == pytest.approx(e_o, rel=1e-5, abs=1e-9 * pot)
        assert br_g[0, 0] == pytest.approx(b0, rel=1e-5, abs=1e-9 * pot)
        assert br_g[0, 1] == pytest.approx(b1, rel=1e-5, abs=1e-9 * pot)
        for i in (0, 1):
            orc.load_profile("average")
            _, _, allv = orc.best_response(i, all_nodes=True)
            for g, o, _ in mapping:
                if g not in inside:
                    close(capi.cfr_read_values(tree, capi.CFR_READ_BR_CFV, g, player=i), allv[o],
                          floor=1e-8 * pot, what=f"best response node {g} player {i}")
    finally:
        capi.cfr_tree_destroy(tree)


def _decisions(tree):
    n_nodes = capi.cfr_tree_info(tree)[0]
    return [n for n in range(n_nodes) if capi.cfr_node_info(tree, n)["type"] == capi.CFR_NODE_DECISION]


def _state(tree, dec):
    return [(capi.cfr_read_values(tree, capi.CFR_READ_REGRET, n), capi.cfr_read_values(tree, capi.CFR_READ_AVG_SUM, n))
            for n in dec]


def _same_step(spec, net=None, iters=4):
    """Both forms after `iters` iterations, then one more from identical state: the board-by-
    board handle's R and S are written into the table handle (same iteration count), both run
    one iteration, and their R and S must agree to the FP32 rounding of the values (1e-5 of
    each node's largest entry).  Free-running runs are not compared: FP32 values that differ
    in summation order flip near-zero regrets, and regret matching is discontinuous there."""
    trees = []
    try:
        for tables in (False, True):
            tree = capi.cfr_tree_create(spec, opts(tables=tables))
            trees.append(tree)
            if net is not None:
                capi.cfr_set_leaf_net(tree, *net)
            capi.cfr_iterate(tree, iters)
        dec = _decisions(trees[0])
        for n, (R, S) in zip(dec, _state(trees[0], dec)):
            capi.cfr_write_values(trees[1], capi.CFR_READ_REGRET, n, R)
            capi.cfr_write_values(trees[1], capi.CFR_READ_AVG_SUM, n, S)
        e0, e1 = capi.cfr_exploitability(trees[0])[0][0], capi.cfr_exploitability(trees[1])[0][0]
        assert e1 == pytest.approx(e0, rel=1e-5, abs=1e-9 * spec.pot)
        for tree in trees:
            capi.cfr_iterate(tree, 1)
        for (R0, S0), (R1, S1) in zip(_state(trees[0], dec), _state(trees[1], dec)):
            close(R1, R0, floor=1e-8 * spec.pot)
            close(S1, S0)
    finally:
        for tree in trees:
            capi.cfr_tree_destroy(tree)


@pytest.mark.parametrize("case", list(CASES))
def test_runout_tables_follow_the_board_by_board_form(case):
    _same_step(CASES[case]())


def test_runout_tables_with_network_leaves():
    """A depth-limited flop: network leaves below the turn cards beside run-outs of the flop's
    all-ins; against the board-by-board form from identical state."""
    spec = synth.flop_subgame(n_hands=24, seed=5, range_seed=6, bet_sizes=(synth.ALL_IN,), max_raises=1)
    spec.depth_limit = 1
    rng = np.random.default_rng(1)
    W, b = [], []
    for k, shape in enumerate(capi.LEAF_SHAPES):
        w = rng.standard_normal(shape).astype(np.float32) * np.float32(2.0 / np.sqrt(shape[1]))
        W.append(ln.bf16_bits(ln.bf16_round(w * (0.2 if k == 3 else 1.0))))
        b.append(rng.standard_normal(shape[0]).astype(np.float32) * 0.05)
    _same_step(spec, net=(W, b))


def test_runout_tables_refusals():
    spec = CASES["turn_allin"]()
    for o in (capi.make_opts(precision="single", schedule="level", runout_tables=True),
              capi.make_opts(precision="pairs", schedule="wide", runout_tables=True)):
        with pytest.raises(capi.CfrError) as e:
            capi.cfr_tree_create(spec, o)
        assert e.value.code == capi.CFR_EINVAL
    with pytest.raises(capi.CfrError) as e:
        capi.cfr_batch_create([spec, CASES["turn_40"]()], opts())
    assert e.value.code == capi.CFR_EINVAL
    # a river has no run-outs: the option changes nothing
    river = synth.river_subgame(n_hands=64, seed=3, range_seed=4)
    out = []
    for tables in (False, True):
        tree = capi.cfr_tree_create(river, opts(tables=tables))
        try:
            capi.cfr_iterate(tree, 3)
            out.append(capi.cfr_read_values(tree, capi.CFR_READ_REGRET, 0))
        finally:
            capi.cfr_tree_destroy(tree)
    assert np.array_equal(out[0], out[1])
