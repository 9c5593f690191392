"""The served depth-limited solve on the GPU (Section 3): the continuation subgames the
judge solves exactly are the states the network was given, and the fallback returns the
full-depth subgame, or, leaf by leaf, one handle with exact river subtrees where the
network failed and network leaves elsewhere."""
import numpy as np
import pytest

from oracle import leafnet as ln
from paper_2605_19928_gb300 import capi, leafnet_train, serve, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2605_19928_gb300 import build as pbuild
    pbuild.build()
    capi.load()


def _samples_are_network_inputs(tree, judgement):
    """Each sampled continuation (ranges, completed board, pot and chips behind) against the
    BF16 input row the network saw for that leaf and river card."""
    for row, cont in judgement.samples:
        x = ln.bf16_from_bits(capi.cfr_read_leaf_rows(tree, 0, row, 1))[0].astype(np.float64)
        sl = leafnet_train.slot_of(cont.hands)
        for p in (0, 1):
            want = cont.ranges[p].astype(np.float64)
            got = x[p * ln.SLOTS + sl]
            # one BF16 rounding of the FP32 input (the FP32 normalisation is far below it)
            assert np.all(np.abs(got - want) <= np.abs(want) * 2.0 ** -8 + 1e-6 * want.max()), (row, p)
            assert abs(x[p * ln.SLOTS:(p + 1) * ln.SLOTS].sum() - got.sum()) <= 1e-12, (row, p)
        on = np.flatnonzero(x[2 * ln.SLOTS:2 * ln.SLOTS + 52])
        assert on.tolist() == cont.board.tolist(), row
        feat = ln.leaf_features(cont.pot, cont.stack)
        for k in (0, 1):
            assert abs(x[2 * ln.SLOTS + 52 + k] - feat[k]) <= abs(feat[k]) * 2.0 ** -8, row


def test_judge_turn_rows_are_the_network_inputs():
    spec = synth.ranked_turn_subgame(depth_limit=1)
    W, b = leafnet_train.load_weights()
    tree = capi.cfr_tree_create(spec, capi.make_opts("dcfr", precision="single"))
    try:
        capi.cfr_set_leaf_net(tree, W, b)
        capi.cfr_iterate(tree, 100)
        capi.cfr_exploitability(tree)
        j = serve.judge_leaves(tree, spec, n_rows=12, iters=200)
        assert j.rows == 12 and j.candidates >= 12
        _samples_are_network_inputs(tree, j)
        assert np.isfinite([j.mean_abs_error, j.reach_weighted_error, j.max_row_error]).all()
        assert 0.0 <= j.reach_weighted_error <= j.max_row_error
        assert 0.0 <= j.continuation_exploitability_mbb < 100.0
    finally:
        capi.cfr_tree_destroy(tree)


def test_judge_flop_rows_are_the_network_inputs():
    spec = synth.ranked_flop_subgame(depth_limit=1)
    W, b = leafnet_train.load_weights()
    tree = capi.cfr_tree_create(spec, capi.make_opts("dcfr", precision="single"))
    try:
        capi.cfr_set_leaf_net(tree, W, b)
        capi.cfr_iterate(tree, 20)
        capi.cfr_exploitability(tree)
        j = serve.judge_leaves(tree, spec, n_rows=8, iters=100, seed=3)
        assert j.rows == 8
        _samples_are_network_inputs(tree, j)
        assert np.isfinite(j.reach_weighted_error)
    finally:
        capi.cfr_tree_destroy(tree)


def test_fallback_returns_the_full_depth_subgame():
    spec = synth.ranked_turn_subgame(depth_limit=1)
    W, b = leafnet_train.load_weights()
    opts = capi.make_opts("dcfr", precision="single")
    kept = serve.solve_depth_limited(spec, W, b, 50, opts, tol=np.inf, judge_rows=4, judge_iters=50, per_leaf=0)
    try:
        assert kept.form == "learned" and len(capi.cfr_leaf_info(kept.tree)) > 0
        n_learned = capi.cfr_tree_info(kept.tree)[0]
    finally:
        capi.cfr_tree_destroy(kept.tree)
    dropped = serve.solve_depth_limited(spec, W, b, 50, opts, tol=0.0, judge_rows=4, judge_iters=50, per_leaf=0)
    try:
        assert dropped.form == "exact" and dropped.judgement.rows == 4
        assert capi.cfr_leaf_info(dropped.tree) == []
        n_nodes, _, done = capi.cfr_tree_info(dropped.tree)
        assert n_nodes > n_learned and done == 50
        e, _ = capi.cfr_exploitability(dropped.tree)
        assert np.isfinite(e[0]) and e[0] >= 0.0
    finally:
        capi.cfr_tree_destroy(dropped.tree)


def _paths(tree):
    n_nodes = capi.cfr_tree_info(tree)[0]
    paths = {0: ()}
    for n in range(1, n_nodes):
        info = capi.cfr_node_info(tree, n)
        paths[n] = paths[info["parent"]] + (info["action"],)
    return paths


def test_per_leaf_fallback_mixes_exact_subtrees_and_network_leaves():
    """With the tolerance at the median judged leaf error, the leaves above it come back as
    exact river-card chance nodes and the rest stay network leaves, in one handle."""
    spec = synth.ranked_turn_subgame(depth_limit=1)
    W, b = leafnet_train.load_weights()
    opts = capi.make_opts("dcfr", precision="single")
    tree = capi.cfr_tree_create(spec, opts)
    try:
        capi.cfr_set_leaf_net(tree, W, b)
        capi.cfr_iterate(tree, 50)
        capi.cfr_exploitability(tree)
        j = serve.judge_leaves(tree, spec, iters=50, per_leaf=2)
        leaf_paths = [_paths(tree)[node] for _, node, _ in capi.cfr_leaf_info(tree)]
    finally:
        capi.cfr_tree_destroy(tree)
    judged = [e for e in j.leaf_errors if e is not None]
    assert len(judged) >= 2 and j.rows <= 2 * len(leaf_paths)
    tol = float(np.median(judged))
    want = serve.fallback_leaves(j.leaf_errors, tol)
    assert 0 < len(want) < len(leaf_paths)
    s = serve.solve_depth_limited(spec, W, b, 50, opts, tol=tol, judge_iters=50, per_leaf=2)
    try:
        assert s.form == "mixed" and list(s.exact_leaves) == want
        paths = _paths(s.tree)
        by_path = {p: n for n, p in paths.items()}
        left = [_paths(s.tree)[node] for _, node, _ in capi.cfr_leaf_info(s.tree)]
        assert left == [p for k, p in enumerate(leaf_paths) if k not in want]
        for k in want:  # the river card is dealt by chance there now
            assert capi.cfr_node_info(s.tree, by_path[leaf_paths[k]])["type"] == capi.CFR_NODE_CHANCE
        assert capi.cfr_tree_info(s.tree)[2] == 50
        e, _ = capi.cfr_exploitability(s.tree)
        assert np.isfinite(e[0])
    finally:
        capi.cfr_tree_destroy(s.tree)
