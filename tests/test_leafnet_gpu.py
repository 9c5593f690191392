"""The leaf network's dense layers on the tensor cores (cfr_gemm_bf16) against the FP64
reference on the same BF16 operands."""
import dataclasses

import numpy as np
import pytest

from oracle import leafnet as ln
from paper_2605_19928_gb300 import capi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2605_19928_gb300 import build as pbuild
    pbuild.build()
    capi.load()


def _gemm(M, N, K, act, out_f32, seed, scale=1.0):
    import torch
    rng = np.random.default_rng(seed)
    a = ln.bf16_round(rng.standard_normal((M, K)).astype(np.float32) * scale)
    w = ln.bf16_round(rng.standard_normal((N, K)).astype(np.float32) / np.sqrt(K))
    b = rng.standard_normal(N).astype(np.float32) * 0.1
    dev = torch.device("cuda")
    A = torch.from_numpy(a).to(dev, torch.bfloat16)
    B = torch.from_numpy(w).to(dev, torch.bfloat16)
    bias = torch.from_numpy(b).to(dev)
    C = torch.full((M, N), float("nan"), dtype=torch.float32 if out_f32 else torch.bfloat16, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    capi.cfr_gemm_bf16(A, B, bias, C, act, err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    return C.float().cpu().numpy(), ln.dense(a, w, b, act=act), ln.abs_terms(a, w)


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (300, 256, 256), (1000, 512, 2752), (77, 2688, 512)])
def test_fp32_output_matches_fp64_reference(M, N, K):
    got, want, terms = _gemm(M, N, K, act=False, out_f32=True, seed=M + N + K)
    # FP32 accumulation: error bounded by a small multiple of eps_32 times sum |a_k w_k|
    assert np.all(np.abs(got - want) <= 2e-6 * (terms + np.abs(want)) + 1e-30), np.max(np.abs(got - want))


@pytest.mark.parametrize("M,N,K", [(200, 512, 2752), (513, 512, 512)])
def test_bf16_gelu_output_matches_reference(M, N, K):
    got, want, terms = _gemm(M, N, K, act=True, out_f32=False, seed=7 * M + N)
    # the GPU rounds its FP32 result to BF16: within one BF16 step of the FP64 value, plus
    # the accumulation error carried through GELU (slope <= 1.13)
    step = np.abs(ln.bf16_round(want).astype(np.float64)) * 2.0 ** -7 + 1e-38
    assert np.all(np.abs(got - want) <= step + 3e-6 * terms), np.max(np.abs(got - want) / step)


def test_shapes_are_checked():
    import torch
    dev = torch.device("cuda")
    A = torch.zeros((16, 64), dtype=torch.bfloat16, device=dev)
    B = torch.zeros((100, 64), dtype=torch.bfloat16, device=dev)  # N not a multiple of 128
    C = torch.zeros((16, 100), dtype=torch.float32, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    with pytest.raises(capi.CfrError) as e:
        capi.cfr_gemm_bf16(A, B, None, C, False, err)
    assert e.value.code == capi.CFR_EINVAL


# ---------------------------------------------------------------- depth-limit leaves in the CFR iteration

from gpu_helpers import compare_player, inject, node_map  # noqa: E402
from paper_2605_19928_gb300 import synth  # noqa: E402


def _leaf_spec(n_hands=40, seed=5, max_raises=2, street="turn"):
    if street == "flop":  # all-in the only bet: 49 turn cards, one leaf below each
        spec = synth.flop_subgame(n_hands=n_hands, seed=seed, range_seed=seed + 1, bet_sizes=(synth.ALL_IN,),
                                  max_raises=1)
    else:
        spec = synth.turn_subgame(n_hands=n_hands, seed=seed, range_seed=seed + 1,
                                  bet_sizes=(1.0, synth.ALL_IN), max_raises=max_raises)
    spec.depth_limit = 1
    return spec


def _node_board(orc, spec, o):
    """The board at oracle node o: the subgame's cards and those dealt on the way."""
    info = orc.nodes()
    dealt = []
    while o > 0:
        if info[o]["deal"] >= 0:
            dealt.append(info[o]["deal"])
        o = info[o]["parent"]
    return [int(c) for c in spec.board] + dealt[::-1]


def _random_net(seed):
    rng = np.random.default_rng(seed)
    W, b = [], []
    for k, shape in enumerate(capi.LEAF_SHAPES):
        w = rng.standard_normal(shape).astype(np.float32) * np.float32(2.0 / np.sqrt(shape[1]))
        W.append(ln.bf16_round(w * (0.2 if k == 3 else 1.0)))
        b.append(rng.standard_normal(shape[0]).astype(np.float32) * 0.05)
    return W, b


def _leaf_rows(tree, orc, spec, mapping, W, b, check_inputs=True, game=0):
    """Check one evaluation's inputs and outputs of one subgame's leaves against the oracle;
    load the GPU's outputs into the oracle's leaves.  Returns the worst output error relative
    to the row maximum."""
    g2o = {g: o for g, o, _ in mapping}
    slots = np.array([ln.pair_slot(int(a), int(c)) for a, c in spec.hands])
    worst = 0.0
    for g_leaf, node, row0 in capi.cfr_leaf_info(tree):
        if g_leaf != game:
            continue
        o = g2o[node]
        board = _node_board(orc, spec, o)
        live = [c for c in range(52) if c not in board]
        assert len(board) == 4 and len(live) == 48
        X = ln.bf16_from_bits(capi.cfr_read_leaf_rows(tree, 0, row0, 48))
        Y = capi.cfr_read_leaf_rows(tree, 1, row0, 48)
        if check_inputs:
            reach = [orc.node_reach("current", p, o) for p in (0, 1)]
            c = capi.cfr_node_info(tree, node, game)["contrib"]
            feat = ln.leaf_features(c[0] + c[1], spec.pot / 2 + spec.stack - c[0])
            for k, r in enumerate(live):
                x = ln.leaf_input(reach, spec.hands, board, r, feat)
                # the GPU rounds its FP32 input to BF16: one BF16 step of the exact value at most
                assert np.all(np.abs(X[k] - x) <= np.abs(x) * 2.0 ** -8 + 1e-30), (node, r)
        Yr = ln.forward(X, list(zip(W, b)))
        scale = np.max(np.abs(Yr), axis=1, keepdims=True)
        # hidden activations are rounded to BF16 on both sides; a rounding that falls the
        # other way moves an output by about one BF16 step of that activation's share
        err = np.max(np.abs(Y[:, :ln.SLOTS * 2] - Yr[:, :ln.SLOTS * 2]) / scale)
        assert err <= 3e-2, (node, err)
        worst = max(worst, float(err))
        y = np.stack([Y[:, :ln.SLOTS][:, slots], Y[:, ln.SLOTS:2 * ln.SLOTS][:, slots]], axis=1)
        orc.set_leaf_values(o, y.astype(np.float64))
    return worst


@pytest.mark.parametrize("schedule,street", [("level", "turn"), ("stream", "turn"), ("wide", "turn"),
                                             ("level", "flop"), ("stream", "flop"), ("wide", "flop")])
def test_leaf_inputs_outputs_and_values_match_oracle(schedule, street):
    from oracle.oracle import Oracle
    spec = _leaf_spec(n_hands=24, street="flop") if street == "flop" else _leaf_spec()
    W, b = _random_net(1)
    tree = capi.cfr_tree_create(spec, capi.make_opts("dcfr", schedule=schedule))
    try:
        capi.cfr_set_leaf_net(tree, [ln.bf16_bits(w) for w in W], b)
        capi.cfr_iterate(tree, 3)
        capi.cfr_eval_leaves(tree)
        orc = Oracle(spec, variant="dcfr")
        mapping = node_map(tree, orc)
        inject(tree, orc, mapping)
        print("output error", _leaf_rows(tree, orc, spec, mapping, W, b))
        for i in (0, 1):
            orc.values_current(i)
            for g, o, info in mapping:
                if info["type"] == capi.CFR_NODE_LEAF:
                    got = capi.cfr_read_values(tree, capi.CFR_READ_CFV, g, player=i)
                    want = orc.cfv(i, o)
                    assert np.max(np.abs(got - want)) <= 1e-5 * np.max(np.abs(want)) + 1e-9 * spec.pot, (i, g)
    finally:
        capi.cfr_tree_destroy(tree)


def _check_leaf_values(tree, orc, spec, mapping, game=0):
    for i in (0, 1):
        orc.values_current(i)
        for g, o, info in mapping:
            if info["type"] == capi.CFR_NODE_LEAF:
                got = capi.cfr_read_values(tree, capi.CFR_READ_CFV, g, player=i, game=game)
                want = orc.cfv(i, o)
                assert np.max(np.abs(got - want)) <= 1e-5 * np.max(np.abs(want)) + 1e-9 * spec.pot, (game, i, g)


def test_leaf_rows_in_slot_order_for_subgames_with_different_hands():
    """Two turn subgames with different hand lists in one handle: no common hand order, so
    the network's range columns and value rows stay in card-pair slot order.  Each subgame's
    inputs, outputs and leaf values match the oracle."""
    from oracle.oracle import Oracle
    specs = [_leaf_spec(n_hands=40, seed=5), _leaf_spec(n_hands=28, seed=9)]
    W, b = _random_net(2)
    tree = capi.cfr_batch_create(specs, capi.make_opts("dcfr"))
    try:
        capi.cfr_set_leaf_net(tree, [ln.bf16_bits(w) for w in W], b)
        capi.cfr_iterate(tree, 3)
        capi.cfr_eval_leaves(tree)
        assert {g for g, _, _ in capi.cfr_leaf_info(tree)} == {0, 1}
        for game, spec in enumerate(specs):
            orc = Oracle(spec, variant="dcfr")
            mapping = node_map(tree, orc, game=game)
            inject(tree, orc, mapping, game=game)
            _leaf_rows(tree, orc, spec, mapping, W, b, game=game)
            _check_leaf_values(tree, orc, spec, mapping, game=game)
    finally:
        capi.cfr_tree_destroy(tree)


@pytest.mark.parametrize("street", ["turn", "flop"])
@pytest.mark.parametrize("reach", ["unreached", "concentrated"])
def test_leaf_rows_with_degenerate_normalisers(street, reach):
    """The root player's regrets set so that the player checks at every later node and, at the
    root,
    - unreached: never checks, so none of the player's hands reaches the leaves below the check
      (every flop leaf), whose rows then hold the uniform range over the live hands (the
      oracle's reading of a zero normaliser);
    - concentrated: checks with the hands holding one card X and with the rest with
      probability 1e-6, so for river card X more than 99.8 % of a leaf's reach sits on hands
      holding X and the normaliser is the small remainder (summed directly, not as the
      difference of two sums).
    Inputs, outputs and leaf values match the oracle."""
    from oracle.oracle import Oracle
    spec = _leaf_spec(n_hands=24, street="flop") if street == "flop" else _leaf_spec()
    W, b = _random_net(3)
    tree = capi.cfr_tree_create(spec, capi.make_opts("dcfr"))
    try:
        capi.cfr_set_leaf_net(tree, [ln.bf16_bits(w) for w in W], b)
        capi.cfr_iterate(tree, 2)
        orc = Oracle(spec, variant="dcfr")
        mapping = node_map(tree, orc)
        assert capi.cfr_node_info(tree, 0)["type"] == capi.CFR_NODE_DECISION
        p0 = capi.cfr_node_info(tree, 0)["player"]
        cards = np.array(spec.hands)
        X = int(np.bincount(cards.ravel(), minlength=52).argmax())
        holds = (cards == X).any(axis=1)
        for g, o, info in mapping:
            if info["type"] != capi.CFR_NODE_DECISION or info["player"] != p0:
                continue
            R = capi.cfr_read_values(tree, capi.CFR_READ_REGRET, g)
            R[:] = -1.0
            if g != 0:
                R[0] = 1.0
            elif reach == "unreached":
                R[1] = 1.0
            else:
                R[0] = np.where(holds, 1.0, 1e-6)
                R[1] = np.where(holds, -1.0, 1.0)
            capi.cfr_write_values(tree, capi.CFR_READ_REGRET, g, R)
        capi.cfr_eval_leaves(tree)
        inject(tree, orc, mapping)
        leaves = [o for g, o, info in mapping if info["type"] == capi.CFR_NODE_LEAF]
        if reach == "unreached":
            assert any(not np.any(orc.node_reach("current", p0, o) > 0) for o in leaves), "no leaf without reach"
        else:  # some row's normaliser is below 2e-3 of the player's total at the leaf
            small = False
            for o in leaves:
                q = orc.node_reach("current", p0, o)
                board = _node_board(orc, spec, o)
                live = np.array([not ({int(a), int(c)} & set(board)) for a, c in spec.hands])
                rest = ~holds
                tot, s_x = q[live].sum(), q[live & rest].sum()
                small |= X not in board and tot > 0 and 0 < s_x < 2e-3 * tot
            assert small, "no row with a concentrated range"
        _leaf_rows(tree, orc, spec, mapping, W, b)
        _check_leaf_values(tree, orc, spec, mapping)
    finally:
        capi.cfr_tree_destroy(tree)


@pytest.mark.parametrize("schedule,variant,street,exact", [
    ("level", "dcfr", "turn", ()), ("stream", "dcfr", "turn", ()), ("level", "cfr+", "turn", ()),
    ("level", "dcfr", "flop", ()), ("wide", "dcfr", "flop", ()), ("wide", "pcfr+", "turn", ()),
    # the per-leaf fallback's trees: network leaves beside exact river subtrees
    ("level", "dcfr", "turn", (1,)), ("stream", "dcfr", "turn", (0, 2)), ("wide", "dcfr", "flop", (0, 20))])
def test_iterations_with_leaves_match_oracle_from_the_same_state(schedule, variant, street, exact):
    from oracle.oracle import Oracle
    spec = _leaf_spec(n_hands=32, seed=9, street=street)
    spec.exact_leaves = exact
    W, b = _random_net(2)
    Wbits = [ln.bf16_bits(w) for w in W]
    tree = capi.cfr_tree_create(spec, capi.make_opts(variant, schedule=schedule))
    try:
        capi.cfr_set_leaf_net(tree, Wbits, b)
        capi.cfr_iterate(tree, 2)
        orc = Oracle(spec, variant=variant)
        mapping = node_map(tree, orc)
        for t in range(3, 6):
            inject(tree, orc, mapping)
            capi.cfr_eval_leaves(tree)  # the evaluation player 0's update is about to see
            _leaf_rows(tree, orc, spec, mapping, W, b, check_inputs=False)
            capi.cfr_iterate(tree, 1)
            orc.update_player(0, t)
            compare_player(tree, orc, mapping, 0)
            inject(tree, orc, mapping, player=0)
            _leaf_rows(tree, orc, spec, mapping, W, b, check_inputs=False)  # player 1's evaluation
            orc.update_player(1, t)
            compare_player(tree, orc, mapping, 1)
            orc.set_iterations(t)
        e, _ = capi.cfr_exploitability(tree)
        assert np.isfinite(e[0])
    finally:
        capi.cfr_tree_destroy(tree)


def test_leaf_handles_need_a_network():
    spec = _leaf_spec(n_hands=20)
    tree = capi.cfr_tree_create(spec)
    try:
        with pytest.raises(capi.CfrError) as e:
            capi.cfr_iterate(tree, 1)
        assert e.value.code == capi.CFR_ESTATE
        assert len(capi.cfr_leaf_info(tree)) > 0
    finally:
        capi.cfr_tree_destroy(tree)


def test_full_size_flop_with_network_leaves():
    """The flop workload at full size (1176 hands, leaves below every turn card): sampled
    network rows against the FP64 forward pass of the same inputs, and input rows that are
    normalised ranges over the hands live on the leaf's board."""
    from paper_2605_19928_gb300 import leafnet_train
    spec = synth.ranked_flop_subgame(depth_limit=1)
    W, b = leafnet_train.load_weights()
    tree = capi.cfr_tree_create(spec, capi.make_opts("dcfr", precision="single"))
    try:
        capi.cfr_set_leaf_net(tree, W, b)
        capi.cfr_iterate(tree, 20)
        e, br = capi.cfr_exploitability(tree)
        assert np.isfinite(e[0]) and np.isfinite(br).all()
        leaves = capi.cfr_leaf_info(tree)
        assert len(leaves) > 1000
        capi.cfr_eval_leaves(tree)
        rng = np.random.default_rng(0)
        for k in rng.choice(len(leaves), size=3, replace=False):
            _, node, row0 = leaves[int(k)]
            X = ln.bf16_from_bits(capi.cfr_read_leaf_rows(tree, 0, row0, 48))
            Y = capi.cfr_read_leaf_rows(tree, 1, row0, 48)
            on = X[:, 2 * ln.SLOTS:2 * ln.SLOTS + 52]
            assert np.all(on.sum(axis=1) == 5)
            for p in (0, 1):
                tot = X[:, p * ln.SLOTS:(p + 1) * ln.SLOTS].astype(np.float64).sum(axis=1)
                assert np.all(np.abs(tot - 1.0) <= 0.01), (node, p)
            Yr = ln.forward(X, list(zip([ln.bf16_from_bits(w) for w in W], b)))  # W: BF16 bit patterns
            scale = np.max(np.abs(Yr), axis=1, keepdims=True)
            assert np.max(np.abs(Y[:, :2 * ln.SLOTS] - Yr[:, :2 * ln.SLOTS]) / scale) <= 3e-2
    finally:
        capi.cfr_tree_destroy(tree)


@pytest.mark.parametrize("schedule", ["level", "wide"])
def test_every_leaf_exact_gives_the_full_depth_bits(schedule):
    """A depth-limited subgame with all its leaves solved exactly is the full-depth subgame:
    the same tree, so the same bits after the same iterations."""
    spec = _leaf_spec(n_hands=24, seed=4)
    probe = capi.cfr_tree_create(spec)
    try:
        n_leaves = len(capi.cfr_leaf_info(probe))
    finally:
        capi.cfr_tree_destroy(probe)
    states = []
    for sp in (dataclasses.replace(spec, exact_leaves=tuple(range(n_leaves))), dataclasses.replace(spec, depth_limit=0)):
        tree = capi.cfr_tree_create(sp, capi.make_opts("dcfr", schedule=schedule))
        try:
            assert capi.cfr_leaf_info(tree) == []
            capi.cfr_iterate(tree, 5)
            n_nodes = capi.cfr_tree_info(tree)[0]
            st = []
            for n in range(n_nodes):
                if capi.cfr_node_info(tree, n)["type"] == capi.CFR_NODE_DECISION:
                    st.append(capi.cfr_read_values(tree, capi.CFR_READ_REGRET, n))
                    st.append(capi.cfr_read_values(tree, capi.CFR_READ_AVG_SUM, n))
            states.append((n_nodes, st, capi.cfr_exploitability(tree)[0][0]))
        finally:
            capi.cfr_tree_destroy(tree)
    assert states[0][0] == states[1][0]
    assert all(np.array_equal(a, b) for a, b in zip(states[0][1], states[1][1]))
    assert states[0][2] == states[1][2]
