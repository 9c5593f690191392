"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same seeded
inputs, element by element, after each of the first 10 iterations, plus exploitability."""
import numpy as np
import pytest

from gpu_helpers import compare_player, compare_state, compare_strategies, forced_step, inject, node_map
from paper_2605_19928_gb300 import capi, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2605_19928_gb300 import build as pbuild
    pbuild.build()
    capi.load()
    import torch
    assert torch.cuda.is_available()
    capi.use_torch_allocator()


def river(n_hands, seed=3, **kw):
    return synth.river_subgame(n_hands=n_hands, seed=seed, range_seed=seed + 1, **kw)


def turn(n_hands, seed=5, **kw):
    kw.setdefault("bet_sizes", (1.0, synth.ALL_IN))
    kw.setdefault("max_raises", 2)
    return synth.turn_subgame(n_hands=n_hands, seed=seed, range_seed=seed + 1, **kw)


def flop(n_hands, seed=5, **kw):
    kw.setdefault("bet_sizes", (synth.ALL_IN,))
    kw.setdefault("max_raises", 1)
    return synth.flop_subgame(n_hands=n_hands, seed=seed, range_seed=seed + 1, **kw)


def kuhn_random(seed=7):
    g = synth.kuhn()
    g.ranges[:] = synth.random_ranges(3, seed)
    return g


def leduc_random(seed=11):
    g = synth.leduc()
    g.ranges[:] = synth.random_ranges(6, seed)
    return g


# Two checks per case.  "forced": every iteration starts the oracle from the GPU's own
# state (gpu_helpers.forced_step), so each player's update is compared from identical
# inputs.  "free": both run 10 iterations independently; this needs inputs whose trajectory
# has no exact ties between action values, which FP64 and double-float may break
# differently (with few hands, or uniform deals, such ties appear within a few iterations
# and send two correct runs down different paths).
CASES = {
    "kuhn": (kuhn_random, ["cfr", "cfr+", "dcfr", "pcfr+"], False),
    "leduc": (leduc_random, ["cfr", "cfr+", "dcfr", "pcfr+"], False),
    "river_203": (lambda: river(203), ["dcfr", "cfr+", "pcfr+"], True),        # 26 blocks, ragged tail
    "river_64_r4": (lambda: river(64, seed=9, bet_sizes=(0.33, 0.75, 1.25, synth.ALL_IN), max_raises=4),
                    ["dcfr"], False),
    "turn_40": (lambda: turn(40), ["dcfr"], False),
}


def check_exploitability(tree, orc, mapping, pot, game=0, n_games=1):
    """The GPU's best-response pass against the oracle's on the GPU's own average strategy."""
    inject(tree, orc, mapping, game)
    expl_g, br_g = capi.cfr_exploitability(tree, n_games=n_games)
    e_o, b0, b1 = orc.exploitability()
    assert expl_g[game] == pytest.approx(e_o, rel=1e-5, abs=1e-9 * pot)
    assert br_g[game, 0] == pytest.approx(b0, rel=1e-5, abs=1e-9 * pot)
    assert br_g[game, 1] == pytest.approx(b1, rel=1e-5, abs=1e-9 * pot)
    for i in (0, 1):
        orc.load_profile("average")
        _, _, allv = orc.best_response(i, all_nodes=True)
        for g, o, info in mapping:
            got = capi.cfr_read_values(tree, capi.CFR_READ_BR_CFV, g, player=i, game=game)
            want = allv[o]
            scale = float(np.max(np.abs(want)))
            assert float(np.max(np.abs(got - want))) <= 1e-5 * scale + 1e-8 * pot, (i, g)


def run_pair(spec, variant, iters=10, alternating=True, chunk=0, forced=True, check_every=1, schedule="auto"):
    from oracle.oracle import Oracle
    tree = capi.cfr_tree_create(spec, capi.make_opts(variant, alternating=alternating, chunk_hands=chunk,
                                                     schedule=schedule))
    try:
        orc = Oracle(spec, variant=variant, alternating=alternating)
        mapping = node_map(tree, orc)
        worst = {}
        for t in range(1, iters + 1):
            if forced:
                w = forced_step(tree, orc, mapping, t, alternating)
            else:
                capi.cfr_iterate(tree, 1)
                orc.iterate(1)
                if t % check_every and t != iters:
                    continue
                w = compare_state(tree, orc, mapping)
            worst = {k: max(worst.get(k, 0.0), v) for k, v in w.items()}
        if not forced:
            e_g, _ = capi.cfr_exploitability(tree)
            assert e_g[0] == pytest.approx(orc.exploitability()[0], rel=1e-2)
        check_exploitability(tree, orc, mapping, spec.pot)
        return worst
    finally:
        capi.cfr_tree_destroy(tree)


@pytest.mark.parametrize("case,variant", [(c, v) for c, (_, vs, _) in CASES.items() for v in vs])
def test_each_iteration_matches_oracle_from_the_same_state(case, variant):
    worst = run_pair(CASES[case][0](), variant, forced=True)
    print(case, variant, "forced", worst)


@pytest.mark.parametrize("case,variant", [(c, v) for c, (_, vs, free) in CASES.items() if free for v in vs])
def test_first_ten_iterations_match_oracle(case, variant):
    worst = run_pair(CASES[case][0](), variant, forced=False)
    print(case, variant, "free", worst)


@pytest.mark.parametrize("game,variant,iters,bound", [
    ("kuhn", "cfr", 1000, 2e-3), ("kuhn", "cfr+", 1000, 1e-3),
    ("leduc", "cfr", 1000, 0.02), ("leduc", "cfr+", 1000, 2e-3), ("leduc", "dcfr", 1000, 2e-3),
    ("leduc", "pcfr+", 1000, 2e-3)])
def test_uniform_kuhn_and_leduc_converge_like_the_oracle(game, variant, iters, bound):
    """Config: Leduc (936 infosets) and Kuhn with uniform deals, 1000 iterations, FP32 GPU vs
    FP64 oracle.  Exact ties make the trajectories differ, so compare what is unique: both
    reach the same small exploitability and the Kuhn game value -1/18."""
    from oracle.oracle import Oracle
    spec = synth.kuhn() if game == "kuhn" else synth.leduc()
    tree = capi.cfr_tree_create(spec, capi.make_opts(variant))
    try:
        orc = Oracle(spec, variant=variant, threads=1)
        capi.cfr_iterate(tree, iters)
        orc.iterate(iters)
        expl, br = capi.cfr_exploitability(tree)
        e_o, b0, b1 = orc.exploitability()
        print(game, variant, "exploitability gpu", expl[0], "oracle", e_o)
        assert 0.0 <= expl[0] < bound and e_o < bound
        # not within 1 % of each other: with uniform deals exact ties between action values
        # recur every iteration, FP64 and double-float break them differently, and the two
        # (equally correct) trajectories end at different points of the same small
        # exploitability; the 1 % bar is met on inputs without such ties (above)
        assert expl[0] < 3.0 * e_o + 1e-4
        if game == "kuhn":
            # BR_0 >= game value >= -BR_1, both within the exploitability of -1/18
            assert br[0, 0] >= -1.0 / 18 - 1e-6 and -br[0, 1] <= -1.0 / 18 + 1e-6
            assert abs(br[0, 0] + 1.0 / 18) <= 2 * expl[0] + 1e-6
    finally:
        capi.cfr_tree_destroy(tree)


def test_full_size_river_ten_iterations():
    """The benchmarked workload itself: 1081 hands, pot 100, stacks 400, {0.5, 1, all-in},
    3 raises, DCFR(1.5, 0, 2), in the benchmark's launch configuration."""
    worst = run_pair(synth.river_subgame(), "dcfr", iters=10, forced=False, check_every=1)
    print("full river", worst)


def free_running_exploitability(spec, variant, iters, precision="pairs", schedule="auto"):
    """Both solvers run `iters` iterations independently from scratch; their final
    exploitabilities (average strategy, in chips)."""
    from oracle.oracle import Oracle
    tree = capi.cfr_tree_create(spec, capi.make_opts(variant, precision=precision, schedule=schedule))
    try:
        orc = Oracle(spec, variant=variant)
        capi.cfr_iterate(tree, iters)
        orc.iterate(iters)
        e_g, _ = capi.cfr_exploitability(tree)
        return float(e_g[0]), orc.exploitability()[0]
    finally:
        capi.cfr_tree_destroy(tree)


@pytest.mark.parametrize("case,iters", [("river_203", 500), ("river_1081", 300)])
def test_converged_exploitability_within_one_percent(case, iters):
    """Spec bar for the final result: after a long free-running solve (DCFR 1.5/0/2,
    default pair values) the GPU's exploitability is within 1 % of the oracle's.  The
    1081-hand river is the single-subgame benchmark workload."""
    spec = river(203) if case == "river_203" else synth.river_subgame()
    e_g, e_o = free_running_exploitability(spec, "dcfr", iters)
    print(case, iters, "exploitability gpu", e_g, "oracle", e_o, "relative", abs(e_g - e_o) / e_o)
    assert e_g == pytest.approx(e_o, rel=1e-2)


def test_long_run_follows_the_oracle_from_its_own_state():
    """Past a few hundred iterations two correct runs can part: near-indifferent hands turn
    rounding-level differences in values into regret differences, and on the 203-hand river
    the GPU's trajectory meets an exploitability spike near iteration 740 (0.011 -> 0.08)
    that the oracle's own trajectory misses.  From the GPU's state at iteration 725 the
    oracle must follow it across the spike: every iteration from identical state within
    1e-10 of the node maximum, and after 75 free-running iterations the same exploitability
    within 1 %."""
    from oracle.oracle import Oracle
    spec = river(203)
    tree = capi.cfr_tree_create(spec, capi.make_opts("dcfr"))
    try:
        free = Oracle(spec, variant="dcfr")
        mapping = node_map(tree, free)
        capi.cfr_iterate(tree, 725)
        inject(tree, free, mapping)
        free.set_iterations(725)
        forced = Oracle(spec, variant="dcfr")
        for t in range(726, 801):
            if t <= 760:  # each of these iterations from identical state
                w = forced_step(tree, forced, mapping, t, rtol=1e-10)
                assert max(w["R"], w["S"]) <= 1e-10, (t, w)
            else:
                capi.cfr_iterate(tree, 1)
        free.iterate(75)
        e_g, _ = capi.cfr_exploitability(tree)
        e_o = free.exploitability()[0]
        print("from iteration 725: exploitability gpu", e_g[0], "oracle", e_o, "(0.011 before the spike)")
        assert e_g[0] == pytest.approx(e_o, rel=1e-2)
    finally:
        capi.cfr_tree_destroy(tree)


def test_batch_subgame_converged_exploitability_within_one_percent():
    """A subgame of the benchmarked batch (its smallest tree) solved for the batch's 500
    iterations in its precision (FP32 values) on the stream schedule, free-running, against
    the oracle: final exploitability within 1 %."""
    specs = synth.batch_rivers(256)
    from oracle.oracle import Oracle
    sizes = [Oracle(s, variant="dcfr", threads=1).n_nodes for s in specs[:32]]
    spec = specs[int(np.argmin(sizes))]
    e_g, e_o = free_running_exploitability(spec, "dcfr", 500, precision="single", schedule="stream")
    print("batch subgame", min(sizes), "nodes: exploitability gpu", e_g, "oracle", e_o, "relative",
          abs(e_g - e_o) / e_o)
    assert e_g == pytest.approx(e_o, rel=1e-2)


def test_simultaneous_updates_match_oracle():
    run_pair(river(97, seed=21), "dcfr", iters=5, alternating=False)


@pytest.mark.parametrize("chunk", [1, 4, 32])
def test_block_shape_does_not_change_results(chunk):
    run_pair(river(77, seed=13), "dcfr", iters=3, chunk=chunk)


def test_all_strengths_equal_gives_zero_showdown_values():
    spec = river(120, seed=17)
    spec.strength[:] = 777
    run_pair(spec, "dcfr", iters=3)


def test_degenerate_ranges_and_tiny_trees():
    spec = river(50, seed=19, max_raises=0)  # check / check only
    spec.ranges[0, ::2] = 0.0
    run_pair(spec, "dcfr", iters=3)
    spec = river(50, seed=23, stack=0.0)     # no chips behind: no bets
    run_pair(spec, "cfr", iters=2)


def test_batch_matches_independent_solves():
    from oracle.oracle import Oracle
    specs = [river(60, seed=31), river(45, seed=32, bet_sizes=(1.0, synth.ALL_IN), max_raises=2),
             leduc_random(seed=5), river(150, seed=33, stack=900.0, bet_sizes=(0.75, synth.ALL_IN))]
    tree = capi.cfr_batch_create(specs, capi.make_opts("dcfr"))
    try:
        orcs = [Oracle(s, variant="dcfr") for s in specs]
        maps = [node_map(tree, o, game=k) for k, o in enumerate(orcs)]
        capi.cfr_iterate(tree, 4)  # reach a non-trivial state first
        # the batch advances all games together, so compare each game's update from its
        # own state: load, iterate the batch once, and check every game
        for t in range(5, 8):
            for k, (o, m) in enumerate(zip(orcs, maps)):
                inject(tree, o, m, game=k)
            capi.cfr_iterate(tree, 1)
            for k, (o, m) in enumerate(zip(orcs, maps)):
                o.update_player(0, t)
                compare_player(tree, o, m, 0, game=k)
                inject(tree, o, m, game=k, player=0)
                o.update_player(1, t)
                compare_player(tree, o, m, 1, game=k)
                o.set_iterations(t)
        for k, (o, m) in enumerate(zip(orcs, maps)):
            check_exploitability(tree, o, m, specs[k].pot, game=k, n_games=len(specs))
    finally:
        capi.cfr_tree_destroy(tree)


def test_average_strategy_readback():
    from oracle.oracle import Oracle
    spec = river(88, seed=41)
    tree = capi.cfr_tree_create(spec, capi.make_opts("dcfr"))
    try:
        orc = Oracle(spec, variant="dcfr")
        mapping = node_map(tree, orc)
        capi.cfr_iterate(tree, 6)
        inject(tree, orc, mapping)
        orc.load_profile("average")
        for g, o, info in mapping:
            if info["type"] == capi.CFR_NODE_DECISION:
                got = capi.cfr_strategy(tree, g, average=True)
                compare_strategies(got, orc.avg_sums(o), what=f"average strategy node {g}", plus_part=False)
                cur = capi.cfr_strategy(tree, g, average=False)
                compare_strategies(cur, orc.regrets(o), what=f"current strategy node {g}")
    finally:
        capi.cfr_tree_destroy(tree)


@pytest.mark.parametrize("schedule", ["level", "stream", "wide"])
def test_flop_matches_oracle_from_the_same_state(schedule):
    """Three streets: turn and river cards by chance, 2352 showdown boards, all-in run-outs
    from the flop and from the turn (31k nodes)."""
    worst = run_pair(flop(12), "dcfr", iters=3, forced=True, schedule=schedule)
    print("flop", schedule, worst)


def test_invalid_specs_are_rejected():
    spec = river(30, seed=5)
    spec.hands[0, 0] = spec.board[0]
    with pytest.raises(capi.CfrError) as e:
        capi.cfr_tree_create(spec)
    assert e.value.code == capi.CFR_EINVAL
    spec = river(30, seed=5)
    spec.ranges[1, :] = 0.0
    with pytest.raises(capi.CfrError):
        capi.cfr_tree_create(spec)
    spec = river(30, seed=5)
    spec.ranges[0, 3] = np.nan
    with pytest.raises(capi.CfrError):
        capi.cfr_tree_create(spec)


def test_batch_reports_the_first_rejected_subgame():
    """Batches of eight or more subgames are built on several host threads; a rejected spec is
    still reported by its index, and the lowest one when several are bad."""
    specs = [river(30, seed=40 + k) for k in range(12)]
    specs[9].ranges[1, :] = 0.0
    specs[6].hands[0, 0] = specs[6].board[0]
    with pytest.raises(capi.CfrError) as e:
        capi.cfr_batch_create(specs)
    assert e.value.code == capi.CFR_EINVAL
    assert "game 6:" in str(e.value), str(e.value)
    good = [river(30, seed=40 + k) for k in range(12)]
    tree = capi.cfr_batch_create(good)
    capi.cfr_tree_destroy(tree)


# ---------------------------------------------------------------- stream schedule
# The one-warp-per-32-hands update (chosen automatically for large batches) must agree with
# the oracle exactly like the level schedule, and with the level schedule bit for bit.

STREAM_CASES = [("kuhn", "cfr"), ("leduc", "cfr+"), ("river_203", "dcfr"), ("turn_40", "dcfr"),
                ("river_64_r4", "dcfr"), ("leduc", "pcfr+"), ("river_203", "pcfr+")]


@pytest.mark.parametrize("case,variant", STREAM_CASES)
def test_stream_schedule_matches_oracle_from_the_same_state(case, variant):
    worst = run_pair(CASES[case][0](), variant, forced=True, schedule="stream")
    print(case, variant, "stream forced", worst)


def test_stream_schedule_first_ten_iterations_match_oracle():
    run_pair(river(203), "dcfr", forced=False, schedule="stream")


def test_stream_schedule_simultaneous_updates_match_oracle():
    run_pair(river(97, seed=21), "dcfr", iters=5, alternating=False, schedule="stream")


# ---------------------------------------------------------------- wide schedule
# One launch per level over every (node, hand) pair of the level (large single trees); the
# same arithmetic as the level schedule.

WIDE_CASES = [("kuhn", "cfr"), ("leduc", "cfr+"), ("river_203", "dcfr"), ("turn_40", "dcfr"),
              ("river_64_r4", "dcfr"), ("river_203", "pcfr+")]


@pytest.mark.parametrize("case,variant", WIDE_CASES)
def test_wide_schedule_matches_oracle_from_the_same_state(case, variant):
    worst = run_pair(CASES[case][0](), variant, forced=True, schedule="wide")
    print(case, variant, "wide forced", worst)


def test_wide_schedule_first_ten_iterations_match_oracle():
    run_pair(river(203), "dcfr", forced=False, schedule="wide")


def test_wide_schedule_simultaneous_updates_match_oracle():
    run_pair(river(97, seed=21), "dcfr", iters=5, alternating=False, schedule="wide")


def _state(tree, n_games, with_pred=False):
    out = []
    for game in range(n_games):
        n_nodes = capi.cfr_tree_info(tree, game)[0]
        for n in range(n_nodes):
            info = capi.cfr_node_info(tree, n, game)
            if info["type"] == capi.CFR_NODE_DECISION:
                out.append(capi.cfr_read_values(tree, capi.CFR_READ_REGRET, n, game=game))
                out.append(capi.cfr_read_values(tree, capi.CFR_READ_AVG_SUM, n, game=game))
                if with_pred:
                    out.append(capi.cfr_read_values(tree, capi.CFR_READ_PREDICTION, n, game=game))
                out.append(capi.cfr_strategy(tree, n, average=False, game=game))
                out.append(capi.cfr_strategy(tree, n, average=True, game=game))
            if n == 0 or info["type"] in (capi.CFR_NODE_FOLD, capi.CFR_NODE_SHOWDOWN):
                for i in (0, 1):
                    out.append(capi.cfr_read_values(tree, capi.CFR_READ_CFV, n, player=i, game=game))
    return out


@pytest.mark.parametrize("warp_hands", [32, 64])
@pytest.mark.parametrize("precision", ["pairs", "single"])
@pytest.mark.parametrize("variant,alternating", [("dcfr", True), ("cfr+", True), ("cfr", False), ("pcfr+", True)])
def test_stream_and_level_schedules_give_the_same_bits(precision, variant, alternating, warp_hands):
    """Both hands-per-warp forms of the stream update.  64 hands per warp (two per lane) needs
    rows padded to 64, so that batch has no one-card games, and rivers only (a turn's chance
    node stacks 48 subtrees per hand, which two hands per lane do not fit); 100 hands leave
    the last warp's second hand of each lane partly beyond the hand list."""
    if warp_hands == 32:
        specs = [river(203, seed=51), river(64, seed=52, bet_sizes=(0.33, 0.75, 1.25, synth.ALL_IN), max_raises=4),
                 leduc_random(seed=53), turn(40, seed=54), kuhn_random(seed=55)]
    else:
        specs = [river(120, seed=51), river(64, seed=52, bet_sizes=(0.33, 0.75, 1.25, synth.ALL_IN), max_raises=4),
                 river(100, seed=56)]
    states, expl = [], []
    for schedule in ("level", "stream"):
        tree = capi.cfr_batch_create(specs, capi.make_opts(variant, alternating=alternating, precision=precision,
                                                           schedule=schedule,
                                                           warp_hands=warp_hands if schedule == "stream" else 0))
        try:
            assert capi.cfr_schedule(tree) == capi.SCHEDULES[schedule]
            capi.cfr_iterate(tree, 7)
            states.append(_state(tree, len(specs), with_pred=variant == "pcfr+"))
            expl.append(capi.cfr_exploitability(tree, len(specs)))
        finally:
            capi.cfr_tree_destroy(tree)
    assert len(states[0]) == len(states[1])
    for a, b in zip(*states):
        assert np.array_equal(a, b)
    assert np.array_equal(expl[0][0], expl[1][0]) and np.array_equal(expl[0][1], expl[1][1])


def test_64_hands_per_warp_needs_rows_padded_to_64():
    with pytest.raises(capi.CfrError) as e:
        capi.cfr_batch_create([river(203)], capi.make_opts("dcfr", schedule="stream", warp_hands=64))
    assert e.value.code == capi.CFR_EINVAL


@pytest.mark.parametrize("precision", ["pairs", "single"])
@pytest.mark.parametrize("variant,alternating", [("dcfr", True), ("cfr+", True), ("cfr", False), ("pcfr+", True)])
def test_wide_and_level_schedules_give_the_same_bits(precision, variant, alternating):
    """Same state bits; the exploitability differs only in the order of its FP64 root sum."""
    for spec in (river(203, seed=51), turn(40, seed=54), leduc_random(seed=53), kuhn_random(seed=55)):
        states, expl = [], []
        for schedule in ("level", "wide"):
            tree = capi.cfr_tree_create(spec, capi.make_opts(variant, alternating=alternating, precision=precision,
                                                             schedule=schedule))
            try:
                assert capi.cfr_schedule(tree) == capi.SCHEDULES[schedule]
                capi.cfr_iterate(tree, 7)
                states.append(_state(tree, 1, with_pred=variant == "pcfr+"))
                expl.append(capi.cfr_exploitability(tree))
            finally:
                capi.cfr_tree_destroy(tree)
        assert len(states[0]) == len(states[1])
        for a, b in zip(*states):
            assert np.array_equal(a, b)
        np.testing.assert_allclose(expl[0][1], expl[1][1], rtol=1e-12, atol=1e-12 * spec.pot)


def test_schedule_selection():
    tree = capi.cfr_tree_create(river(203))
    try:
        assert capi.cfr_schedule(tree) == capi.CFR_SCHEDULE_LEVEL  # one subgame: latency form
    finally:
        capi.cfr_tree_destroy(tree)
    # 36 full rivers = 36 * 34 warps of 32 hands >= 8 per SM: throughput form
    specs = [synth.river_subgame(seed=60 + k, range_seed=61 + k, max_raises=1) for k in range(36)]
    tree = capi.cfr_batch_create(specs)
    try:
        assert capi.cfr_schedule(tree) == capi.CFR_SCHEDULE_STREAM
    finally:
        capi.cfr_tree_destroy(tree)
    # more than 8 actions at a node: the stream form is refused, auto falls back to level
    wide = river(40, seed=62, bet_sizes=(0.25, 0.5, 0.75, 1.0, 1.25, 1.5, 2.0, synth.ALL_IN), max_raises=2)
    with pytest.raises(capi.CfrError) as e:
        capi.cfr_tree_create(wide, capi.make_opts(schedule="stream"))
    assert e.value.code == capi.CFR_EINVAL
    tree = capi.cfr_tree_create(wide, capi.make_opts(schedule="auto"))
    try:
        assert capi.cfr_schedule(tree) == capi.CFR_SCHEDULE_LEVEL
    finally:
        capi.cfr_tree_destroy(tree)
    with pytest.raises(capi.CfrError) as e:  # the wide form takes at most 8 actions too
        capi.cfr_tree_create(wide, capi.make_opts(schedule="wide"))
    assert e.value.code == capi.CFR_EINVAL
    # one tree too large for a block to stage (31k nodes): the wide form; two of them: level
    tree = capi.cfr_tree_create(flop(12))
    try:
        assert capi.cfr_schedule(tree) == capi.CFR_SCHEDULE_WIDE
    finally:
        capi.cfr_tree_destroy(tree)
    tree = capi.cfr_batch_create([flop(12), flop(12, seed=6)])
    try:
        assert capi.cfr_schedule(tree) == capi.CFR_SCHEDULE_LEVEL
    finally:
        capi.cfr_tree_destroy(tree)
    with pytest.raises(capi.CfrError) as e:
        capi.cfr_batch_create([river(30, seed=5), river(30, seed=6)], capi.make_opts(schedule="wide"))
    assert e.value.code == capi.CFR_EINVAL


# ---------------------------------------------------------------- FP32 values
# CFR_PRECISION_SINGLE carries reach, strategies and values in plain FP32 (R and S stay
# FP64).  Compared from the GPU's own state each iteration, it meets the same bar as the
# default precision (1e-5 of the largest oracle magnitude in each node's vector); the test
# prints the worst errors it saw.  Free-running FP32 trajectories drift further, because
# rounding decides near-ties between actions differently from FP64.

@pytest.mark.parametrize("case,variant,schedule", [("river_203", "dcfr", "level"), ("river_203", "dcfr", "stream"),
                                                   ("turn_40", "dcfr", "stream"), ("leduc", "cfr+", "stream"),
                                                   ("turn_40", "dcfr", "wide")])
def test_single_precision_error_against_oracle(case, variant, schedule):
    from oracle.oracle import Oracle
    spec = CASES[case][0]()
    tree = capi.cfr_tree_create(spec, capi.make_opts(variant, precision="single", schedule=schedule))
    try:
        orc = Oracle(spec, variant=variant)
        mapping = node_map(tree, orc)
        worst = {}
        for t in range(1, 11):
            w = forced_step(tree, orc, mapping, t, rtol=1e-5, floor_frac=1e-8)
            worst = {k: max(worst.get(k, 0.0), v) for k, v in w.items()}
        print(case, variant, schedule, "single forced (relative to node max)", worst)
        inject(tree, orc, mapping)
        e_g, _ = capi.cfr_exploitability(tree)
        assert e_g[0] == pytest.approx(orc.exploitability()[0], rel=1e-4, abs=1e-7 * spec.pot)
    finally:
        capi.cfr_tree_destroy(tree)


def test_terminal_runs_match_one_node_blocks():
    """Large handles evaluate up to eight terminal nodes per block; small ones one.  The same
    subgames solved in one large handle and one handle each must agree bit for bit."""
    specs = [river(64, seed=70 + k, bet_sizes=(0.33, 0.75, 1.25, synth.ALL_IN), max_raises=4) for k in range(40)]
    big = capi.cfr_batch_create(specs, capi.make_opts("dcfr", precision="pairs", schedule="level"))
    try:
        n_term = sum(1 for g in range(len(specs)) for n in range(capi.cfr_tree_info(big, g)[0])
                     if capi.cfr_node_info(big, n, g)["type"] in (capi.CFR_NODE_FOLD, capi.CFR_NODE_SHOWDOWN))
        assert n_term >= 4 * 152 * 8  # runs of four
        capi.cfr_iterate(big, 3)
        e_big, _ = capi.cfr_exploitability(big, len(specs))
        for g in (0, 17, 39):
            one = capi.cfr_tree_create(specs[g], capi.make_opts("dcfr", precision="pairs", schedule="level"))
            try:
                capi.cfr_iterate(one, 3)
                e_one, _ = capi.cfr_exploitability(one)
                assert e_one[0] == e_big[g]
                for n in range(capi.cfr_tree_info(one)[0]):
                    info = capi.cfr_node_info(one, n)
                    if info["type"] == capi.CFR_NODE_DECISION:
                        for what in (capi.CFR_READ_REGRET, capi.CFR_READ_AVG_SUM):
                            assert np.array_equal(capi.cfr_read_values(one, what, n),
                                                  capi.cfr_read_values(big, what, n, game=g))
                    elif info["type"] != capi.CFR_NODE_CHANCE:
                        for i in (0, 1):
                            assert np.array_equal(capi.cfr_read_values(one, capi.CFR_READ_CFV, n, player=i),
                                                  capi.cfr_read_values(big, capi.CFR_READ_CFV, n, player=i, game=g))
            finally:
                capi.cfr_tree_destroy(one)
    finally:
        capi.cfr_tree_destroy(big)


@pytest.mark.parametrize("schedule", ["level", "stream"])
def test_fp32_terminal_runs_match_oracle(schedule):
    """A batch whose terminal nodes fill the GPU (runs of four nodes per block) with FP32
    values: each subgame against the oracle from the GPU's own state, and its
    exploitability."""
    from oracle.oracle import Oracle
    specs = [river(64, seed=70 + k, bet_sizes=(0.33, 0.75, 1.25, synth.ALL_IN), max_raises=4) for k in range(40)]
    big = capi.cfr_batch_create(specs, capi.make_opts("dcfr", precision="single", schedule=schedule))
    try:
        capi.cfr_iterate(big, 2)
        for g in (0, 39):
            orc = Oracle(specs[g], variant="dcfr")
            mapping = node_map(big, orc, game=g)
            for t in range(3, 5):
                forced_step(big, orc, mapping, t, game=g, rtol=1e-5, floor_frac=1e-8)
            inject(big, orc, mapping, game=g)
            e_g, _ = capi.cfr_exploitability(big, len(specs))
            assert e_g[g] == pytest.approx(orc.exploitability()[0], rel=1e-4, abs=1e-7 * specs[g].pot)
            capi.cfr_reset(big)
            capi.cfr_iterate(big, 2)
    finally:
        capi.cfr_tree_destroy(big)


def test_autotune_picks_a_layout_with_the_same_results():
    """The launch-tiling autotuner times every layout and returns the fastest; every layout
    gives the same bits, so the tuned handle's state equals the default one's."""
    specs = [river(96, seed=80 + k, max_raises=2) for k in range(12)]
    base = capi.make_opts("dcfr", precision="single")
    best, ms = capi.cfr_autotune(specs, base, iters=3)
    assert ms > 0
    assert best.schedule in (capi.CFR_SCHEDULE_LEVEL, capi.CFR_SCHEDULE_STREAM, capi.CFR_SCHEDULE_RESIDENT)
    assert best.term_nodes in (0, 1, 2, 4, 8) and best.variant == base.variant and best.precision == base.precision
    assert best.warp_hands in (0, 32, 64)
    states = []
    for o in (base, best):
        tree = capi.cfr_batch_create(specs, o)
        try:
            capi.cfr_iterate(tree, 5)
            states.append(_state(tree, len(specs)))
        finally:
            capi.cfr_tree_destroy(tree)
    for a, b in zip(*states):
        assert np.array_equal(a, b)
    with pytest.raises(capi.CfrError) as e:
        capi.cfr_autotune(specs, base, iters=0)
    assert e.value.code == capi.CFR_EINVAL


@pytest.mark.parametrize("schedule", ["level", "stream", "wide"])
def test_fp32_strategy_is_regret_matching_rounded_to_nearest(schedule):
    """FP32 values: the strategy the GPU derives from FP64 regrets is IEEE arithmetic on the
    regrets rounded to FP32 (nearest, ties to even): positive parts, their sum in action
    order, one FP32 reciprocal and products (Eq. rm).  The regrets cover 60 binades, values
    exactly halfway between two floats (both parities of the last mantissa bit) and values
    one FP64 step either side of those midpoints."""
    spec = river(30, seed=5)
    tree = capi.cfr_tree_create(spec, capi.make_opts("dcfr", precision="single", schedule=schedule))
    try:
        info = capi.cfr_node_info(tree, 0)
        A, H = info["n_actions"], spec.n_hands
        assert A >= 3
        rng = np.random.default_rng(17)
        R = np.exp(rng.uniform(-69.0, 69.0, size=(A, H))) * rng.choice([-1.0, 1.0], size=(A, H), p=[0.3, 0.7])
        f = rng.uniform(0.5, 4.0, size=(A, H)).astype(np.float32)
        mid = f.astype(np.float64) + np.spacing(f).astype(np.float64) / 2  # exactly halfway
        cols = np.arange(H) % 4
        R = np.where(cols == 1, mid, R)
        R = np.where(cols == 2, np.nextafter(mid, np.inf), R)
        R = np.where(cols == 3, np.nextafter(mid, -np.inf), R)
        capi.cfr_write_values(tree, capi.CFR_READ_REGRET, 0, R)
        got = capi.cfr_strategy(tree, 0)
        x = np.where(R > 0, R, 0.0).astype(np.float32)  # round to nearest even
        want = np.empty((A, H), np.float32)
        for h in range(H):
            pos = x[:, h] > 0
            if pos.sum() == 1:
                want[:, h] = pos.astype(np.float32)
            elif pos.sum() == 0:
                want[:, h] = np.float32(1) / np.float32(A)
            else:
                tot = np.float32(0)
                for a in range(A):
                    tot = np.float32(tot + x[a, h])
                want[:, h] = x[:, h] * (np.float32(1) / tot)
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    finally:
        capi.cfr_tree_destroy(tree)


def test_full_size_batch_sampled_subgames_match_oracle():
    """The benchmarked batch itself (256 uneven 1081-hand rivers, FP32 values, the stream
    schedule the bench's autotuner picks, terminal runs): two sampled subgames against the
    oracle from the GPU's own state for one iteration, and their exploitability."""
    from oracle.oracle import Oracle
    specs = synth.batch_rivers(256, seed=0)
    tree = capi.cfr_batch_create(specs, capi.make_opts("dcfr", precision="single", schedule="stream"))
    try:
        assert capi.cfr_schedule(tree) == capi.CFR_SCHEDULE_STREAM
        capi.cfr_iterate(tree, 3)
        for g in (0, 255):
            orc = Oracle(specs[g], variant="dcfr")
            mapping = node_map(tree, orc, game=g)
            w = forced_step(tree, orc, mapping, 4, game=g, rtol=1e-5, floor_frac=1e-8)
            print("batch subgame", g, w)
            inject(tree, orc, mapping, game=g)
            e_g, _ = capi.cfr_exploitability(tree, len(specs))
            assert e_g[g] == pytest.approx(orc.exploitability()[0], rel=1e-4, abs=1e-7 * specs[g].pot)
            capi.cfr_reset(tree)
            capi.cfr_iterate(tree, 3)
    finally:
        capi.cfr_tree_destroy(tree)
