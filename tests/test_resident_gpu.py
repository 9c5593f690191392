"""The resident schedule: one cooperative launch runs whole iterations, each block keeping a
chunk of hands of both players in shared memory, with a grid barrier between an iteration's
phases.  Its arithmetic is the level schedule's, so after the same iterations every regret,
strategy sum, strategy and counterfactual value has the same bits, whether the iterations
ran in one launch or several; plus its refusals and its barrier timeout."""
import numpy as np
import pytest

from paper_2605_19928_gb300 import capi, synth
from test_gpu_parity import _state, kuhn_random, leduc_random, river, turn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2605_19928_gb300 import build as pbuild
    pbuild.build()
    capi.load()
    import torch
    assert torch.cuda.is_available()
    capi.use_torch_allocator()


def turn_runout(seed=54):
    """A turn whose all-in call deals the river with no one left to act: showdowns below a
    chance node read the run-out's reach (the terminal pass zeroes the dealt card's hands)."""
    return turn(24, seed=seed, bet_sizes=(synth.ALL_IN,), max_raises=1)


SINGLE = {
    "river_1081": lambda: synth.river_subgame(seed=0, range_seed=1),  # 136 chunks of 8 hands
    "river_203": lambda: river(203, seed=51),                          # ragged last chunk
    "turn_runout": turn_runout,
    "leduc": lambda: leduc_random(seed=53),
    "kuhn": lambda: kuhn_random(seed=55),
}


def _run(specs, opts, splits):
    tree = capi.cfr_batch_create(specs, opts)
    try:
        for k in splits:
            capi.cfr_iterate(tree, k)
        capi.cfr_sync(tree)
        return _state(tree, len(specs), with_pred=opts.variant == capi.VARIANTS["pcfr+"]), \
            capi.cfr_exploitability(tree, len(specs)), capi.cfr_schedule(tree)
    finally:
        capi.cfr_tree_destroy(tree)


@pytest.mark.parametrize("precision", ["pairs", "single"])
@pytest.mark.parametrize("variant,alternating", [("dcfr", True), ("cfr+", True), ("cfr", False), ("pcfr+", True)])
@pytest.mark.parametrize("case", list(SINGLE))
def test_resident_and_level_schedules_give_the_same_bits(case, precision, variant, alternating):
    specs = [SINGLE[case]()]
    level, expl_l, sch_l = _run(specs, capi.make_opts(variant, alternating=alternating, precision=precision,
                                                      schedule="level"), [7])
    res, expl_r, sch_r = _run(specs, capi.make_opts(variant, alternating=alternating, precision=precision,
                                                    schedule="resident"), [3, 4])  # two launches
    assert sch_l == capi.CFR_SCHEDULE_LEVEL and sch_r == capi.CFR_SCHEDULE_RESIDENT
    assert len(level) == len(res)
    for a, b in zip(level, res):
        assert np.array_equal(a, b)
    # same chunks of 8 hands: the best-response root sums run in the same order
    assert np.array_equal(expl_l[0], expl_r[0]) and np.array_equal(expl_l[1], expl_r[1])


def test_resident_batch_of_small_subgames_gives_the_level_bits():
    """Several subgames in one handle: blocks move between games' board tables."""
    specs = [river(64, seed=52, bet_sizes=(0.33, 0.75, 1.25, synth.ALL_IN), max_raises=4), leduc_random(seed=53),
             river(97, seed=21), kuhn_random(seed=55), turn_runout(seed=57)]
    level, expl_l, _ = _run(specs, capi.make_opts("dcfr", schedule="level"), [9])
    res, expl_r, _ = _run(specs, capi.make_opts("dcfr", schedule="resident"), [1, 8])
    for a, b in zip(level, res):
        assert np.array_equal(a, b)
    assert np.array_equal(expl_l[1], expl_r[1])


def test_resident_converges_like_level_over_a_long_run():
    """300 iterations of the 1081-hand river in one launch: the same bits as 300 graph replays."""
    spec = synth.river_subgame(seed=0, range_seed=1)
    out = []
    for schedule in ("level", "resident"):
        tree = capi.cfr_tree_create(spec, capi.make_opts("dcfr", schedule=schedule))
        try:
            capi.cfr_iterate(tree, 300)
            out.append((capi.cfr_exploitability(tree), capi.cfr_tree_info(tree)[2],
                        capi.cfr_read_values(tree, capi.CFR_READ_AVG_SUM, 0)))
        finally:
            capi.cfr_tree_destroy(tree)
    (e0, n0, s0), (e1, n1, s1) = out
    assert n0 == n1 == 300
    assert np.array_equal(s0, s1) and np.array_equal(e0[0], e1[0]) and np.array_equal(e0[1], e1[1])
    print("exploitability after 300 iterations:", e1[0][0])


def test_resident_reset_starts_over():
    spec = river(203, seed=51)
    tree = capi.cfr_tree_create(spec, capi.make_opts("dcfr", schedule="resident"))
    try:
        capi.cfr_iterate(tree, 5)
        first = _state(tree, 1)
        capi.cfr_reset(tree)
        capi.cfr_iterate(tree, 2)
        capi.cfr_iterate(tree, 3)
        again = _state(tree, 1)
    finally:
        capi.cfr_tree_destroy(tree)
    for a, b in zip(first, again):
        assert np.array_equal(a, b)


def test_resident_refusals():
    # a tree whose hand region does not fit shared memory
    with pytest.raises(capi.CfrError) as e:
        capi.cfr_tree_create(turn(40, seed=54), capi.make_opts("dcfr", schedule="resident"))
    assert e.value.code == capi.CFR_EINVAL
    # more chunks than resident blocks (1081 chunks of one hand)
    with pytest.raises(capi.CfrError) as e:
        capi.cfr_tree_create(synth.river_subgame(seed=0, range_seed=1),
                             capi.make_opts("dcfr", schedule="resident", chunk_hands=1))
    assert e.value.code == capi.CFR_EINVAL
    # depth-limit leaves: no leaf-network stage in the resident launch
    spec = synth.turn_subgame(n_hands=6, seed=5, range_seed=6, bet_sizes=(1.0, synth.ALL_IN), max_raises=1)
    spec.depth_limit = 1
    with pytest.raises(capi.CfrError) as e:
        capi.cfr_tree_create(spec, capi.make_opts("dcfr", schedule="resident"))
    assert e.value.code == capi.CFR_EINVAL


def test_resident_barrier_timeout_reports_etimeout_and_the_context_survives():
    """With the first barrier's poll limit at 0, every block but the last to arrive gives up,
    sets the flag and leaves; the rest see the flag at their next barrier.  No kernel is left
    waiting, the call reports CFR_ETIMEOUT, and the next handle solves normally."""
    spec = river(203, seed=51)
    tree = capi.cfr_tree_create(spec, capi.make_opts("dcfr", schedule="resident"))
    try:
        capi.cfr_sync(tree)
        capi.cfr_debug_first_wait_polls(0)
        try:
            capi.cfr_iterate(tree, 4)
            with pytest.raises(capi.CfrError) as e:
                capi.cfr_sync(tree)
            assert e.value.code == capi.CFR_ETIMEOUT
        finally:
            capi.cfr_debug_first_wait_polls(-1)
    finally:
        capi.cfr_tree_destroy(tree)
    ok = capi.cfr_tree_create(spec, capi.make_opts("dcfr", schedule="resident"))
    try:
        capi.cfr_iterate(ok, 4)
        capi.cfr_sync(ok)
        expl, _ = capi.cfr_exploitability(ok)
        assert np.all(np.isfinite(expl)) and np.all(expl > 0)
    finally:
        capi.cfr_tree_destroy(ok)


def test_discount_table_grows_past_its_first_capacity():
    """A handle's discount table covers 2048 iterations and doubles on demand (the iteration
    graph is recorded again, the resident launch reads the new table): 2100 iterations, in
    one call and in calls that cross the boundary, give the same bits on both schedules."""
    spec = river(64, seed=71)
    out = []
    for schedule, splits in (("level", [2100]), ("level", [2000, 100]), ("resident", [1500, 600]),
                             ("resident", [2100])):
        tree = capi.cfr_tree_create(spec, capi.make_opts("dcfr", schedule=schedule))
        try:
            for k in splits:
                capi.cfr_iterate(tree, k)
            out.append((_state(tree, 1), capi.cfr_exploitability(tree)))
        finally:
            capi.cfr_tree_destroy(tree)
    for state, expl in out[1:]:
        for a, b in zip(out[0][0], state):
            assert np.array_equal(a, b)
        assert np.array_equal(out[0][1][0], expl[0])


def test_autotune_picks_the_resident_layout_for_one_river():
    """The autotuner times every layout of the 1081-hand river; whichever wins, the tuned
    handle's state equals the default one's (the bench's river runs the tuned layout)."""
    spec = synth.river_subgame(seed=0, range_seed=1)
    base = capi.make_opts("dcfr", precision="single")
    best, ms = capi.cfr_autotune([spec], base, iters=20)
    assert ms > 0
    assert best.schedule in (capi.CFR_SCHEDULE_LEVEL, capi.CFR_SCHEDULE_STREAM, capi.CFR_SCHEDULE_WIDE,
                             capi.CFR_SCHEDULE_RESIDENT)
    print("autotuned river layout:", best.schedule, best.chunk_hands, best.term_nodes, ms)
    states = []
    for o in (base, best):
        tree = capi.cfr_tree_create(spec, o)
        try:
            capi.cfr_iterate(tree, 5)
            states.append(_state(tree, 1))
        finally:
            capi.cfr_tree_destroy(tree)
    for a, b in zip(*states):
        assert np.array_equal(a, b)
