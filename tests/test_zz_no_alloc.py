"""cfr_exploitability_noalloc (static device scratch, no allocation) against cfr_exploitability
on the same solver state, two calls in a row each, through the C ABI.  Collected last so it
also runs after every other test of the session has used the library."""
import numpy as np
import pytest

from paper_2605_19928_gb300 import capi, synth

pytestmark = pytest.mark.gpu

RTOL = 1e-12  # the two differ only in the summation order of the FP64 root reduction


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2605_19928_gb300 import build as pbuild
    pbuild.build()
    capi.load()
    import torch
    assert torch.cuda.is_available()
    capi.use_torch_allocator()


def _both(tree, n_games):
    e_ref, br_ref = capi.cfr_exploitability(tree, n_games)
    expl = np.full(n_games, np.nan)
    br = np.full((n_games, 2), np.nan)
    before = capi.cfr_counters(tree)["device_bytes"]
    capi.cfr_exploitability_noalloc(tree, expl, br)
    assert capi.cfr_counters(tree)["device_bytes"] == before
    return e_ref, br_ref, expl, br


def _check(tree, n_games, pot):
    e_ref, br_ref, expl, br = _both(tree, n_games)
    scale = np.maximum(np.abs(br_ref), 1e-9 * pot)
    assert np.all(np.abs(br - br_ref) <= RTOL * scale), (br, br_ref)
    assert np.allclose(expl, 0.5 * br.sum(axis=1), rtol=0, atol=0)
    assert np.all(np.abs(expl - e_ref) <= RTOL * np.maximum(np.abs(e_ref), 1e-9 * pot))
    return expl


@pytest.mark.parametrize("precision,schedule", [("pairs", "level"), ("single", "level"), ("pairs", "stream"),
                                                ("single", "stream"), ("pairs", "wide"), ("single", "wide"),
                                                ("pairs", "resident"), ("single", "resident")])
def test_noalloc_matches_on_river_two_calls(precision, schedule):
    """Every launch layout leaves the best-response values where the static reduction reads
    them: the per-hand, stream, wide and resident schedules (the last iterates in one
    cooperative launch and runs its exploitability pass with the per-hand kernels)."""
    spec = synth.river_subgame(n_hands=1081, seed=0, range_seed=1)
    tree = capi.cfr_tree_create(spec, capi.make_opts("dcfr", precision=precision, schedule=schedule))
    try:
        capi.cfr_iterate(tree, 30)
        e1 = _check(tree, 1, spec.pot)
        e1_again = _check(tree, 1, spec.pot)   # second call in a row, same state
        assert e1_again[0] == e1[0]
        capi.cfr_iterate(tree, 20)
        e2 = _check(tree, 1, spec.pot)
        assert e2[0] != e1[0]
    finally:
        capi.cfr_tree_destroy(tree)


def test_noalloc_matches_on_batch_two_calls():
    specs = [synth.river_subgame(n_hands=n, seed=s, range_seed=s + 1) for n, s in ((1081, 2), (203, 3), (64, 4))]
    leduc = synth.leduc()
    leduc.ranges[:] = synth.random_ranges(6, 11)
    specs.append(leduc)
    tree = capi.cfr_batch_create(specs, capi.make_opts("dcfr"))
    try:
        for _ in range(2):
            capi.cfr_iterate(tree, 10)
            _check(tree, len(specs), 100.0)
            _check(tree, len(specs), 100.0)
    finally:
        capi.cfr_tree_destroy(tree)


def test_noalloc_rejects_handles_beyond_its_scratch():
    # 8 rivers at one hand per chunk: 8 * 1081 = 8648 chunks per player > 8192
    specs = [synth.river_subgame(n_hands=1081, seed=s, range_seed=s + 1, max_raises=1) for s in range(8)]
    tree = capi.cfr_batch_create(specs, capi.make_opts("dcfr", chunk_hands=1))
    try:
        expl = np.zeros(8)
        br = np.zeros((8, 2))
        with pytest.raises(capi.CfrError) as ei:
            capi.cfr_exploitability_noalloc(tree, expl, br)
        assert ei.value.code == capi.CFR_EINVAL
        assert "8192" in str(ei.value)
        # the handle still works through the allocating entry point
        e, _ = capi.cfr_exploitability(tree, 8)
        assert np.all(np.isfinite(e))
    finally:
        capi.cfr_tree_destroy(tree)


def _random_net(seed):
    """A random leaf network as BF16 bit patterns (weights) and FP32 biases."""
    from oracle.leafnet import bf16_bits
    rng = np.random.default_rng(seed)
    W, b = [], []
    for k, shape in enumerate(capi.LEAF_SHAPES):
        w = rng.standard_normal(shape).astype(np.float32) * np.float32(2.0 / np.sqrt(shape[1]))
        W.append(bf16_bits(w * (0.2 if k == 3 else 1.0)))
        b.append(rng.standard_normal(shape[0]).astype(np.float32) * 0.05)
    return W, b


@pytest.mark.parametrize("schedule", ["level", "stream", "wide"])
def test_noalloc_matches_with_depth_limit_leaves(schedule):
    """A depth-limited turn (network leaves at the river card): the call also runs the leaf
    network under the average strategy, and counts its launches as the allocating pass
    does (plus its one reduction kernel)."""
    spec = synth.turn_subgame(n_hands=40, seed=5, range_seed=6, bet_sizes=(1.0, synth.ALL_IN), max_raises=2)
    spec.depth_limit = 1
    tree = capi.cfr_tree_create(spec, capi.make_opts("dcfr", schedule=schedule))
    try:
        W, b = _random_net(3)
        capi.cfr_set_leaf_net(tree, W, b)
        capi.cfr_iterate(tree, 6)
        for _ in range(2):
            l0 = capi.cfr_counters(tree)["kernel_launches"]
            e_ref, br_ref = capi.cfr_exploitability(tree, 1)
            l1 = capi.cfr_counters(tree)["kernel_launches"]
            _check(tree, 1, spec.pot)
            l2 = capi.cfr_counters(tree)["kernel_launches"]
            # _check runs cfr_exploitability once more, then the call itself
            assert (l2 - l1) - (l1 - l0) == (l1 - l0) + 1
    finally:
        capi.cfr_tree_destroy(tree)
