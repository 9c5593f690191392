"""Depth-limited subgames with some leaves solved exactly (no GPU): the per-leaf fallback's
trees.  A leaf is named by its index in the breadth-first order of the depth-limited tree
(by action-path length, then lexicographically); naming it expands that position into the
river-card chance node with its exact river subtrees, as the full-depth tree has there.
Checked on the oracle's trees against the full-depth and depth-limited trees built with no
exact leaves; the host builder's mixed trees are compared with the oracle's node by node
in tests/test_host_tree.py."""
import dataclasses

import pytest

from paper_2605_19928_gb300 import synth


def turn6():
    spec = synth.turn_subgame(n_hands=6, seed=5, range_seed=6, bet_sizes=(1.0, synth.ALL_IN), max_raises=1)
    spec.depth_limit = 1
    return spec


def flop4():
    spec = synth.flop_subgame(n_hands=4, seed=3, range_seed=4, bet_sizes=(synth.ALL_IN,), max_raises=1)
    spec.depth_limit = 1
    return spec


def by_path(o):
    """{action path: node info} of an oracle tree."""
    info = o.nodes()
    return {p: info[n] for p, n in o.paths().items()}


def leaf_paths_bfs(o):
    """Leaf paths in the breadth-first order that names leaves."""
    return sorted((p for p, nd in by_path(o).items() if nd["type"] == 4), key=lambda p: (len(p), p))


def same_node(a, b):
    return (a["type"], a["n_actions"], a["player"] if a["type"] in (0, 1) else -1, a["deal"], a["contrib"]) == \
           (b["type"], b["n_actions"], b["player"] if b["type"] in (0, 1) else -1, b["deal"], b["contrib"])


@pytest.mark.parametrize("make", [turn6, flop4])
def test_every_leaf_exact_is_the_full_depth_tree(oracle_mod, make):
    spec = make()
    pure = oracle_mod.Oracle(spec, threads=1)
    n_leaves = len(leaf_paths_bfs(pure))
    assert n_leaves > 1
    mixed = oracle_mod.Oracle(dataclasses.replace(spec, exact_leaves=tuple(range(n_leaves))), threads=1)
    full = oracle_mod.Oracle(dataclasses.replace(spec, depth_limit=0), threads=1)
    a, b = by_path(mixed), by_path(full)
    assert a.keys() == b.keys()
    assert all(same_node(a[p], b[p]) for p in a)


@pytest.mark.parametrize("make", [turn6, flop4])
def test_one_exact_leaf_expands_that_position_only(oracle_mod, make):
    spec = make()
    pure = oracle_mod.Oracle(spec, threads=1)
    full = by_path(oracle_mod.Oracle(dataclasses.replace(spec, depth_limit=0), threads=1))
    leaves = leaf_paths_bfs(pure)
    for k in sorted({0, len(leaves) // 2, len(leaves) - 1}):
        mixed = by_path(oracle_mod.Oracle(dataclasses.replace(spec, exact_leaves=(k,)), threads=1))
        assert leaf_paths_bfs_from(mixed) == leaves[:k] + leaves[k + 1:]
        root = leaves[k]
        below = {p: nd for p, nd in full.items() if p[:len(root)] == root}
        assert mixed[root]["type"] == 3 and below[root]["type"] == 3  # the river-card chance node
        assert all(p in mixed and same_node(mixed[p], nd) for p, nd in below.items())
        # everything else is the depth-limited tree
        rest = {p: nd for p, nd in by_path(pure).items() if p[:len(root)] != root}
        assert all(same_node(mixed[p], nd) for p, nd in rest.items())
        assert len(mixed) == len(rest) + len(below)


def leaf_paths_bfs_from(tree_by_path):
    return sorted((p for p, nd in tree_by_path.items() if nd["type"] == 4), key=lambda p: (len(p), p))


def test_exact_leaves_must_name_distinct_leaves(oracle_mod):
    spec = turn6()
    n = len(leaf_paths_bfs(oracle_mod.Oracle(spec, threads=1)))
    for bad in ((n,), (-1,), (0, 0)):
        with pytest.raises(ValueError):
            oracle_mod.Oracle(dataclasses.replace(spec, exact_leaves=bad), threads=1)
