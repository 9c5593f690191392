"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI next to the
FP64 oracle on the same seeded inputs and compare them node by node."""
from __future__ import annotations

import numpy as np

from paper_2605_19928_gb300 import capi

# Parity bar.  Regrets, average-strategy sums and counterfactual values must agree to
# 1e-5 relative, measured against the largest magnitude in the same node's vector (a
# relative error per element is ill-posed where values cancel to ~0), with an absolute
# floor of 1e-8 of the pot for nodes whose oracle vector is exactly zero.  Strategies
# follow from regrets by regret matching (Eq. rm), so their tolerance is the regret
# tolerance carried through its derivative (see compare_strategies).
RTOL = 1e-5
FLOOR = 1e-8


def node_paths_gpu(tree, n_nodes, game=0):
    """GPU node id -> action path from the root (child indices)."""
    paths = {0: ()}
    for n in range(1, n_nodes):
        info = capi.cfr_node_info(tree, n, game)
        paths[n] = paths[info["parent"]] + (info["action"],)
    return paths


def node_map(tree, oracle, game=0):
    """List of (gpu node, oracle node, info) for every node; checks the two trees agree."""
    n_nodes, n_hands, _ = capi.cfr_tree_info(tree, game)
    assert n_nodes == oracle.n_nodes
    assert n_hands == oracle.n_hands
    gp = node_paths_gpu(tree, n_nodes, game)
    op = oracle.paths()
    out = []
    oinfo = oracle.nodes()
    for g, path in gp.items():
        o = op[path]
        gi = capi.cfr_node_info(tree, g, game)
        oi = oinfo[o]
        assert gi["type"] == oi["type"], (g, path)
        assert gi["n_actions"] == oi["n_actions"], (g, path)
        if gi["type"] in (capi.CFR_NODE_DECISION, capi.CFR_NODE_FOLD):
            assert gi["player"] == oi["player"]
        assert gi["contrib"] == tuple(oi["contrib"])
        out.append((g, o, gi))
    return out


def close(got, want, rtol=RTOL, floor=0.0, what=""):
    """max |got - want| <= rtol * ||want||_inf + floor; returns the normalised error."""
    scale = float(np.max(np.abs(want))) if np.size(want) else 0.0
    err = float(np.max(np.abs(got - want))) if np.size(want) else 0.0
    assert err <= rtol * scale + floor + 1e-15, f"{what}: max error {err:.3e} vs scale {scale:.3e}"
    return err / scale if scale > 0 else 0.0


def compare_strategies(got, R, what="", plus_part=True):
    """A strategy vs the oracle's normalised positive part of R (regret matching, Eq. rm;
    with plus_part=False, R are average-strategy sums S and the result is S / sum S).

    If R is known to RTOL * ||R||_inf, the normalised vector is known to
    2 * RTOL * ||R||_inf / sum(R+) (its derivative), never tighter than 1e-5 absolute.
    Where the oracle's positive mass is zero any valid distribution is accepted."""
    pos = np.maximum(R, 0.0) if plus_part else R
    tot = pos.sum(axis=0)
    scale = float(np.max(np.abs(R))) if R.size else 0.0
    n_act = R.shape[0]
    want = np.where(tot > 0, pos / np.where(tot > 0, tot, 1.0), 1.0 / n_act)
    assert np.allclose(got.sum(axis=0), 1.0, atol=1e-5), what
    assert (got >= 0).all(), what
    live = tot > 0
    if not live.any():
        return 0.0
    tol = np.maximum(1e-5, 2 * RTOL * scale / tot[live])
    err = np.max(np.abs(got[:, live] - want[:, live]), axis=0)
    bad = err > tol
    assert not bad.any(), f"{what}: strategy error {err[bad].max():.3e} above {tol[bad].min():.3e}"
    return float(np.max(err / tol) * 1e-5)


def compare_state(tree, oracle, mapping, game=0, check_cfv=True, check_strategy=True, pot=None):
    """Compare R, S, the current strategy and both players' last counterfactual values."""
    worst = {"R": 0.0, "S": 0.0, "sigma": 0.0, "cfv": 0.0}
    pot = oracle.spec.pot if pot is None else pot
    floor = FLOOR * pot
    for g, o, info in mapping:
        if info["type"] == capi.CFR_NODE_DECISION:
            R_g = capi.cfr_read_values(tree, capi.CFR_READ_REGRET, g, game=game)
            S_g = capi.cfr_read_values(tree, capi.CFR_READ_AVG_SUM, g, game=game)
            R_o, S_o = oracle.regrets(o), oracle.avg_sums(o)
            worst["R"] = max(worst["R"], close(R_g, R_o, floor=floor, what=f"R node {g}"))
            worst["S"] = max(worst["S"], close(S_g, S_o, what=f"S node {g}"))
            if check_strategy:
                # Predictive CFR+ plays regret matching of R + M (regrets plus prediction)
                R_m = R_o + oracle.prediction(o) if oracle.variant == "pcfr+" else R_o
                sig = capi.cfr_strategy(tree, g, average=False, game=game)
                worst["sigma"] = max(worst["sigma"], compare_strategies(sig, R_m, what=f"sigma node {g}"))
        if check_cfv and stored_cfv(tree, g, info):
            for i in (0, 1):
                v_g = capi.cfr_read_values(tree, capi.CFR_READ_CFV, g, player=i, game=game)
                v_o = oracle.cfv(i, o)
                worst["cfv"] = max(worst["cfv"], close(v_g, v_o, floor=floor, what=f"cfv player {i} node {g}"))
    return worst


def inject(tree, oracle, mapping, game=0, player=None):
    """Load the GPU's R and S (and the Predictive CFR+ prediction) of all decision nodes, or
    of one player's, into the oracle."""
    for g, o, info in mapping:
        if info["type"] == capi.CFR_NODE_DECISION and (player is None or info["player"] == player):
            oracle.set_node_state(o, capi.cfr_read_values(tree, capi.CFR_READ_REGRET, g, game=game),
                                  capi.cfr_read_values(tree, capi.CFR_READ_AVG_SUM, g, game=game))
            if oracle.variant == "pcfr+":
                oracle.set_node_pred(o, capi.cfr_read_values(tree, capi.CFR_READ_PREDICTION, g, game=game))


def stored_cfv(tree, g, info):
    """Whether the handle keeps node g's counterfactual values: the level schedule stores
    every node's, the stream schedule the terminals' and the root's."""
    if capi.cfr_schedule(tree) == capi.CFR_SCHEDULE_LEVEL:
        return True
    return g == 0 or info["type"] in (capi.CFR_NODE_FOLD, capi.CFR_NODE_SHOWDOWN, capi.CFR_NODE_LEAF)


def compare_player(tree, oracle, mapping, player, game=0, pot=None, rtol=RTOL, floor_frac=FLOOR, skip=()):
    """R and S of one player's decision nodes and that player's counterfactual values (not at
    the GPU nodes in `skip`, whose values the handle does not keep)."""
    pot = oracle.spec.pot if pot is None else pot
    floor = floor_frac * pot
    worst = {"R": 0.0, "S": 0.0, "cfv": 0.0}
    for g, o, info in mapping:
        if info["type"] == capi.CFR_NODE_DECISION and info["player"] == player:
            R_g = capi.cfr_read_values(tree, capi.CFR_READ_REGRET, g, game=game)
            S_g = capi.cfr_read_values(tree, capi.CFR_READ_AVG_SUM, g, game=game)
            worst["R"] = max(worst["R"], close(R_g, oracle.regrets(o), rtol, floor=floor, what=f"R node {g}"))
            worst["S"] = max(worst["S"], close(S_g, oracle.avg_sums(o), rtol, what=f"S node {g}"))
            if oracle.variant == "pcfr+":
                M_g = capi.cfr_read_values(tree, capi.CFR_READ_PREDICTION, g, game=game)
                close(M_g, oracle.prediction(o), rtol, floor=floor, what=f"prediction node {g}")
        if g in skip or not stored_cfv(tree, g, info):
            continue
        v_g = capi.cfr_read_values(tree, capi.CFR_READ_CFV, g, player=player, game=game)
        worst["cfv"] = max(worst["cfv"], close(v_g, oracle.cfv(player, o), rtol, floor=floor,
                                               what=f"cfv player {player} node {g}"))
    return worst


def forced_step(tree, oracle, mapping, t, alternating=True, game=0, advance_gpu=True, rtol=RTOL, floor_frac=FLOOR,
                skip=()):
    """Iteration t from identical state.

    The GPU's R and S are loaded into the oracle, then the GPU runs one iteration and the
    oracle runs the same updates.  With alternating updates player 0 is compared first;
    the GPU's new player-0 rows are then loaded into the oracle before player 1's update,
    so each player's update is checked from exactly the state the GPU used.  This keeps
    two correct runs from drifting apart where FP64 and double-float break an exact tie
    between action values differently."""
    inject(tree, oracle, mapping, game)
    if advance_gpu:
        capi.cfr_iterate(tree, 1)
    worst = {}
    if alternating:
        oracle.update_player(0, t)
        w0 = compare_player(tree, oracle, mapping, 0, game, rtol=rtol, floor_frac=floor_frac, skip=skip)
        inject(tree, oracle, mapping, game, player=0)
        oracle.update_player(1, t)
        w1 = compare_player(tree, oracle, mapping, 1, game, rtol=rtol, floor_frac=floor_frac, skip=skip)
        worst = {k: max(w0[k], w1[k]) for k in w0}
    else:
        oracle.update_both(t)
        w0 = compare_player(tree, oracle, mapping, 0, game, rtol=rtol, floor_frac=floor_frac, skip=skip)
        w1 = compare_player(tree, oracle, mapping, 1, game, rtol=rtol, floor_frac=floor_frac, skip=skip)
        worst = {k: max(w0[k], w1[k]) for k in w0}
    oracle.set_iterations(t)
    return worst
