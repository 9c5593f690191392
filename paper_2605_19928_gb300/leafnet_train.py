"""Train the depth-limit leaf network on river subgames solved by this library.

    python -m paper_2605_19928_gb300.leafnet_train --samples 100000 --out leafnet_weights.npz

Data (Section 3: the network maps both players' normalised reach and the public state to
counterfactual values): seeded river subgames (synth.leaf_training_rivers: rank-based
showdowns, thinned Dirichlet ranges, pots and chips behind spanning those of turn leaves),
256 at a time in one batched handle, solved by DCFR on the GPU.  Each solve gives one
example per subgame: the input row the leaf kernels build (both ranges over the 1326 card
slots, the 5-card board one-hot, the pot / stack features) and, per player and hand, the
best-response value against the solution divided by pot x (opponent reach sharing no card)
x kappa, i.e. the value per unit pot that the leaf kernels multiply back.  With
--turn-solves, exact turn subgames (synth.leaf_training_turns) are solved too and every
river-card node below a leaf position gives one more example with the ranges the turn's
solution brings there (turn_leaf_examples): the states the network meets in depth-limited
solves.

Training is offline model fitting with PyTorch autograd (Adam, Huber loss on the slots of
hands that exist); the serving path is the library's own kernels (cfr_set_leaf_net).  The
weights are written BF16-rounded (uint16 bit patterns) with FP32 biases.
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2605_19928_gb300 import capi, synth  # noqa: E402

SLOTS, IN, OUT = 1326, 2752, 2688


def slot_of(hands: np.ndarray) -> np.ndarray:
    a, b = np.minimum(hands[:, 0], hands[:, 1]).astype(np.int64), np.maximum(hands[:, 0], hands[:, 1]).astype(np.int64)
    return b * (b - 1) // 2 + a


def bf16(x: np.ndarray) -> np.ndarray:
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32).view(np.float32)


def example(spec, v_root) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """(input row, target row, target mask) of one solved river subgame; v_root[i] is player
    i's root value per hand (counterfactual, kappa = 1/Z included)."""
    hands = spec.hands.astype(np.int64)
    sl = slot_of(hands)
    r = spec.ranges.astype(np.float64)
    r = r / r.sum(axis=1, keepdims=True)
    x = np.zeros(IN, np.float32)
    x[sl] = r[0]
    x[SLOTS + sl] = r[1]
    x[2 * SLOTS + spec.board] = 1.0
    pot, behind = float(spec.pot), float(spec.stack)
    x[2 * SLOTS + 52] = pot / (pot + 2 * behind)
    x[2 * SLOTS + 53] = behind / (pot + 2 * behind)
    # opponent reach sharing no card with each hand (inclusion-exclusion) and Z
    y = np.zeros(OUT, np.float32)
    m = np.zeros(OUT, np.float32)
    cm = np.zeros((hands.shape[0], 52), np.float64)
    cm[np.arange(hands.shape[0])[:, None], hands] = 1.0
    M = []
    for i in (0, 1):
        q = r[1 - i]
        C = cm.T @ q
        M.append(q.sum() - C[hands[:, 0]] - C[hands[:, 1]] + q)
    Z = float(np.dot(r[0], M[0]))  # sum of r0 r1 over pairs of hands sharing no card
    for i in (0, 1):
        ok = M[i] > 1e-12
        val = np.zeros(hands.shape[0])
        val[ok] = v_root[i][ok] * Z / (pot * M[i][ok])
        y[i * SLOTS + sl] = val
        m[i * SLOTS + sl] = ok
    return x, y, m


def generate(n: int, iters: int, seed: int, log=print):
    """n examples from n river solves (DCFR, FP32 values, `iters` iterations each)."""
    X = np.zeros((n, IN), np.float32)
    Y = np.zeros((n, OUT), np.float32)
    Mk = np.zeros((n, OUT), np.float32)
    opts = capi.make_opts("dcfr", precision="single")
    done, t0, chunk, expl = 0, time.time(), 0, []
    while done < n:
        k = min(256, n - done)
        specs = synth.leaf_training_rivers(k, seed=seed * 100_000 + chunk)
        tree = capi.cfr_batch_create(specs, opts)
        try:
            capi.cfr_iterate(tree, iters)
            e, _ = capi.cfr_exploitability(tree, k)
            expl.extend((1000.0 * e / 100.0).tolist())
            for g, spec in enumerate(specs):
                v = [capi.cfr_read_values(tree, capi.CFR_READ_BR_CFV, 0, player=i, game=g) for i in (0, 1)]
                X[done + g], Y[done + g], Mk[done + g] = example(spec, v)
        finally:
            capi.cfr_tree_destroy(tree)
        done += k
        chunk += 1
        if chunk % 20 == 0:
            log(f"  {done} solves, {time.time() - t0:.0f} s, median exploitability {np.median(expl):.3f} mbb")
    return bf16(X), Y, Mk, float(np.median(expl))


def turn_leaf_examples(spec, tree):
    """Examples at the river-card nodes of a solved exact turn subgame: below every river
    chance node with chips behind (where a depth-limited solve puts a leaf), the input row
    the leaf kernels build from both players' reach under the average strategy, and per
    player and hand the best-response value against it, per unit pot (divided by pot x
    kappa / 44 x the opponent reach sharing no card with the hand)."""
    n_nodes = capi.cfr_tree_info(tree)[0]
    infos = [capi.cfr_node_info(tree, n) for n in range(n_nodes)]
    kids = {}
    for n in range(1, n_nodes):
        kids.setdefault(infos[n]["parent"], []).append(n)
    hands = spec.hands.astype(np.int64)
    sl = slot_of(hands)
    r = spec.ranges.astype(np.float64)
    r = r / r.sum(axis=1, keepdims=True)
    cm = np.zeros((hands.shape[0], 52), np.float64)
    cm[np.arange(hands.shape[0])[:, None], hands] = 1.0

    def blocker_free(q):  # opponent reach sharing no card with each hand
        C = cm.T @ q
        return q.sum() - C[hands[:, 0]] - C[hands[:, 1]] + q

    Z = float(np.dot(r[0], blocker_free(r[1])))
    cap = spec.pot / 2 + spec.stack
    xs, ys, ms = [], [], []
    for n, info in enumerate(infos):
        if info["type"] != capi.CFR_NODE_CHANCE or max(info["contrib"]) >= cap:
            continue
        pot, behind = info["contrib"][0] + info["contrib"][1], cap - info["contrib"][0]
        for kid in kids.get(n, []):
            card = infos[kid]["deal"]
            q = [capi.cfr_read_values(tree, capi.CFR_READ_AVG_REACH, kid, player=p) for p in (0, 1)]
            if min(q[0].sum(), q[1].sum()) <= 0.0:
                continue
            v = [capi.cfr_read_values(tree, capi.CFR_READ_BR_CFV, kid, player=i) for i in (0, 1)]
            x = np.zeros(IN, np.float32)
            for p in (0, 1):
                x[p * SLOTS + sl] = q[p] / q[p].sum()
            x[2 * SLOTS + spec.board] = 1.0
            x[2 * SLOTS + card] = 1.0
            x[2 * SLOTS + 52] = pot / (pot + 2 * behind)
            x[2 * SLOTS + 53] = behind / (pot + 2 * behind)
            live = ~np.any(hands == card, axis=1)
            y = np.zeros(OUT, np.float32)
            m = np.zeros(OUT, np.float32)
            for i in (0, 1):
                M = blocker_free(q[1 - i])
                ok = live & (M > 1e-12 * q[1 - i].sum())
                val = np.zeros(hands.shape[0])
                val[ok] = v[i][ok] * Z * 44.0 / (pot * M[ok])
                y[i * SLOTS + sl] = val
                m[i * SLOTS + sl] = ok
            xs.append(x)
            ys.append(y)
            ms.append(m)
    return xs, ys, ms


def generate_turns(n_solves: int, iters: int, seed: int, log=print):
    """Leaf examples from n_solves exact turn solves (DCFR, FP32 values, `iters` iterations)."""
    opts = capi.make_opts("dcfr", precision="single")
    X, Y, Mk, expl = [], [], [], []
    t0 = time.time()
    for k, spec in enumerate(synth.leaf_training_turns(n_solves, seed=seed)):
        tree = capi.cfr_tree_create(spec, opts)
        try:
            capi.cfr_iterate(tree, iters)
            e, _ = capi.cfr_exploitability(tree)
            expl.append(1000.0 * float(e[0]) / 100.0)
            xs, ys, ms = turn_leaf_examples(spec, tree)
            X += xs
            Y += ys
            Mk += ms
        finally:
            capi.cfr_tree_destroy(tree)
        if (k + 1) % 25 == 0:
            log(f"  {k + 1} turn solves, {len(X)} leaf examples, {time.time() - t0:.0f} s, "
                f"median exploitability {np.median(expl):.3f} mbb")
    return bf16(np.array(X, np.float32)), np.array(Y, np.float32), np.array(Mk, np.float32), float(np.median(expl))


def train(X, Y, Mk, epochs: int, seed: int, log=print):
    import torch
    torch.manual_seed(seed)
    dev = torch.device("cuda")
    n = X.shape[0]
    n_val = max(1, n // 20)
    Xt, Yt, Mt = (torch.from_numpy(a).to(dev) for a in (X, Y, Mk))
    net = torch.nn.Sequential(torch.nn.Linear(IN, 512), torch.nn.GELU(), torch.nn.Linear(512, 512), torch.nn.GELU(),
                              torch.nn.Linear(512, 512), torch.nn.GELU(), torch.nn.Linear(512, OUT)).to(dev)
    opt = torch.optim.Adam(net.parameters(), lr=1e-3)
    steps = epochs * ((n - n_val) // 1024 + 1)
    sched = torch.optim.lr_scheduler.OneCycleLR(opt, max_lr=1e-3, total_steps=steps)

    def loss_of(xb, yb, mb):
        out = net(xb)
        return (torch.nn.functional.huber_loss(out * mb, yb * mb, reduction="sum", delta=0.5) /
                mb.sum().clamp_min(1.0))

    for ep in range(epochs):
        perm = torch.randperm(n - n_val, device=dev) + n_val
        net.train()
        for s in range(0, n - n_val, 1024):
            idx = perm[s:s + 1024]
            opt.zero_grad()
            loss = loss_of(Xt[idx], Yt[idx], Mt[idx])
            loss.backward()
            opt.step()
            sched.step()
        net.eval()
        with torch.no_grad():
            out = net(Xt[:n_val])
            mae = float(((out - Yt[:n_val]).abs() * Mt[:n_val]).sum() / Mt[:n_val].sum())
        if ep % 5 == 4 or ep == epochs - 1:
            log(f"  epoch {ep + 1}: train loss {float(loss.detach()):.4f}, validation mean |error| {mae:.4f} pot")
    layers = [m for m in net if isinstance(m, torch.nn.Linear)]
    W = [bf16(l.weight.detach().float().cpu().numpy()) for l in layers]
    b = [l.bias.detach().float().cpu().numpy() for l in layers]
    Wbits = [(w.view(np.uint32) >> 16).astype(np.uint16) for w in W]
    return Wbits, b, mae


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--samples", type=int, default=100_000, help="river solves (one example each)")
    ap.add_argument("--turn-solves", type=int, default=0,
                    help="exact turn solves whose river-card nodes give leaf examples (many each)")
    ap.add_argument("--iters", type=int, default=300)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "leafnet_weights.npz"))
    args = ap.parse_args(argv)
    import torch
    capi.load()
    capi.use_torch_allocator()
    t0 = time.time()
    X, Y, Mk, med = generate(args.samples, args.iters, args.seed)
    t1 = time.time()
    print(f"generated {args.samples} river solves in {t1 - t0:.0f} s (median exploitability {med:.3f} mbb/hand)")
    n_turn = 0
    if args.turn_solves > 0:
        Xt, Yt, Mt, med_t = generate_turns(args.turn_solves, args.iters, args.seed)
        n_turn = Xt.shape[0]
        print(f"generated {n_turn} leaf examples from {args.turn_solves} turn solves in {time.time() - t1:.0f} s "
              f"(median exploitability {med_t:.3f} mbb/hand)")
        # interleave so that the validation slice (the first 5 %) holds both kinds
        X, Y, Mk = (np.concatenate([a, b]) for a, b in ((X, Xt), (Y, Yt), (Mk, Mt)))
        order = np.random.default_rng(args.seed).permutation(X.shape[0])
        X, Y, Mk = X[order], Y[order], Mk[order]
        t1 = time.time()
    Wbits, b, mae = train(X, Y, Mk, args.epochs, args.seed)
    t2 = time.time()
    print(f"trained in {t2 - t1:.0f} s, validation mean |error| {mae:.4f} of the pot")
    np.savez_compressed(args.out, **{f"W{k}": w for k, w in enumerate(Wbits)}, **{f"b{k}": x for k, x in enumerate(b)},
                        meta=np.array([args.samples, args.iters, args.epochs, args.seed, med, mae, args.turn_solves,
                                       n_turn], np.float64))
    torch.cuda.synchronize()
    print("wrote", args.out)


def load_weights(path: str | None = None):
    """(W, b) lists for capi.cfr_set_leaf_net from a file written by main()."""
    path = path or os.path.join(os.path.dirname(os.path.abspath(__file__)), "leafnet_weights.npz")
    d = np.load(path)
    return [d[f"W{k}"] for k in range(4)], [d[f"b{k}"] for k in range(4)]


if __name__ == "__main__":
    main()
