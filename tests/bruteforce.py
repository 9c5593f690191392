"""Independent brute-force poker games, written from the games' rules.

Histories are explicit tuples of tokens ('k' check, 'c' call, 'f' fold, ('b', amount) bet
or raise to `amount` chips, ('d', card) public card dealt).  Nothing here is shared with the
oracle or the CUDA path.  Every quantity is computed from its definition by enumerating
histories, which pins the oracle's tree rules, utilities, chance weights, counterfactual
values (Section 3, Eq. cfv), regrets (Section 3), regret matching (Section 3, Eq. rm) and
best responses on games small enough to enumerate.

Counterfactual weighting: a subgame starts with a chance deal of (h0, h1) with probability
r0(h0) r1(h1) / Z over pairs that share no card.  Player i's own r_i(h_i) counts as player
i's reach; the counterfactual weight of a history is r_{-i}(h_{-i}) / Z times the
opponent's action probabilities times the public-card chance probabilities.
"""
from __future__ import annotations

import itertools

import numpy as np

KUHN, LEDUC, HOLDEM = "kuhn", "leduc", "holdem"


class Game:
    """Heads-up poker subgame: Kuhn, Leduc, or a hold'em flop/turn/river subgame."""

    def __init__(self, kind, hands=None, ranges=None, board=(), strength=None, pot=2.0, stack=0.0,
                 sizes=(), max_raises=1):
        self.kind = kind
        if kind == KUHN:
            self.deck, self.hands, self.n_streets = 3, [(c,) for c in range(3)], 1
            self.bets, self.max_raises, self.base = [1.0], 1, 1.0
        elif kind == LEDUC:
            self.deck, self.hands, self.n_streets = 6, [(c,) for c in range(6)], 2
            self.bets, self.max_raises, self.base = [2.0, 4.0], 2, 1.0
        else:
            self.deck, self.hands = 52, [tuple(int(c) for c in h) for h in hands]
            self.n_streets = 6 - len(board)  # river 1, turn 2, flop 3
            self.bets, self.max_raises, self.base = None, max_raises, pot / 2.0
            self.cap = pot / 2.0 + stack
            self.sizes = list(sizes)
            self.strength = np.asarray(strength)
        self.board0 = tuple(int(c) for c in board)
        n = len(self.hands)
        if ranges is None:
            ranges = np.full((2, n), 1.0 / n)
        r = np.asarray(ranges, dtype=np.float64)
        self.r = r / r.sum(axis=1, keepdims=True)
        self.Z = sum(self.r[0][a] * self.r[1][b] for a in range(n) for b in range(n) if self.compatible(a, b))

    # ------------------------------------------------------------ cards
    def compatible(self, a, b):
        return not (set(self.hands[a]) & set(self.hands[b]))

    def deals(self):
        n = len(self.hands)
        return [(a, b) for a in range(n) for b in range(n) if self.compatible(a, b)]

    # ------------------------------------------------------------ betting state
    def state(self, hist):
        c = [self.base, self.base]
        street, to_act, raises, street_acts = 0, 0, 0, []
        board = list(self.board0)
        folded = -1
        for tok in hist:
            if tok[0] == "d":
                board.append(tok[1])
                street, to_act, raises, street_acts = street + 1, 0, 0, []
                continue
            p = to_act
            if tok == "c":
                c[p] = c[1 - p]
            elif tok == "f":
                folded = p
            elif tok[0] == "b":
                c[p] = tok[1]
                raises += 1
            street_acts.append(tok)
            to_act = 1 - p
        over = bool(street_acts) and (street_acts[-1] == "c" or street_acts[-2:] == ["k", "k"])
        if not street_acts and street > 0 and self.kind == HOLDEM and max(c) >= self.cap:
            over = True  # all-in: no betting on later streets
        return dict(c=c, street=street, to_act=to_act, raises=raises, board=board, folded=folded, over=over)

    def legal(self, hist):
        s = self.state(hist)
        c, p = s["c"], s["to_act"]
        facing = c[1 - p] > c[p]
        acts = ["f", "c"] if facing else ["k"]
        if s["raises"] < self.max_raises:
            if self.kind != HOLDEM:
                acts.append(("b", c[1 - p] + self.bets[s["street"]]))
            elif c[1 - p] < self.cap and c[p] < self.cap:
                d = c[1 - p] - c[p]
                pot = c[0] + c[1]
                targets = []
                for x in self.sizes:
                    t = self.cap if x <= 0 else min(c[p] + (d + x * (pot + d)), self.cap)
                    if t not in targets and t > c[1 - p]:
                        targets.append(t)
                acts += [("b", t) for t in sorted(targets)]
        return acts

    def strength_of(self, h, board):
        if self.kind == KUHN:
            return self.hands[h][0]
        if self.kind == LEDUC:
            r, br = self.hands[h][0] // 2, board[0] // 2
            return 10 + r if r == br else r
        if len(self.board0) == 5:
            row = 0
        elif len(self.board0) == 4:
            row = board[4]
        else:
            row = board[3] * 52 + board[4]
        return int(self.strength[row][h])

    def utility(self, hands, hist, i):
        """u_i at a terminal history, else None."""
        s = self.state(hist)
        c = s["c"]
        if s["folded"] >= 0:
            f = s["folded"]
            return -c[i] if f == i else c[f]
        if s["over"] and s["street"] == self.n_streets - 1:
            si = self.strength_of(hands[i], s["board"])
            so = self.strength_of(hands[1 - i], s["board"])
            return c[1 - i] if si > so else (-c[i] if si < so else 0.0)
        return None

    def chance_cards(self, hands, hist):
        """Live public cards when the betting round is over and a card is to come, else None."""
        s = self.state(hist)
        if s["folded"] >= 0 or not s["over"] or s["street"] == self.n_streets - 1:
            return None
        dead = set(s["board"]) | set(self.hands[hands[0]]) | set(self.hands[hands[1]])
        return [x for x in range(self.deck) if x not in dead]


class Profile:
    """Behaviour strategy: infoset key -> list of action probabilities; missing = uniform."""

    def __init__(self, table=None):
        self.table = dict(table or {})

    def probs(self, key, n):
        return self.table.get(key, [1.0 / n] * n)


def infoset_key(player, hand, hist):
    return (player, hand, tuple(hist))


def expected_utility(g, prof, hands, hist, i, memo=None):
    """E[u_i | history] under the profile, chance below the history included.

    `memo` caches results for one fixed profile."""
    if memo is not None:
        key = (hands, hist, i)
        if key in memo:
            return memo[key]
    u = g.utility(hands, hist, i)
    if u is not None:
        out = float(u)
    else:
        live = g.chance_cards(hands, hist)
        if live is not None:
            out = sum(expected_utility(g, prof, hands, hist + (("d", x),), i, memo) for x in live) / len(live)
        else:
            p = g.state(hist)["to_act"]
            acts = g.legal(hist)
            pr = prof.probs(infoset_key(p, hands[p], hist), len(acts))
            out = sum(pr[k] * expected_utility(g, prof, hands, hist + (a,), i, memo) for k, a in enumerate(acts))
    if memo is not None:
        memo[key] = out
    return out


def decision_histories(g, prof):
    """(hands, hist, pi0, pi1, pc) for every decision history; pi_i excludes the deal."""
    out = []

    def rec(hands, hist, pi, pc):
        if g.utility(hands, hist, 0) is not None:
            return
        live = g.chance_cards(hands, hist)
        if live is not None:
            for x in live:
                rec(hands, hist + (("d", x),), pi, pc / len(live))
            return
        out.append((hands, hist, pi[0], pi[1], pc))
        p = g.state(hist)["to_act"]
        acts = g.legal(hist)
        pr = prof.probs(infoset_key(p, hands[p], hist), len(acts))
        for k, a in enumerate(acts):
            npi = list(pi)
            npi[p] *= pr[k]
            rec(hands, hist + (a,), npi, pc)

    for h0, h1 in g.deals():
        rec((h0, h1), (), [1.0, 1.0], 1.0)
    return out


def regrets_and_values(g, prof, i):
    """r_i(I, a) = v_i(sigma_{I->a}, I) - v_i(sigma, I) and v_i(sigma, I) for player i."""
    reg, val = {}, {}
    memo = {}
    for hands, hist, pi0, pi1, pc in decision_histories(g, prof):
        if g.state(hist)["to_act"] != i:
            continue
        key = infoset_key(i, hands[i], hist)
        w = g.r[1 - i][hands[1 - i]] / g.Z * (pi1 if i == 0 else pi0) * pc
        eu = expected_utility(g, prof, hands, hist, i, memo)
        val[key] = val.get(key, 0.0) + w * eu
        acts = g.legal(hist)
        r = reg.setdefault(key, [0.0] * len(acts))
        for k, a in enumerate(acts):
            r[k] += w * (expected_utility(g, prof, hands, hist + (a,), i, memo) - eu)
    return reg, val


def own_reach(g, prof, i):
    """pi_i(I), including player i's range weight r_i(h_i)."""
    out = {}
    for hands, hist, pi0, pi1, pc in decision_histories(g, prof):
        if g.state(hist)["to_act"] == i:
            out[infoset_key(i, hands[i], hist)] = g.r[i][hands[i]] * (pi0 if i == 0 else pi1)
    return out


def regret_matching(R):
    table = {}
    for key, ra in R.items():
        pos = [max(v, 0.0) for v in ra]
        s = sum(pos)
        table[key] = [x / s if s > 0 else 1.0 / len(ra) for x in pos]
    return Profile(table)


def profile_value(g, prof, i=0):
    memo = {}
    return sum(g.r[0][h0] * g.r[1][h1] / g.Z * expected_utility(g, prof, (h0, h1), (), i, memo)
               for h0, h1 in g.deals())


def run_cfr(g, iterations, variant="cfr", alpha=1.5, beta=0.0, gamma=2.0, alternating=True):
    """CFR by definition: regrets from profile deviations, then the variant update.
    Predictive CFR+ ("pcfr+") plays regret matching on R + M with M the last instantaneous
    regret, keeps R non-negative and weighs the average by t^2."""
    R, S, M = {}, {}, {}

    def strategy():
        if variant != "pcfr+":
            return regret_matching(R)
        return regret_matching({k: [R[k][a] + M.get(k, [0.0] * len(R[k]))[a] for a in range(len(R[k]))] for k in R})

    for t in range(1, iterations + 1):
        ta, tb = t ** alpha, t ** beta
        dpos, dneg, dS = ta / (ta + 1.0), tb / (tb + 1.0), (t / (t + 1.0)) ** gamma
        players = [0, 1]
        snap = strategy() if not alternating else None
        for i in players:
            prof = strategy() if alternating else snap
            reg, _ = regrets_and_values(g, prof, i)
            reach = own_reach(g, prof, i)
            for key, r in reg.items():
                old = R.get(key, [0.0] * len(r))
                new = []
                for a in range(len(r)):
                    x = old[a] + r[a]
                    if variant == "dcfr":
                        x *= dpos if x > 0 else dneg
                    if variant in ("cfr+", "pcfr+"):
                        x = max(x, 0.0)
                    new.append(x)
                R[key] = new
                if variant == "pcfr+":
                    M[key] = list(r)
            for key, pi in reach.items():
                n = len(reg[key])
                sig = prof.probs(key, n)
                old = S.get(key, [0.0] * n)
                wS = {"cfr+": float(t), "pcfr+": float(t) * t}.get(variant, 1.0)
                S[key] = [(old[a] * (dS if variant == "dcfr" else 1.0)) + wS * pi * sig[a] for a in range(n)]
    return R, S


def average_profile(S):
    table = {}
    for key, s in S.items():
        tot = sum(s)
        table[key] = [x / tot if tot > 0 else 1.0 / len(s) for x in s]
    return Profile(table)


def kuhn_pure_strategies(player):
    """All 2^6 pure strategies of a Kuhn player, as infoset -> action probabilities."""
    hists = [(), ("k", ("b", 2.0))] if player == 0 else [("k",), (("b", 2.0),)]
    slots = [(card, h) for card in range(3) for h in hists]
    for choice in itertools.product([0, 1], repeat=len(slots)):
        yield {infoset_key(player, card, h): [float(k == c) for k in range(2)] for (card, h), c in zip(slots, choice)}


def kuhn_best_response_bruteforce(opp_profile, i):
    """max over the 64 pure strategies of player i of E[u_i] against the opponent profile."""
    g = Game(KUHN)
    best = -1e300
    for table in kuhn_pure_strategies(i):
        merged = dict(opp_profile.table)
        merged.update(table)
        best = max(best, profile_value(g, Profile(merged), i))
    return best


# ------------------------------------------------------------ hold'em best response and reach

def pure_best_response(g, prof, i):
    """Best-response value of player i by definition: the largest expected utility of player
    i over every pure strategy (one action at each of its infosets), the opponent playing
    `prof`.  Only for games with a handful of infosets."""
    keys = sorted({infoset_key(i, hands[i], hist) for hands, hist, *_ in decision_histories(g, prof)
                   if g.state(hist)["to_act"] == i}, key=repr)
    n_acts = [len(g.legal(k[2])) for k in keys]
    best = -1e300
    for choice in itertools.product(*[range(a) for a in n_acts]):
        table = dict(prof.table)
        table.update({k: [float(j == c) for j in range(a)] for k, a, c in zip(keys, n_acts, choice)})
        best = max(best, profile_value(g, Profile(table), i))
    return best


def best_response(g, prof, i):
    """Best response of player i against the opponent's behaviour in `prof`, as a maximum at
    each of player i's infosets (own hand h, public history).  The value of an infoset is the
    sum, over the opponent's hands o that share no card with h and over the public cards to
    come, of u_i weighted by r_{-i}(o) / Z, the opponent's action probabilities and the
    chance probability of each card -- 1 / (live cards of the pair (h, o)), a card held by o
    not being dealt to that pair at all.  Returns (BR_i, {(h, hist): v*_i(h, hist)}) with
    BR_i = sum_h r_i(h) v*_i(h, ()); histories below a card that h holds get no entry."""
    n = len(g.hands)
    vals = {}

    def pair(h, o):
        return (h, o) if i == 0 else (o, h)

    def rec(h, hist, w):
        if not w:
            vals[(h, hist)] = 0.0
            return 0.0
        o0 = next(iter(w))
        u = g.utility(pair(h, o0), hist, i)
        if u is not None:
            v = sum(wo * g.utility(pair(h, o), hist, i) for o, wo in w.items())
        elif g.chance_cards(pair(h, o0), hist) is not None:
            s = g.state(hist)
            v = 0.0
            for x in range(g.deck):
                if x in s["board"] or x in g.hands[h]:
                    continue
                w2 = {}
                for o, wo in w.items():
                    live = g.chance_cards(pair(h, o), hist)
                    if x in live:
                        w2[o] = wo / len(live)
                v += rec(h, hist + (("d", x),), w2)
        else:
            s = g.state(hist)
            acts = g.legal(hist)
            if s["to_act"] == i:
                v = max(rec(h, hist + (a,), w) for a in acts)
            else:
                v = 0.0
                for k, a in enumerate(acts):
                    w2 = {o: wo * prof.probs(infoset_key(1 - i, o, hist), len(acts))[k] for o, wo in w.items()}
                    v += rec(h, hist + (a,), w2)
        vals[(h, hist)] = v
        return v

    br = 0.0
    for h in range(n):
        w = {o: g.r[1 - i][o] / g.Z for o in range(n) if g.compatible(h, o)}
        br += g.r[i][h] * rec(h, (), w)
    return br, vals


def reach_at_histories(g, prof, p):
    """pi_p at every history (decision, chance and terminal), including player p's range
    weight r_p(h): {(h, hist): r_p(h) times p's action probabilities on the path}, from the
    enumeration of every deal and every history of it (a card dealt on the path is live for
    the deal, so a hand holding it never gets an entry)."""
    out = {}

    def rec(hands, hist, pi):
        key = (hands[p], hist)
        if key in out:
            assert out[key] == pi, (key, out[key], pi)
        out[key] = pi
        if g.utility(hands, hist, 0) is not None:
            return
        live = g.chance_cards(hands, hist)
        if live is not None:
            for x in live:
                rec(hands, hist + (("d", x),), pi)
            return
        s = g.state(hist)
        acts = g.legal(hist)
        if s["to_act"] == p:
            pr = prof.probs(infoset_key(p, hands[p], hist), len(acts))
            for k, a in enumerate(acts):
                rec(hands, hist + (a,), pi * pr[k])
        else:
            for a in acts:
                rec(hands, hist + (a,), pi)

    for h0, h1 in g.deals():
        rec((h0, h1), (), g.r[p][(h0, h1)[p]])
    return out
