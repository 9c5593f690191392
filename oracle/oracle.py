"""ctypes wrapper around the plain-C FP64 oracle (cfr_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the benchmark's
``cpu_baseline`` / ``--impl reference`` legs may use this module; the product path may not.

The oracle walks every history (every private deal x every public action path) in FP64 and
follows the paper's definitions: counterfactual values (Section 3, Eq. cfv), regrets
(Section 3), regret matching (Section 3, Eq. rm), the Stage 6 backward values (Section 4.4,
Eq. backward) and the Stage 7 variant update (Section 4.4; CFR, CFR+, DCFR from Section 2).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cfr_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

T_DEC, T_FOLD, T_SHOW, T_CHANCE, T_LEAF = 0, 1, 2, 3, 4
VARIANTS = {"cfr": 0, "cfr+": 1, "dcfr": 2, "pcfr+": 3}


def build(force: bool = False) -> str:
    """Compile cfr_oracle.c into liboracle.so next to it (gcc, no CUDA)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load(path: str | None = None):
    """The oracle library, bound once per process; `path` binds another build of the same
    source instead (the tests compile copies with planted mistakes to check the pins)."""
    global _lib
    with _lock:
        if path is None and _lib is not None:
            return _lib
        lib = C.CDLL(path or build())
        P, I, D = C.c_void_p, C.c_int, C.c_double
        pi = C.POINTER(C.c_int)
        pd = C.POINTER(C.c_double)
        lib.ocfr_create.restype = P
        lib.ocfr_create.argtypes = [I, I, pi, I, pi, pd, pd, pi, I, D, D, I, pd, I, I, D, D, D, I, I, I, pi, I]
        lib.ocfr_destroy.argtypes = [P]
        lib.ocfr_error.restype = C.c_char_p
        lib.ocfr_iterate.argtypes = [P, I]
        for f in ("ocfr_n_nodes", "ocfr_n_hands", "ocfr_n_rows", "ocfr_iters"):
            getattr(lib, f).argtypes = [P]
            getattr(lib, f).restype = I
        lib.ocfr_Z.argtypes = [P]
        lib.ocfr_Z.restype = D
        lib.ocfr_node.argtypes = [P, I, pi, pd]
        lib.ocfr_child.argtypes = [P, I, I]
        lib.ocfr_child.restype = I
        lib.ocfr_get_node.argtypes = [P, I, I, pd]
        lib.ocfr_get_node.restype = I
        lib.ocfr_get_cfv.argtypes = [P, I, I, pd]
        lib.ocfr_load_profile.argtypes = [P, I]
        lib.ocfr_set_profile_node.argtypes = [P, I, pd]
        lib.ocfr_set_profile_node.restype = I
        lib.ocfr_profile_value.argtypes = [P, pd]
        lib.ocfr_best_response.argtypes = [P, I, pd, pd]
        lib.ocfr_best_response.restype = D
        lib.ocfr_exploitability.argtypes = [P, pd]
        lib.ocfr_exploitability.restype = D
        lib.ocfr_values_current.argtypes = [P, I]
        lib.ocfr_update_player.argtypes = [P, I, I]
        lib.ocfr_update_both.argtypes = [P, I]
        lib.ocfr_set_node_state.argtypes = [P, I, pd, pd]
        lib.ocfr_set_node_state.restype = I
        lib.ocfr_set_iterations.argtypes = [P, I]
        lib.ocfr_set_node_pred.argtypes = [P, I, pd]
        lib.ocfr_set_node_pred.restype = I
        lib.ocfr_node_reach.argtypes = [P, I, I, I, pd]
        lib.ocfr_node_reach.restype = I
        lib.ocfr_set_leaf_values.argtypes = [P, I, pd]
        lib.ocfr_set_leaf_values.restype = I
        if path is None:
            _lib = lib
        return lib


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


class Oracle:
    """FP64 CFR over one subgame (a ``synth.GameSpec``)."""

    def __init__(self, spec, variant: str = "dcfr", alpha: float = 1.5, beta: float = 0.0, gamma: float = 2.0,
                 alternating: bool = True, threads: int | None = None, lib_path: str | None = None):
        lib = _load(lib_path)
        self._lib = lib
        self.spec = spec
        nh = spec.n_hands
        cards = np.ascontiguousarray(spec.hands, dtype=np.int32).reshape(-1)
        r0 = np.ascontiguousarray(spec.ranges[0], dtype=np.float64)
        r1 = np.ascontiguousarray(spec.ranges[1], dtype=np.float64)
        board = np.ascontiguousarray(spec.board, dtype=np.int32)
        if spec.strength is not None:
            strength = np.ascontiguousarray(spec.strength, dtype=np.int32)
            nstr = strength.shape[0]
        else:
            strength = np.zeros(1, np.int32)
            nstr = 0
        sizes = np.ascontiguousarray(np.array(spec.bet_sizes, dtype=np.float64).reshape(-1))
        if sizes.size == 0:
            sizes = np.zeros(1, np.float64)
        if threads is None:
            threads = os.cpu_count() or 1
        self.threads = int(threads)
        flags = self._exact_flags(spec, lib_path)
        self._keep = (cards, r0, r1, board, strength, sizes, flags)
        self.variant = variant
        self._h = lib.ocfr_create(spec.game, int(board.size), _ptr(board, C.c_int), nh, _ptr(cards, C.c_int),
                                  _ptr(r0, C.c_double), _ptr(r1, C.c_double), _ptr(strength, C.c_int), nstr,
                                  float(spec.pot), float(spec.stack), len(spec.bet_sizes), _ptr(sizes, C.c_double),
                                  int(spec.max_raises), VARIANTS[variant], alpha, beta, gamma, int(alternating),
                                  self.threads, int(getattr(spec, "depth_limit", 0)),
                                  _ptr(flags, C.c_int) if flags.size else None, int(flags.size))
        if not self._h:
            raise ValueError("oracle: " + lib.ocfr_error().decode())
        self.n_nodes = lib.ocfr_n_nodes(self._h)
        self.n_hands = nh
        self._info = None

    @staticmethod
    def _exact_flags(spec, lib_path=None) -> np.ndarray:
        """Leaves the spec asks to solve exactly (`exact_leaves`: indices in the breadth-first
        order of the depth-limited tree -- by action-path length, then lexicographically) as
        flags in the order this oracle's depth-first builder meets leaf positions."""
        exact = sorted(int(k) for k in getattr(spec, "exact_leaves", ()) or ())
        if not exact:
            return np.zeros(0, np.int32)
        import dataclasses
        pure = Oracle(dataclasses.replace(spec, exact_leaves=()), variant="cfr", threads=1, lib_path=lib_path)
        paths = {n: p for p, n in pure.paths().items()}
        leaves = [n for n in range(pure.n_nodes) if pure.node(n)["type"] == T_LEAF]  # depth first: by id
        rank = {n: k for k, n in enumerate(sorted(leaves, key=lambda n: (len(paths[n]), paths[n])))}
        if exact[-1] >= len(leaves) or exact[0] < 0 or len(set(exact)) != len(exact):
            raise ValueError("exact_leaves must be distinct leaf indices")
        want = set(exact)
        return np.array([1 if rank[n] in want else 0 for n in leaves], np.int32)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.ocfr_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    # ---------------------------------------------------------------- tree
    def node(self, n: int) -> dict:
        out = np.zeros(9, np.int32)
        c = np.zeros(2, np.float64)
        self._lib.ocfr_node(self._h, n, _ptr(out, C.c_int), _ptr(c, C.c_double))
        kids = [self._lib.ocfr_child(self._h, n, k) for k in range(int(out[4]))]
        return {"type": int(out[0]), "player": int(out[1]), "parent": int(out[2]), "action": int(out[3]),
                "n_actions": int(out[4]), "street": int(out[5]), "deal": int(out[6]), "n_board": int(out[7]),
                "contrib": (float(c[0]), float(c[1])), "kids": kids}

    def nodes(self) -> list[dict]:
        if self._info is None:
            self._info = [self.node(n) for n in range(self.n_nodes)]
        return self._info

    def paths(self) -> dict:
        """Map from action path (tuple of child indices from the root) to node id."""
        info = self.nodes()
        out = {}
        stack = [(0, ())]
        while stack:
            n, p = stack.pop()
            out[p] = n
            for k, kid in enumerate(info[n]["kids"]):
                stack.append((kid, p + (k,)))
        return out

    @property
    def Z(self) -> float:
        return self._lib.ocfr_Z(self._h)

    @property
    def iterations(self) -> int:
        return self._lib.ocfr_iters(self._h)

    # ---------------------------------------------------------------- solving
    def iterate(self, n: int = 1):
        self._lib.ocfr_iterate(self._h, int(n))

    def _node_rows(self, what: int, n: int) -> np.ndarray:
        a = self.nodes()[n]["n_actions"]
        out = np.zeros((a, self.n_hands), np.float64)
        if self._lib.ocfr_get_node(self._h, what, n, _ptr(out, C.c_double)) != 0:
            raise ValueError(f"node {n} is not a decision node")
        return out

    def regrets(self, n: int) -> np.ndarray:
        return self._node_rows(0, n)

    def avg_sums(self, n: int) -> np.ndarray:
        return self._node_rows(1, n)

    def strategy(self, n: int) -> np.ndarray:
        return self._node_rows(2, n)

    def prediction(self, n: int) -> np.ndarray:
        """Predictive CFR+: the prediction M (last instantaneous regret) at node n."""
        return self._node_rows(4, n)

    def set_node_pred(self, n: int, M):
        M = np.ascontiguousarray(M, dtype=np.float64)
        if self._lib.ocfr_set_node_pred(self._h, n, _ptr(M, C.c_double)) != 0:
            raise ValueError(f"node {n} is not a decision node")

    def profile(self, n: int) -> np.ndarray:
        return self._node_rows(3, n)

    def cfv(self, i: int, n: int) -> np.ndarray:
        out = np.zeros(self.n_hands, np.float64)
        self._lib.ocfr_get_cfv(self._h, i, n, _ptr(out, C.c_double))
        return out

    def update_player(self, i: int, t: int):
        """Player i's update at iteration t (regret matching, traversal, update)."""
        self._lib.ocfr_update_player(self._h, int(i), int(t))

    def update_both(self, t: int):
        """Both players' updates at iteration t from one strategy (simultaneous)."""
        self._lib.ocfr_update_both(self._h, int(t))

    def set_node_state(self, n: int, R, S):
        """Overwrite a decision node's regrets and average sums ([n_actions][n_hands])."""
        R = np.ascontiguousarray(R, dtype=np.float64)
        S = np.ascontiguousarray(S, dtype=np.float64)
        if self._lib.ocfr_set_node_state(self._h, n, _ptr(R, C.c_double), _ptr(S, C.c_double)) != 0:
            raise ValueError(f"node {n} is not a decision node")

    def set_iterations(self, t: int):
        self._lib.ocfr_set_iterations(self._h, int(t))

    def node_reach(self, kind: str, p: int, n: int) -> np.ndarray:
        """Player p's own reach at node n per hand, under the current ("current") or average
        ("average") strategy."""
        out = np.zeros(self.n_hands, np.float64)
        if self._lib.ocfr_node_reach(self._h, {"current": 0, "average": 1}[kind], p, n, _ptr(out, C.c_double)) != 0:
            raise ValueError(f"bad node {n}")
        return out

    def set_leaf_values(self, n: int, y):
        """Network outputs at depth-limit leaf n: y [K][2][n_hands], K the river cards not on
        the leaf's board in ascending order, values per unit pot."""
        y = np.ascontiguousarray(y, dtype=np.float64)
        if self._lib.ocfr_set_leaf_values(self._h, n, _ptr(y, C.c_double)) != 0:
            raise ValueError(f"node {n} is not a leaf")

    def values_current(self, i: int):
        """Counterfactual values of player i under the current strategy (no update)."""
        self._lib.ocfr_values_current(self._h, i)

    # ---------------------------------------------------------------- profiles, best response
    def load_profile(self, kind: str):
        self._lib.ocfr_load_profile(self._h, {"current": 0, "average": 1}[kind])

    def set_profile_node(self, n: int, vals):
        v = np.ascontiguousarray(vals, dtype=np.float64)
        if self._lib.ocfr_set_profile_node(self._h, n, _ptr(v, C.c_double)) != 0:
            raise ValueError(f"node {n} is not a decision node")

    def profile_value(self) -> np.ndarray:
        out = np.zeros(2, np.float64)
        self._lib.ocfr_profile_value(self._h, _ptr(out, C.c_double))
        return out

    def best_response(self, i: int, all_nodes: bool = False):
        root = np.zeros(self.n_hands, np.float64)
        allv = np.zeros((self.n_nodes, self.n_hands), np.float64) if all_nodes else None
        br = self._lib.ocfr_best_response(self._h, i, _ptr(root, C.c_double),
                                          _ptr(allv, C.c_double) if all_nodes else None)
        return (br, root, allv) if all_nodes else (br, root)

    def exploitability(self) -> tuple[float, float, float]:
        """(exploitability, BR_0, BR_1) of the average strategy, in chips."""
        br = np.zeros(2, np.float64)
        e = self._lib.ocfr_exploitability(self._h, _ptr(br, C.c_double))
        return float(e), float(br[0]), float(br[1])
