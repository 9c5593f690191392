"""Thin Python binding of libpcfr.so (include/pcfr.h): the same entry points, argument
marshalling only.  Every step of the CFR iteration runs in the library's CUDA kernels; if
the library is missing or no GB300 is present, calls raise instead of falling back.

PyTorch supplies device memory (its caching allocator, through ``cfr_set_allocator``) and
streams; nothing here computes.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libpcfr.so")

CFR_OK, CFR_EINVAL, CFR_ENOMEM, CFR_ECUDA, CFR_ETIMEOUT, CFR_ESTATE = 0, -1, -2, -3, -4, -5
CFR_GAME_HOLDEM, CFR_GAME_KUHN, CFR_GAME_LEDUC = 0, 1, 2
CFR_VARIANT_CFR, CFR_VARIANT_CFRPLUS, CFR_VARIANT_DCFR, CFR_VARIANT_PCFRPLUS = 0, 1, 2, 3
CFR_NODE_DECISION, CFR_NODE_FOLD, CFR_NODE_SHOWDOWN, CFR_NODE_CHANCE, CFR_NODE_LEAF = 0, 1, 2, 3, 4
LEAF_SLOTS, LEAF_IN, LEAF_HIDDEN, LEAF_OUT, LEAF_CARDS = 1326, 2752, 512, 2688, 48
LEAF_SHAPES = ((LEAF_HIDDEN, LEAF_IN), (LEAF_HIDDEN, LEAF_HIDDEN), (LEAF_HIDDEN, LEAF_HIDDEN), (LEAF_OUT, LEAF_HIDDEN))
CFR_READ_REGRET, CFR_READ_AVG_SUM, CFR_READ_CFV, CFR_READ_BR_CFV, CFR_READ_PREDICTION = 0, 1, 2, 3, 4
CFR_READ_AVG_REACH = 5
CFR_PRECISION_PAIRS, CFR_PRECISION_SINGLE = 0, 1
PRECISIONS = {"pairs": CFR_PRECISION_PAIRS, "single": CFR_PRECISION_SINGLE}
CFR_SCHEDULE_AUTO, CFR_SCHEDULE_LEVEL, CFR_SCHEDULE_STREAM, CFR_SCHEDULE_WIDE, CFR_SCHEDULE_RESIDENT = 0, 1, 2, 3, 4
SCHEDULES = {"auto": CFR_SCHEDULE_AUTO, "level": CFR_SCHEDULE_LEVEL, "stream": CFR_SCHEDULE_STREAM,
             "wide": CFR_SCHEDULE_WIDE, "resident": CFR_SCHEDULE_RESIDENT}
VARIANTS = {"cfr": CFR_VARIANT_CFR, "cfr+": CFR_VARIANT_CFRPLUS, "dcfr": CFR_VARIANT_DCFR,
            "pcfr+": CFR_VARIANT_PCFRPLUS}
CFR_STAGES = ("terminal", "update", "avg_reach", "br_terminal", "br", "leaf")
EXPORTS = ("cfr_set_allocator", "cfr_tree_create", "cfr_batch_create", "cfr_iterate", "cfr_strategy",
           "cfr_exploitability", "cfr_tree_info", "cfr_node_info", "cfr_read_values", "cfr_sync",
           "cfr_stage_times", "cfr_counters", "cfr_exploitability_async", "cfr_exploitability_result",
           "cfr_reset", "cfr_tree_destroy", "cfr_last_error", "cfr_exploitability_noalloc", "cfr_schedule",
           "cfr_gemm_bf16", "cfr_set_leaf_net", "cfr_leaf_info", "cfr_read_leaf_rows",
           "cfr_eval_leaves", "cfr_write_values", "cfr_autotune", "cfr_debug_first_wait_polls")


class CfrError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (code {code})")
        self.code = code


class cfr_game_spec(C.Structure):
    _fields_ = [("game", C.c_int), ("n_board", C.c_int), ("board", C.POINTER(C.c_int32)), ("n_hands", C.c_int),
                ("hands", C.POINTER(C.c_uint8)), ("range", C.POINTER(C.c_float) * 2),
                ("strength", C.POINTER(C.c_int32)), ("n_strength_rows", C.c_int), ("pot", C.c_double),
                ("stack", C.c_double), ("n_bet_sizes", C.c_int), ("bet_sizes", C.POINTER(C.c_double)),
                ("max_raises", C.c_int), ("depth_limit", C.c_int), ("exact_leaves", C.POINTER(C.c_int32)),
                ("n_exact_leaves", C.c_int)]


class cfr_solver_opts(C.Structure):
    _fields_ = [("variant", C.c_int), ("alpha", C.c_double), ("beta", C.c_double), ("gamma", C.c_double),
                ("alternating", C.c_int), ("chunk_hands", C.c_int), ("precision", C.c_int), ("schedule", C.c_int),
                ("term_nodes", C.c_int), ("warp_hands", C.c_int), ("runout_tables", C.c_int)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)

_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH):
    """Load libpcfr.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with `python -m paper_2605_19928_gb300.build`")
        lib = C.CDLL(path)
        I, P, S = C.c_int, C.c_void_p, C.c_size_t
        pd = C.POINTER(C.c_double)
        pi = C.POINTER(C.c_int)
        lib.cfr_set_allocator.argtypes = [ALLOC_FN, FREE_FN, P]
        lib.cfr_tree_create.argtypes = [C.POINTER(cfr_game_spec), C.POINTER(cfr_solver_opts), P, C.POINTER(P)]
        lib.cfr_batch_create.argtypes = [C.POINTER(cfr_game_spec), I, C.POINTER(cfr_solver_opts), P, C.POINTER(P)]
        lib.cfr_autotune.argtypes = [C.POINTER(cfr_game_spec), I, C.POINTER(cfr_solver_opts), P, I,
                                     C.POINTER(cfr_solver_opts), C.POINTER(C.c_double)]
        lib.cfr_iterate.argtypes = [P, I]
        lib.cfr_strategy.argtypes = [P, I, I, I, C.POINTER(C.c_float), S]
        lib.cfr_exploitability.argtypes = [P, pd, pd]
        lib.cfr_tree_info.argtypes = [P, I, pi, pi, pi]
        lib.cfr_node_info.argtypes = [P, I, I, pi, pi, pi, pi, pi, pi, pd]
        lib.cfr_read_values.argtypes = [P, I, I, I, I, pd, S]
        lib.cfr_sync.argtypes = [P]
        pl = C.POINTER(C.c_int64)
        lib.cfr_stage_times.argtypes = [P, I, pd, pl]
        lib.cfr_counters.argtypes = [P, pl, pl, pl]
        lib.cfr_exploitability_async.argtypes = [P]
        lib.cfr_exploitability_result.argtypes = [P, pd, pd]
        lib.cfr_reset.argtypes = [P]
        lib.cfr_exploitability_noalloc.argtypes = [P, pd, pd]
        lib.cfr_schedule.argtypes = [P]
        lib.cfr_gemm_bf16.argtypes = [P, P, P, P, I, I, I, I, I, P, P]
        lib.cfr_debug_first_wait_polls.argtypes = [C.c_long]
        lib.cfr_set_leaf_net.argtypes = [P, C.POINTER(P), C.POINTER(P)]
        lib.cfr_leaf_info.argtypes = [P, I, pi, pi, pi, pi]
        lib.cfr_read_leaf_rows.argtypes = [P, I, I, I, P]
        lib.cfr_eval_leaves.argtypes = [P, I]
        lib.cfr_write_values.argtypes = [P, I, I, I, pd, S]
        lib.cfr_tree_destroy.argtypes = [P]
        lib.cfr_tree_destroy.restype = None
        lib.cfr_last_error.restype = C.c_char_p
        _lib = lib
        return lib


def _check(rc: int):
    if rc != CFR_OK:
        raise CfrError(rc, _lib.cfr_last_error().decode())


# ---------------------------------------------------------------- allocator hook

_hooks = None


def cfr_set_allocator(alloc=None, free=None, ctx=None):
    """Install Python callables alloc(bytes, stream) -> int pointer and free(pointer)."""
    global _hooks
    lib = load()
    if alloc is None:
        _hooks = None
        _check(lib.cfr_set_allocator(ALLOC_FN(), FREE_FN(), None))
        return

    def _a(nbytes, stream, _ctx):
        try:
            return int(alloc(int(nbytes), stream))
        except Exception:  # reported to the library as an allocation failure
            return None

    def _f(ptr, _ctx):
        free(ptr)

    _hooks = (ALLOC_FN(_a), FREE_FN(_f))
    _check(lib.cfr_set_allocator(_hooks[0], _hooks[1], None))


def use_torch_allocator():
    """Route the library's device allocations through PyTorch's caching allocator."""
    import torch

    def alloc(nbytes, stream):
        return torch.cuda.caching_allocator_alloc(nbytes, stream=stream or 0)

    def free(ptr):
        torch.cuda.caching_allocator_delete(ptr)

    cfr_set_allocator(alloc, free)


# ---------------------------------------------------------------- marshalling

def make_spec(g) -> tuple[cfr_game_spec, tuple]:
    """cfr_game_spec for a ``synth.GameSpec`` (plus the arrays it points into)."""
    board = np.ascontiguousarray(g.board, dtype=np.int32)
    hands = np.ascontiguousarray(g.hands, dtype=np.uint8)
    r0 = np.ascontiguousarray(g.ranges[0], dtype=np.float32)
    r1 = np.ascontiguousarray(g.ranges[1], dtype=np.float32)
    strength = None if g.strength is None else np.ascontiguousarray(g.strength, dtype=np.int32)
    sizes = np.ascontiguousarray(np.array(g.bet_sizes, dtype=np.float64).reshape(-1))
    s = cfr_game_spec()
    s.game = int(g.game)
    holdem = g.game == CFR_GAME_HOLDEM
    s.n_board = int(board.size) if holdem else 0
    s.board = board.ctypes.data_as(C.POINTER(C.c_int32)) if holdem else None
    s.n_hands = int(hands.shape[0]) if holdem else 0
    s.hands = hands.ctypes.data_as(C.POINTER(C.c_uint8)) if holdem else None
    s.range[0] = r0.ctypes.data_as(C.POINTER(C.c_float))
    s.range[1] = r1.ctypes.data_as(C.POINTER(C.c_float))
    s.strength = strength.ctypes.data_as(C.POINTER(C.c_int32)) if strength is not None else None
    s.n_strength_rows = int(strength.shape[0]) if strength is not None else 0
    s.pot = float(g.pot)
    s.stack = float(g.stack)
    s.n_bet_sizes = int(sizes.size)
    s.bet_sizes = sizes.ctypes.data_as(C.POINTER(C.c_double))
    s.max_raises = int(g.max_raises)
    s.depth_limit = int(getattr(g, "depth_limit", 0))
    exact = np.ascontiguousarray(np.array(getattr(g, "exact_leaves", ()), dtype=np.int32).reshape(-1))
    s.n_exact_leaves = int(exact.size)
    s.exact_leaves = exact.ctypes.data_as(C.POINTER(C.c_int32)) if exact.size else None
    return s, (board, hands, r0, r1, strength, sizes, exact)


def make_opts(variant="dcfr", alpha=1.5, beta=0.0, gamma=2.0, alternating=True, chunk_hands=0,
              precision="pairs", schedule="auto", term_nodes=0, warp_hands=0, runout_tables=False) -> cfr_solver_opts:
    return cfr_solver_opts(VARIANTS[variant] if isinstance(variant, str) else int(variant), alpha, beta, gamma,
                           int(alternating), int(chunk_hands),
                           PRECISIONS[precision] if isinstance(precision, str) else int(precision),
                           SCHEDULES[schedule] if isinstance(schedule, str) else int(schedule), int(term_nodes),
                           int(warp_hands), int(runout_tables))


def _stream_arg(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return None
    return C.c_void_p(int(stream))


# ---------------------------------------------------------------- entry points

def cfr_tree_create(spec, opts: cfr_solver_opts | None = None, stream=None) -> C.c_void_p:
    lib = load()
    s, keep = make_spec(spec)
    out = C.c_void_p()
    _check(lib.cfr_tree_create(C.byref(s), C.byref(opts) if opts else None, _stream_arg(stream), C.byref(out)))
    del keep
    return out


def cfr_batch_create(specs, opts: cfr_solver_opts | None = None, stream=None) -> C.c_void_p:
    lib = load()
    arr = (cfr_game_spec * len(specs))()
    keep = []
    for k, g in enumerate(specs):
        arr[k], kk = make_spec(g)
        keep.append(kk)
    out = C.c_void_p()
    _check(lib.cfr_batch_create(arr, len(specs), C.byref(opts) if opts else None, _stream_arg(stream),
                                C.byref(out)))
    del keep
    return out


def cfr_autotune(specs, opts: cfr_solver_opts | None = None, iters: int = 20, stream=None):
    """(best options, ms per iteration) of the launch-tiling autotuner over these subgames."""
    lib = load()
    arr = (cfr_game_spec * len(specs))()
    keep = []
    for k, g in enumerate(specs):
        arr[k], kk = make_spec(g)
        keep.append(kk)
    best, ms = cfr_solver_opts(), C.c_double()
    _check(lib.cfr_autotune(arr, len(specs), C.byref(opts if opts else make_opts()), _stream_arg(stream), int(iters),
                            C.byref(best), C.byref(ms)))
    del keep
    return best, float(ms.value)


def cfr_iterate(tree, n_iters: int = 1):
    _check(load().cfr_iterate(tree, int(n_iters)))


def cfr_sync(tree):
    _check(load().cfr_sync(tree))


def cfr_gemm_bf16(A, B, bias, C, act: bool, err, stream=None):
    """C = act(A B^T + bias) on the tensor cores; A [M, K] and B [N, K] bfloat16 CUDA tensors,
    bias float32 [N] or None, C bfloat16 or float32 [M, N], err an int32 CUDA tensor."""
    M, K = A.shape
    N = B.shape[0]
    assert B.shape[1] == K and tuple(C.shape) == (M, N)
    import torch
    out_f32 = C.dtype == torch.float32
    _check(load().cfr_gemm_bf16(A.data_ptr(), B.data_ptr(), None if bias is None else bias.data_ptr(), C.data_ptr(),
                                M, N, K, int(bool(act)), int(out_f32), err.data_ptr(), _stream_arg(stream)))


def cfr_set_leaf_net(tree, weights, biases):
    """weights: 4 uint16 arrays of BF16 bit patterns (as leafnet_train writes them) of shapes
    LEAF_SHAPES; biases: 4 float32 arrays."""
    Ws, bs = [], []
    for k, (w, b) in enumerate(zip(weights, biases)):
        w = np.asarray(w)
        if w.dtype != np.uint16:
            raise TypeError(f"layer {k}: weights must be BF16 bit patterns (uint16), not {w.dtype}")
        assert w.shape == LEAF_SHAPES[k], (k, w.shape)
        Ws.append(np.ascontiguousarray(w))
        bs.append(np.ascontiguousarray(b, dtype=np.float32).reshape(LEAF_SHAPES[k][0]))
    Wp = (C.c_void_p * 4)(*[w.ctypes.data for w in Ws])
    bp = (C.c_void_p * 4)(*[b.ctypes.data for b in bs])
    _check(load().cfr_set_leaf_net(tree, Wp, bp))


def cfr_debug_first_wait_polls(polls: int):
    """Testing aid: polls of the terminal kernel's first bulk-copy wait (< 0: the default)."""
    _check(load().cfr_debug_first_wait_polls(int(polls)))


def cfr_eval_leaves(tree, average: bool = False):
    _check(load().cfr_eval_leaves(tree, int(bool(average))))


def cfr_leaf_info(tree):
    """[(game, node, row0)] of every depth-limit leaf."""
    lib = load()
    n = C.c_int()
    _check(lib.cfr_leaf_info(tree, -1, C.byref(n), None, None, None))
    out = []
    for k in range(n.value):
        g, nd, r0 = C.c_int(), C.c_int(), C.c_int()
        _check(lib.cfr_leaf_info(tree, k, None, C.byref(g), C.byref(nd), C.byref(r0)))
        out.append((g.value, nd.value, r0.value))
    return out


def cfr_read_leaf_rows(tree, what: int, row0: int, n_rows: int) -> np.ndarray:
    """what 0: network inputs (uint16 BF16 bits [n_rows, LEAF_IN]); 1: outputs (float32 [n_rows, LEAF_OUT])."""
    out = np.empty((n_rows, LEAF_IN), np.uint16) if what == 0 else np.empty((n_rows, LEAF_OUT), np.float32)
    _check(load().cfr_read_leaf_rows(tree, int(what), int(row0), int(n_rows), out.ctypes.data))
    return out


def cfr_schedule(tree) -> int:
    rc = load().cfr_schedule(tree)
    if rc < 0:
        _check(rc)
    return rc


def cfr_tree_info(tree, game: int = 0):
    a, b, c = C.c_int(), C.c_int(), C.c_int()
    _check(load().cfr_tree_info(tree, game, C.byref(a), C.byref(b), C.byref(c)))
    return a.value, b.value, c.value


def cfr_node_info(tree, node: int, game: int = 0) -> dict:
    v = [C.c_int() for _ in range(6)]
    contrib = (C.c_double * 2)()
    _check(load().cfr_node_info(tree, game, node, *[C.byref(x) for x in v], contrib))
    return {"type": v[0].value, "player": v[1].value, "n_actions": v[2].value, "parent": v[3].value,
            "action": v[4].value, "deal": v[5].value, "contrib": (contrib[0], contrib[1])}


def cfr_strategy(tree, node: int, average: bool = False, game: int = 0, out: np.ndarray | None = None):
    info = cfr_node_info(tree, node, game)
    nh = cfr_tree_info(tree, game)[1]
    if out is None:
        out = np.empty((info["n_actions"], nh), np.float32)
    _check(load().cfr_strategy(tree, game, node, int(bool(average)), out.ctypes.data_as(C.POINTER(C.c_float)),
                               out.size))
    return out


def cfr_exploitability(tree, n_games: int = 1):
    expl = np.zeros(n_games, np.float64)
    br = np.zeros((n_games, 2), np.float64)
    _check(load().cfr_exploitability(tree, expl.ctypes.data_as(C.POINTER(C.c_double)),
                                     br.ctypes.data_as(C.POINTER(C.c_double))))
    return expl, br


def cfr_exploitability_async(tree):
    _check(load().cfr_exploitability_async(tree))


def cfr_exploitability_result(tree, n_games: int = 1):
    expl = np.zeros(n_games, np.float64)
    br = np.zeros((n_games, 2), np.float64)
    _check(load().cfr_exploitability_result(tree, expl.ctypes.data_as(C.POINTER(C.c_double)),
                                            br.ctypes.data_as(C.POINTER(C.c_double))))
    return expl, br


def cfr_exploitability_noalloc(tree, expl: np.ndarray, br: np.ndarray):
    """cfr_exploitability into caller-owned float64 arrays expl [n_games] and br [n_games, 2]
    (the library allocates nothing during the call)."""
    for a, n in ((expl, br.shape[0]), (br, 2 * br.shape[0])):
        if a.dtype != np.float64 or not a.flags.c_contiguous or a.size != n:
            raise ValueError("expl must be float64 [n_games] and br float64 [n_games, 2], C-contiguous")
    _check(load().cfr_exploitability_noalloc(tree, expl.ctypes.data_as(C.POINTER(C.c_double)),
                                             br.ctypes.data_as(C.POINTER(C.c_double))))
    return expl, br


def cfr_reset(tree):
    _check(load().cfr_reset(tree))


def cfr_read_values(tree, what: int, node: int, player: int = 0, game: int = 0) -> np.ndarray:
    info = cfr_node_info(tree, node, game)
    nh = cfr_tree_info(tree, game)[1]
    shape = (info["n_actions"], nh) if what in (CFR_READ_REGRET, CFR_READ_AVG_SUM, CFR_READ_PREDICTION) else (nh,)
    out = np.zeros(shape, np.float64)
    _check(load().cfr_read_values(tree, game, what, player, node, out.ctypes.data_as(C.POINTER(C.c_double)),
                                  out.size))
    return out


def cfr_write_values(tree, what: int, node: int, values, game: int = 0):
    v = np.ascontiguousarray(values, dtype=np.float64)
    _check(load().cfr_write_values(tree, game, int(what), int(node), v.ctypes.data_as(C.POINTER(C.c_double)), v.size))


def cfr_stage_times(tree, n_iters: int = 1) -> dict:
    """Mean device ms per launch of each stage over n_iters un-graphed iterations plus one
    exploitability pass: {stage: (ms, launches)}."""
    ms = np.zeros(len(CFR_STAGES), np.float64)
    cnt = np.zeros(len(CFR_STAGES), np.int64)
    _check(load().cfr_stage_times(tree, int(n_iters), ms.ctypes.data_as(C.POINTER(C.c_double)),
                                  cnt.ctypes.data_as(C.POINTER(C.c_int64))))
    return {name: (float(ms[k]), int(cnt[k])) for k, name in enumerate(CFR_STAGES)}


def cfr_counters(tree) -> dict:
    a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
    _check(load().cfr_counters(tree, C.byref(a), C.byref(b), C.byref(c)))
    return {"kernel_launches": a.value, "device_bytes": b.value, "h2d_bytes": c.value}


def cfr_tree_destroy(tree):
    if tree:
        load().cfr_tree_destroy(tree)


def cfr_last_error() -> str:
    return load().cfr_last_error().decode()
