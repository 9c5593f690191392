"""C-ABI checks that need no GPU: the library builds, loads and exports every function that
include/pcfr.h declares, and refuses to run (no CPU fallback) when no GB300 is present."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2605_19928_gb300 import build as pbuild
from paper_2605_19928_gb300 import capi, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pcfr.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:int|void|const char\*)\s+\*?\s*(cfr_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    pbuild.build()
    return capi.load()


def test_header_declares_the_documented_entry_points():
    names = declared_functions()
    for n in ("cfr_tree_create", "cfr_iterate", "cfr_strategy", "cfr_exploitability", "cfr_tree_destroy"):
        assert n in names
    assert sorted(capi.EXPORTS) == names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", capi.LIB_PATH], capture_output=True, text=True, check=True)
    exported = set(re.findall(r"\sT\s+(cfr_\w+)", out.stdout))
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(lib, name)


def test_kernels_are_built_for_sm_103a(lib):
    out = subprocess.run(["strings", capi.LIB_PATH], capture_output=True, text=True)
    assert "sm_103a" in out.stdout or "sm_103" in out.stdout


def have_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except ImportError:
        return False


@pytest.mark.skipif(have_gpu(), reason="checks the no-GPU failure path")
def test_create_fails_loudly_without_a_gpu(lib):
    with pytest.raises(capi.CfrError) as e:
        capi.cfr_tree_create(synth.kuhn())
    assert e.value.code == capi.CFR_ECUDA


def test_argument_checks_need_no_gpu(lib):
    assert lib.cfr_tree_info(None, 0, None, None, None) == capi.CFR_EINVAL
    assert "NULL" in capi.cfr_last_error()
    assert lib.cfr_iterate(None, 1) == capi.CFR_EINVAL
    assert lib.cfr_exploitability(None, None, None) == capi.CFR_EINVAL
    out = C.c_void_p()
    assert lib.cfr_tree_create(None, None, None, C.byref(out)) == capi.CFR_EINVAL
    assert lib.cfr_batch_create(None, 0, None, None, C.byref(out)) == capi.CFR_EINVAL
    lib.cfr_tree_destroy(None)  # ignored


def test_bad_options_are_rejected_before_any_device_call(lib):
    s, keep = capi.make_spec(synth.kuhn())
    out = C.c_void_p()
    bad = capi.make_opts(chunk_hands=3)
    assert lib.cfr_tree_create(C.byref(s), C.byref(bad), None, C.byref(out)) == capi.CFR_EINVAL
    bad = capi.make_opts(variant=7)
    assert lib.cfr_tree_create(C.byref(s), C.byref(bad), None, C.byref(out)) == capi.CFR_EINVAL
    bad = capi.make_opts(precision=5)
    assert lib.cfr_tree_create(C.byref(s), C.byref(bad), None, C.byref(out)) == capi.CFR_EINVAL
    bad = capi.make_opts(schedule=5)
    assert lib.cfr_tree_create(C.byref(s), C.byref(bad), None, C.byref(out)) == capi.CFR_EINVAL
    for tn in (-1, 9):  # terminal nodes per block: 0 (automatic) to 8
        bad = capi.make_opts(term_nodes=tn)
        assert lib.cfr_tree_create(C.byref(s), C.byref(bad), None, C.byref(out)) == capi.CFR_EINVAL
    best, ms = capi.cfr_solver_opts(), C.c_double()
    good = capi.make_opts()
    assert lib.cfr_autotune(C.byref(s), 1, C.byref(good), None, 0, C.byref(best), C.byref(ms)) == capi.CFR_EINVAL
    assert lib.cfr_autotune(None, 1, C.byref(good), None, 5, C.byref(best), C.byref(ms)) == capi.CFR_EINVAL


def test_leaf_net_setter_only_marshals_bf16_bit_patterns():
    """The binding does no arithmetic on the network: FP32 weights are refused, not rounded
    in Python (the training script writes BF16 bit patterns)."""
    import numpy as np
    W = [np.zeros(s, np.float32) for s in capi.LEAF_SHAPES]
    b = [np.zeros(s[0], np.float32) for s in capi.LEAF_SHAPES]
    with pytest.raises(TypeError):
        capi.cfr_set_leaf_net(None, W, b)
