"""The leaf network's dense layers on the tensor cores (cfr_gemm_bf16) against the FP64
reference on the same BF16 operands."""
import numpy as np
import pytest

from oracle import leafnet as ln
from paper_2605_19928_gb300 import capi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2605_19928_gb300 import build as pbuild
    pbuild.build()
    capi.load()


def _gemm(M, N, K, act, out_f32, seed, scale=1.0):
    import torch
    rng = np.random.default_rng(seed)
    a = ln.bf16_round(rng.standard_normal((M, K)).astype(np.float32) * scale)
    w = ln.bf16_round(rng.standard_normal((N, K)).astype(np.float32) / np.sqrt(K))
    b = rng.standard_normal(N).astype(np.float32) * 0.1
    dev = torch.device("cuda")
    A = torch.from_numpy(a).to(dev, torch.bfloat16)
    B = torch.from_numpy(w).to(dev, torch.bfloat16)
    bias = torch.from_numpy(b).to(dev)
    C = torch.full((M, N), float("nan"), dtype=torch.float32 if out_f32 else torch.bfloat16, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    capi.cfr_gemm_bf16(A, B, bias, C, act, err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    return C.float().cpu().numpy(), ln.dense(a, w, b, act=act), ln.abs_terms(a, w)


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (300, 256, 256), (1000, 512, 2752), (77, 2688, 512)])
def test_fp32_output_matches_fp64_reference(M, N, K):
    got, want, terms = _gemm(M, N, K, act=False, out_f32=True, seed=M + N + K)
    # FP32 accumulation: error bounded by a small multiple of eps_32 times sum |a_k w_k|
    assert np.all(np.abs(got - want) <= 2e-6 * (terms + np.abs(want)) + 1e-30), np.max(np.abs(got - want))


@pytest.mark.parametrize("M,N,K", [(200, 512, 2752), (513, 512, 512)])
def test_bf16_gelu_output_matches_reference(M, N, K):
    got, want, terms = _gemm(M, N, K, act=True, out_f32=False, seed=7 * M + N)
    # the GPU rounds its FP32 result to BF16: within one BF16 step of the FP64 value, plus
    # the accumulation error carried through GELU (slope <= 1.13)
    step = np.abs(ln.bf16_round(want).astype(np.float64)) * 2.0 ** -7 + 1e-38
    assert np.all(np.abs(got - want) <= step + 3e-6 * terms), np.max(np.abs(got - want) / step)


def test_shapes_are_checked():
    import torch
    dev = torch.device("cuda")
    A = torch.zeros((16, 64), dtype=torch.bfloat16, device=dev)
    B = torch.zeros((100, 64), dtype=torch.bfloat16, device=dev)  # N not a multiple of 128
    C = torch.zeros((16, 100), dtype=torch.float32, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    with pytest.raises(capi.CfrError) as e:
        capi.cfr_gemm_bf16(A, B, None, C, False, err)
    assert e.value.code == capi.CFR_EINVAL
