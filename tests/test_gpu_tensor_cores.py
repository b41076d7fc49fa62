"""The tcgen05 tensor-core product of the mixed path (tt_tc_gemm: kind::tf32 MMAs from shared-memory
descriptors into a TMEM accumulator) against an FP64 product of the same FP32 operands.

Bars, relative to sum_k |a_ik| |b_jk| (the scale of each output's rounding errors):
  * split TF32 (3 passes): 1e-6 + K 2^-24, i.e. FP32-level products (each hi/lo product exact in
    FP32, the truncation of lo and the dropped lo lo term below 2^-20 of a product) plus the bound
    of FP32 accumulation over K terms;
  * plain TF32 (1 pass): 2e-3 (two roundings to 11 significant bits), and at least 30 times the
    3-pass error on the same data, which shows that the lo passes are really summed.
Shapes cover ragged M (not a multiple of the 128-row tile), every N the accumulator layout takes
from 16 to 256 in steps that exercise partial 32-column TMEM loads, and K not a multiple of the
32-value staging chunk."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tt():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2602_00290_gb300 as mod
    return mod


def _err(tt, M, N, K, passes, seed=0):
    g = torch.Generator(device="cpu").manual_seed(seed)
    A = torch.randn(M, K, generator=g, dtype=torch.float32)
    B = torch.randn(N, K, generator=g, dtype=torch.float32)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    D = tt.tc_gemm(A.cuda(), B.cuda(), passes=passes, status=status).cpu().double()
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    ref = A.double() @ B.double().T
    scale = A.double().abs() @ B.double().abs().T
    return float(torch.max(torch.abs(D - ref) / scale))


@pytest.mark.parametrize("M,N,K", [(128, 32, 160), (1000, 16, 8), (257, 48, 33), (384, 256, 64), (130, 112, 1),
                                   (128, 208, 100)])
def test_tc_gemm_split_tf32_matches_fp64(tt, M, N, K):
    e3 = _err(tt, M, N, K, 3)
    assert e3 < 1e-6 + K * 2.0 ** -24, e3
    e1 = _err(tt, M, N, K, 1)
    assert e1 < 2e-3, e1
    if K >= 8:
        assert e1 > 30 * e3, (e1, e3)


def test_tc_gemm_rejects_bad_shapes(tt):
    A = torch.zeros(128, 8, device="cuda")
    for N in (8, 24, 272):
        with pytest.raises(tt.TTError) as e:
            tt.tc_gemm(A, torch.zeros(N, 8, device="cuda"))
        assert e.value.status == tt.TT_ERR_ARG


@pytest.mark.parametrize("kind,iters", [("fp64", 20000), ("fp32", 20000), ("tf32_tensor", 20000)])
def test_peak_probes_report_work(tt, kind, iters):
    flops, ms = tt.peak_probe(kind, iters)
    assert flops > 0 and ms > 0
    tf = flops / (ms * 1e-3) / 1e12
    # far below or above the part's nominal rates means the probe did not run the work it counts
    lo, hi = {"fp64": (0.3, 2.0), "fp32": (20.0, 120.0), "tf32_tensor": (200.0, 1600.0)}[kind]
    assert lo < tf < hi, (kind, tf)
