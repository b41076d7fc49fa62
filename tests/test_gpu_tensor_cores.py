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


# ------------------------------------------------------------- the mixed step on the tensor cores

from oracle import naive_tt as nt, problem  # noqa: E402
from paper_2602_00290_gb300.workloads import cube_config, plane_config1, slab_config0  # noqa: E402


def fro_rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _plane(**kw):
    args = dict(nx=12, ny=10, G=5, ntheta=4, nphi=8, rmax=8, tol=1e-6)
    args.update(kw)
    return plane_config1(**args)


TC_CASES = {
    "small_r8": _plane(),
    "r16_inflow": _plane(nx=14, ny=12, G=6, ntheta=8, nphi=16, rmax=16).with_(
        inflow_temperature=(0.9, None, 0.6, None, None, None)),
    "r32": _plane(nx=20, ny=16, G=8, ntheta=8, nphi=16, rmax=32),
    "rusanov_r16": _plane(rmax=16).with_(flux="rusanov"),
    "central_r8": _plane().with_(flux="central"),
    "cube_r8_inflow": cube_config().with_(inflow_temperature=(0.9, None, None, None, 0.6, None)),
    "slab_r8_rusanov": slab_config0().with_(flux="rusanov", tol=1e-6),
}


@pytest.mark.parametrize("name", list(TC_CASES))
def test_mixed_3xtf32_step_matches_oracle(tt, name):
    """Steps with the update pass on the tensor cores (FP32 state): energy density within 1e-6 of
    the FP64 oracle after every step, as the benchmark spec asks of the mixed path; and not bit-identical
    to the FP32-SIMT mixed step from the same state (the tensor-core kernel really ran) while within
    1e-6 of it."""
    wl = TC_CASES[name]
    ctx = tt.Context(0)
    coef = problem.build(wl)
    plan = tt.Plan(ctx, wl)
    rc = [wl.rmax] if wl.ndim == 1 else [wl.rmax, wl.rmax]
    x = tt.initial_state(plan, rc, "f32")
    ref = nt.initial_tt(problem.initial_rows(wl, coef), coef)
    errs = []
    for _ in range(5):
        y = tt.TT.from_cores(x.to_cores(), rcap=rc, dtype="f32")
        tt.tt_step(ctx, plan, x, wl.tol, wl.rmax, "mixed_3xtf32")
        tt.tt_step(ctx, plan, y, wl.tol, wl.rmax, "mixed")
        ref = nt.step(ref, coef, wl.tol, wl.rmax)
        ctx.sync()
        E = tt.tt_energy_density(ctx, plan, x).cpu().numpy()
        Ey = tt.tt_energy_density(ctx, plan, y).cpu().numpy()
        errs.append(fro_rel(E, nt.energy_density_rows(ref, coef)))
        assert fro_rel(E, Ey) <= 1e-6
    assert max(errs) <= 1e-6, errs
    assert not np.array_equal(E, Ey), "the tensor-core update did not run"
    plan.close()
    ctx.close()


def test_mixed_3xtf32_with_fp64_storage_runs_the_fp32_kernels(tt):
    """FP64 storage of the merged core cannot feed the FP32 tensor-core operands: the pass runs the
    FP32-SIMT kernels, bit for bit as TT_PREC_MIXED."""
    wl = _plane()
    ctx = tt.Context(0)
    plan = tt.Plan(ctx, wl)
    x = tt.initial_state(plan, [wl.rmax, wl.rmax], "f64")
    y = tt.initial_state(plan, [wl.rmax, wl.rmax], "f64")
    for _ in range(3):
        tt.tt_step(ctx, plan, x, wl.tol, wl.rmax, "mixed_3xtf32")
        tt.tt_step(ctx, plan, y, wl.tol, wl.rmax, "mixed")
    ctx.sync()
    for a, b in zip(x.to_cores(), y.to_cores()):
        assert np.array_equal(a, b)
    plan.close()
    ctx.close()


def test_mixed_3xtf32_graph_replay_equals_eager(tt):
    wl = _plane(rmax=16)
    out = []
    for graphs in (False, True):
        ctx = tt.Context(0)
        ctx.set_graphs(graphs)
        plan = tt.Plan(ctx, wl)
        x = tt.initial_state(plan, [wl.rmax, wl.rmax], "f32")
        for _ in range(5):
            tt.tt_step(ctx, plan, x, wl.tol, wl.rmax, "mixed_3xtf32")
        ctx.sync()
        out.append(x.to_cores())
        if graphs:
            d = ctx.diagnostics()
            assert d["graph_replays"] == 4 and d["graph_failures"] == 0
        plan.close()
        ctx.close()
    for a, b in zip(*out):
        assert np.array_equal(a, b)
