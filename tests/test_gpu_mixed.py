"""Mixed precision (FP32 passes over the merged core, FP64 small cores) against the FP64 oracle.

Target (the benchmark spec): relative error <= 1e-6 in the angle-integrated energy density at rounding
tolerance 1e-6, with the error stated for every result; the FP32 round-off (6e-8 per stored
value and per pass) leaves about an order of magnitude of room over a few steps.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import naive_tt as nt, problem  # noqa: E402
from paper_2602_00290_gb300.workloads import plane_config1, random_tt  # noqa: E402


@pytest.fixture(scope="module")
def tt():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2602_00290_gb300 as mod
    return mod


@pytest.fixture(scope="module")
def ctx(tt):
    return tt.Context(0)


def fro_rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("kw", [dict(), dict(nx=20, ny=16, G=8, ntheta=8, nphi=16, rmax=12),
                                dict(nx=16, ny=12, G=6, ntheta=8, nphi=16, rmax=48)],
                         ids=["small", "medium", "rank_capacity_48"])
def test_mixed_step_energy_density_within_1e6(tt, ctx, dtype, kw):
    args = dict(nx=12, ny=10, G=5, ntheta=4, nphi=8, rmax=8, tol=1e-6)
    args.update(kw)
    wl = plane_config1(**args)
    coef = problem.build(wl)
    plan = tt.Plan(ctx, wl)
    x = tt.initial_state(plan, [wl.rmax, wl.rmax], dtype)
    ref = nt.initial_tt(problem.initial_rows(wl, coef), coef)
    errs = []
    for _ in range(5):
        tt.tt_step(ctx, plan, x, wl.tol, wl.rmax, "mixed")
        ref = nt.step(ref, coef, wl.tol, wl.rmax)
        ctx.sync()
        E = tt.tt_energy_density(ctx, plan, x).cpu().numpy()
        errs.append(fro_rel(E, nt.energy_density_rows(ref, coef)))
    assert max(errs) <= 1e-6, errs


def test_mixed_round_reconstruction(tt, ctx):
    a = random_tt([700, 6, 9], [5, 4], seed=3)
    for dtype in ("f64", "f32"):
        x = tt.TT.from_cores(a, rcap=[8, 8], dtype=dtype)
        tt.tt_round(ctx, x, 1e-12, 8, "mixed")
        ctx.sync()
        assert x.ranks() == [1, 5, 4, 1]
        assert fro_rel(nt.full(x.to_cores()), nt.full(a)) < 1e-6


@pytest.mark.parametrize("seed0", [20, 40])
@pytest.mark.parametrize("tol", [1e-2, 1e-4, 3e-6])
def test_mixed_round_ranks_match_oracle(tt, ctx, seed0, tol):
    """Mixed rounding keeps the oracle's ranks wherever the oracle's tail is farther from the
    threshold than the FP32 resolution of the singular values (about 6e-8 |X| each): a relative
    gap of 0.2 at tol 3e-6, 0.01 above."""
    n = [233, 5, 9]
    terms = [nt.scale(random_tt(n, [3, 2], seed=seed0 + i), 10.0 ** -i) for i in range(6)]
    a = nt.add_many(terms)
    info = {}
    want = nt.round_tt(a, tol, 20, info)
    need = 0.2 if tol < 1e-5 else 0.01
    assert all(b["gap"] > need for b in info["bonds"])
    x = tt.TT.from_cores(a, rcap=[20, 20])
    tt.tt_round(ctx, x, tol, 20, "mixed")
    ctx.sync()
    assert x.ranks() == nt.ranks(want)
    assert fro_rel(nt.full(x.to_cores()), nt.full(want)) < 1e-5


@pytest.mark.parametrize("prec,dtype,bound", [("mixed", "f32", 2e-6), ("mixed", "f64", 1e-10), ("fp64", "f64", 1e-10)])
def test_step_leaves_angular_cores_right_orthonormal(tt, ctx, prec, dtype, bound):
    """A rounded state keeps its angular cores right-orthonormal (Sec. 3.1: the R->L sweep leaves
    C_k <- V_k^T); in the mixed path the phi core's columns come from FP32 Jacobi vectors that the
    Newton-Schulz steps (FP32, then FP64) make orthonormal, so every bound here is the storage
    precision's."""
    wl = plane_config1(nx=12, ny=10, G=5, ntheta=4, nphi=8, rmax=8, tol=1e-6)
    plan = tt.Plan(ctx, wl)
    x = tt.initial_state(plan, [wl.rmax, wl.rmax], dtype)
    worst = []
    for _ in range(4):
        tt.tt_step(ctx, plan, x, wl.tol, wl.rmax, prec)
        ctx.sync()
        C = x.to_cores()
        th = C[1].reshape(C[1].shape[0], -1)
        ph = C[2].reshape(C[2].shape[0], -1)
        worst.append(max(np.abs(th @ th.T - np.eye(th.shape[0])).max(),
                         np.abs(ph @ ph.T - np.eye(ph.shape[0])).max()))
    assert x.ranks()[2] > 1, x.ranks()
    assert max(worst) <= bound, worst
