"""Degenerate cases of tt_step on the GPU against the oracle:

* the zero state with no absorption (nothing emits) stays exactly zero, with every rank 1 and no
  latched error, in both precisions;
* grids with fewer merged rows than transport-sum columns (2x2, 1x1 and 1x3 cells, 2 groups:
  8, 2 and 6 rows against 5 r columns), where the TSQR leaves are mostly zero rows;
* a rank cap of 1 (every rounding truncates to rank 1).

FP64 against the naive TT oracle to 1e-10 with identical ranks (every seeded case asserted tie-free);
mixed to 1e-6 in energy density."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import naive_tt as nt, problem  # noqa: E402
from paper_2602_00290_gb300.workloads import plane_config1  # noqa: E402
from tie import STEP_KEYS, assert_tie_free  # noqa: E402



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


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b)))) / max(float(np.max(np.abs(np.asarray(b)))), 1e-300)


@pytest.mark.parametrize("prec,dtype", [("fp64", "f64"), ("mixed", "f32"), ("mixed", "f64")])
def test_zero_state_without_absorption_stays_zero(tt, ctx, prec, dtype):
    wl = plane_config1(nx=6, ny=5, G=3, ntheta=4, nphi=8, rmax=8, tol=1e-6)
    wl = wl.with_(rho_kappa_a=np.zeros(wl.nrow))
    plan = tt.Plan(ctx, wl)
    zero = [np.zeros((1, wl.nrow, 2)), np.zeros((2, wl.ntheta, 2)), np.zeros((2, wl.nphi, 1))]
    x = tt.TT.from_cores(zero, rcap=[wl.rmax, wl.rmax], dtype=dtype)
    for _ in range(3):
        tt.tt_step(ctx, plan, x, wl.tol, wl.rmax, prec)
    ctx.sync()  # raises on a latched device error (e.g. a non-finite value)
    assert x.ranks() == [1, 1, 1, 1]
    assert not np.any(nt.full(x.to_cores()))
    assert not np.any(tt.tt_energy_density(ctx, plan, x).cpu().numpy())
    plan.close()


TINY = [(2, 2), (1, 1), (1, 3)]


@pytest.mark.parametrize("nx,ny", TINY, ids=["2x2", "1x1", "1x3"])
def test_tiny_grid_fp64_matches_naive_tt(tt, ctx, nx, ny):
    wl = plane_config1(nx=nx, ny=ny, G=2, ntheta=4, nphi=8, rmax=8, tol=1e-12)
    coef = problem.build(wl)
    plan = tt.Plan(ctx, wl)
    x = tt.initial_state(plan, [wl.rmax, wl.rmax], "f64")
    ref = nt.initial_tt(problem.initial_rows(wl, coef), coef)
    for s in range(4):
        info = {}
        tt.tt_step(ctx, plan, x, wl.tol, wl.rmax, "fp64")
        ref = nt.step(ref, coef, wl.tol, wl.rmax, info)
        ctx.sync()
        assert_tie_free(info, STEP_KEYS, where=f"step {s}")
        assert x.ranks() == nt.ranks(ref), s
        assert rel(nt.to_dense_rows(x.to_cores()), nt.to_dense_rows(ref)) < 1e-10, s
    plan.close()


@pytest.mark.parametrize("nx,ny", TINY, ids=["2x2", "1x1", "1x3"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_tiny_grid_mixed_energy_within_1e6(tt, ctx, nx, ny, dtype):
    wl = plane_config1(nx=nx, ny=ny, G=2, ntheta=4, nphi=8, rmax=8, tol=1e-6)
    coef = problem.build(wl)
    plan = tt.Plan(ctx, wl)
    x = tt.initial_state(plan, [wl.rmax, wl.rmax], dtype)
    ref = nt.initial_tt(problem.initial_rows(wl, coef), coef)
    for s in range(4):
        tt.tt_step(ctx, plan, x, wl.tol, wl.rmax, "mixed")
        ref = nt.step(ref, coef, wl.tol, wl.rmax)
        ctx.sync()
        E = tt.tt_energy_density(ctx, plan, x).cpu().numpy()
        Er = nt.energy_density_rows(ref, coef)
        assert np.linalg.norm(E - Er) <= 1e-6 * np.linalg.norm(Er), s
    plan.close()


@pytest.mark.parametrize("prec,dtype", [("fp64", "f64"), ("mixed", "f32")])
def test_rank_cap_one(tt, ctx, prec, dtype):
    wl = plane_config1(nx=6, ny=5, G=3, ntheta=4, nphi=8, rmax=8, tol=1e-6)
    coef = problem.build(wl)
    plan = tt.Plan(ctx, wl)
    x = tt.initial_state(plan, [wl.rmax, wl.rmax], dtype)
    ref = nt.initial_tt(problem.initial_rows(wl, coef), coef)
    for s in range(4):
        tt.tt_step(ctx, plan, x, wl.tol, 1, prec)
        ref = nt.step(ref, coef, wl.tol, 1)
        ctx.sync()
        assert x.ranks() == [1, 1, 1, 1]
        if prec == "fp64":
            assert rel(nt.to_dense_rows(x.to_cores()), nt.to_dense_rows(ref)) < 1e-10, s
        else:
            E = tt.tt_energy_density(ctx, plan, x).cpu().numpy()
            Er = nt.energy_density_rows(ref, coef)
            assert np.linalg.norm(E - Er) <= 1e-6 * np.linalg.norm(Er), s
    plan.close()


@pytest.mark.gpu
@pytest.mark.parametrize("topology", ["merged_nux_y", "split_x"])
def test_plan_refuses_unbuilt_topologies(tt, ctx, topology):
    # the d = 4 layouts have a place in the problem description but no CUDA path
    wl = plane_config1(nx=4, ny=4, G=2, ntheta=2, nphi=4).with_(topology=topology)
    with pytest.raises(tt.TTError) as e:
        tt.Plan(ctx, wl)
    assert "unsupported" in str(e.value).lower() or "TT_ERR_UNSUPPORTED" in str(e.value)
    ok = tt.Plan(ctx, wl.with_(topology="merged"))
    assert ok.d == 3
