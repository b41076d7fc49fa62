"""Three spatial dimensions (d_X = 3: six upwind or Rusanov terms, three central terms, inflow
columns on x and z faces) on the GPU against the oracle: the transport sum against the explicit
TT sum (1e-13), rounded FP64 steps against the naive TT oracle (1e-10, identical ranks; every seeded
case is asserted tie-free), and the mixed path in energy density (1e-6) with FP32 and FP64 storage of the merged core.
The mixed update passes stage seven row blocks per tile here (the centre and +-s_a on three axes)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import naive_tt as nt, problem  # noqa: E402
from paper_2602_00290_gb300.workloads import cube_config, random_tt  # noqa: E402
from tie import STEP_KEYS, assert_tie_free  # noqa: E402

CASES = [("upwind", (0.9, None, None, None, 0.6, None)), ("rusanov", (None,) * 6), ("central", (None,) * 6)]
IDS = ["upwind_inflow", "rusanov", "central"]


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


@pytest.mark.parametrize("flux,inflow", CASES, ids=IDS)
def test_3d_apply_transport_matches_explicit_sum(tt, ctx, flux, inflow):
    wl = cube_config().with_(flux=flux, inflow_temperature=inflow)
    coef = problem.build(wl)
    plan = tt.Plan(ctx, wl)
    a = random_tt(plan.n, [3, 2], seed=6)
    x = tt.TT.from_cores(a, rcap=[4, 3])
    want = nt.transport_sum(a, coef)
    R = nt.ranks(want)[1:-1]
    out = tt.TT(plan.n, [q + 2 for q in R])
    tt.tt_apply_transport(ctx, plan, x, out)
    ctx.sync()
    assert out.ranks()[1:-1] == R
    assert rel(nt.full(out.to_cores()), nt.full(want)) < 1e-13


@pytest.mark.parametrize("flux,inflow", CASES, ids=IDS)
@pytest.mark.parametrize("kw", [dict(), dict(nx=5, ny=7, nz=6, G=4, ntheta=6, nphi=12, rmax=10, tol=1e-8)],
                         ids=["6x5x4", "5x7x6"])
def test_3d_step_matches_naive_tt(tt, ctx, flux, inflow, kw):
    wl = cube_config(**kw).with_(flux=flux, inflow_temperature=inflow)
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


@pytest.mark.parametrize("flux,inflow", CASES, ids=IDS)
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_3d_mixed_energy_within_1e6(tt, ctx, flux, inflow, dtype):
    wl = cube_config(nx=8, ny=6, nz=5, G=4, ntheta=6, nphi=12, rmax=12).with_(flux=flux, inflow_temperature=inflow)
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
