"""The Rusanov flux on the GPU against the oracle (tolerances as for the upwind flux: 1e-13 for
the exact transport sum, 1e-10 and identical ranks for rounded FP64 steps, 1e-6 in energy
density for the mixed path)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import dense, naive_tt as nt, problem  # noqa: E402
from paper_2602_00290_gb300.workloads import plane_config1, random_tt, slab_config0  # noqa: E402
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


def _plane(**kw):
    args = dict(nx=12, ny=10, G=5, ntheta=4, nphi=8, rmax=8, tol=1e-6)
    args.update(kw)
    return plane_config1(**args).with_(flux="rusanov")


@pytest.mark.parametrize("wl", [_plane(), slab_config0().with_(flux="rusanov")], ids=["plane", "slab"])
def test_rusanov_apply_transport_matches_explicit_sum(tt, ctx, wl):
    coef = problem.build(wl)
    plan = tt.Plan(ctx, wl)
    n = plan.n
    r = [3] if len(n) == 2 else [3, 2]
    a = random_tt(n, r, seed=6)
    x = tt.TT.from_cores(a, rcap=[q + 1 for q in r])
    want = nt.transport_sum(a, coef)
    R = nt.ranks(want)[1:-1]
    out = tt.TT(n, [q + 2 for q in R])
    tt.tt_apply_transport(ctx, plan, x, out)
    ctx.sync()
    assert out.ranks()[1:-1] == R
    assert rel(nt.full(out.to_cores()), nt.full(want)) < 1e-13


@pytest.mark.parametrize("kw", [dict(), dict(tol=1e-8, rmax=12), dict(nx=7, ny=9, G=3, ntheta=6, nphi=12, rmax=10)])
def test_rusanov_step_matches_naive_tt(tt, ctx, kw):
    wl = _plane(**kw)
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


def test_rusanov_slab_exact_rank_matches_dense(tt, ctx):
    wl = slab_config0().with_(flux="rusanov")
    coef = problem.build(wl)
    S = dense.DenseSolver(wl, coef)
    I = S.initial()
    plan = tt.Plan(ctx, wl)
    x = tt.initial_state(plan, [wl.rmax], "f64")
    for _ in range(wl.steps):
        I = S.step(I)
        tt.tt_step(ctx, plan, x, wl.tol, wl.rmax, "fp64")
    ctx.sync()
    assert rel(nt.to_dense_rows(x.to_cores()), I) < 1e-10


def test_rusanov_mixed_energy_within_1e6(tt, ctx):
    wl = _plane()
    coef = problem.build(wl)
    plan = tt.Plan(ctx, wl)
    x = tt.initial_state(plan, [wl.rmax, wl.rmax], "f32")
    ref = nt.initial_tt(problem.initial_rows(wl, coef), coef)
    for s in range(4):
        tt.tt_step(ctx, plan, x, wl.tol, wl.rmax, "mixed")
        ref = nt.step(ref, coef, wl.tol, wl.rmax)
        ctx.sync()
        E = tt.tt_energy_density(ctx, plan, x).cpu().numpy()
        Er = nt.energy_density_rows(ref, coef)
        assert np.linalg.norm(E - Er) <= 1e-6 * np.linalg.norm(Er), s


def test_rusanov_plan_refuses_inflow(tt, ctx):
    wl = _plane().with_(inflow_temperature=(0.8, None, None, None, None, None))
    with pytest.raises(tt.TTError) as e:
        tt.Plan(ctx, wl)
    assert e.value.status == tt.TT_ERR_UNSUPPORTED
