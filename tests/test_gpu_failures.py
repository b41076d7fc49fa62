"""Failure paths of the C ABI on the GPU, made on the host or by a bounded wait that runs out; no
test faults, traps or hangs the GPU.

* A NaN (or Inf) written into a core by the host: the step or rounding latches TT_ERR_NONFINITE
  (the update pass that writes the new merged core sees the non-finite rows; a non-finite column
  norm gives no reflector, so the factorisation itself passes over them), every index the kernels
  form from non-finite values stays in range (ranks of NaN sort last), and the context then steps a
  clean state exactly as the oracle does.
* The FP64 Jacobi sweep cap set to 1 (tt_context_set_limits): the SVD is still rotating when it
  stops, TT_ERR_TIMEOUT is latched, and the default cap restores parity.
* Every grid-wide barrier of the cooperative Jacobi told to wait for one arrival that never comes,
  with a spin limit of 2000: every wait runs out (well under a millisecond), all CTAs leave,
  TT_ERR_TIMEOUT is latched, and the next launch starts a fresh barrier.
* A workspace too small for the step while the caller's stream is being captured (the library
  cannot grow it then): TT_ERR_WORKSPACE before anything is enqueued."""
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


WL = plane_config1(nx=12, ny=10, G=5, ntheta=4, nphi=8, rmax=8, tol=1e-6)


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b)))) / max(float(np.max(np.abs(np.asarray(b)))), 1e-300)


def _clean_step_matches_oracle(tt, ctx, plan, prec="fp64", dtype="f64"):
    """One step of a fresh state from I0 against the oracle (the context is still usable)."""
    coef = problem.build(WL)
    x = tt.initial_state(plan, [WL.rmax, WL.rmax], dtype)
    ref = nt.step(nt.initial_tt(problem.initial_rows(WL, coef), coef), coef, WL.tol, WL.rmax)
    tt.tt_step(ctx, plan, x, WL.tol, WL.rmax, prec)
    ctx.sync()
    if prec == "fp64":
        assert x.ranks() == nt.ranks(ref)
        assert rel(nt.to_dense_rows(x.to_cores()), nt.to_dense_rows(ref)) < 1e-10
    else:
        E = tt.tt_energy_density(ctx, plan, x).cpu().numpy()
        Er = nt.energy_density_rows(ref, coef)
        assert np.linalg.norm(E - Er) <= 1e-6 * np.linalg.norm(Er)


@pytest.mark.parametrize("prec,dtype", [("fp64", "f64"), ("mixed", "f32"), ("mixed", "f64")])
@pytest.mark.parametrize("core,graphs", [(0, False), (1, False), (0, True)])
def test_nan_in_a_core_latches_nonfinite(tt, prec, dtype, core, graphs):
    ctx = tt.Context(0)
    ctx.set_graphs(graphs)
    plan = tt.Plan(ctx, WL)
    x = tt.initial_state(plan, [WL.rmax, WL.rmax], dtype)
    for _ in range(3 if graphs else 1):  # with graphs: eager, capture, replay of a clean state
        tt.tt_step(ctx, plan, x, WL.tol, WL.rmax, prec)
    ctx.sync()
    x.cores[core][3, 0] = float("nan")
    tt.tt_step(ctx, plan, x, WL.tol, WL.rmax, prec)
    with pytest.raises(tt.TTError) as e:
        ctx.sync()
    assert e.value.status == tt.TT_ERR_NONFINITE
    r = x.ranks()
    assert all(1 <= q <= WL.rmax for q in r[1:-1])  # ranks stay inside the capacity
    ctx.sync()  # the status was cleared by the sync that reported it
    _clean_step_matches_oracle(tt, ctx, plan, prec, dtype)
    plan.close()
    ctx.close()


def test_nan_in_round_latches_nonfinite(tt):
    ctx = tt.Context(0)
    a = random_tt([300, 6, 7], [5, 4], seed=8)
    x = tt.TT.from_cores(a, rcap=[8, 8])
    x.cores[2][9, 0] = float("inf")  # the last core is [rcap_2 n_2][1]
    tt.tt_round(ctx, x, 1e-8, 8)
    with pytest.raises(tt.TTError) as e:
        ctx.sync()
    assert e.value.status == tt.TT_ERR_NONFINITE
    y = tt.TT.from_cores(a, rcap=[8, 8])
    tt.tt_round(ctx, y, 1e-12, 8)
    ctx.sync()
    assert y.ranks()[1:-1] == [5, 4]
    assert rel(nt.full(y.to_cores()), nt.full(a)) < 1e-11
    ctx.close()


def test_jacobi_sweep_cap_latches_timeout(tt):
    ctx = tt.Context(0)
    plan = tt.Plan(ctx, WL)
    x = tt.initial_state(plan, [WL.rmax, WL.rmax], "f64")
    tt.tt_step(ctx, plan, x, WL.tol, WL.rmax, "fp64")  # rank > 1 from here on: the SVDs rotate
    ctx.sync()
    ctx.set_limits(jacobi_sweeps=1)
    tt.tt_step(ctx, plan, x, WL.tol, WL.rmax, "fp64")
    with pytest.raises(tt.TTError) as e:
        ctx.sync()
    assert e.value.status == tt.TT_ERR_TIMEOUT
    ctx.set_limits()
    _clean_step_matches_oracle(tt, ctx, plan)
    plan.close()
    ctx.close()


@pytest.mark.parametrize("graphs", [False, True])
def test_grid_barrier_wait_runs_out(tt, graphs):
    ctx = tt.Context(0)
    ctx.set_graphs(graphs)
    plan = tt.Plan(ctx, WL)
    x = tt.initial_state(plan, [WL.rmax, WL.rmax], "f64")
    for _ in range(3 if graphs else 1):
        tt.tt_step(ctx, plan, x, WL.tol, WL.rmax, "fp64")
    ctx.sync()
    ctx.set_limits(barrier_spins=2000, barrier_extra=1)
    tt.tt_step(ctx, plan, x, WL.tol, WL.rmax, "fp64")
    with pytest.raises(tt.TTError) as e:
        ctx.sync()
    assert e.value.status == tt.TT_ERR_TIMEOUT
    ctx.set_limits()
    _clean_step_matches_oracle(tt, ctx, plan)
    plan.close()
    ctx.close()


def test_workspace_too_small_under_capture(tt):
    s = torch.cuda.Stream()
    ctx = tt.Context(0, stream=s, workspace_bytes=4096)
    plan = tt.Plan(ctx, WL)
    x = tt.initial_state(plan, [WL.rmax, WL.rmax], "f64")
    buf = torch.zeros(1, device="cuda")
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    err = None
    with torch.cuda.graph(g, stream=s, capture_error_mode="relaxed"):
        buf.add_(1.0)  # the caller's own work in the capture
        try:
            tt.tt_step(ctx, plan, x, WL.tol, WL.rmax, "fp64")
        except tt.TTError as e:
            err = e
    assert err is not None and err.status == tt.TT_ERR_WORKSPACE
    torch.cuda.synchronize()
    # outside the capture the library sizes its workspace and steps as usual
    with torch.cuda.stream(s):
        _clean_step_matches_oracle(tt, ctx, plan)
    plan.close()
    ctx.close()
