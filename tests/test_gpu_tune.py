"""TSQR kernel choice (tt_context_set_tsqr) and autotuning (tt_autotune).

The row-split TSQR (four lanes per column) runs the same reflector sequence as the column-owner
kernels in a different summation order, so it must meet the same parity bars against the
oracle: FP64 1e-10 relative with identical ranks unless the oracle's tail is within 1e-9 of
the threshold, mixed 1e-6 in energy density.  Leaf caps of 3 and 7 give a ragged last leaf and
odd merge levels (the pass-through copy of the merge tree).  The autotuner must leave the
caller's state and a coupled plan's temperature untouched and store choices that keep parity.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import coupled, naive_tt as nt, problem  # noqa: E402
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


@pytest.fixture
def ctx(tt):
    c = tt.Context(0)
    yield c
    c.close()


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b)))) / max(float(np.max(np.abs(np.asarray(b)))), 1e-300)


def force(ctx, prec, variant, leaves, ncaps=range(1, 257)):
    for n in ncaps:
        ctx.set_tsqr(prec, n, variant, leaves)


@pytest.mark.parametrize("leaves", [0, 3, 7])
@pytest.mark.parametrize("tol,rmax", [(1e-6, 20), (1e-3, 4)])
def test_rowsplit_round_matches_oracle(tt, ctx, leaves, tol, rmax):
    n = [2333, 5, 9]
    a = nt.add_many([nt.scale(random_tt(n, [3, 2], seed=40 + i), 10.0 ** -i) for i in range(6)])
    info = {}
    want = nt.round_tt(a, tol, rmax, info)
    force(ctx, "fp64", "rowsplit", leaves)
    x = tt.TT.from_cores(a, rcap=[20, 20])
    tt.tt_round(ctx, x, tol, rmax)
    ctx.sync()
    assert_tie_free(info)
    assert x.ranks() == nt.ranks(want)
    assert rel(nt.full(x.to_cores()), nt.full(want)) < 1e-10


def test_rowsplit_round_exact_rank_slab(tt, ctx):
    """d = 2 and a wide pass (R = 60 columns, 240 lanes) on 7 leaves."""
    a = random_tt([4100, 24], [17], seed=5)
    force(ctx, "fp64", "rowsplit", 7)
    x = tt.TT.from_cores(a, rcap=[60])
    tt.tt_round(ctx, x, 0.0, 60)
    ctx.sync()
    assert x.ranks()[1:-1] == [17]
    assert rel(nt.full(x.to_cores()), nt.full(a)) < 1e-10


@pytest.mark.parametrize("leaves", [0, 3, 7])
@pytest.mark.parametrize("kw", [dict(), dict(inflow_temperature=(0.9, None, 0.6, None, None, None))])
def test_rowsplit_step_matches_oracle(tt, ctx, leaves, kw):
    wl = plane_config1(nx=12, ny=10, G=5, ntheta=4, nphi=8, rmax=8, tol=1e-6)
    if kw:
        wl = wl.with_(**kw)
    coef = problem.build(wl)
    force(ctx, "fp64", "rowsplit", leaves)
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


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_rowsplit_mixed_step_energy_within_1e6(tt, ctx, dtype):
    wl = plane_config1(nx=12, ny=10, G=5, ntheta=4, nphi=8, rmax=8, tol=1e-6)
    coef = problem.build(wl)
    force(ctx, "mixed", "rowsplit", 3)
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


def test_rowsplit_slab_step_matches_oracle(tt, ctx):
    wl = slab_config0()
    coef = problem.build(wl)
    force(ctx, "fp64", "rowsplit", 3)
    plan = tt.Plan(ctx, wl)
    x = tt.initial_state(plan, [wl.rmax], "f64")
    ref = nt.initial_tt(problem.initial_rows(wl, coef), coef)
    for s in range(3):
        info = {}
        tt.tt_step(ctx, plan, x, wl.tol, wl.rmax, "fp64")
        ref = nt.step(ref, coef, wl.tol, wl.rmax, info)
        ctx.sync()
        assert_tie_free(info, STEP_KEYS, where=f"step {s}")
        assert x.ranks() == nt.ranks(ref), s
        assert rel(nt.to_dense_rows(x.to_cores()), nt.to_dense_rows(ref)) < 1e-10, s


def test_get_tsqr_defaults_and_clear(tt, ctx):
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    assert ctx.get_tsqr("fp64", 41) == ("column", 2 * nsm)
    assert ctx.get_tsqr("mixed", 41) == ("column", 3 * nsm)
    ctx.set_tsqr("mixed", 41, "rowsplit", 10)
    assert ctx.get_tsqr("mixed", 41) == ("rowsplit", 10)
    assert ctx.get_tsqr("fp64", 41) == ("column", 2 * nsm)
    ctx.set_tsqr("mixed", 41, "rowsplit", 10 ** 6)  # above six per SM: clamped
    assert ctx.get_tsqr("mixed", 41) == ("rowsplit", 6 * nsm)
    ctx.set_tsqr("mixed", 300, "rowsplit", 0)  # 4 x 300 lanes > 1024: column kernels run
    assert ctx.get_tsqr("mixed", 300) == ("column", 3 * nsm)
    ctx.set_tsqr("mixed", 200, "column", 0)  # 224 threads: column kernels
    assert ctx.get_tsqr("mixed", 200)[0] == "column"
    ctx.set_tsqr("mixed", 250, "column", 0)  # 256 threads: still column
    assert ctx.get_tsqr("mixed", 250)[0] == "column"
    ctx.set_tsqr("mixed", 161, "column_dense", 0)  # 192 threads > 160: column kernels
    assert ctx.get_tsqr("mixed", 161)[0] == "column"
    ctx.set_tsqr("fp64", 60, "column_dense", 0)  # FP64: column kernels
    assert ctx.get_tsqr("fp64", 60)[0] == "column"
    ctx.set_tsqr("mixed", 160, "column_dense", 4 * nsm)
    assert ctx.get_tsqr("mixed", 160) == ("column_dense", 4 * nsm)
    ctx.set_tsqr("mixed", 0)
    assert ctx.get_tsqr("mixed", 41) == ("column", 3 * nsm)
    ctx.set_tsqr("mixed", 224, "blocked", 0)  # the blocked leaf takes up to 224 columns in FP32
    assert ctx.get_tsqr("mixed", 224)[0] == "blocked"
    ctx.set_tsqr("mixed", 232, "blocked", 0)
    assert ctx.get_tsqr("mixed", 232)[0] == "column"
    ctx.set_tsqr("fp64", 64, "blocked", 0)
    assert ctx.get_tsqr("fp64", 64)[0] == "column"
    ctx.set_tsqr("mixed", 0)
    assert tt.lib().tt_context_set_tsqr(ctx.handle, tt.TT_PREC_MIXED, 41, 4, 0) == tt.TT_ERR_ARG
    assert tt.lib().tt_context_set_tsqr(ctx.handle, 9, 41, 0, 0) == tt.TT_ERR_ARG


def _snapshot(x):
    return x.ranks(), [c.cpu().numpy().copy() for c in x.cores]


@pytest.mark.parametrize("prec,dtype", [("mixed", "f32"), ("fp64", "f64")])
def test_autotune_keeps_state_and_parity(tt, ctx, prec, dtype):
    wl = plane_config1(nx=24, ny=20, G=6, ntheta=4, nphi=8, rmax=8, tol=1e-6)
    coef = problem.build(wl)
    plan = tt.Plan(ctx, wl)
    x = tt.initial_state(plan, [wl.rmax, wl.rmax], dtype)
    ref = nt.initial_tt(problem.initial_rows(wl, coef), coef)
    tt.tt_step(ctx, plan, x, wl.tol, wl.rmax, prec)
    ref = nt.step(ref, coef, wl.tol, wl.rmax)
    ctx.sync()
    before = _snapshot(x)
    res = ctx.autotune(plan, x, wl.tol, wl.rmax, prec, steps=1)
    after = _snapshot(x)
    assert before[0] == after[0]
    for a, b in zip(before[1], after[1]):
        assert np.array_equal(a, b)
    K1 = wl.rmax
    ncaps = {"transport": 5 * K1, "source": K1 + 1}
    for role, ncap in ncaps.items():
        v, l = res[role]
        assert v in ("column", "rowsplit", "column_dense", "blocked") and l > 0
        assert ctx.get_tsqr(prec, ncap) == (v, l)
    assert 0 < res["ms_tuned"] <= res["ms_default"]
    for s in range(3):
        tt.tt_step(ctx, plan, x, wl.tol, wl.rmax, prec)
        info = {}
        ref = nt.step(ref, coef, wl.tol, wl.rmax, info)
        ctx.sync()
        if prec == "fp64":
            assert_tie_free(info, STEP_KEYS, where=f"step {s}")
            assert x.ranks() == nt.ranks(ref), s
            assert rel(nt.to_dense_rows(x.to_cores()), nt.to_dense_rows(ref)) < 1e-10, s
        else:
            E = tt.tt_energy_density(ctx, plan, x).cpu().numpy()
            Er = nt.energy_density_rows(ref, coef)
            assert np.linalg.norm(E - Er) <= 1e-6 * np.linalg.norm(Er), s


def test_autotune_restores_coupled_temperature(tt, ctx):
    wl = plane_config1(nx=12, ny=10, G=5, ntheta=4, nphi=8, rmax=8, tol=1e-6)
    rho_cv = np.full(wl.nx * wl.ny, 0.5)
    wl = wl.with_(rho_cv=rho_cv)
    plan = tt.Plan(ctx, wl)
    x = tt.initial_state(plan, [wl.rmax, wl.rmax], "f64")
    T0 = np.array(plan.temperature(), copy=True)
    ctx.autotune(plan, x, wl.tol, wl.rmax, "fp64", steps=1)
    assert np.array_equal(plan.temperature(), T0)
    # the tuned stepper still advances the material like the oracle
    coef = problem.build(wl)
    edges = np.asarray(wl.group_edges)
    ref = nt.initial_tt(problem.initial_rows(wl, coef), coef)
    T = np.asarray(wl.temperature, dtype=float).copy()
    for s in range(2):
        tt.tt_step(ctx, plan, x, wl.tol, wl.rmax, "fp64")
        ref, T, _ = coupled.tt_step(ref, coef, T, rho_cv, edges, wl.tol, wl.rmax)
        ctx.sync()
        assert rel(plan.temperature(), T) < 1e-10, s


def test_autotune_rejects_other_roundings(tt, ctx):
    wl = plane_config1(nx=6, ny=5, G=3, ntheta=4, nphi=8, rmax=6, tol=1e-6)
    plan = tt.Plan(ctx, wl)
    x = tt.initial_state(plan, [wl.rmax, wl.rmax], "f64")
    ctx.set_rounding("gram")
    with pytest.raises(tt.TTError) as e:
        ctx.autotune(plan, x, wl.tol, wl.rmax, "fp64", steps=1)
    assert e.value.status == tt.TT_ERR_UNSUPPORTED
    ctx.set_rounding("tsqr")
    with pytest.raises(tt.TTError) as e:
        ctx.autotune(plan, x, wl.tol, wl.rmax, "fp64", steps=0)
    assert e.value.status == tt.TT_ERR_ARG
