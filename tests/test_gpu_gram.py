"""Gram-based rounding on the GPU (tt_context_set_rounding(..., TT_ROUND_GRAM)) against the
oracle's Gram rounding and against the TSQR route.

Tolerance 1e-9 relative (FP64): both sides form G = A^T A, whose eigenvalues carry an absolute
error of about eps sigma_1^2, i.e. an absolute error of about eps sigma_1^2 / sigma_k on a kept
singular value sigma_k; with sigma_k >= 1e-6 sigma_1 that is at most ~1e-10 sigma_1.  Ranks
must agree wherever the oracle's tail is not within 1e-6 (relative) of the threshold.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import naive_tt as nt, problem  # noqa: E402
from paper_2602_00290_gb300.workloads import plane_config1, random_tt  # noqa: E402
from tie import STEP_KEYS, assert_tie_free  # noqa: E402

TOL = 1e-9
GAP = 1e-6


@pytest.fixture(scope="module")
def tt():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2602_00290_gb300 as mod
    return mod


@pytest.fixture
def gctx(tt):
    c = tt.Context(0)
    c.set_rounding("gram")
    yield c
    c.close()


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b)))) / max(float(np.max(np.abs(np.asarray(b)))), 1e-300)


@pytest.mark.parametrize("tol,rmax", [(1e-2, 20), (1e-4, 20), (1e-6, 20), (1e-3, 4)])
def test_gram_round_matches_oracle(tt, gctx, tol, rmax):
    n = [233, 5, 9]
    a = nt.add_many([nt.scale(random_tt(n, [3, 2], seed=20 + i), 10.0 ** -i) for i in range(6)])
    info = {}
    want = nt.round_tt_gram(a, tol, rmax, info)
    x = tt.TT.from_cores(a, rcap=[20, 20])
    tt.tt_round(gctx, x, tol, rmax)
    gctx.sync()
    assert_tie_free(info, tie=GAP)
    assert x.ranks() == nt.ranks(want)
    assert rel(nt.full(x.to_cores()), nt.full(want)) < TOL


def test_gram_round_exact_rank(tt, gctx):
    a = random_tt([1000, 16, 32], [12, 9], seed=8)
    x = tt.TT.from_cores(a, rcap=[15, 12])
    tt.tt_round(gctx, x, 1e-6, 12)
    gctx.sync()
    assert x.ranks()[1:-1] == [12, 9]
    assert rel(nt.full(x.to_cores()), nt.full(a)) < 1e-9


@pytest.mark.parametrize("kw", [dict(), dict(inflow_temperature=(0.9, None, 0.6, None, None, None)),
                                dict(nx=7, ny=9, G=3, ntheta=6, nphi=12, rmax=10)])
def test_gram_step_matches_oracle(tt, gctx, kw):
    infl = kw.pop("inflow_temperature", None)
    args = dict(nx=12, ny=10, G=5, ntheta=4, nphi=8, rmax=8, tol=1e-6)
    args.update(kw)
    wl = plane_config1(**args)
    if infl is not None:
        wl = wl.with_(inflow_temperature=infl)
    coef = problem.build(wl)
    plan = tt.Plan(gctx, wl)
    x = tt.initial_state(plan, [wl.rmax, wl.rmax], "f64")
    ref = nt.initial_tt(problem.initial_rows(wl, coef), coef)
    for s in range(4):
        info = {}
        tt.tt_step(gctx, plan, x, wl.tol, wl.rmax, "fp64")
        ref = nt.step(ref, coef, wl.tol, wl.rmax, info, rounding="gram")
        gctx.sync()
        assert_tie_free(info, STEP_KEYS, tie=GAP, where=f"step {s}")
        assert x.ranks() == nt.ranks(ref), s
        assert rel(nt.to_dense_rows(x.to_cores()), nt.to_dense_rows(ref)) < TOL, s
        E = tt.tt_energy_density(gctx, plan, x).cpu().numpy()
        assert rel(E, nt.energy_density_rows(ref, coef)) < TOL, s


def test_gram_mixed_step_energy_within_1e6(tt, gctx):
    wl = plane_config1(nx=12, ny=10, G=5, ntheta=4, nphi=8, rmax=8, tol=1e-6)
    coef = problem.build(wl)
    plan = tt.Plan(gctx, wl)
    x = tt.initial_state(plan, [wl.rmax, wl.rmax], "f32")
    ref = nt.initial_tt(problem.initial_rows(wl, coef), coef)
    for s in range(4):
        tt.tt_step(gctx, plan, x, wl.tol, wl.rmax, "mixed")
        ref = nt.step(ref, coef, wl.tol, wl.rmax)
        gctx.sync()
        E = tt.tt_energy_density(gctx, plan, x).cpu().numpy()
        Er = nt.energy_density_rows(ref, coef)
        assert np.linalg.norm(E - Er) <= 1e-6 * np.linalg.norm(Er), s


def test_rounding_method_rejects_unknown(tt):
    c = tt.Context(0)
    st = tt.lib().tt_context_set_rounding(c.handle, 7)
    assert st == tt.TT_ERR_ARG
    c.close()
