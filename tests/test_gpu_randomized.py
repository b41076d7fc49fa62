"""Randomized rounding on the GPU (TT_ROUND_RANDOMIZED with a caller-drawn sketch) against the
oracle's randomized rounding with the same sketch: 1e-10 relative and identical ranks in FP64
(the two QR factors of the sketch differ only by column signs, which the SVD sweep does not
see), 1e-6 in energy density for the mixed path."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import naive_tt as nt, problem  # noqa: E402
from paper_2602_00290_gb300.workloads import plane_config1, random_tt, sketch_matrix  # noqa: E402
from tie import STEP_KEYS, assert_tie_free  # noqa: E402



@pytest.fixture(scope="module")
def tt():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2602_00290_gb300 as mod
    return mod


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b)))) / max(float(np.max(np.abs(np.asarray(b)))), 1e-300)


def _ctx(tt, omega):
    c = tt.Context(0)
    c.set_sketch(omega)
    c.set_rounding("randomized")
    return c


@pytest.mark.parametrize("tol,ell", [(1e-2, 10), (1e-4, 14), (1e-6, 20), (1e-8, 8)])
def test_randomized_round_matches_oracle(tt, tol, ell):
    n = [233, 5, 9]
    a = nt.add_many([nt.scale(random_tt(n, [3, 2], seed=20 + i), 10.0 ** -i) for i in range(6)])
    om = sketch_matrix(45, ell, seed=4)
    c = _ctx(tt, om)
    info = {}
    want = nt.round_tt_randomized(a, tol, 20, om, info)
    x = tt.TT.from_cores(a, rcap=[20, 20])
    tt.tt_round(c, x, tol, 20)
    c.sync()
    assert_tie_free(info)
    assert x.ranks() == nt.ranks(want)
    assert rel(nt.full(x.to_cores()), nt.full(want)) < 1e-10
    c.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_randomized_step_matches_oracle(tt, prec):
    wl = plane_config1(nx=12, ny=10, G=5, ntheta=4, nphi=8, rmax=8, tol=1e-6)
    coef = problem.build(wl)
    om = sketch_matrix(32, 12, seed=11)
    c = _ctx(tt, om)
    plan = tt.Plan(c, wl)
    x = tt.initial_state(plan, [wl.rmax, wl.rmax], "f64" if prec == "fp64" else "f32")
    ref = nt.initial_tt(problem.initial_rows(wl, coef), coef)
    for s in range(4):
        info = {}
        tt.tt_step(c, plan, x, wl.tol, wl.rmax, prec)
        ref = nt.step(ref, coef, wl.tol, wl.rmax, info, rounding="randomized", omega=om)
        c.sync()
        if prec == "fp64":
            assert_tie_free(info, STEP_KEYS, where=f"step {s}")
            assert x.ranks() == nt.ranks(ref), s
            assert rel(nt.to_dense_rows(x.to_cores()), nt.to_dense_rows(ref)) < 1e-10, s
        E = tt.tt_energy_density(c, plan, x).cpu().numpy()
        Er = nt.energy_density_rows(ref, coef)
        assert np.linalg.norm(E - Er) <= (1e-10 if prec == "fp64" else 1e-6) * np.linalg.norm(Er), s
    plan.close()
    c.close()


def test_randomized_sketch_shape_is_checked(tt):
    c = _ctx(tt, sketch_matrix(10, 8, seed=1))
    x = tt.TT.from_cores(random_tt([50, 5, 9], [3, 2], seed=2), rcap=[6, 6])
    with pytest.raises(tt.TTError) as e:
        tt.tt_round(c, x, 1e-6, 6)
    assert e.value.status == tt.TT_ERR_SHAPE
    c.close()
