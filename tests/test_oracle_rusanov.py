"""Pins of the Rusanov flux in the oracle (Appendix A, 'Value of n': two rank-1 terms per axis,
the central difference times n_a and the isotropic diffusion term), read with vacuum ghost cells:

* with the local speed |n_a| in place of alpha = 1 the Rusanov flux is the upwind flux, so the
  dense stepper must reproduce its own upwind update;
* conservation: with no material, the one-step change of sum_i I_i along a slab is the
  difference of the two boundary fluxes, F_{N-1/2} = (n + 1) I_{N-1} / 2 and F_{-1/2} = (n - 1) I_0 / 2;
* the naive TT transport sum equals the dense operator, and the exact-rank TT step the dense step.
"""
import dataclasses

import numpy as np
import pytest

from oracle import dense, naive_tt as nt, problem
from paper_2602_00290_gb300.workloads import plane_config1, random_tt, slab_config0


def _plane(flux="upwind", **kw):
    args = dict(nx=6, ny=5, G=3, ntheta=4, nphi=8, rmax=64, tol=0.0)
    args.update(kw)
    return plane_config1(**args).with_(flux=flux)


def _no_material(coef):
    c = dataclasses.replace(coef)
    c.acoef = np.zeros_like(coef.acoef)
    c.scoef = np.zeros_like(coef.scoef)
    c.eps = np.zeros_like(coef.eps)
    return c


@pytest.mark.parametrize("wl", [slab_config0(), _plane()], ids=["slab", "plane"])
def test_rusanov_with_local_speed_is_upwind(wl):
    coef_up = problem.build(wl)
    coef_ru = dataclasses.replace(problem.build(wl.with_(flux="rusanov")), alpha_local=True)
    rng = np.random.default_rng(3)
    I = rng.random((wl.nrow, coef_up.nang))
    a = dense.DenseSolver(wl, coef_up).step(I)
    b = dense.DenseSolver(wl, coef_ru).step(I)
    assert np.max(np.abs(a - b)) <= 1e-14 * np.max(np.abs(a))
    # alpha = 1 is strictly more diffusive: the two differ
    c = dense.DenseSolver(wl, problem.build(wl.with_(flux="rusanov"))).step(I)
    assert np.max(np.abs(c - a)) > 1e-3 * np.max(np.abs(a))


def test_rusanov_conservation_slab():
    wl = slab_config0().with_(flux="rusanov")
    coef = _no_material(problem.build(wl))
    rng = np.random.default_rng(4)
    I = rng.random((wl.nrow, coef.nang))
    out = dense.DenseSolver(wl, coef).step(I)
    n = coef.dirs["nx"]
    lam = coef.lam[0]
    G = wl.ngroup
    for g in range(G):
        rows = np.arange(g, wl.nrow, G)          # the cells of group g in x order
        before = I[rows].sum(axis=0)
        after = out[rows].sum(axis=0)
        flux_out = 0.5 * (n + 1.0) * I[rows[-1]] - 0.5 * (n - 1.0) * I[rows[0]]
        assert np.allclose(after, before - lam * flux_out, rtol=0, atol=1e-13 * np.max(np.abs(before)))


def test_rusanov_transport_sum_matches_dense_operator():
    wl = _plane(flux="rusanov")
    coef = problem.build(wl)
    x = random_tt([wl.nrow, wl.ntheta, wl.nphi], [3, 2], seed=13)
    ref = dense.DenseSolver(wl, _no_material(coef)).step(nt.to_dense_rows(x))
    t = nt.transport_sum(x, coef)
    assert nt.ranks(t)[1] == (2 * wl.ndim + 1) * 3
    assert np.max(np.abs(nt.to_dense_rows(t) - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("wl", [slab_config0(), _plane()], ids=["slab", "plane"])
def test_rusanov_exact_rank_tt_step_equals_dense(wl):
    wl = wl.with_(flux="rusanov", tol=0.0, rmax=64)
    coef = problem.build(wl)
    S = dense.DenseSolver(wl, coef)
    I = S.initial()
    x = nt.initial_tt(problem.initial_rows(wl, coef), coef)
    for _ in range(4):
        I = S.step(I)
        x = nt.step(x, coef, 0.0, 10 ** 6)
        assert np.max(np.abs(nt.to_dense_rows(x) - I)) <= 1e-12 * np.max(np.abs(I))


def test_rusanov_refuses_inflow():
    with pytest.raises(ValueError):
        problem.build(_plane(flux="rusanov").with_(inflow_temperature=(0.8, None, None, None, None, None)))
