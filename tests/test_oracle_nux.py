"""Pins of the split-topology oracle [Z(nu x)][y][theta][phi] (oracle/naive_tt_nux.py), the
topology of the configuration with ranks up to 256 and a separate y core:

* exact rank (tol 0): three steps equal the dense stepper for the upwind, Rusanov and central
  fluxes (the dense row k = g + G (ix + Nx iy) is the split (g, ix) x iy);
* the transport sum equals the dense operator applied to the full tensor, with ranks
  (n + 1) r at every bond;
* the source sum equals the dense source step (transport switched off);
* at tol 1e-6 the energy density stays within 1e-5 of the merged-topology oracle's;
* opacities that depend on y are refused (the source is a row scaling of core 0 only when they
  do not).
"""
import dataclasses

import numpy as np
import pytest

from oracle import dense, naive_tt as nt, naive_tt_nux as nux, problem
from paper_2602_00290_gb300.workloads import nux_config, plane_config1, random_tt


@pytest.mark.parametrize("flux", ["upwind", "rusanov", "central"])
def test_exact_rank_split_topology_step_equals_dense(flux):
    wl = nux_config().with_(flux=flux)
    coef = problem.build(wl)
    S = dense.DenseSolver(wl, coef)
    I = S.initial()
    x = nux.from_rows(problem.initial_rows(wl, coef), coef)
    assert np.max(np.abs(nux.to_dense_rows(x) - I)) <= 1e-14 * np.max(np.abs(I))
    for _ in range(3):
        I = S.step(I)
        x = nux.step(x, coef, 0.0, 10 ** 6)
        assert np.max(np.abs(nux.to_dense_rows(x) - I)) <= 1e-12 * np.max(np.abs(I))
        E = S.energy_density(I)
        assert np.max(np.abs(nux.energy_density_rows(x, coef) - E)) <= 1e-12 * np.max(np.abs(E))


def _no_material(coef):
    c = dataclasses.replace(coef)
    c.acoef = np.zeros_like(coef.acoef)
    c.scoef = np.zeros_like(coef.scoef)
    c.eps = np.zeros_like(coef.eps)
    return c


@pytest.mark.parametrize("flux,nterm", [("upwind", 4), ("rusanov", 4), ("central", 2)])
def test_split_topology_transport_sum_equals_dense_operator(flux, nterm):
    wl = nux_config().with_(flux=flux)
    coef = problem.build(wl)
    x = random_tt([wl.ngroup * wl.nx, wl.ny, wl.ntheta, wl.nphi], [3, 2, 2], seed=19)
    t = nux.transport_sum(x, coef)
    assert nt.ranks(t)[1:-1] == [(nterm + 1) * 3, (nterm + 1) * 2, (nterm + 1) * 2]
    ref = dense.DenseSolver(wl, _no_material(coef)).step(nux.to_dense_rows(x))
    assert np.max(np.abs(nux.to_dense_rows(t) - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_split_topology_source_sum_equals_dense_source():
    wl = nux_config()
    coef = problem.build(wl)
    no_transport = dataclasses.replace(coef)
    no_transport.lam = np.zeros(3)
    x = random_tt([wl.ngroup * wl.nx, wl.ny, wl.ntheta, wl.nphi], [3, 2, 2], seed=23)
    x[0] = np.abs(x[0])
    got = nux.to_dense_rows(nux.source_sum(x, coef))
    ref = dense.DenseSolver(wl, no_transport).step(nux.to_dense_rows(x))
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_rounded_split_topology_tracks_the_merged_topology():
    wl = nux_config(tol=1e-6, rmax=64)
    coef = problem.build(wl)
    x4 = nux.from_rows(problem.initial_rows(wl, coef), coef)
    x3 = nt.initial_tt(problem.initial_rows(wl, coef), coef)
    for _ in range(4):
        x4 = nux.step(x4, coef, wl.tol, wl.rmax)
        x3 = nt.step(x3, coef, wl.tol, wl.rmax)
    E4 = nux.energy_density_rows(x4, coef)
    E3 = nt.energy_density_rows(x3, coef)
    assert np.linalg.norm(E4 - E3) <= 1e-5 * np.linalg.norm(E3)


def test_y_dependent_opacities_are_refused():
    wl = plane_config1(nx=6, ny=5, G=3, ntheta=4, nphi=8)     # blob density depends on y
    coef = problem.build(wl)
    x = random_tt([wl.ngroup * wl.nx, wl.ny, wl.ntheta, wl.nphi], [2, 2, 2], seed=3)
    with pytest.raises(AssertionError):
        nux.source_sum(x, coef)
