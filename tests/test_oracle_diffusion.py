"""Pins of the central flux (the Rusanov flux with wavespeed S+ = 0 that Sec. 4.3 runs its
multigroup Gaussian-diffusion test with) in the oracle.

* Eq. (diffusion): with pure scattering rho*kappa_s[f] in [1000, 2000] the S_N solution of an
  isotropic Gaussian diffuses with D_f = c / (3 rho kappa_s,f); after 4000 steps at CFL 1 the
  oracle's energy density must match E_f(t, x; t_0) of Eq. (diffusion) in every group.  The
  paper's t_0 = 1e-3 / D_f gives a Gaussian narrower than one of 128 cells on [-5, 5]; the pin
  takes t_0 = 0.25 / D_f (identical initial data in every group, as in the paper, but resolved).
  The upwind and alpha = 1 Rusanov fluxes carry numerical diffusion of order c dx and miss the
  same solution by far more: the pin tells the fluxes apart.
* conservation: with no material, the one-step change of sum_i I_i along a slab is the difference
  of the boundary fluxes F_{N-1/2} = n I_{N-1} / 2 and F_{-1/2} = n I_0 / 2 (vacuum ghost cells);
* one rank-1 term per axis: the naive TT transport sum has rank (d_X + 1) r and equals the dense
  operator, and the exact-rank TT step equals the dense step.
"""
import dataclasses
import math

import numpy as np
import pytest

from oracle import dense, naive_tt as nt, problem
from paper_2602_00290_gb300.workloads import (gaussian_diffusion_config, plane_config1, random_tt,
                                              slab_config0)

DT0 = 0.25


def diffusion_energy(wl, t):
    """E_f(t, x; t_0) of Eq. (diffusion) with A = 1, at the cell centres of [-5, 5], per merged row."""
    G = wl.ngroup
    dx = wl.extent[0] / wl.nx
    x = -0.5 * wl.extent[0] + (np.arange(wl.nx) + 0.5) * dx
    D = wl.c / (3.0 * np.asarray(wl.rho_kappa_s[:G]))
    s = 4.0 * D[None, :] * (DT0 / D[None, :] + t)
    return (np.exp(-x[:, None] ** 2 / s) / np.sqrt(math.pi * s)).reshape(-1)


def _no_material(coef):
    c = dataclasses.replace(coef)
    c.acoef = np.zeros_like(coef.acoef)
    c.scoef = np.zeros_like(coef.scoef)
    c.eps = np.zeros_like(coef.eps)
    return c


def _run_dense(wl, flux, steps):
    coef = problem.build(wl.with_(flux=flux))
    S = dense.DenseSolver(wl, coef)
    I = np.repeat((diffusion_energy(wl, 0.0) / (4.0 * np.pi))[:, None], coef.nang, axis=1)
    for _ in range(steps):
        I = S.step(I)
    return S.energy_density(I)


def _group_errors(wl, E, t):
    G = wl.ngroup
    want = diffusion_energy(wl, t).reshape(wl.nx, G)
    got = E.reshape(wl.nx, G)
    return np.max(np.abs(got - want), axis=0) / np.max(want, axis=0), want


def test_central_flux_matches_gaussian_diffusion():
    wl = gaussian_diffusion_config()
    steps = wl.steps
    t = steps * wl.dt
    err, want = _group_errors(wl, _run_dense(wl, "central", steps), t)
    assert np.max(err) < 5e-3, err
    # the solution did move: each group's peak fell by more than 8 %, by a group-dependent amount
    decay = np.max(want, axis=0) / np.max(diffusion_energy(wl, 0.0).reshape(wl.nx, -1), axis=0)
    assert np.all(decay < 0.92) and np.ptp(decay) > 0.02
    for flux in ("upwind", "rusanov"):
        err_other, _ = _group_errors(wl, _run_dense(wl, flux, steps), t)
        assert np.min(err_other) > 0.1, (flux, err_other)


def test_central_conservation_slab():
    wl = slab_config0().with_(flux="central")
    coef = _no_material(problem.build(wl))
    rng = np.random.default_rng(4)
    I = rng.random((wl.nrow, coef.nang))
    out = dense.DenseSolver(wl, coef).step(I)
    n = coef.dirs["nx"]
    lam = coef.lam[0]
    for g in range(wl.ngroup):
        rows = np.arange(g, wl.nrow, wl.ngroup)
        before = I[rows].sum(axis=0)
        after = out[rows].sum(axis=0)
        flux_out = 0.5 * n * I[rows[-1]] - 0.5 * n * I[rows[0]]
        assert np.allclose(after, before - lam * flux_out, rtol=0, atol=1e-13 * np.max(np.abs(before)))


def test_central_transport_sum_matches_dense_operator():
    wl = plane_config1(nx=6, ny=5, G=3, ntheta=4, nphi=8, rmax=64, tol=0.0).with_(flux="central")
    coef = problem.build(wl)
    x = random_tt([wl.nrow, wl.ntheta, wl.nphi], [3, 2], seed=13)
    ref = dense.DenseSolver(wl, _no_material(coef)).step(nt.to_dense_rows(x))
    t = nt.transport_sum(x, coef)
    assert nt.ranks(t)[1] == (wl.ndim + 1) * 3
    assert np.max(np.abs(nt.to_dense_rows(t) - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("wl", [gaussian_diffusion_config(nx=32, G=4, ntheta=8),
                                plane_config1(nx=6, ny=5, G=3, ntheta=4, nphi=8)],
                         ids=["diffusion", "plane"])
def test_central_exact_rank_tt_step_equals_dense(wl):
    wl = wl.with_(flux="central", tol=0.0, rmax=64)
    coef = problem.build(wl)
    S = dense.DenseSolver(wl, coef)
    I = S.initial()
    I = I + np.random.default_rng(8).random(I.shape)     # an anisotropic state of full angular rank
    U, s, Vt = np.linalg.svd(I, full_matrices=False)      # the state as an exact TT
    r = len(s)
    if wl.nphi == 1:
        x = [(U * s).reshape(1, wl.nrow, r), Vt.reshape(r, wl.ntheta, 1)]
    else:
        W = Vt.reshape(r, wl.ntheta, wl.nphi)
        U2, s2, V2 = np.linalg.svd(W.reshape(r * wl.ntheta, wl.nphi), full_matrices=False)
        x = [(U * s).reshape(1, wl.nrow, r), (U2 * s2).reshape(r, wl.ntheta, -1), V2.reshape(-1, wl.nphi, 1)]
    assert np.max(np.abs(nt.to_dense_rows(x) - I)) <= 1e-13 * np.max(np.abs(I))
    for _ in range(3):
        I = S.step(I)
        x = nt.step(x, coef, 0.0, 10 ** 6)
        assert np.max(np.abs(nt.to_dense_rows(x) - I)) <= 1e-12 * np.max(np.abs(I))


def test_central_refuses_inflow():
    with pytest.raises(ValueError):
        problem.build(slab_config0().with_(flux="central", inflow_temperature=(0.8,) + (None,) * 5))
