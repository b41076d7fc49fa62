"""Pins of the oracle in three spatial dimensions (d_X = 3, lat/long ordinates, merged rows
k = g + G (ix + Nx (iy + Ny iz))):

* conservation: with no material, the one-step change of sum_cells I along every axis line is
  the difference of the two boundary fluxes, for the upwind flux F_{N-1/2} = n^+ I_{N-1},
  F_{-1/2} = n^- I_0 (vacuum ghost cells), the Rusanov flux (n + 1) I_{N-1} / 2 and (n - 1) I_0 / 2
  and the central flux n I_{N-1} / 2 and n I_0 / 2, summed over the three axes with lambda_a;
* symmetry: exchanging x and y (transposed grid and materials) maps the solution onto itself with
  the azimuth reflected, phi -> pi/2 - phi, which on the midpoint grid phi_p = (2p + 1) pi / N_phi
  is p -> N_phi/4 - 1 - p (mod N_phi);
* the naive TT transport sum has (2 d_X + 1) r + n_bc columns (d_X + 1 for the central flux) and
  the exact-rank TT step equals the dense step, with an inflow face on z.
"""
import dataclasses

import numpy as np
import pytest

from oracle import dense, naive_tt as nt, problem
from paper_2602_00290_gb300.workloads import cube_config, plane_config1, random_tt


def _no_material(coef):
    c = dataclasses.replace(coef)
    c.acoef = np.zeros_like(coef.acoef)
    c.scoef = np.zeros_like(coef.scoef)
    c.eps = np.zeros_like(coef.eps)
    return c


def _boundary_flux(flux, n, first, last):
    if flux == "upwind":
        return np.maximum(n, 0.0) * last - np.minimum(n, 0.0) * first
    if flux == "rusanov":
        return 0.5 * (n + 1.0) * last - 0.5 * (n - 1.0) * first
    return 0.5 * n * last - 0.5 * n * first


@pytest.mark.parametrize("flux", ["upwind", "rusanov", "central"])
def test_3d_conservation(flux):
    wl = cube_config().with_(flux=flux)
    coef = _no_material(problem.build(wl))
    G, nx, ny, nz = wl.ngroup, wl.nx, wl.ny, wl.nz
    rng = np.random.default_rng(7)
    I = rng.random((wl.nrow, coef.nang))
    out = dense.DenseSolver(wl, coef).step(I)
    A = I.reshape(nz, ny, nx, G, -1)          # [iz, iy, ix, g, q]
    B = out.reshape(nz, ny, nx, G, -1)
    d = coef.dirs
    expect = A.sum(axis=(0, 1, 2))
    for ax, n in ((2, d["nx"]), (1, d["ny"]), (0, d["nz"])):   # array axis of x, y, z
        lam = coef.lam[2 - ax]
        first = np.take(A, 0, axis=ax).sum(axis=(0, 1))
        last = np.take(A, -1, axis=ax).sum(axis=(0, 1))
        expect = expect - lam * _boundary_flux(flux, n[None, :], first, last)
    got = B.sum(axis=(0, 1, 2))
    assert np.allclose(got, expect, rtol=0, atol=1e-13 * np.max(np.abs(expect)))


def _swap_xy(wl):
    """The same problem with x and y exchanged (materials transposed cell by cell)."""
    G = wl.ngroup

    def tr_rows(a):
        return np.asarray(a).reshape(wl.nz, wl.ny, wl.nx, G).transpose(0, 2, 1, 3).reshape(-1)

    def tr_cells(a):
        return np.asarray(a).reshape(wl.nz, wl.ny, wl.nx).transpose(0, 2, 1).reshape(-1)

    ext = (wl.extent[1], wl.extent[0], wl.extent[2])
    return wl.with_(nx=wl.ny, ny=wl.nx, extent=ext, rho_kappa_a=tr_rows(wl.rho_kappa_a),
                    rho_kappa_s=tr_rows(wl.rho_kappa_s), temperature=tr_cells(wl.temperature))


@pytest.mark.parametrize("wl", [cube_config(nx=6, ny=5, nz=3, nphi=8), plane_config1(nx=7, ny=5, G=3, ntheta=4, nphi=8)],
                         ids=["cube", "plane"])
@pytest.mark.parametrize("flux", ["upwind", "rusanov"])
def test_xy_swap_symmetry(wl, flux):
    wl = wl.with_(flux=flux)
    ws = _swap_xy(wl)
    S, Ss = dense.DenseSolver(wl), dense.DenseSolver(ws)
    rng = np.random.default_rng(11)
    I = S.initial() * (1.0 + 0.5 * rng.random((wl.nrow, S.coef.nang)))   # anisotropic start
    nth, nph, G = wl.ntheta, wl.nphi, wl.ngroup
    perm_p = (nph // 4 - 1 - np.arange(nph)) % nph

    def to_swapped(X):
        X = X.reshape(wl.nz, wl.ny, wl.nx, G, nth, nph).transpose(0, 2, 1, 3, 4, 5)
        return X[..., perm_p].reshape(wl.nrow, -1)

    Is = to_swapped(I)
    for _ in range(3):
        I = S.step(I)
        Is = Ss.step(Is)
    want = to_swapped(I)
    assert np.max(np.abs(Is - want)) <= 1e-12 * np.max(np.abs(want))


@pytest.mark.parametrize("flux,inflow", [("upwind", (None, None, None, None, 0.7, None)),
                                         ("upwind", (0.9, None, None, 0.4, None, None)),
                                         ("rusanov", (None,) * 6), ("central", (None,) * 6)])
def test_3d_exact_rank_tt_step_equals_dense(flux, inflow):
    wl = cube_config(tol=0.0, rmax=10 ** 6).with_(flux=flux, inflow_temperature=inflow)
    coef = problem.build(wl)
    S = dense.DenseSolver(wl, coef)
    I = S.initial()
    x = nt.initial_tt(problem.initial_rows(wl, coef), coef)
    for _ in range(3):
        I = S.step(I)
        x = nt.step(x, coef, 0.0, 10 ** 6)
        assert np.max(np.abs(nt.to_dense_rows(x) - I)) <= 1e-12 * np.max(np.abs(I))


@pytest.mark.parametrize("flux,nterm", [("upwind", 6), ("rusanov", 6), ("central", 3)])
def test_3d_transport_sum_rank_and_values(flux, nterm):
    inflow = (None, None, None, None, 0.7, None) if flux == "upwind" else (None,) * 6
    wl = cube_config().with_(flux=flux, inflow_temperature=inflow)
    coef = problem.build(wl)
    x = random_tt([wl.nrow, wl.ntheta, wl.nphi], [3, 2], seed=17)
    t = nt.transport_sum(x, coef)
    nbc = sum(b is not None for b in coef.inflow)
    assert nt.ranks(t)[1] == (nterm + 1) * 3 + nbc
    c0 = _no_material(coef)
    ref = dense.DenseSolver(wl, c0).step(nt.to_dense_rows(x))
    assert np.max(np.abs(nt.to_dense_rows(t) - ref)) <= 1e-13 * np.max(np.abs(ref))
