"""Pins of the dense FP64 S_N stepper (oracle) against closed forms and invariants."""
import math

import numpy as np
import pytest
from scipy.special import comb

from oracle import dense, planck, problem
from paper_2602_00290_gb300.workloads import Workload, group_edges, plane_config1, slab_config0


def _slab(nx=32, G=2, nmu=4, sigma=(2.0, 5.0), T=0.0, inflow_T=None, dt=0.01, ks=None):
    edges = group_edges(G, 0.5, 2.0) if G > 1 else np.array([0.0, np.inf])
    ka = np.tile(np.asarray(sigma, float), nx)
    return Workload(name="slab", ndim=1, nx=nx, ny=1, nz=1, ngroup=G, quad="gauss_legendre_mu",
                    ntheta=nmu, nphi=1, extent=(1.0, 1.0, 1.0), c=1.0, dt=dt, group_edges=edges,
                    temperature=np.full(nx, T), rho_kappa_a=ka,
                    rho_kappa_s=np.zeros_like(ka) if ks is None else np.tile(np.asarray(ks, float), nx),
                    inflow_temperature=(inflow_T, None, None, None, None, None), tol=0.0, rmax=8)


def test_beer_lambert_discrete_steady_state():
    """Pure absorption with inflow on the left: steady state I_i = I_{i-1}/(1 + sigma dx/mu)
    for mu > 0 (forward-Euler upwind + backward-Euler absorption), 0 for mu < 0."""
    wl = _slab(inflow_T=1.0)
    S = dense.DenseSolver(wl)
    I = np.zeros((wl.nrow, wl.ntheta))
    for _ in range(4000):
        I = S.step(I)
    mu = S.coef.dirs["mu"]
    b = S.coef.inflow[0]
    dx = 1.0 / wl.nx
    for g in range(wl.ngroup):
        sig = wl.rho_kappa_a[g]
        for q in range(wl.ntheta):
            col = I[g::wl.ngroup, q]
            if mu[q] > 0:
                expect = b[g] * (1.0 + sig * dx / mu[q]) ** -(np.arange(wl.nx) + 1.0)
                assert np.max(np.abs(col - expect)) <= 1e-12 * b[g]
            else:
                assert np.max(np.abs(col)) == 0.0


def test_beer_lambert_first_order_convergence():
    """The discrete profile approaches I_0 exp(-sigma x / mu) at first order in dx."""
    errs = []
    for nx in (32, 64, 128):
        sig, mu = 2.0, 0.8
        xr = 1.0  # right edge
        disc = (1.0 + sig * (xr / nx) / mu) ** -nx
        errs.append(abs(disc - math.exp(-sig * xr / mu)))
    assert 1.8 < errs[0] / errs[1] < 2.2 and 1.8 < errs[1] / errs[2] < 2.2


def test_free_streaming_binomial():
    """sigma = 0: I_i^m = sum_k C(m,k) lam^k (1-lam)^(m-k) I^0_{i-k} (zero ghost), per mu > 0."""
    wl = _slab(nx=40, G=1, nmu=6, sigma=(0.0,), dt=0.01)
    S = dense.DenseSolver(wl)
    x = (np.arange(wl.nx) + 0.5) / wl.nx
    f0 = np.exp(-((x - 0.3) / 0.08) ** 2)
    I = np.repeat(f0[:, None], wl.ntheta, axis=1)
    m = 7
    for _ in range(m):
        I = S.step(I)
    mu = S.coef.dirs["mu"]
    for q in range(wl.ntheta):
        lam = wl.c * wl.dt * mu[q] * wl.nx
        if mu[q] > 0:
            exp_ = np.zeros(wl.nx)
            for k in range(m + 1):
                sh = np.zeros(wl.nx)
                sh[k:] = f0[:wl.nx - k]
                exp_ += comb(m, k) * lam ** k * (1 - lam) ** (m - k) * sh
        else:
            lm = -lam
            exp_ = np.zeros(wl.nx)
            for k in range(m + 1):
                sh = np.zeros(wl.nx)
                sh[:wl.nx - k] = f0[k:]
                exp_ += comb(m, k) * lm ** k * (1 - lm) ** (m - k) * sh
        assert np.max(np.abs(I[:, q] - exp_)) < 1e-14


def test_planck_equilibrium_fixed_point():
    """Uniform T, isotropic I = epsilon(T), inflow epsilon(T) on every face: exact fixed point."""
    wl = plane_config1(nx=6, ny=5, G=4, ntheta=4, nphi=8)
    wl = wl.with_(temperature=np.full(wl.ncell, 0.7), inflow_temperature=(0.7,) * 4 + (None, None))
    S = dense.DenseSolver(wl)
    I = S.initial()
    I1 = S.step(I)
    assert np.max(np.abs(I1 - I)) <= 1e-14 * np.max(np.abs(I))


def _boundary_transport_energy(S, I):
    """-dt * net outflow through the faces, from the telescoped upwind differences."""
    c = S.coef
    wl = S.wl
    A = I.reshape(wl.nz, wl.ny, wl.nx, wl.ngroup, c.nang)
    dom = c.dirs["domega"]
    tot = 0.0
    for ax, key in enumerate(("nx", "ny", "nz")[:wl.ndim]):
        n = c.dirs[key]
        axis = 2 - ax
        last = np.take(A, -1, axis=axis)
        first = np.take(A, 0, axis=axis)
        gm = np.zeros(wl.ngroup) if c.inflow[2 * ax] is None else c.inflow[2 * ax]
        gp = np.zeros(wl.ngroup) if c.inflow[2 * ax + 1] is None else c.inflow[2 * ax + 1]
        pos = n >= 0
        # n >= 0 lines: sum_i (I_i - I_{i-1}) = I_last - ghost_minus
        tpos = (last - gm[None, None, :, None]) * (n * pos * dom)
        tneg = (gp[None, None, :, None] - first) * (n * (~pos) * dom)
        tot += -wl.dt * c.dA[ax] * float(np.sum(tpos) + np.sum(tneg))
    return tot


@pytest.mark.parametrize("inflow", [None, 0.9])
def test_energy_balance_per_step(inflow):
    """dE = -dt (net boundary outflow) + (4pi/c) sum dV a (eps - J^{m+1}); scattering cancels."""
    wl = plane_config1(nx=8, ny=7, G=5, ntheta=4, nphi=8)
    if inflow is not None:
        wl = wl.with_(inflow_temperature=(inflow, None, None, 0.5, None, None))
    S = dense.DenseSolver(wl)
    I = S.initial()
    rng = np.random.default_rng(5)
    I = I * (1.0 + 0.5 * rng.random(I.shape))
    for _ in range(3):
        I1, Is = S.step(I, return_star=True)
        E0, Es, E1 = S.total_energy(I), S.total_energy(Is), S.total_energy(I1)
        bt = _boundary_transport_energy(S, I)
        assert abs((Es - E0) - bt) <= 1e-13 * E0
        J1 = S.J(I1)
        ex = 4 * math.pi / wl.c * S.coef.dV * float(np.sum(S.coef.acoef * (S.coef.eps - J1)))
        assert abs((E1 - Es) - ex) <= 1e-13 * E0
        I = I1


def test_slab_config_runs_and_is_finite():
    wl = slab_config0()
    S = dense.DenseSolver(wl)
    I = S.initial()
    for _ in range(wl.steps):
        I = S.step(I)
    assert np.all(np.isfinite(I)) and np.all(I >= 0)
