"""Coupled material temperature on the GPU (tt_problem.rho_cv, Sec. 2.1) against the oracle's
coupled stepper, and the paper's thermal relaxation (Sec. 4.2, N_nu = 3) run to equilibrium.
Tolerances: FP64 1e-10 relative on the state, T^dagger and T (as for the fixed-T steps);
mixed 1e-6 relative in energy density and temperature."""
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import coupled, naive_tt as nt, planck, problem  # noqa: E402
from paper_2602_00290_gb300.workloads import plane_config1  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
TIE = 1e-9


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


def _wl(**kw):
    args = dict(nx=12, ny=10, G=5, ntheta=4, nphi=8, rmax=8, tol=1e-6)
    args.update(kw)
    wl = plane_config1(**args)
    return wl.with_(rho_cv=np.full(wl.nx * wl.ny, 0.5))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-6)])
def test_coupled_step_matches_oracle(tt, ctx, prec, tol):
    wl = _wl()
    coef = problem.build(wl)
    plan = tt.Plan(ctx, wl)
    x = tt.initial_state(plan, [wl.rmax, wl.rmax], "f64" if prec == "fp64" else "f32")
    ref = nt.initial_tt(problem.initial_rows(wl, coef), coef)
    T = np.asarray(wl.temperature, dtype=float).copy()
    edges = np.asarray(wl.group_edges)
    for s in range(3):
        tt.tt_step(ctx, plan, x, wl.tol, wl.rmax, prec)
        ref, T, Td = coupled.tt_step(ref, coef, T, wl.rho_cv, edges, wl.tol, wl.rmax)
        ctx.sync()
        if prec == "fp64":
            assert rel(nt.to_dense_rows(x.to_cores()), nt.to_dense_rows(ref)) < tol, s
        E = tt.tt_energy_density(ctx, plan, x).cpu().numpy()
        Er = nt.energy_density_rows(ref, coef)
        assert np.linalg.norm(E - Er) <= tol * np.linalg.norm(Er), s
        assert rel(plan.t_dagger(), Td) < tol, s
        assert rel(plan.temperature(), T) < tol, s
    assert np.max(np.abs(T - np.asarray(wl.temperature))) > 1e-3


def _golden(name):
    out = {}
    with open(os.path.join(HERE, "golden", name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                out[k] = float(v)
    return out


def test_thermal_relaxation_on_the_gpu(tt, ctx):
    """One cell of a 1e14-wide domain (lambda = 5e-15: negligible transport), the paper's N_nu = 3
    relaxation: T -> 2.77 and group fractions 0.31 / 0.47 / 0.22 (printed values, 2 digits)."""
    g = _golden("thermal_relaxation_nu3.txt")
    x1 = g["h_cgs"] / g["kB_cgs"] * g["k_hz"]
    edges = np.array([0.0, x1, 2.0 * x1, np.inf])
    wl = plane_config1(nx=1, ny=1, G=3, ntheta=4, nphi=8, rmax=2, tol=1e-10)
    wl = wl.with_(group_edges=edges, temperature=np.array([g["T_initial"]]), rho_kappa_a=np.ones(3),
                  rho_kappa_s=np.zeros(3), extent=(1e14, 1e14, 1.0), dt=0.5, rho_cv=np.array([g["rho_cv"]]))
    plan = tt.Plan(ctx, wl)
    eps_r = planck.emission(g["Tr_initial"], edges)
    cores = [eps_r.reshape(1, 3, 1), np.ones((1, 4, 1)), np.ones((1, 8, 1))]
    x = tt.TT.from_cores(cores, rcap=[2, 2])
    dom = plan.array(1)
    for _ in range(400):
        tt.tt_step(ctx, plan, x, wl.tol, wl.rmax, "fp64")
    ctx.sync()
    T = plan.temperature()[0]
    assert round(T, 2) == g["T_eq"]
    rows = nt.to_dense_rows(x.to_cores())          # (3 groups, 32 angles)
    E = rows @ dom
    frac = E / E.sum()
    for f, key in enumerate(("E1", "E2", "E3")):
        assert round(frac[f], 2) == g[key]
    # total energy rho c_v T + sum_f E_f (per unit volume, c = 1) is conserved
    e0 = g["rho_cv"] * g["T_initial"] + 4 * math.pi * float(eps_r.sum())
    assert abs(g["rho_cv"] * T + float(E.sum()) - e0) <= 1e-8 * e0
