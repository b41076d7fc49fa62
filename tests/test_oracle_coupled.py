"""Pins of the coupled-temperature oracle (Sec. 2.1, Eq. Tupdate and the f(T^dagger) root):

* the paper's multigroup thermal relaxation (Sec. 4.2, N_nu = 3): an infinite medium at
  rho c_v = 8, T = 10 with Planckian radiation at T_r = 1 relaxes to T_eq = 2.77 with group
  energy fractions 0.31 / 0.47 / 0.22 (the printed values, tests/golden), conserving
  rho c_v T + sum_f E_f at every step;
* the gray limit (one group over [0, inf)): T^dagger is the positive root of the quartic
  T^m + C w (J* - c a T^4 / 4 pi) - T = 0;
* the exact-rank TT coupled step equals the dense coupled step.
"""
import math
import os

import numpy as np
import pytest

from oracle import coupled, dense, naive_tt as nt, planck, problem
from paper_2602_00290_gb300.workloads import plane_config1, slab_config0

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden(name):
    out = {}
    with open(os.path.join(HERE, "golden", name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                out[k] = float(v)
    return out


def _single_cell(edges, T0, kappa, dt):
    G = len(edges) - 1
    wl = slab_config0().with_(nx=1, ngroup=G, group_edges=np.asarray(edges, dtype=float),
                              temperature=np.array([T0]), rho_kappa_a=np.full(G, kappa),
                              rho_kappa_s=np.zeros(G), dt=dt)
    return wl, problem.build(wl)


def test_thermal_relaxation_reaches_printed_equilibrium():
    g = _golden("thermal_relaxation_nu3.txt")
    x1 = g["h_cgs"] / g["kB_cgs"] * g["k_hz"]       # nu_1 in temperature units (h = k_B = 1)
    edges = [0.0, x1, 2.0 * x1, np.inf]
    wl, coef = _single_cell(edges, g["T_initial"], 1.0, 0.5)
    rho_cv = np.array([g["rho_cv"]])
    T = np.array([g["T_initial"]])
    I = np.repeat(planck.emission(g["Tr_initial"], np.asarray(edges))[:, None], coef.nang, axis=1)
    dom = coef.dirs["domega"]

    def total(I, T):
        return rho_cv[0] * T[0] + 4.0 * math.pi / coef.c * float(np.sum(I @ dom / (4.0 * math.pi)))

    e0 = total(I, T)
    for _ in range(400):
        I, T, _ = coupled.dense_step(None, coef, I, T, rho_cv, np.asarray(edges), transport=False)
        assert abs(total(I, T) - e0) <= 1e-12 * e0
    assert round(T[0], 2) == g["T_eq"]
    E = I @ dom
    frac = E / E.sum()
    for f, key in enumerate(("E1", "E2", "E3")):
        assert round(frac[f], 2) == g[key]
    assert np.allclose(I @ dom / (4 * math.pi), planck.emission(T[0], np.asarray(edges)), rtol=1e-9)


def test_gray_t_dagger_is_the_quartic_root():
    edges = np.array([0.0, np.inf])
    for Tm, J, a, rcv in ((10.0, 0.02, 0.7, 8.0), (0.5, 3.0, 5.0, 0.3), (2.0, 0.0, 1e-3, 1.0)):
        Td = coupled.t_dagger(Tm, np.array([J]), np.array([a]), rcv, edges)
        C = 4.0 * math.pi / rcv
        w = a / (1.0 + a)
        roots = np.roots([-C * w / (4.0 * math.pi), 0.0, 0.0, -1.0, Tm + C * w * J])
        real = [r.real for r in roots if abs(r.imag) < 1e-9 and r.real > 0]
        assert len(real) == 1
        assert abs(Td - real[0]) <= 1e-12 * real[0]


def test_exact_rank_tt_coupled_step_equals_dense():
    wl = plane_config1(nx=5, ny=4, G=3, ntheta=4, nphi=8, rmax=64, tol=0.0)
    coef = problem.build(wl)
    coef0 = problem.build(wl)
    coef0.acoef[:] = 0.0
    coef0.scoef[:] = 0.0
    coef0.eps[:] = 0.0
    S0 = dense.DenseSolver(wl, coef0)
    rho_cv = np.full(wl.nx * wl.ny, 0.5)
    edges = np.asarray(wl.group_edges)
    T = np.asarray(wl.temperature, dtype=float).copy()
    Tt = T.copy()
    I = dense.DenseSolver(wl, coef).initial()
    x = nt.initial_tt(problem.initial_rows(wl, coef), coef)
    for _ in range(3):
        I, T, Td = coupled.dense_step(S0, coef, I, T, rho_cv, edges)
        x, Tt, Tdt = coupled.tt_step(x, coef, Tt, rho_cv, edges, 0.0, 10 ** 6)
        assert np.max(np.abs(nt.to_dense_rows(x) - I)) <= 1e-11 * np.max(np.abs(I))
        assert np.max(np.abs(Tt - T)) <= 1e-11 * np.max(np.abs(T))
        assert np.max(np.abs(Tdt - Td)) <= 1e-11 * np.max(np.abs(Td))
    # the material actually moved
    assert np.max(np.abs(T - np.asarray(wl.temperature))) > 1e-3
