"""Pins of the oracle's quadrature and Planck emission against closed forms and printed values."""
import math
import os

import numpy as np
import pytest
from scipy.optimize import brentq

from oracle import planck, quadrature

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        lines = fh.readlines()
    for line in lines:
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, v = line.split()
        vals[k] = float(v)
    return vals


def test_gauss_legendre_moments():
    mu, w = quadrature.gauss_legendre_mu(8)
    assert abs(w.sum() - 2.0) < 1e-14
    # exact for degree <= 15: int_{-1}^{1} mu^(2m) = 2/(2m+1)
    for m in range(8):
        assert abs(np.sum(w * mu ** (2 * m)) - 2.0 / (2 * m + 1)) < 1e-14
    assert abs(np.sum(w * mu ** 3)) < 1e-15


def test_latlong_midpoint_moments():
    nt, nph = 16, 32
    mu, phi, dom = quadrature.latlong_midpoint(nt, nph)
    assert abs(dom.sum() - 4 * math.pi) < 1e-13
    # midpoint rule for mu^2 on [-1,1]: 2/3 - 2/(3 N^2)
    assert abs(np.sum(2.0 / nt * mu ** 2) - (2.0 / 3 - 2.0 / (3 * nt * nt))) < 1e-14
    # azimuthal midpoint sums of cos^2 are exact: (2 pi / N) sum cos^2 = pi
    assert abs(np.sum(2 * math.pi / nph * np.cos(phi) ** 2) - math.pi) < 1e-13
    assert np.all(np.abs(np.cos(phi)) > 1e-3)  # no azimuthal node on the n_x = 0 plane


def test_directions_unit_and_odd_moments():
    from paper_2602_00290_gb300.workloads import plane_config1
    wl = plane_config1(nx=4, ny=4, G=2, ntheta=8, nphi=16)
    d = quadrature.directions(wl)
    n2 = d["nx"] ** 2 + d["ny"] ** 2 + d["nz"] ** 2
    assert np.max(np.abs(n2 - 1.0)) < 1e-14
    for comp in ("nx", "ny", "nz"):
        assert abs(np.sum(d["domega"] * d[comp])) < 1e-13


def test_planck_gray_limit():
    """sum_f epsilon_f = c a T^4 / (4 pi): the whole spectrum integrates to pi^4/15 (Sec. 2)."""
    edges = np.array([0.0, 0.05, 0.3, 1.0, 2.5, 7.0, 20.0, np.inf])
    for T in (0.1, 0.37, 1.0, 3.0):
        e = planck.emission(T, edges)
        assert abs(e.sum() / (T ** 4 / (4 * math.pi)) - 1.0) < 2e-14
        assert np.all(e > 0)


def test_planck_wien_and_rayleigh_jeans_closed_forms():
    x = 40.0  # e^{-2x} corrections are below 1e-34 relative
    wien = math.exp(-x) * (x ** 3 + 3 * x ** 2 + 6 * x + 6)
    assert abs(planck.planck_segment(x, math.inf) / wien - 1.0) < 1e-14
    x = 1e-3  # t^3/(e^t-1) = t^2 - t^3/2 + t^4/12 - ...
    rj = x ** 3 / 3 - x ** 4 / 8 + x ** 5 / 60
    assert abs(planck.planck_segment(0.0, x) / rj - 1.0) < 1e-13


def test_planck_flush_far_wien_tail():
    e = planck.emission(0.1, np.array([0.0, 50.0, 100.0, np.inf]))
    assert e[2] == 0.0 and e[0] > 0


def test_thermal_relaxation_fractions_golden():
    """Paper's worked example (Sec. 4.2, N_nu = 3): T_eq ~ 2.77 and equilibrium group
    fractions 0.31 / 0.47 / 0.22 follow from energy conservation and the Planck integrals."""
    g = _golden("thermal_relaxation_nu3.txt")
    # rho c_v T + a T^4 conserved, a = 1
    T_eq = brentq(lambda T: T ** 4 + g["rho_cv"] * T - (g["rho_cv"] * g["T_initial"] + g["Tr_initial"] ** 4), 1, 10)
    assert round(T_eq, 2) == g["T_eq"]
    x1 = g["h_cgs"] / g["kB_cgs"] * g["k_hz"] / T_eq
    edges = np.array([0.0, x1, 2 * x1, np.inf])
    frac = planck.emission(1.0, edges) / (1.0 / (4 * math.pi))
    for f, key in enumerate(("E1", "E2", "E3")):
        assert round(frac[f], 2) == g[key]
