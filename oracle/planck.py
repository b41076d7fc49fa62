"""Group emission coefficients for the oracle (test infrastructure; see oracle/__init__).

Eqs. (Ttoeps1)-(Ttoeps2), Sec. 2: epsilon_f = (c/4pi) int_{nu_{f-1}}^{nu_f} B(nu,T) dnu with
B = (8 pi h nu^3/c^3) / (exp(h nu/kT) - 1).  In the unit system h = k = c = a = 1 read
from Sec. 4.2 (a = c = 1) and normalised so that the gray limit is c a T^4/(4 pi):

    epsilon_f(T) = (c a T^4 / 4 pi) (15 / pi^4) int_{nu_{f-1}/T}^{nu_f/T} t^3/(e^t - 1) dt .

The oracle integrates the Planck integrand directly with adaptive quadrature
(scipy.integrate.quad); the paper's own route (polylogarithms, end of Sec. 2.1) is
not used here, so the two sides are independent.  Values below 1e-300 are
flushed to 0.
"""
import math

import numpy as np
from scipy import integrate

FLUSH = 1e-300


def _integrand(t):
    if t == 0.0:
        return 0.0
    if t > 1.0:
        return t ** 3 * math.exp(-t) / -math.expm1(-t)
    return t ** 3 / math.expm1(t)


def planck_segment(x1, x2):
    """int_{x1}^{x2} t^3/(e^t-1) dt for 0 <= x1 < x2 <= inf."""
    if not (x2 > x1):
        return 0.0
    if x1 > 740.0:  # e^{-x1} underflows in double
        return 0.0
    if np.isinf(x2):
        # beyond x1 + 100 the integrand is below e^{-100} of its value at x1: negligible in FP64
        x2 = x1 + 100.0
    # split at points where the integrand changes scale so quad stays accurate
    pts = [x1]
    for p in (1.0, 3.0, 10.0, 30.0, 60.0, 100.0, 200.0, 300.0, 500.0):
        if x1 < p < x2:
            pts.append(p)
    total = 0.0
    for a, b in zip(pts, pts[1:] + [x2]):
        val, _ = integrate.quad(_integrand, a, b, epsabs=0.0, epsrel=2e-14, limit=400)
        total += val
    return total


def emission(T, edges, c=1.0, a_rad=1.0):
    """epsilon_f(T) for every group f; T scalar >= 0."""
    G = len(edges) - 1
    out = np.zeros(G)
    if T <= 0.0:
        return out
    pref = c * a_rad * T ** 4 / (4.0 * math.pi) * 15.0 / math.pi ** 4
    for f in range(G):
        x1 = edges[f] / T
        x2 = edges[f + 1] / T if np.isfinite(edges[f + 1]) else np.inf
        if x1 > 30.0:
            # upper bound of the whole Wien tail, e^{-x}(x^3+3x^2+6x+6)/(1-e^{-x}); skip what flushes
            bound = math.exp(-x1) * (x1 ** 3 + 3 * x1 ** 2 + 6 * x1 + 6) * 1.01
            if pref * bound < FLUSH:
                continue
        v = pref * planck_segment(x1, x2)
        out[f] = v if v >= FLUSH else 0.0
    return out


def emission_rows(temperature, edges, c=1.0, a_rad=1.0):
    """epsilon per merged row k = g + G*cell."""
    cache = {}
    G = len(edges) - 1
    out = np.empty(len(temperature) * G)
    for i, T in enumerate(np.asarray(temperature, dtype=float)):
        key = float(T)
        if key not in cache:
            cache[key] = emission(key, edges, c, a_rad)
        out[i * G:(i + 1) * G] = cache[key]
    return out
