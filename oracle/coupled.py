"""Coupled material temperature (Sec. 2.1): the backward-Euler source stage with
epsilon^{m+1} = epsilon(T^dagger), where T^dagger is the root of the paper's f(T^dagger), and the
temperature advanced by total energy conservation,

    rho c_v (T^{m+1} - T^m) = (4 pi / c) sum_f [ J*_f - J^{m+1}_f ],

on top of the dense stepper and the naive TT.  TEST INFRASTRUCTURE: only tests, smoke() and the
bench's CPU baseline use this package.

Reading of f(T^dagger): with a_f = c dt rho kappa_{a,f} the printed bracket
eps_f - [(c dt)^-1 + rho kappa_a]^-1 (J_f / (c dt) + rho kappa_a eps_f) equals (eps_f - J_f)/(1 + a_f),
so f(T) = T^m - T - (4 pi / (c rho c_v)) sum_f a_f (eps_f(T) - J*_f) / (1 + a_f), where J*_f is the
group mean intensity entering the source stage (after transport) and kappa_a / c_v =
(rho kappa_a) / (rho c_v).  f is strictly decreasing in T, f(0) >= 0: one root on [0, inf).
J^{m+1}_f of the energy update is the mean intensity of the state carried to the next step (after
the rounding, in the TT stepper), so the step conserves material plus radiation energy.
"""
import dataclasses
import math

import numpy as np
from scipy.optimize import brentq

from . import naive_tt as nt
from . import planck


def t_dagger(Tm, Jstar, acoef, rho_cv, edges, c=1.0, a_rad=1.0):
    """Root of f(T) for one cell: Jstar and acoef over the cell's G groups."""
    C = 4.0 * math.pi / (c * rho_cv)
    w = acoef / (1.0 + acoef)

    def f(T):
        return Tm + C * float(np.sum(w * (Jstar - planck.emission(T, edges, c, a_rad)))) - T

    f0 = f(0.0)
    if f0 <= 0.0:
        return 0.0
    hi = max(Tm, 1e-3)
    while f(hi) > 0.0:
        hi *= 2.0
    return brentq(f, 0.0, hi, xtol=1e-15 * hi, rtol=1e-15, maxiter=500)


def source_temperature(Jstar, coef, T, rho_cv, edges):
    """Per cell: T^dagger and epsilon_f(T^dagger) on the cell's rows (row k = g + G cell)."""
    G = coef.G
    ncell = len(T)
    eps = np.empty(ncell * G)
    Td = np.empty(ncell)
    for cell in range(ncell):
        rows = slice(cell * G, cell * G + G)
        Td[cell] = t_dagger(T[cell], Jstar[rows], coef.acoef[rows], rho_cv[cell], edges, coef.c)
        eps[rows] = planck.emission(Td[cell], edges, coef.c)
    return eps, Td


def temperature_update(T, Jstar, Jnew, rho_cv, coef):
    """rho c_v (T^{m+1} - T^m) = (4 pi / c) sum_f (J*_f - J^{m+1}_f), per cell."""
    G = coef.G
    dJ = (Jstar - Jnew).reshape(len(T), G).sum(axis=1)
    return T + 4.0 * math.pi / (coef.c * rho_cv) * dJ


def dense_step(S0, coef, I, T, rho_cv, edges, transport=True):
    """One coupled step on the full grid.  S0: DenseSolver whose source stage is switched off
    (a = s = eps = 0), used for the transport; transport=False skips it (infinite medium)."""
    Istar = S0.step(I) if transport else I.copy()
    dom = coef.dirs["domega"]
    Js = Istar @ dom / (4.0 * math.pi)
    eps, Td = source_temperature(Js, coef, T, rho_cv, edges)
    a, s = coef.acoef, coef.scoef
    Jn = (Js + a * eps) / (1.0 + a)
    Inew = (Istar + (a * eps + s * Jn)[:, None]) / (1.0 + a + s)[:, None]
    J1 = Inew @ dom / (4.0 * math.pi)
    return Inew, temperature_update(T, Js, J1, rho_cv, coef), Td


def tt_step(tt, coef, T, rho_cv, edges, tol, rmax, rounding="svd"):
    """One coupled step-then-truncate step of the naive TT: transport, round, T^dagger, source,
    round, energy-conserving temperature update."""
    rnd = nt.round_tt_gram if rounding == "gram" else nt.round_tt
    x = rnd(nt.transport_sum(tt, coef), tol, rmax)
    Js = x[0][0] @ nt.angular_weights_vector(x, coef)
    eps, Td = source_temperature(Js, coef, T, rho_cv, edges)
    x = rnd(nt.source_sum(x, dataclasses.replace(coef, eps=eps)), tol, rmax)
    J1 = x[0][0] @ nt.angular_weights_vector(x, coef)
    return x, temperature_update(T, Js, J1, rho_cv, coef), Td
