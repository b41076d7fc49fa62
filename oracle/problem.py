"""Derived coefficients of one operator-split time step, for the oracle (test infrastructure).

From a raw ``Workload`` this builds what Sec. 2.1 needs per step:

* lambda_a = c dt / dx_a, the forward-Euler transport factor of the upwind update
  (Sec. 2.1 first paragraph and Appendix A, 'Value of n');
* a_k = c dt rho kappa_a and s_k = c dt rho kappa_s per merged row, the backward-Euler
  source coefficients of Eq. (discRTsource);
* epsilon_k = epsilon_f(T(cell)) per merged row (Eqs. Ttoeps1-2, fixed material T);
* the inflow spectrum per face (isotropic Planck at the face temperature) or None;
* direction cosines and solid-angle weights.
"""
from dataclasses import dataclass
from typing import List, Optional

import numpy as np

from . import planck, quadrature


@dataclass
class StepCoefficients:
    ndim: int
    nx: int
    ny: int
    nz: int
    G: int
    ntheta: int
    nphi: int
    lam: np.ndarray            # (3,)
    acoef: np.ndarray          # (N_Z,)
    scoef: np.ndarray          # (N_Z,)
    eps: np.ndarray            # (N_Z,)
    inflow: List[Optional[np.ndarray]]  # 6 faces
    dirs: dict
    dV: float
    dA: np.ndarray             # face area per axis (3,)
    c: float
    dt: float
    flux: str = "upwind"       # "upwind", "rusanov" or "central" (Appendix A, 'Value of n';
                               # "central" is the Rusanov flux with wavespeed S+ = 0, Sec. 4.3)
    alpha_local: bool = False  # Rusanov with the local speed |n_a| (reduces to upwind; a pin)

    @property
    def nrow(self):
        return self.nx * self.ny * self.nz * self.G

    @property
    def nang(self):
        return self.ntheta * self.nphi


def build(wl) -> StepCoefficients:
    dx = np.array(wl.spacing, dtype=float)
    lam = np.zeros(3)
    for a in range(wl.ndim):
        lam[a] = wl.c * wl.dt / dx[a]
    acoef = wl.c * wl.dt * np.asarray(wl.rho_kappa_a, dtype=float)
    scoef = wl.c * wl.dt * np.asarray(wl.rho_kappa_s, dtype=float)
    eps = planck.emission_rows(wl.temperature, wl.group_edges, wl.c, wl.a_rad)
    inflow = []
    for f in range(6):
        Tb = wl.inflow_temperature[f] if f < len(wl.inflow_temperature) else None
        if Tb is None or f // 2 >= wl.ndim:
            inflow.append(None)
        else:
            inflow.append(planck.emission(float(Tb), wl.group_edges, wl.c, wl.a_rad))
    dV = float(np.prod(dx[:wl.ndim]))
    dA = np.array([dV / dx[a] for a in range(3)])
    flux = getattr(wl, "flux", "upwind")
    if flux not in ("upwind", "rusanov", "central"):
        raise ValueError(f"unknown flux {flux!r}")
    if flux in ("rusanov", "central") and any(b is not None for b in inflow):
        raise ValueError("the Rusanov flux is read with vacuum ghost cells only")
    return StepCoefficients(wl.ndim, wl.nx, wl.ny, wl.nz, wl.ngroup, wl.ntheta, wl.nphi,
                            lam, acoef, scoef, eps, inflow, quadrature.directions(wl),
                            dV, dA, wl.c, wl.dt, flux)


def initial_rows(wl, coef: StepCoefficients) -> np.ndarray:
    """I^0 = epsilon_f(T) isotropic (the unspecified initial condition read as equilibrium
    with the material, or with ``wl.initial_temperature`` when given)."""
    if wl.initial_temperature is None:
        return coef.eps.copy()
    return planck.emission_rows(wl.initial_temperature, wl.group_edges, wl.c, wl.a_rad)
