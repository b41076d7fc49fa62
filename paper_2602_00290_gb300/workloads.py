"""Seeded synthetic workloads for the multigroup S_N tensor-train transport step.

This module produces raw problem inputs only: grid sizes, frequency-group edges,
fixed material temperature per cell, absorption and scattering opacities per
merged (cell, group) row, boundary temperatures, time step, rounding tolerance
and rank cap, plus random TT cores for the rounding tests.  It holds none of the
method's arithmetic (no quadrature, no Planck integrals, no transport or source
update); both the CUDA path and the CPU oracle consume these arrays and derive
everything else on their own.

Conventions shared by every consumer:

* merged spatio-spectral row index ``k = g + G * (ix + Nx * (iy + Ny * iz))``
  (group fastest, then x, y, z), the row order of the merged core Z of Eq.
  (tensor_decomp_mer) in Sec. 3.1;
* frequency groups ``[nu_{f-1}, nu_f)`` with ``nu_0 = 0`` and ``nu_G = inf`` and
  log-spaced interior edges (Sec. 2 and Sec. 4 preamble);
* units ``h = k_B = c = a = 1`` so that ``x = nu / T`` (the a = c = 1 unit
  system of the thermal-relaxation test in Sec. 4.2);
* face order ``(x-, x+, y-, y+, z-, z+)``; a face temperature of ``None`` means
  vacuum, otherwise isotropic Planck inflow at that temperature.

Opacity recipe (synthetic stand-in for the paper's tabulated opacities, which
are not available): ``rho*kappa_a[cell, f] = rho(cell) * kappa0 * (nu_f/nu0)^-3
* L_f`` with ``L_f = exp(z_f)``, ``z_f ~ N(0, 1)`` seeded, ``nu_f`` the
geometric mean of the group edges (end groups use the log grid extended by one
step), ``kappa0 = 10``, ``nu0 = 1``.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import Optional, Sequence, Tuple

import numpy as np

FACES = ("x-", "x+", "y-", "y+", "z-", "z+")


@dataclass
class Workload:
    name: str
    ndim: int                      # number of spatial axes d_X (1, 2 or 3)
    nx: int
    ny: int
    nz: int
    ngroup: int                    # G
    quad: str                      # "gauss_legendre_mu" (slab) or "latlong_midpoint"
    ntheta: int                    # polar nodes (mu nodes for the slab)
    nphi: int                      # azimuthal nodes (1 for the slab)
    extent: Tuple[float, float, float]
    c: float
    dt: float
    group_edges: np.ndarray        # (G+1,), [0, ..., inf]
    temperature: np.ndarray        # (N_X,) material temperature per cell (fixed)
    rho_kappa_a: np.ndarray        # (N_X*G,) per merged row
    rho_kappa_s: np.ndarray        # (N_X*G,) per merged row
    rho_cv: Optional[np.ndarray] = None  # per cell: couples the material temperature
    flux: str = "upwind"            # "upwind", "rusanov" or "central" (vacuum boundaries only)
    topology: str = "merged"        # TT layout of the state: "merged" (built), "merged_nux_y", "split_x"
    inflow_temperature: Tuple[Optional[float], ...] = (None,) * 6
    initial_temperature: Optional[np.ndarray] = None  # radiation temperature per cell for I^0
    tol: float = 1e-6
    rmax: int = 32
    steps: int = 20
    a_rad: float = 1.0
    seed: int = 0
    notes: str = ""

    @property
    def ncell(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def nrow(self) -> int:
        """Rows of the merged spatio-spectral core (N_X * N_nu)."""
        return self.ncell * self.ngroup

    @property
    def spacing(self) -> Tuple[float, float, float]:
        n = (self.nx, self.ny, self.nz)
        return tuple(self.extent[a] / n[a] for a in range(3))

    @property
    def nangle(self) -> int:
        return self.ntheta * self.nphi

    def full_unknowns(self) -> int:
        return self.nrow * self.nangle

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


def group_edges(G: int, lo: float = 0.01, hi: float = 100.0) -> np.ndarray:
    """G groups: nu_0 = 0, G-1 log-spaced interior edges on [lo, hi], nu_G = inf."""
    e = np.empty(G + 1)
    e[0] = 0.0
    e[G] = np.inf
    if G >= 2:
        e[1:G] = np.logspace(np.log10(lo), np.log10(hi), G - 1)
    return e


def representative_nu(edges: np.ndarray) -> np.ndarray:
    """Geometric-mean group frequency used only by the synthetic opacity law."""
    G = len(edges) - 1
    inner = np.array(edges[1:G], dtype=float)
    if G == 1:
        return np.array([1.0])
    if G == 2:
        return np.array([inner[0] / 2.0, inner[0] * 2.0])
    step = inner[1] / inner[0]
    ext = np.concatenate([[inner[0] / step], inner, [inner[-1] * step]])
    return np.sqrt(ext[:-1] * ext[1:])


def line_factors(G: int, seed: int, sd: float = 1.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.exp(sd * rng.standard_normal(G))


def blob_density(nx: int, ny: int, seed: int, nblob: int = 8, contrast: float = 100.0) -> np.ndarray:
    """rho = 1 + (contrast-1) * min(1, sum_b exp(-|x-c_b|^2 / (2 w_b^2))) on [0,1]^2 cell centres.

    Returned with x fastest: rho[ix + nx*iy]."""
    rng = np.random.default_rng(seed)
    cb = rng.uniform(0.1, 0.9, size=(nblob, 2))
    wb = rng.uniform(0.03, 0.1, size=nblob)
    xc = (np.arange(nx) + 0.5) / nx
    yc = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(xc, yc, indexing="xy")  # shape (ny, nx)
    s = np.zeros_like(X)
    for b in range(nblob):
        s += np.exp(-((X - cb[b, 0]) ** 2 + (Y - cb[b, 1]) ** 2) / (2.0 * wb[b] ** 2))
    rho = 1.0 + (contrast - 1.0) * np.minimum(1.0, s)
    return rho.reshape(-1)


def blob_density3(nx: int, ny: int, nz: int, seed: int, nblob: int = 8, contrast: float = 100.0) -> np.ndarray:
    """3-D counterpart of blob_density on [0,1]^3 cell centres, x fastest: rho[ix + nx*(iy + ny*iz)]."""
    rng = np.random.default_rng(seed)
    cb = rng.uniform(0.1, 0.9, size=(nblob, 3))
    wb = rng.uniform(0.05, 0.15, size=nblob)
    xc, yc, zc = [(np.arange(n) + 0.5) / n for n in (nx, ny, nz)]
    Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")  # shape (nz, ny, nx)
    s = np.zeros_like(X)
    for b in range(nblob):
        s += np.exp(-((X - cb[b, 0]) ** 2 + (Y - cb[b, 1]) ** 2 + (Z - cb[b, 2]) ** 2) / (2.0 * wb[b] ** 2))
    rho = 1.0 + (contrast - 1.0) * np.minimum(1.0, s)
    return rho.reshape(-1)


def linear_temperature(nx: int, ny: int = 1, nz: int = 1, t0: float = 1.0, t1: float = 0.1) -> np.ndarray:
    """T linear in x over cell centres from t0 to t1, constant in y and z."""
    xc = (np.arange(nx) + 0.5) / nx
    tx = t0 + (t1 - t0) * xc
    return np.tile(tx, ny * nz)


def opacity_rows(rho_cell: np.ndarray, edges: np.ndarray, lf: np.ndarray,
                 kappa0: float = 10.0, nu0: float = 1.0) -> np.ndarray:
    """rho*kappa_a per merged row k = g + G*cell."""
    nu = representative_nu(edges)
    kg = kappa0 * (nu / nu0) ** -3.0 * lf
    return (rho_cell[:, None] * kg[None, :]).reshape(-1)


def slab_config0() -> Workload:
    """1-D planar slab: Nx=64 on [0,1], G=16, 8 Gauss-Legendre mu, rho=1, kappa_s=0,
    T linear 1 -> 0.1, vacuum, dt=0.01, 10 steps, exact rank (tol 0, rank cap 8)."""
    nx, G = 64, 16
    edges = group_edges(G)
    lf = line_factors(G, seed=0)
    rho = np.ones(nx)
    ka = opacity_rows(rho, edges, lf)
    return Workload(
        name="slab1d_nx64_g16_mu8", ndim=1, nx=nx, ny=1, nz=1, ngroup=G,
        quad="gauss_legendre_mu", ntheta=8, nphi=1, extent=(1.0, 1.0, 1.0),
        c=1.0, dt=0.01, group_edges=edges, temperature=linear_temperature(nx),
        rho_kappa_a=ka, rho_kappa_s=np.zeros_like(ka), tol=0.0, rmax=8, steps=10, seed=0)


def plane_config1(nx: int = 128, ny: int = 128, G: int = 64, ntheta: int = 16, nphi: int = 32,
                  rmax: int = 32, tol: float = 1e-6, steps: int = 20, seed: int = 1,
                  cfl: float = 0.5) -> Workload:
    """2-D (x,y) on [0,1]^2, Gaussian-blob density (8 blobs, contrast 100), kappa_s = 0.1 kappa_a,
    T linear in x 1 -> 0.1, vacuum, CFL 0.5, lat/long ordinates."""
    edges = group_edges(G)
    lf = line_factors(G, seed=seed + 1000)
    rho = blob_density(nx, ny, seed=seed)
    ka = opacity_rows(rho, edges, lf)
    dx = 1.0 / nx
    return Workload(
        name=f"plane2d_{nx}x{ny}_g{G}_{ntheta}x{nphi}_r{rmax}", ndim=2, nx=nx, ny=ny, nz=1,
        ngroup=G, quad="latlong_midpoint", ntheta=ntheta, nphi=nphi, extent=(1.0, 1.0, 1.0),
        c=1.0, dt=cfl * dx, group_edges=edges, temperature=linear_temperature(nx, ny),
        rho_kappa_a=ka, rho_kappa_s=0.1 * ka, tol=tol, rmax=rmax, steps=steps, seed=seed)


def cube_config(nx: int = 6, ny: int = 5, nz: int = 4, G: int = 3, ntheta: int = 4, nphi: int = 8,
                rmax: int = 8, tol: float = 1e-6, steps: int = 4, seed: int = 5, cfl: float = 0.3) -> Workload:
    """3-D (x,y,z) on [0,1]^3: the plane workload's recipe in three dimensions (Gaussian-blob
    density, kappa_s = 0.1 kappa_a, T linear in x 1 -> 0.1), vacuum, lat/long ordinates; the
    time step dt = cfl * min(dx) keeps the forward-Euler transport step stable (sum over axes of
    lambda_a <= 3 cfl)."""
    edges = group_edges(G)
    lf = line_factors(G, seed=seed + 1000)
    rho = blob_density3(nx, ny, nz, seed=seed)
    ka = opacity_rows(rho, edges, lf)
    h = min(1.0 / nx, 1.0 / ny, 1.0 / nz)
    return Workload(
        name=f"cube3d_{nx}x{ny}x{nz}_g{G}_{ntheta}x{nphi}_r{rmax}", ndim=3, nx=nx, ny=ny, nz=nz,
        ngroup=G, quad="latlong_midpoint", ntheta=ntheta, nphi=nphi, extent=(1.0, 1.0, 1.0),
        c=1.0, dt=cfl * h, group_edges=edges, temperature=linear_temperature(nx, ny, nz),
        rho_kappa_a=ka, rho_kappa_s=0.1 * ka, tol=tol, rmax=rmax, steps=steps, seed=seed)


def nux_config(nx: int = 8, ny: int = 6, G: int = 6, ntheta: int = 4, nphi: int = 8, rmax: int = 16,
               tol: float = 1e-6, steps: int = 4, seed: int = 7, cfl: float = 0.5,
               contrast: float = 1000.0) -> Workload:
    """2-D problem on [0,1]^2 whose density, temperature and opacities depend on x only (so that
    the source step is a row scaling of a core over (group, x), the topology [Z(nu x)][y][theta]
    [phi]): rho(x) = 1 + 99 min(1, sum_b exp(-(x - c_b)^2 / (2 w_b^2))) with 4 blobs,
    c_b ~ U[0.1, 0.9], w_b ~ U[0.03, 0.1]; rho*kappa_a = rho(x) kappa0 (nu_f/nu0)^-3 (1 + contrast
    1[f is a line group]) with min(16, G/2) seeded line groups; kappa_s = 0.1 kappa_a; T linear in
    x 1 -> 0.1; vacuum; lat/long ordinates; dt = cfl dx."""
    rng = np.random.default_rng(seed)
    cb = rng.uniform(0.1, 0.9, 4)
    wb = rng.uniform(0.03, 0.1, 4)
    xc = (np.arange(nx) + 0.5) / nx
    s_ = np.zeros(nx)
    for b in range(4):
        s_ += np.exp(-(xc - cb[b]) ** 2 / (2.0 * wb[b] ** 2))
    rho_x = 1.0 + 99.0 * np.minimum(1.0, s_)
    edges = group_edges(G)
    lines = np.zeros(G)
    nl = max(1, min(16, G // 2))
    lines[rng.choice(G, nl, replace=False)] = contrast
    ka = opacity_rows(np.tile(rho_x, ny), edges, 1.0 + lines)
    return Workload(
        name=f"nux2d_{nx}x{ny}_g{G}_{ntheta}x{nphi}_r{rmax}", ndim=2, nx=nx, ny=ny, nz=1,
        ngroup=G, quad="latlong_midpoint", ntheta=ntheta, nphi=nphi, extent=(1.0, 1.0, 1.0),
        c=1.0, dt=cfl / max(nx, ny), group_edges=edges, temperature=linear_temperature(nx, ny),
        rho_kappa_a=ka, rho_kappa_s=0.1 * ka, tol=tol, rmax=rmax, steps=steps, seed=seed)


def batch_config3(nprob: int = 256, seed: int = 3, scale: int = 1, tol: float = 1e-6,
                  steps: int = 20) -> list:
    """Independent 2-D problems of uneven shape stepped as one batch: Nx = Ny ~ U{32, 64, ..., 192},
    G ~ U{16, 32, ..., 96}, ordinates ~ U{8x16, 12x24, 16x32}, r_max ~ U{8, ..., 48}, each with its
    own seeded density blobs and line factors, and isotropic Planck inflow on the x- face at
    T_b ~ U[0.1, 1] (the rest vacuum).  `scale` > 1 divides the cell counts and group counts by
    `scale` and halves the ordinates (floor 4 x 8), for parity runs the oracle can finish."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(nprob):
        n = int(rng.choice([32, 64, 96, 128, 160, 192]))
        G = int(rng.choice([16, 32, 48, 64, 80, 96]))
        nth, nph = [(8, 16), (12, 24), (16, 32)][int(rng.integers(3))]
        rmax = int(rng.integers(8, 49))
        Tb = float(rng.uniform(0.1, 1.0))
        pseed = int(rng.integers(1, 1 << 30))
        if scale > 1:
            n, G = max(4, n // scale), max(2, G // scale)
            nth, nph = max(4, nth // 2), max(8, nph // 2)
            rmax = max(2, min(rmax // scale + 2, nth))
        wl = plane_config1(nx=n, ny=n, G=G, ntheta=nth, nphi=nph, rmax=rmax, tol=tol, steps=steps, seed=pseed)
        out.append(replace(wl, name=f"batch{i}_{n}x{n}_g{G}_{nth}x{nph}_r{rmax}",
                           inflow_temperature=(Tb, None, None, None, None, None)))
    return out


def gaussian_diffusion_config(nx: int = 128, G: int = 8, kappa_max: float = 2000.0, ntheta: int = 16,
                              rmax: int = 16, tol: float = 1e-6, steps: int = 4000,
                              seed: int = 4) -> Workload:
    """The multigroup Gaussian-diffusion slab of Sec. 4.3 at reduced size: nx cells on [-5, 5],
    rho = c = 1, pure scattering with rho*kappa_s[f] ~ U[1000, kappa_max] (seeded, the same in
    every cell), no absorption, CFL = 1 (dt = dx), vacuum faces, the central flux (Rusanov with
    wavespeed 0).  The temperature is irrelevant (kappa_a = 0) and set to 1.  The initial field
    (an isotropic Gaussian per group) is built by the consumer, not here."""
    rng = np.random.default_rng(seed)
    ks = rng.uniform(1000.0, kappa_max, G)
    L = 10.0
    return Workload(
        name=f"diffusion1d_nx{nx}_g{G}_mu{ntheta}_kmax{int(kappa_max)}", ndim=1, nx=nx, ny=1, nz=1,
        ngroup=G, quad="gauss_legendre_mu", ntheta=ntheta, nphi=1, extent=(L, 1.0, 1.0),
        c=1.0, dt=L / nx, group_edges=group_edges(G), temperature=np.ones(nx),
        rho_kappa_a=np.zeros(nx * G), rho_kappa_s=np.tile(ks, nx), flux="central",
        tol=tol, rmax=rmax, steps=steps, seed=seed)


def sketch_matrix(nang: int, ell: int, seed: int = 11) -> np.ndarray:
    """Gaussian N(0, 1) sketch omega (nang x ell) for randomized rounding, seeded."""
    return np.random.default_rng(seed).standard_normal((nang, ell))


def graded_state(wl: Workload, seed: int = 21):
    """A seeded state of full rank r_max with geometrically graded cores (factors 0.55^j on the
    merged core's columns, 0.7^j on the polar core's), so that every rank decision of a step is far
    from a tie: iid N(0,1) cores, shapes of the workload's TT (d = 3)."""
    a = random_tt([wl.nrow, wl.ntheta, wl.nphi], [wl.rmax, wl.rmax], seed=seed)
    a[0] = a[0] * (0.55 ** np.arange(wl.rmax))[None, None, :]
    a[1] = a[1] * (0.7 ** np.arange(wl.rmax))[None, None, :]
    return a


def random_tt(n: Sequence[int], ranks: Sequence[int], seed: int, scale: float = 1.0):
    """Cores with iid N(0,1) entries, core k of shape (r_{k-1}, n_k, r_k)."""
    rng = np.random.default_rng(seed)
    r = [1] + list(ranks) + [1]
    assert len(r) == len(n) + 1
    return [scale * rng.standard_normal((r[k], n[k], r[k + 1])) for k in range(len(n))]
