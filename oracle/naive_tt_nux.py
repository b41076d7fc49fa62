"""Naive explicit-sum TT step in the split topology [Z(nu x)][y][theta][phi] (test infrastructure;
see oracle/__init__).

Sec. 5.2 compares the merged spatio-spectral core of Eq. (tensor_decomp_mer) with orderings that
give space its own cores (Fig. 3d4dtt); this module takes the one whose first core merges
frequency with x and keeps y as a core of its own, for 2-D problems:

    I[(g, ix), iy, l, p] = C0[(g, ix)] C1[iy] C2[l] C3[p],   core-0 row k0 = g + G ix,

so the full-grid row of the dense stepper is k = k0 + G Nx iy.  The step is the merged one's,
step-then-truncate (end of Sec. 3.1), with the operators acting on the cores they touch:

* transport (Appendix A, 'Value of n'): an x-term differences core-0 rows G apart (cells ix and
  ix -+ 1), a y-term differences core 1 along its mode; both scale the angular cores by the
  term's factors, exactly as in the merged topology; vacuum faces only;
* source, Eq. (discRTsource) at fixed T, for opacities and emission that depend on (g, x) only:
  1/(1 + a + s) scales the rows of core 0, and the isotropic term
  g = (a eps + s J^{m+1}) / (1 + a + s) with J^{m+1} = (J* + a eps)/(1 + a) is
  g = a eps / (1 + a) + s / ((1 + a)(1 + a + s)) J*, a TT of rank 1 + r_1 at the first bond
  (J* = C0 C1 w, w the angular weights contracted through C2 C3);
* rounding: the SVD rounding of oracle.naive_tt over the four cores.
"""
import numpy as np

from . import naive_tt as nt


def _dims(coef):
    assert coef.ndim == 2 and coef.nz == 1, "the [Z(nu x)][y][theta][phi] topology is for 2-D problems"
    return coef.G * coef.nx, coef.ny


def _row_field(arr, coef):
    """A per-merged-row field that depends on (g, x) only, as its core-0 rows (length G Nx)."""
    n0, ny = _dims(coef)
    a = np.asarray(arr, dtype=float).reshape(ny, n0)
    assert np.all(a == a[0]), "opacities and emission must not depend on y in this topology"
    return a[0].copy()


def from_rows(rows, coef):
    """Isotropic TT of a per-merged-row field: the (G Nx) x Ny matrix split by an SVD (exact),
    angular cores all ones."""
    n0, ny = _dims(coef)
    M = np.asarray(rows, dtype=float).reshape(ny, n0).T          # [k0, iy]
    U, S, Vt = np.linalg.svd(M, full_matrices=False)
    r = max(1, int(np.sum(S > S[0] * 1e-15))) if S[0] > 0 else 1
    return [(U[:, :r] * S[:r]).reshape(1, n0, r), Vt[:r].reshape(r, ny, 1),
            np.ones((1, coef.ntheta, 1)), np.ones((1, coef.nphi, 1))]


def to_dense_rows(tt):
    """Full tensor as the dense stepper's (N_Z, N_theta N_phi) array, row k = k0 + G Nx iy."""
    F = nt.full(tt)                                             # (G Nx, Ny, N_theta, N_phi)
    n0, ny = F.shape[0], F.shape[1]
    return F.transpose(1, 0, 2, 3).reshape(ny * n0, -1)


def _shift_x(C0, coef, sgn):
    """Core-0 row k0 -> row k0 + sgn G (cell ix + sgn), zero past the x faces."""
    out = np.zeros_like(C0)
    ix = (np.arange(C0.shape[1]) // coef.G)
    valid = (ix + sgn >= 0) & (ix + sgn < coef.nx)
    rows = np.nonzero(valid)[0]
    out[:, rows, :] = C0[:, rows + sgn * coef.G, :]
    return out


def _shift_y(C1, sgn):
    """Core-1 mode iy -> iy + sgn, zero past the y faces."""
    out = np.zeros_like(C1)
    if sgn > 0:
        out[:, :-1, :] = C1[:, 1:, :]
    else:
        out[:, 1:, :] = C1[:, :-1, :]
    return out


def _difference(core, shift, w):
    """The term's difference of a core along its axis (upwind, Rusanov central / diffusion)."""
    if w == 2:
        return 0.5 * (shift(+1) - shift(-1))
    if w == -2:
        return -0.5 * (shift(+1) - 2.0 * core + shift(-1))
    if w > 0:
        return core - shift(-1)
    return shift(+1) - core


def transport_sum(tt, coef):
    """Explicit TT sum [X, T_1 X, ..., T_n X] of the forward-Euler update (vacuum faces)."""
    assert all(b is None for b in coef.inflow), "vacuum faces only in this topology"
    C0, C1, C2, C3 = tt
    summands = [tt]
    for (ax, w, facs) in nt.angular_terms(coef):
        lam = coef.lam[ax]
        if ax == 0:
            c0 = -lam * _difference(C0, lambda s: _shift_x(C0, coef, s), w)
            c1 = C1.copy()
        else:
            c0 = -lam * C0
            c1 = _difference(C1, lambda s: _shift_y(C1, s), w)
        summands.append([c0, c1, C2 * facs[0][None, :, None], C3 * facs[1][None, :, None]])
    return nt.add_many(summands)


def angular_weights(tt, coef):
    """w (length r_2) with J = (1/4 pi) sum dOmega I = C0 C1 w."""
    dom = coef.dirs["domega"].reshape(coef.ntheta, coef.nphi)
    right = np.tensordot(tt[2], tt[3], axes=([-1], [0]))[:, :, :, 0]   # (r2, N_theta, N_phi)
    return np.tensordot(right, dom, axes=([1, 2], [0, 1])) / (4.0 * np.pi)


def source_sum(tt, coef):
    """Eq. (discRTsource) at fixed T as the TT sum [row-scaled X, g (x) 1 (x) 1]."""
    C0, C1, C2, C3 = tt
    a = _row_field(coef.acoef, coef)
    s = _row_field(coef.scoef, coef)
    e = _row_field(coef.eps, coef)
    dinv = 1.0 / (1.0 + a + s)
    alpha = a * e / (1.0 + a)
    beta = s / ((1.0 + a) * (1.0 + a + s))
    w = angular_weights(tt, coef)
    Jy = np.tensordot(C1, w, axes=([2], [0]))                     # (r1, Ny): C1 w
    n0, ny = C0.shape[1], C1.shape[1]
    r1 = C0.shape[2]
    g0 = np.concatenate([alpha[:, None], beta[:, None] * C0[0]], axis=1).reshape(1, n0, 1 + r1)
    g1 = np.concatenate([np.ones((1, ny)), Jy], axis=0).reshape(1 + r1, ny, 1)
    iso = [g0, g1, np.ones((1, coef.ntheta, 1)), np.ones((1, coef.nphi, 1))]
    scaled = [C0 * dinv[None, :, None], C1.copy(), C2.copy(), C3.copy()]
    return nt.add(scaled, iso)


def step(tt, coef, tol, rmax, info=None):
    """Transport, round, source, round (step-then-truncate, end of Sec. 3.1)."""
    i1, i2 = {}, {}
    x = nt.round_tt(transport_sum(tt, coef), tol, rmax, i1)
    x = nt.round_tt(source_sum(x, coef), tol, rmax, i2)
    if info is not None:
        info["transport_round"] = i1
        info["source_round"] = i2
    return x


def energy_density_rows(tt, coef):
    """E_f = (4 pi / c) J per merged row k = k0 + G Nx iy."""
    J = np.tensordot(tt[0][0], np.tensordot(tt[1], angular_weights(tt, coef), axes=([2], [0])), axes=([1], [0]))
    return 4.0 * np.pi / coef.c * J.T.reshape(-1)
