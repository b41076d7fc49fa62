"""Naive explicit-sum tensor-train arithmetic in FP64 (test infrastructure; see oracle/__init__).

TT format of Eq. (tensor_decomp_mer), Sec. 3.1: I_{k l p} = Z_k Theta_l Phi_p, generalised to
a list of cores G_j of shape (r_{j-1}, n_j, r_j) with r_0 = r_d = 1.  The merged
spatio-spectral core Z is core 0 (rows k = g + G*cell).  The slab case has d = 2 with a
single mu core; the plane case has d = 3 with polar and azimuthal cores.

Operations (all written from their definitions, with LAPACK through numpy for QR/SVD):

* ``add``      TT addition by rank concatenation (Sec. 3.1, basic TT operations; Appendix A,
               summands of the post-transport tensor): first core side by side, middle cores
               block diagonal, last core stacked.
* ``dot``      <X, Y> by left-to-right contraction of the cores.
* ``round``    SVD-based rounding (Sec. 3.1 footnote, Oseledets 2011): left-to-right
               Householder QR sweep, then right-to-left truncated-SVD sweep with
               delta = tol * ||X||_F / sqrt(d-1); at each bond keep the smallest k >= 1 whose
               discarded tail sqrt(sum_{j>k} sigma_j^2) <= delta, then cap at rmax.  tol == 0
               keeps the full rank of every unfolding (the 'exact rank' case).
* ``transport_sum``  the forward-Euler upwind update as the explicit sum of the solution, its
               n = 2 d_X rank-1-operator images and the rank-n_b Dirichlet inflow tensor
               (Appendix A, 'Value of n' and the transport-update figure): ranks
               (n+1) r + n_b before rounding.
* ``source_sum``     the backward-Euler source update of Eq. (discRTsource) at fixed T as
               diag(1/(1+a+s)) Z plus the rank-1 isotropic term g (x) 1 (x) 1 (Sec. 3.1:
               rank-1 lift of a spatio-spectral field; Appendix A: source adds to the ranks).
* ``step``     transport -> round -> source -> round (step-then-truncate, end of Sec. 3.1).
"""
import math

import numpy as np


# --- basic TT arithmetic -------------------------------------------------------------------

def ranks(tt):
    return [1] + [c.shape[2] for c in tt[:-1]] + [1]


def full(tt):
    """Dense tensor of shape (n_0, ..., n_{d-1})."""
    out = tt[0].reshape(tt[0].shape[1], tt[0].shape[2])
    for c in tt[1:]:
        out = np.tensordot(out, c, axes=([-1], [0]))
    return out.reshape([c.shape[1] for c in tt])


def scale(tt, alpha):
    out = [c.copy() for c in tt]
    out[0] = out[0] * alpha
    return out


def add(x, y):
    d = len(x)
    assert len(y) == d
    if d == 1:
        return [x[0] + y[0]]
    out = []
    for j in range(d):
        a, b = x[j], y[j]
        assert a.shape[1] == b.shape[1]
        if j == 0:
            out.append(np.concatenate([a, b], axis=2))
        elif j == d - 1:
            out.append(np.concatenate([a, b], axis=0))
        else:
            m = np.zeros((a.shape[0] + b.shape[0], a.shape[1], a.shape[2] + b.shape[2]))
            m[:a.shape[0], :, :a.shape[2]] = a
            m[a.shape[0]:, :, a.shape[2]:] = b
            out.append(m)
    return out


def add_many(terms):
    acc = terms[0]
    for t in terms[1:]:
        acc = add(acc, t)
    return acc


def dot(x, y):
    W = np.ones((1, 1))
    for a, b in zip(x, y):
        # W'[p, q] = sum_{i, s, t} W[s, t] a[s, i, p] b[t, i, q]
        W = np.einsum("st,sip,tiq->pq", W, a, b)
    return float(W[0, 0])


def norm(x):
    return math.sqrt(max(dot(x, x), 0.0))


# --- SVD-based rounding --------------------------------------------------------------------

def _tail(S):
    """t[k] = sqrt(sum_{j>=k} S_j^2) for k = 0..len(S) (t[len] = 0), summed from the small end."""
    sq = S[::-1] ** 2
    cs = np.concatenate([[0.0], np.cumsum(sq)])[::-1]
    return np.sqrt(cs)


def choose_rank(S, delta, rmax, exact):
    """Truncation rule shared by every bond (see module docstring)."""
    n = len(S)
    if exact:
        k = n
    else:
        t = _tail(S)
        k = n
        for kk in range(1, n + 1):
            if t[kk] <= delta:
                k = kk
                break
    return max(1, min(k, rmax)), k


def round_tt(tt, tol, rmax=1 << 30, info=None):
    """SVD-based rounding: L->R Householder QR sweep, R->L truncated SVD sweep."""
    d = len(tt)
    cores = [c.copy() for c in tt]
    # left-to-right orthogonalisation
    for j in range(d - 1):
        r0, n, r1 = cores[j].shape
        Q, R = np.linalg.qr(cores[j].reshape(r0 * n, r1), mode="reduced")
        cores[j] = Q.reshape(r0, n, Q.shape[1])
        cores[j + 1] = np.tensordot(R, cores[j + 1], axes=([1], [0]))
    nrm = float(np.linalg.norm(cores[d - 1]))
    delta = tol * nrm / math.sqrt(max(d - 1, 1))
    exact = (tol == 0.0)
    bonds = []
    # right-to-left truncation
    for j in range(d - 1, 0, -1):
        r0, n, r1 = cores[j].shape
        U, S, Vt = np.linalg.svd(cores[j].reshape(r0, n * r1), full_matrices=False)
        k, kuncapped = choose_rank(S, delta, rmax, exact)
        t = _tail(S)
        gap = np.inf
        if not exact and delta > 0:
            for kk in (kuncapped - 1, kuncapped):
                if 1 <= kk <= len(S):
                    gap = min(gap, abs(t[kk] - delta) / delta)
        bonds.append(dict(bond=j, sigma=S.copy(), rank=k, uncapped=kuncapped, gap=gap))
        cores[j] = Vt[:k].reshape(k, n, r1)
        cores[j - 1] = np.tensordot(cores[j - 1], U[:, :k] * S[:k], axes=([2], [0]))
    if info is not None:
        info["norm"] = nrm
        info["delta"] = delta
        info["bonds"] = bonds[::-1]
        info["ranks"] = ranks(cores)
    return cores


def right_part(cores):
    """Contraction of cores (r0, n_1, r_1) ... (r_{m-1}, n_m, 1) into an r0 x (n_1 ... n_m) matrix."""
    B = cores[0]
    for c in cores[1:]:
        B = np.tensordot(B, c, axes=([B.ndim - 1], [0]))
    return B.reshape(B.shape[0], -1)


def round_tt_gram(tt, tol, rmax=1 << 30, info=None):
    """Gram-based rounding of the first bond (the Gram method among the three rounding methods
    of Sec. 3.1): the left unfolding A of the first core enters only through its Gram matrix
    G = A^T A = V diag(lam) V^T, whose square root R = diag(lam^(1/2)) V^T stands in for the QR
    factor (R^T R = A^T A, so every unfolding of X' = R x (cores 2..d) has the singular values and
    right singular vectors of the same unfolding of X).  X' is rounded by round_tt; its new
    cores 2..d are those of X, and the new first core is A projected onto the new right frame,
    A (B_old B_new^T) (the Q U S of the QR route).  Accuracy: Gram squares the condition number,
    so singular values below about sqrt(eps) |X| are not resolved."""
    d = len(tt)
    r0, n, r1 = tt[0].shape
    A = tt[0].reshape(r0 * n, r1)
    lam, V = np.linalg.eigh(A.T @ A)
    R = np.sqrt(np.clip(lam, 0.0, None))[:, None] * V.T
    small = [R.reshape(1, r1, r1)] + [c.copy() for c in tt[1:]]
    out = round_tt(small, tol, rmax, info)
    Bold = right_part(tt[1:])
    Bnew = right_part(out[1:])
    first = (A @ (Bold @ Bnew.T)).reshape(r0, n, Bnew.shape[0])
    return [first] + out[1:]


# --- merged-topology transport and source (upwind, vacuum or Dirichlet inflow) -------------

def angular_terms(coef):
    """Transport terms of the TT operator (Appendix A, 'Value of n').

    Returns a list of (axis, w, factors) where factors is one diagonal per angular core
    such that n_axis * 1[n_axis (>=|<) 0] = prod of the factors over the angular nodes (upwind,
    w = +1 / -1).  For the Rusanov flux the two terms of an axis are w = +2 (the central
    difference, factors of the full n_axis) and w = -2 (the diffusion term, factors 1); the
    central flux (Rusanov with wavespeed S+ = 0, Sec. 4.3) keeps the w = +2 term only."""
    d = coef.dirs
    terms = []
    flux = getattr(coef, "flux", "upwind")
    if flux in ("rusanov", "central"):
        diffusion = flux == "rusanov"
        if coef.ntheta > 0 and coef.nphi == 1 and "w" in d:
            terms.append((0, +2, [d["mu"]]))
            if diffusion:
                terms.append((0, -2, [np.ones_like(d["mu"])]))
            return terms
        mu, phi, st = d["mu"], d["phi"], d["sintheta"]
        full = {0: [st, np.cos(phi)], 1: [st, np.sin(phi)], 2: [mu, np.ones(coef.nphi)]}
        for ax in range(coef.ndim):
            terms.append((ax, +2, full[ax]))
            if diffusion:
                terms.append((ax, -2, [np.ones(coef.ntheta), np.ones(coef.nphi)]))
        return terms
    if coef.ntheta > 0 and coef.nphi == 1 and "w" in d:   # planar slab, single mu core
        mu = d["mu"]
        terms.append((0, +1, [np.where(mu >= 0.0, mu, 0.0)]))
        terms.append((0, -1, [np.where(mu < 0.0, mu, 0.0)]))
        return terms
    mu, phi, st = d["mu"], d["phi"], d["sintheta"]
    cph, sph = np.cos(phi), np.sin(phi)
    for ax in range(coef.ndim):
        if ax == 0:
            terms.append((0, +1, [st, np.where(cph >= 0.0, cph, 0.0)]))
            terms.append((0, -1, [st, np.where(cph < 0.0, cph, 0.0)]))
        elif ax == 1:
            terms.append((1, +1, [st, np.where(sph >= 0.0, sph, 0.0)]))
            terms.append((1, -1, [st, np.where(sph < 0.0, sph, 0.0)]))
        else:
            terms.append((2, +1, [np.where(mu >= 0.0, mu, 0.0), np.ones(coef.nphi)]))
            terms.append((2, -1, [np.where(mu < 0.0, mu, 0.0), np.ones(coef.nphi)]))
    return terms


def _cell_index(coef):
    nrow = coef.nrow
    cell = np.arange(nrow) // coef.G
    ix = cell % coef.nx
    iy = (cell // coef.nx) % coef.ny
    iz = cell // (coef.nx * coef.ny)
    return (ix, iy, iz)


def _shift_rows(Z, coef, axis, sgn):
    """Row k -> Z[k + sgn*stride] with zero where the neighbour cell leaves the grid."""
    stride = [coef.G, coef.G * coef.nx, coef.G * coef.nx * coef.ny][axis]
    ext = [coef.nx, coef.ny, coef.nz][axis]
    idx = _cell_index(coef)[axis]
    out = np.zeros_like(Z)
    valid = (idx + sgn >= 0) & (idx + sgn < ext)
    rows = np.nonzero(valid)[0]
    out[rows] = Z[rows + sgn * stride]
    return out


def _apply_diag(core, diag):
    return core * diag[None, :, None]


def transport_sum(tt, coef):
    """Explicit TT sum [X, T_1 X, ..., T_n X, sum_t BC_t] of the upwind forward-Euler update."""
    Z = tt[0][0]                      # (N_Z, r)
    summands = [tt]
    bc_terms = []
    idx = _cell_index(coef)
    for (ax, w, facs) in angular_terms(coef):
        lam = coef.lam[ax]
        if w == 2:      # Rusanov central part: lam n (I_{i+1} - I_{i-1}) / 2
            DZ = 0.5 * (_shift_rows(Z, coef, ax, +1) - _shift_rows(Z, coef, ax, -1))
        elif w == -2:   # Rusanov diffusion part: -lam (I_{i+1} - 2 I_i + I_{i-1}) / 2
            DZ = -0.5 * (_shift_rows(Z, coef, ax, +1) - 2.0 * Z + _shift_rows(Z, coef, ax, -1))
        elif w > 0:
            DZ = Z - _shift_rows(Z, coef, ax, -1)          # I_i - I_{i-1}
        else:
            DZ = _shift_rows(Z, coef, ax, +1) - Z          # I_{i+1} - I_i
        cores = [(-lam * DZ)[None, :, :]]
        for j, f in enumerate(facs):
            cores.append(_apply_diag(tt[1 + j], f))
        summands.append(cores)
        if abs(w) == 2:
            continue    # Rusanov: vacuum ghost cells only
        face = 2 * ax + (0 if w > 0 else 1)
        b = coef.inflow[face]
        if b is not None:
            ext = [coef.nx, coef.ny, coef.nz][ax]
            at_face = (idx[ax] == 0) if w > 0 else (idx[ax] == ext - 1)
            g = np.arange(coef.nrow) % coef.G
            z = np.where(at_face, (lam if w > 0 else -lam) * b[g], 0.0)
            bc = [z.reshape(1, -1, 1)] + [f.reshape(1, -1, 1) for f in facs]
            bc_terms.append(bc)
    return add_many(summands + bc_terms)


def angular_weights_vector(tt, coef):
    """v such that J*(k) = Z[k, :] . v, with J = (1/4pi) sum dOmega I (Sec. 2)."""
    dom = coef.dirs["domega"].reshape([c.shape[1] for c in tt[1:]])
    right = tt[1]
    for c in tt[2:]:
        right = np.tensordot(right, c, axes=([-1], [0]))
    right = right.reshape(right.shape[0], -1)       # (r1, n_1*...*n_{d-1})
    return right @ dom.reshape(-1) / (4.0 * np.pi)


def source_sum(tt, coef):
    """Eq. (discRTsource) at fixed T as the explicit TT sum [diag(1/(1+a+s)) Z, g]."""
    Z = tt[0][0]
    v = angular_weights_vector(tt, coef)
    Js = Z @ v
    a, s, e = coef.acoef, coef.scoef, coef.eps
    Jn = (Js + a * e) / (1.0 + a)
    dinv = 1.0 / (1.0 + a + s)
    g = (a * e + s * Jn) * dinv
    scaled = [(dinv[:, None] * Z)[None, :, :]] + [c.copy() for c in tt[1:]]
    iso = [g.reshape(1, -1, 1)] + [np.ones((1, c.shape[1], 1)) for c in tt[1:]]
    return add(scaled, iso)


def step(tt, coef, tol, rmax, info=None, rounding="svd", omega=None):
    """One step-then-truncate time step: transport, round, source, round (end of Sec. 3.1).
    rounding: "svd" (round_tt), "gram" (round_tt_gram) or "randomized" (round_tt_randomized with
    the sketch omega), used for both roundings."""
    if rounding == "randomized":
        def rnd(x, t, r, i=None):
            return round_tt_randomized(x, t, r, omega, i)
    else:
        rnd = round_tt_gram if rounding == "gram" else round_tt
    i1, i2 = {}, {}
    x = rnd(transport_sum(tt, coef), tol, rmax, i1)
    x = rnd(source_sum(x, coef), tol, rmax, i2)
    if info is not None:
        info["transport_round"] = i1
        info["source_round"] = i2
    return x


def initial_tt(rows, coef):
    """Rank-1 isotropic TT of a per-row field: Z = rows, angular cores all ones (Sec. 3.1)."""
    if coef.nphi == 1 and "w" in coef.dirs:
        return [rows.reshape(1, -1, 1), np.ones((1, coef.ntheta, 1))]
    return [rows.reshape(1, -1, 1), np.ones((1, coef.ntheta, 1)), np.ones((1, coef.nphi, 1))]


def to_dense_rows(tt):
    """Full tensor as an (N_Z, N_angles) matrix with angle index q = l*N_phi + p."""
    F = full(tt)
    return F.reshape(F.shape[0], -1)


def energy_density_rows(tt, coef):
    """E_f = (4 pi / c) J_f per merged row."""
    return 4.0 * np.pi / coef.c * (tt[0][0] @ angular_weights_vector(tt, coef))


def compression(nX, nnu, ntheta, nphi, rzt, rtp):
    """Eq. (compression), Sec. 3.2."""
    return (nX * nnu * ntheta * nphi) / (nX * nnu * rzt + ntheta * rzt * rtp + nphi * rtp)


# --- internal structure of the merged core (Sec. 5.2) --------------------------------------

def delta_rank(S, delta_rel):
    """Smallest k with sqrt(sum_{j >= k} sigma_j^2) <= delta_rel * ||sigma||_2 (the delta-SVD of
    Sec. 5.4: relative Frobenius error below delta)."""
    S = np.asarray(S, dtype=float)
    tot = math.sqrt(float(np.sum(S ** 2)))
    if tot == 0.0:
        return 1
    t = _tail(S)
    for k in range(1, len(S) + 1):
        if t[k] <= delta_rel * tot:
            return k
    return len(S)


def internal_ranks(Z, G, delta_rel):
    """Internal delta-ranks of the merged core Z (N_X G x r, row k = g + G cell), Sec. 5.2:
    r1 (frequency-leading) of reshape(Z, [N_nu, N_X r]) and r1x (space-leading) of
    reshape(Z, [N_X, N_nu r]).  The angular cores must be right-orthonormal (a rounded state), so
    that these local errors are global ones.  Returns (r1, r1x, sigma_nu, sigma_x)."""
    nrow, r = Z.shape
    nX = nrow // G
    Z3 = Z.reshape(nX, G, r)                              # [cell][g][q]
    M_nu = np.transpose(Z3, (1, 0, 2)).reshape(G, nX * r)
    M_x = Z3.reshape(nX, G * r)
    s_nu = np.linalg.svd(M_nu, compute_uv=False)
    s_x = np.linalg.svd(M_x, compute_uv=False)
    return delta_rank(s_nu, delta_rel), delta_rank(s_x, delta_rel), s_nu, s_x


def relative_compression(nX, nnu, ntheta, nphi, r1, r1x, r2, r3):
    """Eqs. (rel_compression_nu) and (rel_compression_x): (C_rel^nu, C_rel^x), with N_TT the
    parameter count of the merged-core TT."""
    ntt = nX * nnu * r2 + ntheta * r2 * r3 + nphi * r3
    c_nu = ntt / (nnu * r1 + nX * r1 * r2 + ntheta * r2 * r3 + nphi * r3)
    c_x = ntt / (nX * r1x + nnu * r1x * r2 + ntheta * r2 * r3 + nphi * r3)
    return c_nu, c_x


def round_tt_randomized(tt, tol, rmax, omega, info=None):
    """Randomized rounding of the first bond (the randomized method among the three rounding
    methods of Sec. 3.1): the first unfolding X_(1) = A B (A the first core's left unfolding, B the
    right part) is sketched as Y = X_(1) omega = A (B omega) with a caller-drawn omega
    (n_2 ... n_d x l); Q from the QR of Y spans the sketch, and C = Q^T A stands in for the QR
    factor of A (X' = C x (cores 2..d) = Q^T X).  X' is rounded by round_tt (the SVD-based
    truncation at the same tolerance); its new cores 2..d are X's, and the new first core is A
    projected onto the new right frame, A (B_old B_new^T).  With l >= rank(A) this is SVD rounding;
    otherwise it keeps what the sketch captured (randomized range finder)."""
    r0, n, r1 = tt[0].shape
    A = tt[0].reshape(r0 * n, r1)
    Bold = right_part(tt[1:])
    Y = A @ (Bold @ omega)
    Q, _ = np.linalg.qr(Y, mode="reduced")
    C = Q.T @ A
    small = [C.reshape(1, C.shape[0], r1)] + [c.copy() for c in tt[1:]]
    out = round_tt(small, tol, rmax, info)
    Bnew = right_part(out[1:])
    first = (A @ (Bold @ Bnew.T)).reshape(r0, n, Bnew.shape[0])
    return [first] + out[1:]
