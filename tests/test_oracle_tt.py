"""Pins of the naive TT oracle: brute force, closed forms and the dense stepper."""
import math

import numpy as np
import pytest

from oracle import dense, naive_tt as nt, problem
from paper_2602_00290_gb300.workloads import Workload, plane_config1, random_tt, slab_config0


def test_full_and_dot_brute_force():
    x = random_tt([5, 3, 4], [2, 3], seed=1)
    y = random_tt([5, 3, 4], [3, 2], seed=2)
    Fx, Fy = nt.full(x), nt.full(y)
    # brute-force element loop for the full tensor
    ref = np.zeros((5, 3, 4))
    for i in range(5):
        for j in range(3):
            for k in range(4):
                ref[i, j, k] = (x[0][0, i, :] @ x[1][:, j, :] @ x[2][:, k, 0])
    assert np.allclose(Fx, ref, rtol=0, atol=1e-13)
    assert abs(nt.dot(x, y) - float(np.sum(Fx * Fy))) < 1e-12 * abs(np.sum(Fx * Fy)) + 1e-14
    assert abs(nt.norm(x) - np.linalg.norm(Fx)) < 1e-12 * np.linalg.norm(Fx)


def test_add_is_elementwise_sum_and_ranks_add():
    x = random_tt([6, 3, 4], [2, 3], seed=3)
    y = random_tt([6, 3, 4], [3, 2], seed=4)
    s = nt.add(x, y)
    assert nt.ranks(s) == [1, 5, 5, 1]
    assert np.allclose(nt.full(s), nt.full(x) + nt.full(y), atol=1e-13)


@pytest.mark.parametrize("d,n,r", [(3, [40, 6, 7], [5, 4]), (2, [30, 9], [6]), (4, [12, 3, 4, 5], [4, 5, 3])])
def test_round_exact_reconstruction(d, n, r):
    x = random_tt(n, r, seed=7)
    info = {}
    y = nt.round_tt(x, 1e-12, info=info)
    assert nt.ranks(y)[1:-1] == list(r)
    err = np.linalg.norm(nt.full(y) - nt.full(x))
    assert err <= 1e-12 * np.linalg.norm(nt.full(x))


def test_round_x_plus_x_and_x_minus_x():
    x = random_tt([20, 5, 6], [3, 4], seed=9)
    y = nt.round_tt(nt.add(x, x), 1e-10)
    assert nt.ranks(y) == nt.ranks(x)
    assert np.allclose(nt.full(y), 2 * nt.full(x), atol=1e-10 * np.abs(nt.full(x)).max())
    # X - X is zero up to round-off; a relative tolerance then resolves the round-off itself,
    # so only the size of the result is fixed, not its ranks
    z = nt.round_tt(nt.add(x, nt.scale(x, -1.0)), 1e-8)
    assert np.max(np.abs(nt.full(z))) < 1e-14 * np.abs(nt.full(x)).max()
    # an exactly zero tensor rounds to ranks 1 with zero cores
    zero = [np.zeros_like(c) for c in nt.add(x, x)]
    z = nt.round_tt(zero, 1e-8)
    assert nt.ranks(z) == [1, 1, 1, 1] and all(not np.any(c) for c in z[:1])
    assert not np.any(nt.full(z))


def test_round_matrix_known_spectrum():
    """d = 2 with prescribed singular values: the kept rank and the error follow the tail rule
    exactly (Eckart-Young): error = sqrt(sum of discarded sigma^2) <= tol * ||X||."""
    rng = np.random.default_rng(0)
    m, n = 30, 12
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    s = 10.0 ** -np.arange(n, dtype=float)          # 1, 0.1, ..., 1e-11
    A = (U * s) @ V.T
    x = [A.reshape(1, m, n) @ np.eye(n)[None], np.eye(n).reshape(n, n, 1)]
    x = [A.reshape(1, m, n), np.eye(n).reshape(n, n, 1)]
    nrm = math.sqrt(np.sum(s ** 2))
    for tol, kexp in ((3e-3, 3), (3e-6, 6), (3e-9, 9)):
        y = nt.round_tt(x, tol)
        k = nt.ranks(y)[1]
        assert k == kexp
        err = np.linalg.norm(nt.full(y) - A)
        assert abs(err - math.sqrt(np.sum(s[k:] ** 2))) < 1e-14 * nrm
        assert err <= tol * nrm
    y = nt.round_tt(x, 1e-3, rmax=2)
    assert nt.ranks(y)[1] == 2


def test_round_error_bound_d4():
    """Oseledets' guarantee: ||X - round(X)|| <= tol ||X|| with delta = tol ||X|| / sqrt(d-1)."""
    x = random_tt([10, 4, 5, 6], [6, 8, 5], seed=11)
    nx = np.linalg.norm(nt.full(x))
    for tol in (0.3, 0.1, 0.01):
        y = nt.round_tt(x, tol)
        assert np.linalg.norm(nt.full(y) - nt.full(x)) <= tol * nx * (1 + 1e-12)


def _small_plane(inflow=False, ks=True):
    wl = plane_config1(nx=6, ny=5, G=3, ntheta=4, nphi=8, rmax=64, tol=0.0)
    if inflow:
        wl = wl.with_(inflow_temperature=(0.8, None, None, 0.6, None, None))
    if not ks:
        wl = wl.with_(rho_kappa_s=np.zeros_like(wl.rho_kappa_s))
    return wl


@pytest.mark.parametrize("inflow", [False, True])
def test_transport_sum_matches_dense_operator(inflow):
    """Brute force: full(TT transport sum) equals the dense upwind update of full(TT).
    The dense stepper's source stage is switched off (a = s = eps = 0)."""
    wl = _small_plane(inflow)
    coef = problem.build(wl)
    coef0 = problem.build(wl)
    coef0.acoef[:] = 0.0
    coef0.scoef[:] = 0.0
    coef0.eps[:] = 0.0
    x = random_tt([wl.nrow, wl.ntheta, wl.nphi], [3, 2], seed=13)
    S = dense.DenseSolver(wl, coef0)
    ref = S.step(nt.to_dense_rows(x))
    t = nt.transport_sum(x, coef)
    n = 2 * wl.ndim
    nb = 2 if inflow else 0
    assert nt.ranks(t)[1] == (n + 1) * 3 + nb and nt.ranks(t)[2] == (n + 1) * 2 + nb
    assert np.max(np.abs(nt.to_dense_rows(t) - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_source_sum_adds_one_rank_per_bond():
    wl = _small_plane()
    coef = problem.build(wl)
    x = random_tt([wl.nrow, wl.ntheta, wl.nphi], [3, 2], seed=14)
    s = nt.source_sum(x, coef)
    assert nt.ranks(s) == [1, 4, 3, 1]


@pytest.mark.parametrize("inflow", [False, True])
def test_exact_rank_tt_step_equals_dense_plane(inflow):
    """tol = 0 (no truncation): the TT step reproduces the dense step (transport + source)."""
    wl = _small_plane(inflow)
    coef = problem.build(wl)
    S = dense.DenseSolver(wl, coef)
    I = S.initial()
    x = nt.initial_tt(problem.initial_rows(wl, coef), coef)
    for _ in range(4):
        I = S.step(I)
        x = nt.step(x, coef, 0.0, 10 ** 6)
        D = nt.to_dense_rows(x)
        assert np.max(np.abs(D - I)) <= 1e-12 * np.max(np.abs(I))


def test_exact_rank_slab_config_equals_dense():
    """The 1-D slab workload (exact rank, 10 steps) matches the dense stepper to 1e-12."""
    wl = slab_config0()
    coef = problem.build(wl)
    S = dense.DenseSolver(wl, coef)
    I = S.initial()
    x = nt.initial_tt(problem.initial_rows(wl, coef), coef)
    for _ in range(wl.steps):
        I = S.step(I)
        x = nt.step(x, coef, wl.tol, wl.rmax)
    D = nt.to_dense_rows(x)
    assert nt.ranks(x)[1] <= wl.rmax
    assert np.max(np.abs(D - I)) <= 1e-12 * np.max(np.abs(I))
    E = nt.energy_density_rows(x, coef)
    assert np.max(np.abs(E - S.energy_density(I))) <= 1e-12 * np.max(np.abs(E))


def test_planck_equilibrium_stays_rank_one():
    wl = _small_plane()
    wl = wl.with_(temperature=np.full(wl.ncell, 0.7), inflow_temperature=(0.7,) * 4 + (None, None), tol=1e-10)
    coef = problem.build(wl)
    x = nt.initial_tt(problem.initial_rows(wl, coef), coef)
    F0 = nt.full(x)
    y = nt.step(x, coef, 1e-10, 32)
    assert nt.ranks(y) == [1, 1, 1, 1]
    assert np.max(np.abs(nt.full(y) - F0)) <= 1e-13 * np.max(np.abs(F0))


def test_compression_counts_parameters():
    """Eq. (compression): dense size over the parameter count of the cores."""
    n = [7 * 3, 4, 8]
    x = random_tt(n, [5, 3], seed=1)
    params = sum(c.size for c in x)
    assert nt.compression(7, 3, 4, 8, 5, 3) == pytest.approx(np.prod(n) / params, rel=1e-15)


# --- Gram-based rounding (the Gram method of Sec. 3.1) -------------------------------------

@pytest.mark.parametrize("tol", [1e-2, 1e-4, 3e-6])
def test_round_gram_equals_svd_rounding_on_resolved_spectra(tol):
    """Where every kept singular value is far above sqrt(eps)|X|, the Gram route is the SVD
    route: same ranks, same result to round-off."""
    n = [233, 5, 9]
    a = nt.add_many([nt.scale(random_tt(n, [3, 2], seed=20 + i), 10.0 ** -i) for i in range(4)])
    i1, i2 = {}, {}
    w = nt.round_tt(a, tol, 20, i1)
    g = nt.round_tt_gram(a, tol, 20, i2)
    assert nt.ranks(g) == nt.ranks(w)
    assert np.linalg.norm(nt.full(g) - nt.full(w)) <= 1e-12 * np.linalg.norm(nt.full(w))
    for b1, b2 in zip(i1["bonds"], i2["bonds"]):
        k = b1["rank"]
        assert np.allclose(b2["sigma"][:k], b1["sigma"][:k], rtol=1e-10, atol=0)


def test_round_gram_known_spectrum_and_exact_rank():
    """A matrix with a prescribed spectrum (d = 2): Gram rounding recovers the singular values
    to 1e-10 relative while they stay above 1e-4 of the largest; at a tolerance above its
    sqrt(eps) noise floor (1e-6) it keeps the exact rank of a rank-6 tensor and reconstructs it."""
    rng = np.random.default_rng(5)
    m, k = 300, 6
    U, _ = np.linalg.qr(rng.standard_normal((m, k)))
    V, _ = np.linalg.qr(rng.standard_normal((40, k)))
    s = 10.0 ** -np.arange(k) * 0.5
    A = (U * s) @ V.T
    tt = [A.reshape(1, m, 40), np.eye(40).reshape(40, 40, 1)]
    info = {}
    g = nt.round_tt_gram(tt, 1e-6, 40, info)
    assert nt.ranks(g) == [1, k, 1]
    assert np.allclose(info["bonds"][0]["sigma"][:4], s[:4], rtol=1e-10, atol=0)
    assert np.linalg.norm(nt.full(g).reshape(m, 40) - A) <= 1e-10 * np.linalg.norm(A)


def test_round_gram_loses_the_squared_condition_tail():
    """The paper's caution: forming A^T A squares the condition number.  Singular values near
    1e-10 |A| are not resolved by the Gram route (they are by the SVD route)."""
    rng = np.random.default_rng(6)
    m = 200
    U, _ = np.linalg.qr(rng.standard_normal((m, 5)))
    V, _ = np.linalg.qr(rng.standard_normal((30, 5)))
    s = np.array([1.0, 1e-2, 1e-4, 1e-10, 1e-11])
    tt = [((U * s) @ V.T).reshape(1, m, 30), np.eye(30).reshape(30, 30, 1)]
    i1, i2 = {}, {}
    nt.round_tt(tt, 1e-14, 30, i1)
    nt.round_tt_gram(tt, 1e-14, 30, i2)
    sv, sg = i1["bonds"][0]["sigma"], i2["bonds"][0]["sigma"]
    assert np.allclose(sv[:5], s, rtol=1e-5, atol=0)
    assert np.allclose(sg[:3], s[:3], rtol=1e-8, atol=0)
    assert abs(sg[3] - s[3]) > 1e-2 * s[3]


def test_round_gram_zero_tensor():
    z = [np.zeros((1, 20, 3)), np.zeros((3, 4, 2)), np.zeros((2, 5, 1))]
    g = nt.round_tt_gram(z, 1e-6)
    assert nt.ranks(g) == [1, 1, 1, 1]
    assert not np.any(nt.full(g))


# --- randomized rounding (the randomized method of Sec. 3.1) --------------------------------

def test_round_randomized_equals_svd_rounding_when_the_sketch_spans_the_range():
    """With l >= rank of the first unfolding the sketch's range is the whole range: the
    randomized route is the SVD route (ranks and result)."""
    from paper_2602_00290_gb300.workloads import sketch_matrix
    n = [233, 5, 9]
    a = nt.add_many([nt.scale(random_tt(n, [3, 2], seed=20 + i), 10.0 ** -i) for i in range(4)])
    om = sketch_matrix(5 * 9, 14, seed=3)          # rank of the first unfolding <= 12
    for tol in (1e-2, 1e-4, 1e-8):
        i1, i2 = {}, {}
        w = nt.round_tt(a, tol, 20, i1)
        g = nt.round_tt_randomized(a, tol, 20, om, i2)
        assert nt.ranks(g) == nt.ranks(w)
        assert np.linalg.norm(nt.full(g) - nt.full(w)) <= 1e-11 * np.linalg.norm(nt.full(w))


def test_round_randomized_range_finder_error_bound():
    """Sketching with l = k + p columns: the discarded part of the sketch obeys the randomized
    range-finder bound E|X - Q Q^T X| <= (1 + sqrt(k/(p-1))) (sum_{j>k} s_j^2)^(1/2) (Halko,
    Martinsson, Tropp); a seeded draw stays within 10x that, and the leading singular values
    are recovered when the spectrum decays fast."""
    from paper_2602_00290_gb300.workloads import sketch_matrix
    rng = np.random.default_rng(9)
    m, ncol, k, p = 400, 60, 6, 6
    U, _ = np.linalg.qr(rng.standard_normal((m, ncol)))
    V, _ = np.linalg.qr(rng.standard_normal((ncol, ncol)))
    s = 10.0 ** (-0.5 * np.arange(ncol))
    A = (U * s) @ V.T
    tt = [A.reshape(1, m, ncol), np.eye(ncol).reshape(ncol, ncol, 1)]
    om = sketch_matrix(ncol, k + p, seed=5)
    info = {}
    g = nt.round_tt_randomized(tt, 0.0, k, om, info)
    err = np.linalg.norm(nt.full(g).reshape(m, ncol) - A)
    bound = (1 + math.sqrt(k / (p - 1))) * math.sqrt(np.sum(s[k:] ** 2))
    assert err <= 10 * bound
    assert np.allclose(info["bonds"][0]["sigma"][:3], s[:3], rtol=1e-3)
