"""Pins of the internal-rank analysis (Sec. 5.2): closed forms for separable and known-rank merged
cores, the delta rule on a prescribed spectrum, and the relative compression ratios counted by
hand."""
import numpy as np

from oracle import naive_tt as nt


def test_separable_cores():
    """Z[g + G cell][q] = a_g b_{cell,q}: frequency separates (r1 = 1) while the space-leading
    rank is rank(b) = min(N_X, r); with b = c d^T as well both internal ranks are 1."""
    rng = np.random.default_rng(1)
    G, nX, r = 7, 30, 4
    a = rng.random(G) + 0.5
    b = rng.standard_normal((nX, r))
    Z = (b[:, None, :] * a[None, :, None]).reshape(nX * G, r)
    r1, r1x, s_nu, _ = nt.internal_ranks(Z, G, 1e-12)
    assert (r1, r1x) == (1, r)
    assert s_nu[1] <= 1e-13 * s_nu[0]
    b1 = np.outer(rng.standard_normal(nX), rng.standard_normal(r))
    Z1 = (b1[:, None, :] * a[None, :, None]).reshape(nX * G, r)
    r1, r1x, s_nu, s_x = nt.internal_ranks(Z1, G, 1e-12)
    assert (r1, r1x) == (1, 1)
    assert s_x[1] <= 1e-13 * s_x[0]


def test_known_internal_ranks():
    """Z = sum_{i<k} a_i(g) b_i(cell, q) has r1 = k; with b_i(cell, q) = c_i(cell) d_i(q) and
    cross terms the space-leading rank follows the rank of the [cell] x [g, q] unfolding."""
    rng = np.random.default_rng(2)
    G, nX, r, k = 9, 40, 5, 3
    A = rng.standard_normal((k, G))
    B = rng.standard_normal((k, nX, r))
    Z3 = np.einsum("ig,icq->cgq", A, B)
    Z = Z3.reshape(nX * G, r)
    r1, r1x, _, _ = nt.internal_ranks(Z, G, 1e-12)
    assert r1 == k
    assert r1x == min(nX, G * r, np.linalg.matrix_rank(Z3.reshape(nX, G * r)))


def test_delta_rule_on_prescribed_spectrum():
    S = 10.0 ** -np.arange(8)
    tot = np.sqrt(np.sum(S ** 2))
    for delta, kexp in ((2e-3, 3), (2e-5, 5), (1e-9, 8)):
        k = nt.delta_rank(S, delta)
        assert k == kexp
        assert np.sqrt(np.sum(S[k:] ** 2)) <= delta * tot < np.sqrt(np.sum(S[k - 1:] ** 2))
    assert nt.delta_rank(np.zeros(4), 1e-6) == 1


def test_relative_compression_counts():
    nX, nnu, nth, nph = 100, 10, 8, 16
    r1, r1x, r2, r3 = 3, 20, 12, 6
    c_nu, c_x = nt.relative_compression(nX, nnu, nth, nph, r1, r1x, r2, r3)
    ntt = 100 * 10 * 12 + 8 * 12 * 6 + 16 * 6
    assert np.isclose(c_nu, ntt / (10 * 3 + 100 * 3 * 12 + 8 * 12 * 6 + 16 * 6))
    assert np.isclose(c_x, ntt / (100 * 20 + 10 * 20 * 12 + 8 * 12 * 6 + 16 * 6))
