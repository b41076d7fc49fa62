"""Angular quadrature sets for the oracle (test infrastructure; see oracle/__init__).

Sec. 4 preamble: latitude/longitude discretization with N_phi = 2 N_theta and
nodes uniformly spaced in cos(theta) and in phi.  Reading: midpoint rule in both,
mu_l = -1 + (2l+1)/N_theta, phi_p = (2p+1) pi / N_phi, Delta Omega = (2/N_theta)(2 pi/N_phi),
summing to 4 pi.  The planar-slab case uses Gauss-Legendre nodes in mu with
Delta Omega_j = 2 pi w_j (sum w = 2), i.e. J = (1/2) sum_j w_j I_j.

Directions: polar axis z, n = (sin th cos ph, sin th sin ph, cos th); in the slab the
transport axis is x with direction cosine n_x = mu.
"""
import numpy as np


def gauss_legendre_mu(n):
    """Nodes mu_j, weights w_j (sum 2) of n-point Gauss-Legendre (numpy's leggauss)."""
    mu, w = np.polynomial.legendre.leggauss(n)
    return mu, w


def latlong_midpoint(ntheta, nphi):
    """Return (mu[ntheta], phi[nphi], domega[ntheta, nphi])."""
    mu = -1.0 + (2.0 * np.arange(ntheta) + 1.0) / ntheta
    phi = (2.0 * np.arange(nphi) + 1.0) * np.pi / nphi
    dom = np.full((ntheta, nphi), (2.0 / ntheta) * (2.0 * np.pi / nphi))
    return mu, phi, dom


def directions(wl):
    """Direction cosines and solid-angle weights flattened over angles a = l*N_phi + p.

    Returns dict with nx, ny, nz, domega (each length N_theta*N_phi) plus the separable
    factors used by the TT form of the operator (Appendix A, 'Value of n'):
    theta-factor and phi-factor per transport term."""
    if wl.quad == "gauss_legendre_mu":
        mu, w = gauss_legendre_mu(wl.ntheta)
        return dict(nx=mu.copy(), ny=np.zeros_like(mu), nz=np.zeros_like(mu),
                    domega=2.0 * np.pi * w, mu=mu, w=w)
    if wl.quad == "latlong_midpoint":
        mu, phi, dom = latlong_midpoint(wl.ntheta, wl.nphi)
        st = np.sqrt(1.0 - mu * mu)
        nx = np.outer(st, np.cos(phi)).reshape(-1)
        ny = np.outer(st, np.sin(phi)).reshape(-1)
        nz = np.outer(mu, np.ones_like(phi)).reshape(-1)
        return dict(nx=nx, ny=ny, nz=nz, domega=dom.reshape(-1), mu=mu, phi=phi, sintheta=st)
    raise ValueError(wl.quad)
