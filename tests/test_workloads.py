"""Seeded workload generators: shapes, determinism and the stated value ranges (no GPU)."""
import numpy as np

from paper_2602_00290_gb300.workloads import cube_config, gaussian_diffusion_config, plane_config1, slab_config0


def test_generators_are_seeded():
    for make in (plane_config1, cube_config, gaussian_diffusion_config, slab_config0):
        a, b = make(), make()
        assert np.array_equal(a.rho_kappa_a, b.rho_kappa_a)
        assert np.array_equal(a.rho_kappa_s, b.rho_kappa_s)
        assert np.array_equal(a.temperature, b.temperature)


def test_cube_config_shapes_and_stable_step():
    wl = cube_config(nx=6, ny=5, nz=4, G=3)
    assert wl.ndim == 3 and wl.nrow == 6 * 5 * 4 * 3
    assert wl.rho_kappa_a.shape == (wl.nrow,) and wl.temperature.shape == (wl.ncell,)
    lam = [wl.c * wl.dt / h for h in wl.spacing]
    assert sum(lam) <= 1.0  # forward-Euler transport: sum of the axis Courant numbers within 1
    assert np.all(wl.rho_kappa_a > 0) and np.allclose(wl.rho_kappa_s, 0.1 * wl.rho_kappa_a)


def test_gaussian_diffusion_config_matches_its_recipe():
    wl = gaussian_diffusion_config(nx=128, G=8, kappa_max=2000.0)
    ks = wl.rho_kappa_s.reshape(wl.nx, wl.ngroup)
    assert np.all(ks == ks[0])                       # the same opacities in every cell
    assert np.all((ks[0] >= 1000.0) & (ks[0] <= 2000.0))
    assert not np.any(wl.rho_kappa_a)                # pure scattering
    assert wl.flux == "central" and wl.extent[0] == 10.0
    assert wl.dt == wl.extent[0] / wl.nx             # CFL 1
