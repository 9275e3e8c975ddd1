"""The seeded input generators (no GPU): the recipes stated for the
synthetic workloads hold -- normalisations (on the grid, or in the continuum
for the paper's analytic initial data), the phase-only perturbation of the
seeded Gaussian, determinism per seed, parameter ranges of the ensemble, and
the masses of the adjoint target."""
import math

import numpy as np
import pytest

from paper_2603_25282_gb300 import inputs


def _grid_mass(psi, n, L):
    _, h = inputs.coords(n, L)
    return float(np.prod(h)) * float(np.sum(np.abs(psi) ** 2))


@pytest.mark.parametrize("n,L", [((64, 48), (8.0, 6.0)), ((16, 32, 24), (4.0, 5.0, 6.0))])
def test_gaussian_random_phase_recipe(n, L):
    a = inputs.gaussian_random_phase(n, L, seed=3, amp=0.5)
    assert a.shape == (5,) + n[::-1] and a.dtype == np.complex128
    assert abs(_grid_mass(a, n, L) - 1.0) < 1e-13
    # the perturbation is a phase: every component has the Gaussian's modulus
    X, _ = inputs.coords(n, L)
    G = np.exp(-0.5 * sum(x * x for x in X))
    G = G / math.sqrt(5 * _grid_mass(G[None], n, L))
    for comp in range(5):
        assert np.abs(np.abs(a[comp]) - G).max() < 1e-14
    # the components carry different phases, the same seed the same field
    assert np.abs(np.angle(a[0]) - np.angle(a[1])).max() > 1e-3
    assert np.array_equal(a, inputs.gaussian_random_phase(n, L, seed=3, amp=0.5))
    assert not np.array_equal(a, inputs.gaussian_random_phase(n, L, seed=4, amp=0.5))
    b = inputs.gaussian_random_phase(n, L, seed=3, amp=0.0)
    assert np.abs(b.imag).max() == 0.0 and b.real.min() > 0.0


def test_paper_initial_data_have_unit_mass_in_the_continuum():
    # ini1 (Examples 1, 2): psi_{+-2} = psi_{+-1} = phi, psi_0 = 2 phi,
    # phi = exp(-|x|^2/2)/(sqrt(8) pi^(d/4)): (1+1+4+1+1)/8 = 1
    for n, L in [((128, 128), 12.0), ((48, 48, 48), 12.0)]:
        psi = inputs.ini_example1(n, L)
        assert abs(_grid_mass(psi, n, L) - 1.0) < 1e-12
        assert np.allclose(psi[2], 2 * psi[0]) and np.array_equal(psi[1], psi[0])
    # Example 3: psi_0 = 6 sqrt(7) phi, phi = exp(-|x|^2/8)/(32 sqrt(pi)):
    # (4 + 252) * (4 pi)/(1024 pi) = 1
    psi = inputs.ini_example3((192, 192), 24.0)
    assert abs(_grid_mass(psi, (192, 192), 24.0) - 1.0) < 1e-12


def test_vortex_state_is_normalised_in_the_weighted_components():
    psi = inputs.vortex_state((64, 64), 8.0, weights=(0, 1, 0, 0, 1))
    assert abs(_grid_mass(psi, (64, 64), 8.0) - 1.0) < 1e-13
    assert np.abs(psi[0]).max() == 0.0 and np.abs(psi[2]).max() == 0.0
    assert np.allclose(psi[1], psi[4])


def test_ensemble_members_ranges_and_determinism():
    m = inputs.ensemble_members(256, seed=4)
    assert m == inputs.ensemble_members(256, seed=4)
    assert {r["n"] for r in m} <= {64, 96, 128, 192, 256}
    assert len({r["n"] for r in m}) == 5
    for r in m:
        assert 0.0 <= r["omega"] <= 0.9 and 0.0 <= r["gamma"] <= 2.0
        assert 50.0 <= r["c0"] <= 1000.0 and -5.0 <= r["c1"] <= 5.0 and 0.0 <= r["c2"] <= 10.0
    assert len({r["seed"] for r in m}) == 256


def test_density_target_masses():
    n, L = (64, 64), 8.0
    centres, weights = inputs.density_target(n, L, seed=9)
    assert centres.shape == (5, 2) and np.abs(centres).max() <= 0.5
    X, h = inputs.coords(n, L)
    cell = float(np.prod(h))
    for comp in range(5):
        r2 = sum((x - c) ** 2 for x, c in zip(X, centres[comp]))
        assert abs(cell * weights[comp] * np.sum(np.exp(-r2)) - 0.2) < 1e-14
