"""Pins of the oracle's clover term (oracle/clover.py) against what the definition fixes: the
closed form on a constant abelian field, the free field, Hermiticity and chirality, gauge
covariance, gamma_5-hermiticity of D_sw, c_sw = 0, and BiCGStab against dense LU."""

import numpy as np
import pytest

import inputs
from oracle import clover, dirac, solve


def _lat(u, dims):
    return u.reshape((4,) + dirac.lattice_shape(dims) + (3, 3))


@pytest.mark.parametrize("plane", [(0, 1), (1, 3), (2, 3)])
def test_constant_abelian_field_closed_form(plane):
    """Every plaquette of the (mu, nu) plane is e^{iB} and the others are 1, so the four leaves
    add to 4 e^{iB}, F_{mu nu} = (4 e^{iB} - 4 e^{-iB}) / (8i) = sin B, the other F vanish, and
    C(x) = (c_sw / 2) sin B (i gamma_mu gamma_nu) (x) 1_3 at every site (sigma_{mu nu} =
    i gamma_mu gamma_nu for mu != nu). A wrong leaf orientation, normalisation or sign fails."""
    mu, nu = plane
    dims = (4, 6, 4, 4)
    u, b = inputs.abelian_field(dims, n=1, mu=mu, nu=nu)
    c_sw = 1.37
    cterm = clover.clover_term(_lat(u, dims), c_sw)
    g = dirac.GAMMA
    expect = 0.5 * c_sw * np.sin(b) * np.kron(1j * g[mu] @ g[nu], np.eye(3))
    blocks = clover.site_blocks(cterm)
    assert np.abs(blocks - expect[None]).max() < 1e-13
    # the field strength itself
    f = clover.field_strength(_lat(u, dims), mu, nu)
    assert np.abs(f - np.sin(b) * np.eye(3)).max() < 1e-13
    other = (0, 2) if plane != (0, 2) else (1, 2)
    assert np.abs(clover.field_strength(_lat(u, dims), *other)).max() < 1e-13


def test_free_field_has_no_clover_term():
    dims = (4, 4, 2, 4)
    cterm = clover.clover_term(_lat(inputs.unit_gauge(dims), dims), 1.9)
    assert np.abs(cterm).max() == 0.0


def test_hermitian_and_chiral_blocks():
    """C(x) is Hermitian and commutes with gamma_5: no entries between the chiralities."""
    dims = (4, 2, 4, 4)
    u = inputs.gauge_field(dims, "haar", seed=61)
    blocks = clover.site_blocks(clover.clover_term(_lat(u, dims), 1.0))
    assert np.abs(blocks - np.conj(np.swapaxes(blocks, 1, 2))).max() < 1e-13
    g5 = np.kron(dirac.GAMMA5, np.eye(3))
    assert np.abs(blocks @ g5 - g5 @ blocks).max() < 1e-13
    assert np.abs(blocks[:, :6, 6:]).max() < 1e-13 and np.abs(blocks[:, 6:, :6]).max() < 1e-13
    assert np.abs(blocks).max() > 0.1  # a Haar field carries a large field strength


def test_gauge_covariance():
    """C[U^g](x) = g(x) C[U](x) g(x)^dag (colour indices), U^g_mu(x) = g(x) U_mu(x) g(x+mu)^dag."""
    dims = (2, 4, 2, 4)
    u = inputs.gauge_field(dims, "haar", seed=62)
    g = inputs.random_gauge_rotation(dims, 63)
    ug = inputs.gauge_transform(u, g, dims)
    c0 = clover.clover_term(_lat(u, dims), 0.8).reshape(-1, 4, 3, 4, 3)
    c1 = clover.clover_term(_lat(ug, dims), 0.8).reshape(-1, 4, 3, 4, 3)
    rot = np.einsum("xab,xsbtc,xdc->xsatd", g, c0, np.conj(g))
    assert np.abs(c1 - rot).max() < 1e-12


def test_dsw_gamma5_hermitian_and_reduces_to_wilson():
    dims = (2, 2, 2, 4)
    u = inputs.gauge_field(dims, "haar", seed=64)
    cterm = clover.clover_term(_lat(u, dims), 1.2)
    d = solve.dense_operator(u, -0.3, 0.1, dims, -1, cterm)
    g5 = solve.dense_gamma5(dims)
    assert np.abs(g5 @ d @ g5 - np.conj(d.T)).max() < 1e-12
    dw = solve.dense_operator(u, -0.3, 0.1, dims, -1)
    c0 = clover.clover_term(_lat(u, dims), 0.0)
    assert np.abs(solve.dense_operator(u, -0.3, 0.1, dims, -1, c0) - dw).max() == 0.0
    assert np.abs(d - dw).max() > 0.05
    # the matrix-free operator agrees with the dense one
    psi = inputs.random_spinor(dims, 65)
    shp = dirac.lattice_shape(dims)
    mf = clover.apply_Dsw(_lat(u, dims), psi.reshape(shp + (4, 3)), -0.3, 0.1, -1, cterm)
    assert np.abs(mf.ravel() - d @ psi.ravel()).max() < 1e-12


def test_bicgstab_with_clover_against_dense():
    dims = (2, 2, 2, 4)
    u = inputs.gauge_field(dims, "smooth", seed=66, eps=0.4)
    cterm = clover.clover_term(_lat(u, dims), 1.0)
    b = inputs.random_spinor(dims, 67)
    res = solve.shifted_solve(u, b, -0.25, 0.05, dims, -1, tol=1e-12, cterm=cterm)
    assert res.converged
    x = np.linalg.solve(solve.dense_operator(u, -0.25, 0.05, dims, -1, cterm), b.ravel())
    assert np.abs(res.x.ravel() - x).max() < 1e-9 * np.abs(x).max()
