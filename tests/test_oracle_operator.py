"""Pins of the oracle's operator layer against facts fixed by mathematics.

Each test is chosen so that a plausible slip in oracle/dirac.py or
oracle/solve.py (a dropped hop, a wrong projector sign, U in place of U^dag,
a reversed Wilson line, a wrong boundary phase) fails at least one of them.
"""

import numpy as np
import pytest

import inputs
from oracle import dirac, freefield, solve


def _lat(a, dims, inner):
    return a.reshape(dirac.lattice_shape(dims) + inner)


def test_gamma_algebra():
    g = dirac.GAMMA
    for a in range(4):
        assert np.allclose(g[a], g[a].conj().T)
        for b in range(4):
            ac = g[a] @ g[b] + g[b] @ g[a]
            assert np.allclose(ac, 2.0 * np.eye(4) * (a == b))
    # chiral basis: gamma_5 = g1 g2 g3 g4 = diag(1, 1, -1, -1)
    assert np.allclose(dirac.GAMMA5, np.diag([1, 1, -1, -1]))
    for a in range(4):
        assert np.allclose(dirac.GAMMA5 @ g[a], -g[a] @ dirac.GAMMA5)


@pytest.mark.parametrize("bc_t", [-1, 1])
@pytest.mark.parametrize("dims", [(4, 4, 2, 4), (2, 2, 4, 6)])
def test_free_field_trace_closed_form(dims, bc_t):
    """Dense position-space inverse against the momentum-space closed form."""
    u = inputs.unit_gauge(dims)
    m, sigma = -0.4, 0.1
    inv = solve.dense_inverse(u, m, sigma, dims, bc_t)
    gammas = [dirac.IDENT4, dirac.GAMMA[2], dirac.gamma_product(["g5", "g3"]),
              dirac.GAMMA[3], dirac.gamma_product(["g1", "g2"]), dirac.GAMMA5]
    for g in gammas:
        for p in (0, 1, 2, 3):
            go = solve.dense_GammaOmega(u, g, p, dims)
            tr = np.trace(go @ inv)
            ref = freefield.free_trace(g, p, m, sigma, dims, bc_t)
            assert abs(tr - ref) <= 1e-10 * max(1.0, abs(ref)), (p, tr, ref)


def test_free_field_value_4444():
    """Tr(gamma_3 Pi_1 D^-1) at 4^4, m=-0.4, sigma=0.1, antiperiodic t: the sign of the
    displacement matters (the value flips sign for Pi_{-1})."""
    dims = (4, 4, 4, 4)
    u = inputs.unit_gauge(dims)
    inv = solve.dense_inverse(u, -0.4, 0.1, dims, -1)
    tr = np.trace(solve.dense_GammaOmega(u, dirac.GAMMA[2], 1, dims) @ inv)
    ref = freefield.free_trace(dirac.GAMMA[2], 1, -0.4, 0.1, dims, -1)
    assert abs(tr - ref) < 1e-10 * abs(ref)
    assert abs(ref.real - 126.1282269) < 1e-6
    back = freefield.free_trace(dirac.GAMMA[2], -1, -0.4, 0.1, dims, -1)
    assert abs(back + ref) < 1e-9 * abs(ref)


def test_free_field_spectrum():
    dims = (2, 2, 2, 4)
    u = inputs.unit_gauge(dims)
    ev = np.linalg.eigvals(solve.dense_operator(u, -0.3, 0.2, dims, -1))
    ref = freefield.free_spectrum(-0.3, 0.2, dims, -1)
    key = lambda z: (np.round(z.real, 8), np.round(z.imag, 8))
    a = sorted(ev, key=key)
    b = sorted(ref, key=key)
    assert np.allclose(a, b, atol=1e-9)


def test_apply_matches_dense_assembly():
    """apply_D (rolls) and dense_operator (block assembly) are two renderings of D."""
    dims = (4, 2, 4, 2)
    u = inputs.gauge_field(dims, "haar", seed=11)
    psi = inputs.random_spinor(dims, 12)
    for bc_t in (-1, 1):
        d = solve.dense_operator(u, -0.2, 0.05, dims, bc_t)
        a = dirac.apply_D(u.reshape((4,) + dirac.lattice_shape(dims) + (3, 3)),
                          _lat(psi, dims, (4, 3)), -0.2, 0.05, bc_t).ravel()
        assert np.abs(a - d @ psi.ravel()).max() < 1e-13


def test_gamma5_hermiticity():
    """gamma_5 D gamma_5 = D^dag on random SU(3) links (Sec. 3.1 relies on it)."""
    dims = (4, 4, 2, 2)
    u = inputs.gauge_field(dims, "haar", seed=21)
    d = solve.dense_operator(u, -0.4, 0.3, dims, -1)
    g5 = solve.dense_gamma5(dims)
    assert np.abs(g5 @ d @ g5 - d.conj().T).max() < 1e-13
    # apply_Ddag is the adjoint as an operator
    ul = u.reshape((4,) + dirac.lattice_shape(dims) + (3, 3))
    a = inputs.random_spinor(dims, 1)
    b = inputs.random_spinor(dims, 2)
    lhs = np.vdot(a.ravel(), dirac.apply_D(ul, _lat(b, dims, (4, 3)), -0.4, 0.3, -1).ravel())
    rhs = np.vdot(dirac.apply_Ddag(ul, _lat(a, dims, (4, 3)), -0.4, 0.3, -1).ravel(), b.ravel())
    assert abs(lhs - rhs) < 1e-11


def test_gauge_covariance():
    """D[U^g] (g psi) = g (D[U] psi), U^g_mu(x) = g(x) U_mu(x) g(x+mu)^dag."""
    dims = (4, 2, 4, 4)
    u = inputs.gauge_field(dims, "haar", seed=31)
    g = inputs.random_gauge_rotation(dims, 32)
    ug = inputs.gauge_transform(u, g, dims)
    psi = inputs.random_spinor(dims, 33)
    shp = dirac.lattice_shape(dims)
    gpsi = np.einsum("xab,xsb->xsa", g, psi)
    lhs = dirac.apply_D(ug.reshape((4,) + shp + (3, 3)), gpsi.reshape(shp + (4, 3)), -0.3, 0.0, -1)
    rhs = dirac.apply_D(u.reshape((4,) + shp + (3, 3)), psi.reshape(shp + (4, 3)), -0.3, 0.0, -1)
    rhs = np.einsum("xab,xsb->xsa", g, rhs.reshape(-1, 4, 3))
    assert np.abs(lhs.reshape(-1, 4, 3) - rhs).max() < 1e-12


@pytest.mark.parametrize("p", [0, 1, 2, 3])
def test_gauge_invariant_trace(p):
    """Tr(Gamma Omega_p D^-1) is gauge invariant only with the Wilson line ordered as
    U_z(x) ... U_z(x+(p-1)z) (Sec. 1)."""
    dims = (2, 2, 4, 4)
    u = inputs.gauge_field(dims, "haar", seed=41)
    g = inputs.random_gauge_rotation(dims, 42)
    ug = inputs.gauge_transform(u, g, dims)
    gam = dirac.gamma_product(["g5", "g3"])
    t0 = np.trace(solve.dense_GammaOmega(u, gam, p, dims) @ solve.dense_inverse(u, -0.4, 0.2, dims))
    t1 = np.trace(solve.dense_GammaOmega(ug, gam, p, dims) @ solve.dense_inverse(ug, -0.4, 0.2, dims))
    assert abs(t0 - t1) < 1e-10 * max(1.0, abs(t0))
    # a wrongly ordered line (reversed product) is not invariant for p >= 2
    if p >= 2:
        shp = dirac.lattice_shape(dims)
        ul = u.reshape((4,) + shp + (3, 3))
        w = np.broadcast_to(np.eye(3), ul[2].shape).copy()
        link = ul[2]
        for _ in range(p):
            w = np.einsum("...ab,...bc->...ac", link, w)  # reversed order
            link = dirac.shift_forward(link, 2, 1)
        assert not np.allclose(w, dirac.wilson_line(ul, p))


def test_wilson_line_composition():
    """Omega_{p+q} = Omega_p Omega_q (Wilson lines compose along z)."""
    dims = (2, 2, 6, 2)
    u = inputs.gauge_field(dims, "smooth", seed=51, eps=0.7)
    shp = dirac.lattice_shape(dims)
    ul = u.reshape((4,) + shp + (3, 3))
    psi = inputs.random_spinor(dims, 52).reshape(shp + (4, 3))
    a = dirac.apply_Omega(ul, psi, 5)
    b = dirac.apply_Omega(ul, dirac.apply_Omega(ul, psi, 3), 2)
    assert np.abs(a - b).max() < 1e-12
    # Omega_Lz is the closed Polyakov-type loop: trace-class, not the identity
    c = dirac.apply_Omega(ul, psi, 6)
    assert not np.allclose(c, psi)


def test_bicgstab_against_dense():
    dims = (4, 4, 2, 2)
    u = inputs.gauge_field(dims, "haar", seed=61)
    z = inputs.random_spinor(dims, 62)
    for sigma in (0.0, 0.25):
        res = solve.shifted_solve(u, z, -0.4, sigma, dims, -1, tol=1e-12)
        assert res.converged and res.rel_resid < 1e-11
        ref = np.linalg.solve(solve.dense_operator(u, -0.4, sigma, dims, -1), z.ravel())
        assert np.abs(res.x.ravel() - ref).max() < 1e-9 * np.abs(ref).max()


def test_smoothed_and_haar_links_are_su3():
    for kind in ("haar", "smooth"):
        u = inputs.gauge_field((2, 2, 2, 2), kind, seed=71, eps=0.4).reshape(-1, 3, 3)
        uu = np.einsum("nab,ncb->nac", u, u.conj())
        assert np.abs(uu - np.eye(3)).max() < 1e-13
        assert np.abs(np.linalg.det(u) - 1.0).max() < 1e-13
