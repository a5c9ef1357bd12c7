"""Clover (Sheikholeslami-Wohlert) term of the Wilson-clover operator (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper computes with "the Clover discretization with even-odd preconditioning" (Sec. 4) and
gives neither the term's normalisation nor c_sw. The reading used here, by the oracle and the
CUDA path alike:

    D_sw = D_W + C,    C(x) = (c_sw / 2) sum_{mu < nu} sigma_{mu nu} (x) F_{mu nu}(x)

    sigma_{mu nu} = (i/2) [gamma_mu, gamma_nu]                       (Hermitian, 4x4)
    F_{mu nu}(x)  = (Q_{mu nu}(x) - Q_{mu nu}(x)^dag) / (8 i)       (Hermitian, 3x3)
    Q_{mu nu}(x)  = the four plaquettes of the (mu, nu) plane that touch x, each a closed
                    path from x, taken counter-clockwise (the mu step before the nu step):
        U_mu(x)     U_nu(x+mu)      U_mu(x+nu)^dag     U_nu(x)^dag
        U_nu(x)     U_mu(x+nu-mu)^dag U_nu(x-mu)^dag   U_mu(x-mu)
        U_mu(x-mu)^dag U_nu(x-mu-nu)^dag U_mu(x-mu-nu) U_nu(x-nu)
        U_nu(x-nu)^dag U_mu(x-nu)   U_nu(x-nu+mu)      U_mu(x)^dag

with D_W the Wilson operator of `dirac`. C is local and Hermitian, commutes with gamma_5 (so D_sw
stays gamma_5-Hermitian and C is block diagonal in the chiral basis), transforms covariantly
under gauge transformations, and vanishes on the free field (U = 1). D_sw + sigma I keeps the
hopping term of D_W and puts (4 + m + sigma) I + C(x) on the diagonal. The links carry no
boundary phase: the antiperiodic t condition belongs to the fermion field.

Arrays: the term is complex128[Lt, Lz, Ly, Lx, 4, 3, 4, 3] (row spin, row colour, column spin,
column colour), i.e. a 12x12 matrix per site with index 3 spin + colour.
"""

import numpy as np

from . import dirac


def _mm(a, b):
    return np.einsum("...ab,...bc->...ac", a, b)


def _dag(a):
    return np.conj(np.swapaxes(a, -1, -2))


def _fwd(f, mu):
    """f(x + mu_hat), periodic (links carry no boundary phase)."""
    return dirac.shift_forward(f, mu, 1, inner=2)


def _bwd(f, mu):
    """f(x - mu_hat), periodic."""
    return dirac.shift_backward(f, mu, 1, inner=2)


def leaves(u, mu, nu):
    """Q_{mu nu}(x): the sum of the four counter-clockwise plaquettes at x (module docstring)."""
    um, un = u[mu], u[nu]
    l1 = _mm(_mm(_mm(um, _fwd(un, mu)), _dag(_fwd(um, nu))), _dag(un))
    l2 = _mm(_mm(_mm(un, _dag(_bwd(_fwd(um, nu), mu))), _dag(_bwd(un, mu))), _bwd(um, mu))
    l3 = _mm(_mm(_mm(_dag(_bwd(um, mu)), _dag(_bwd(_bwd(un, mu), nu))), _bwd(_bwd(um, mu), nu)), _bwd(un, nu))
    l4 = _mm(_mm(_mm(_dag(_bwd(un, nu)), _bwd(um, nu)), _fwd(_bwd(un, nu), mu)), _dag(um))
    return l1 + l2 + l3 + l4


def field_strength(u, mu, nu):
    """F_{mu nu}(x) = (Q - Q^dag) / (8 i), Hermitian 3x3 per site."""
    q = leaves(u, mu, nu)
    return (q - _dag(q)) / 8j


def sigma_munu(mu, nu):
    """sigma_{mu nu} = (i/2) [gamma_mu, gamma_nu]."""
    g = dirac.GAMMA
    return 0.5j * (g[mu] @ g[nu] - g[nu] @ g[mu])


def clover_term(u, c_sw):
    """C(x) = (c_sw / 2) sum_{mu<nu} sigma_{mu nu} (x) F_{mu nu}(x): [Lt, Lz, Ly, Lx, 4, 3, 4, 3].

    u: gauge complex128[4, Lt, Lz, Ly, Lx, 3, 3]."""
    shp = u.shape[1:5]
    c = np.zeros(shp + (4, 3, 4, 3), dtype=np.complex128)
    for mu in range(4):
        for nu in range(mu + 1, 4):
            f = field_strength(u, mu, nu)
            c += 0.5 * c_sw * np.einsum("st,...ab->...satb", sigma_munu(mu, nu), f)
    return c


def apply_clover(cterm, psi):
    """(C psi)(x) for psi [..., Lt, Lz, Ly, Lx, 4, 3]."""
    return np.einsum("...satb,...tb->...sa", cterm, psi)


def apply_Dsw(u, psi, m, sigma, bc_t, cterm):
    """(D_sw + sigma I) psi = (D_W + sigma I) psi + C psi."""
    return dirac.apply_D(u, psi, m, sigma, bc_t) + apply_clover(cterm, psi)


def site_blocks(cterm):
    """The term as 12x12 blocks per canonical site: complex128[V, 12, 12]."""
    v = int(np.prod(cterm.shape[:4]))
    return cterm.reshape(v, 12, 12)
