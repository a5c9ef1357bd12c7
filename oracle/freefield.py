"""Free-field (U = 1) closed forms in momentum space (oracle pins).

Not in the paper: derived here from the operator definition in `dirac`. On a
plane wave psi(x) = exp(i k.x) u the Wilson operator acts as the 4x4 matrix
    D(k) = M(k) + i sum_mu gamma_mu sin k_mu,  M(k) = m + sigma + sum_mu (1 - cos k_mu),
with k_mu = 2 pi n / L_mu (periodic) and k_t = (2n + 1) pi / L_t (antiperiodic).
Hence D(k)^-1 = (M - i gamma.sin k) / (M^2 + sum_mu sin^2 k_mu), and since
Pi_p multiplies a plane wave by exp(i k_z p),
    Tr(Gamma Pi_p (D + sigma)^-1) = 3 sum_k exp(i k_z p) tr[Gamma D(k)^-1],
the factor 3 being the colour trace. The spectrum of D + sigma is
M(k) +- i |sin k|, each with multiplicity 2 (spin) x 3 (colour).
"""

import itertools

import numpy as np

from .dirac import GAMMA


def momenta(dims, bc_t=-1):
    ks = []
    for mu, L in enumerate(dims):
        n = np.arange(L)
        if mu == 3 and bc_t == -1:
            ks.append((2 * n + 1) * np.pi / L)
        else:
            ks.append(2 * n * np.pi / L)
    return ks


def free_trace(gamma, p, m, sigma, dims, bc_t=-1):
    """Tr(Gamma Pi_p (D + sigma)^-1) for the free Wilson operator."""
    ks = momenta(dims, bc_t)
    total = 0j
    for k in itertools.product(*ks):
        k = np.array(k)
        s = np.sin(k)
        mk = m + sigma + np.sum(1.0 - np.cos(k))
        num = mk * np.eye(4) - 1j * sum(GAMMA[mu] * s[mu] for mu in range(4))
        inv = num / (mk * mk + np.sum(s * s))
        total += np.exp(1j * k[2] * p) * np.trace(gamma @ inv)
    return 3.0 * total


def free_spectrum(m, sigma, dims, bc_t=-1):
    """Eigenvalues of the free D + sigma I (each listed with its multiplicity 6)."""
    ks = momenta(dims, bc_t)
    ev = []
    for k in itertools.product(*ks):
        k = np.array(k)
        mk = m + sigma + np.sum(1.0 - np.cos(k))
        sn = np.sqrt(np.sum(np.sin(k) ** 2))
        ev.extend([mk + 1j * sn] * 6 + [mk - 1j * sn] * 6)
    return np.array(ev)
