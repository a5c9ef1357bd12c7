"""Shared helpers for the parity tests (no method arithmetic here: the oracle
does that; these only reshape arrays and compare)."""

import numpy as np

from oracle import dirac


def lattice_u(u, dims):
    return u.reshape((4,) + dirac.lattice_shape(dims) + (3, 3))


def oracle_D(u, psi, m, sigma, dims, bc_t=-1):
    """(D + sigma) psi with the oracle, canonical flat in/out [..., V, 4, 3]."""
    shp = dirac.lattice_shape(dims)
    lead = psi.shape[:-3]
    out = dirac.apply_D(lattice_u(u, dims), psi.reshape(lead + shp + (4, 3)), m, sigma, bc_t)
    return out.reshape(psi.shape)


def rel_resid(u, x, b, m, sigma, dims, bc_t=-1):
    """||b - (D + sigma) x|| / ||b|| computed by the oracle."""
    r = b - oracle_D(u, x, m, sigma, dims, bc_t)
    return float(np.linalg.norm(r.ravel()) / np.linalg.norm(b.ravel()))


def rel_err(a, b):
    """max |a - b| / max |b| (elementwise, normalised by the largest reference entry)."""
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def sample_err(gpu, ref):
    """Level-sample error |c_gpu - c_ref| / max(|T_ref|, mean_s |c_ref|): traces whose mean is
    near zero are compared on the scale of the samples."""
    gpu = np.asarray(gpu)
    ref = np.asarray(ref)
    scale = max(abs(ref.mean()), np.abs(ref).mean(), 1e-300)
    return float(np.abs(gpu - ref).max() / scale)
