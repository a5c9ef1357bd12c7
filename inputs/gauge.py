"""Seeded gauge-field and spinor generators (inputs only, see package doc).

Recipes:
  * Haar-random SU(3): QR decomposition of a complex Gaussian matrix
    G = (A + iB)/sqrt(2), A,B ~ N(0,1), with the phases of R's diagonal moved
    into Q (Mezzadri, Notices AMS 54 (2007) 592) so Q is Haar on U(3), then the
    determinant phase removed: Q <- Q * exp(-i arg(det Q)/3), arg in (-pi, pi].
  * Smoothed SU(3): U = exp(i eps H) with H the traceless Hermitian part of a
    complex Gaussian matrix, H = (G + G^dag)/2 - tr(.)/3, exponentiated through
    the Hermitian eigendecomposition H = Q diag(l) Q^dag.
Draw order: links are generated mu-major, then site, from one PCG64 stream.
"""

import numpy as np


def lattice_volume(dims):
    dims = tuple(int(d) for d in dims)
    if len(dims) != 4:
        raise ValueError("dims must have 4 entries (Lx, Ly, Lz, Lt)")
    v = 1
    for d in dims:
        v *= d
    return v


def _complex_gaussian(rng, shape):
    a = rng.standard_normal(shape)
    b = rng.standard_normal(shape)
    return (a + 1j * b) / np.sqrt(2.0)


def haar_su3(rng, n):
    """n Haar-random SU(3) matrices, complex128[n,3,3]."""
    g = _complex_gaussian(rng, (n, 3, 3))
    q, r = np.linalg.qr(g)
    d = np.diagonal(r, axis1=1, axis2=2)
    ph = d / np.abs(d)
    q = q * ph[:, None, :]
    det = np.linalg.det(q)
    q = q * np.exp(-1j * np.angle(det) / 3.0)[:, None, None]
    return q


def smoothed_su3(rng, n, eps):
    """n matrices exp(i eps H), H traceless Hermitian from a complex Gaussian."""
    g = _complex_gaussian(rng, (n, 3, 3))
    h = 0.5 * (g + np.conj(np.swapaxes(g, 1, 2)))
    tr = np.trace(h, axis1=1, axis2=2).real / 3.0
    h = h - tr[:, None, None] * np.eye(3)[None]
    lam, q = np.linalg.eigh(h)
    ph = np.exp(1j * eps * lam)
    return np.einsum("nab,nb,ncb->nac", q, ph, np.conj(q))


def unit_gauge(dims):
    """Free field: every link is the identity."""
    v = lattice_volume(dims)
    u = np.zeros((4, v, 3, 3), dtype=np.complex128)
    u[:, :, 0, 0] = u[:, :, 1, 1] = u[:, :, 2, 2] = 1.0
    return u


def gauge_field(dims, kind="haar", seed=0, eps=0.3):
    """Gauge field complex128[4][V][3][3] in the canonical layout.

    kind: "haar" (Haar-random SU(3) links), "smooth" (exp(i eps H)) or "unit".
    """
    v = lattice_volume(dims)
    if kind == "unit":
        return unit_gauge(dims)
    rng = np.random.Generator(np.random.PCG64(seed))
    if kind == "haar":
        links = haar_su3(rng, 4 * v)
    elif kind == "smooth":
        links = smoothed_su3(rng, 4 * v, eps)
    else:
        raise ValueError("unknown gauge kind %r" % (kind,))
    return np.ascontiguousarray(links.reshape(4, v, 3, 3))


def abelian_field(dims, n=1, mu=0, nu=1):
    """A constant abelian field strength in the (mu, nu) plane, embedded as a phase times the
    3x3 identity: every plaquette U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag equals e^{iB},
    B = 2 pi n / (L_mu L_nu) (the flux through each periodic plane is quantised). Landau gauge:
    U_nu(x) = e^{i B x_mu}, U_mu(x) = 1 except on the last mu slice, U_mu = e^{-i B L_mu x_nu}
    there; the other links are 1. Returns (links complex128[4][V][3][3], B)."""
    lx, ly, lz, lt = dims
    L = (lx, ly, lz, lt)
    v = lattice_volume(dims)
    s = np.arange(v)
    c = np.stack([s % lx, (s // lx) % ly, (s // (lx * ly)) % lz, s // (lx * ly * lz)])
    b = 2.0 * np.pi * n / (L[mu] * L[nu])
    ph = np.ones((4, v), dtype=np.complex128)
    ph[nu] = np.exp(1j * b * c[mu])
    last = c[mu] == L[mu] - 1
    ph[mu] = np.where(last, np.exp(-1j * b * L[mu] * c[nu]), 1.0)
    links = ph[:, :, None, None] * np.eye(3, dtype=np.complex128)
    return np.ascontiguousarray(links), b


def random_gauge_rotation(dims, seed):
    """Haar-random g(x) in SU(3) per site, complex128[V][3][3]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return haar_su3(rng, lattice_volume(dims))


def gauge_transform(u, g, dims):
    """Gauge-transformed links U'_mu(x) = g(x) U_mu(x) g(x+mu)^dag (periodic wrap)."""
    lx, ly, lz, lt = dims
    shp = (lt, lz, ly, lx, 3, 3)
    g4 = g.reshape(shp)
    out = np.empty_like(u)
    for mu in range(4):
        axis = 3 - mu
        g_fwd = np.roll(g4, -1, axis=axis)
        u4 = u[mu].reshape(shp)
        out[mu] = np.einsum("...ab,...bc,...dc->...ad", g4, u4, np.conj(g_fwd)).reshape(-1, 3, 3)
    return out


def random_spinor(dims, seed, nvec=None):
    """Complex Gaussian spinor field(s), complex128[V][4][3] (or [nvec][V][4][3])."""
    rng = np.random.Generator(np.random.PCG64(seed))
    v = lattice_volume(dims)
    shape = (v, 4, 3) if nvec is None else (nvec, v, 4, 3)
    return _complex_gaussian(rng, shape)


def as_real_view(a):
    """Contiguous float64 view with a trailing (re, im) axis, as the C-ABI expects."""
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a.view(np.float64).reshape(a.shape + (2,))
