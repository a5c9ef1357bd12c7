"""Wilson-Dirac operator, Gamma insertions and the displacement Omega_p (oracle).

Conventions (the paper fixes the operator only as "the lattice Dirac operator
D" (Sec. 1) and runs clover in Chroma (Sec. 4); the readings used here are):
  * Wilson, r = 1:
      (D psi)(x) = (4 + m) psi(x)
                   - 1/2 sum_mu [ (1 - gamma_mu) U_mu(x) psi(x + mu)
                                + (1 + gamma_mu) U_mu(x - mu)^dag psi(x - mu) ]
  * DeGrand-Rossi chiral gamma basis (Chroma's), gamma_5 = g1 g2 g3 g4
    = diag(1, 1, -1, -1); mu = 0,1,2,3 is x,y,z,t (gamma_1..gamma_4).
  * Boundary: periodic in x, y, z; the t-hop that wraps picks up a factor
    bc_t (-1 antiperiodic, +1 periodic). The links never carry the phase.
  * Omega_p = W Pi_p (Sec. 1): (Pi_p psi)(x) = psi(x + p z_hat), and
    W(x) = U_z(x) U_z(x + z_hat) ... U_z(x + (p-1) z_hat), the Wilson line of
    z-links from x to x + p z_hat (periodic in z).

Fields are numpy arrays on the 4-d lattice, leading batch axes allowed:
  spinor  complex128[..., Lt, Lz, Ly, Lx, 4, 3]
  gauge   complex128[4, Lt, Lz, Ly, Lx, 3, 3]
which is the canonical flat layout (site = x + Lx(y + Ly(z + Lz t))) reshaped.
"""

import numpy as np

# ---- gamma matrices (DeGrand-Rossi basis), written out element by element ----
_i = 1j
GAMMA = np.zeros((4, 4, 4), dtype=np.complex128)
# gamma_1
GAMMA[0][0, 3] = _i
GAMMA[0][1, 2] = _i
GAMMA[0][2, 1] = -_i
GAMMA[0][3, 0] = -_i
# gamma_2
GAMMA[1][0, 3] = -1
GAMMA[1][1, 2] = 1
GAMMA[1][2, 1] = 1
GAMMA[1][3, 0] = -1
# gamma_3
GAMMA[2][0, 2] = _i
GAMMA[2][1, 3] = -_i
GAMMA[2][2, 0] = -_i
GAMMA[2][3, 1] = _i
# gamma_4
GAMMA[3][0, 2] = 1
GAMMA[3][1, 3] = 1
GAMMA[3][2, 0] = 1
GAMMA[3][3, 1] = 1

GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
IDENT4 = np.eye(4, dtype=np.complex128)


def gamma_product(names):
    """Product of gamma matrices named left to right, e.g. ("g5", "g3") -> gamma_5 gamma_3.

    Names: "g1".."g4", "g5", "I".
    """
    table = {"g1": GAMMA[0], "g2": GAMMA[1], "g3": GAMMA[2], "g4": GAMMA[3],
             "g5": GAMMA5, "I": IDENT4}
    out = IDENT4.copy()
    for n in names:
        out = out @ table[n]
    return out


def lattice_shape(dims):
    lx, ly, lz, lt = (int(d) for d in dims)
    return (lt, lz, ly, lx)


def to_lattice(flat, dims, inner):
    """Canonical flat field [..., V, *inner] -> [..., Lt, Lz, Ly, Lx, *inner]."""
    lead = flat.shape[: flat.ndim - 1 - len(inner)]
    return flat.reshape(lead + lattice_shape(dims) + tuple(inner))


def to_flat(field, inner):
    """[..., Lt, Lz, Ly, Lx, *inner] -> canonical flat [..., V, *inner]."""
    lead = field.shape[: field.ndim - 4 - len(inner)]
    v = int(np.prod(field.shape[len(lead): len(lead) + 4]))
    return field.reshape(lead + (v,) + tuple(inner))


def _axis(f, mu, inner):
    """Array axis of direction mu (0=x..3=t) for a field with `inner` trailing axes."""
    return f.ndim - inner - 1 - mu


def shift_forward(f, mu, bc_t, inner=2):
    """g(x) = f(x + mu_hat), with the t wrap multiplied by bc_t."""
    ax = _axis(f, mu, inner)
    g = np.roll(f, -1, axis=ax)
    if mu == 3 and bc_t != 1:
        idx = [slice(None)] * g.ndim
        idx[ax] = g.shape[ax] - 1
        g[tuple(idx)] *= bc_t
    return g


def shift_backward(f, mu, bc_t, inner=2):
    """g(x) = f(x - mu_hat), with the t wrap multiplied by bc_t."""
    ax = _axis(f, mu, inner)
    g = np.roll(f, 1, axis=ax)
    if mu == 3 and bc_t != 1:
        idx = [slice(None)] * g.ndim
        idx[ax] = 0
        g[tuple(idx)] *= bc_t
    return g


def color_mul(u, psi):
    """(U psi)(x) per site: u[..., a, b] psi[..., s, b] -> [..., s, a]."""
    return np.einsum("...ab,...sb->...sa", u, psi)


def color_mul_dag(u, psi):
    """(U^dag psi)(x) per site."""
    return np.einsum("...ba,...sb->...sa", np.conj(u), psi)


def spin_mul(g, psi):
    """(Gamma psi)(x): g[s, t] psi[..., t, c] -> [..., s, c]."""
    return np.einsum("st,...tc->...sc", g, psi)


def apply_D(u, psi, m, sigma=0.0, bc_t=-1):
    """(D + sigma I) psi for the Wilson operator defined in the module docstring.

    u: gauge complex128[4, Lt, Lz, Ly, Lx, 3, 3]; psi: [..., Lt, Lz, Ly, Lx, 4, 3].
    The shifted operator D + sigma I of Eq. (shifted_linear_systems).
    """
    out = (4.0 + m + sigma) * psi
    for mu in range(4):
        # forward hop: (1 - gamma_mu) U_mu(x) psi(x + mu)
        fwd = color_mul(u[mu], shift_forward(psi, mu, bc_t))
        out = out - 0.5 * spin_mul(IDENT4 - GAMMA[mu], fwd)
        # backward hop: (1 + gamma_mu) U_mu(x - mu)^dag psi(x - mu)
        bwd = shift_backward(color_mul_dag(u[mu], psi), mu, bc_t)
        out = out - 0.5 * spin_mul(IDENT4 + GAMMA[mu], bwd)
    return out


def apply_Ddag(u, psi, m, sigma=0.0, bc_t=-1):
    """(D + sigma I)^dag psi, written from the adjoint of each term of apply_D.

    The adjoint of  -1/2 (1 - g_mu) U_mu(x) delta_{x+mu, y}  is
    -1/2 (1 - g_mu) U_mu(y - mu)^dag delta_{y-mu, x} (gamma_mu is Hermitian),
    i.e. the backward hop carries (1 - g_mu) and the forward hop (1 + g_mu).
    """
    out = (4.0 + m + sigma) * psi
    for mu in range(4):
        fwd = color_mul(u[mu], shift_forward(psi, mu, bc_t))
        out = out - 0.5 * spin_mul(IDENT4 + GAMMA[mu], fwd)
        bwd = shift_backward(color_mul_dag(u[mu], psi), mu, bc_t)
        out = out - 0.5 * spin_mul(IDENT4 - GAMMA[mu], bwd)
    return out


def wilson_line(u, p):
    """W(x) = U_z(x) U_z(x+z) ... U_z(x+(p-1)z), complex128[Lt, Lz, Ly, Lx, 3, 3] (Sec. 1)."""
    uz = u[2]
    w = np.broadcast_to(np.eye(3, dtype=np.complex128), uz.shape).copy()
    link = uz
    for _ in range(p):
        w = np.einsum("...ab,...bc->...ac", w, link)
        link = shift_forward(link, 2, 1, inner=2)  # U_z(x + (q+1) z_hat), z periodic
    return w


def apply_Omega(u, psi, p):
    """(Omega_p psi)(x) = W(x) psi(x + p z_hat), Omega_p = W Pi_p (Sec. 1)."""
    pi_p = psi
    for _ in range(p):
        pi_p = shift_forward(pi_p, 2, 1, inner=2)
    return color_mul(wilson_line(u, p), pi_p)


def apply_GammaOmega(u, gamma, psi, p):
    """Gamma Omega_p psi."""
    return spin_mul(gamma, apply_Omega(u, psi, p))


def gamma5(psi):
    return spin_mul(GAMMA5, psi)
