"""Clover-improved Wilson Dirac operator D of Sec. 2.2 (oracle; test infrastructure only).

(D psi)(x) = [(m0+4) I_12 - c_sw/32 sum_{mu,nu} (gamma_mu gamma_nu) (x) (Q_mu,nu(x) - Q_nu,mu(x))] psi(x)
             - 1/2 sum_mu ((I_4 - gamma_mu) (x) U_mu(x))        psi(x + mu)
             - 1/2 sum_mu ((I_4 + gamma_mu) (x) U_mu(x - mu)^H) psi(x - mu)
with lattice spacing a = 1 (Sec. 2.3), the chiral gamma basis printed in
Sec. 2.2 and the four-leaf clover Q_mu,nu (Sec. 2.2, clover term).  A spinor
psi(x) is indexed [spin, colour] with colour fastest, so operators on the 12
components are kron(spin matrix, colour matrix).

Pins (tests/test_oracle_dirac.py): Clifford relations and gamma5 = diag(1,1,-1,-1);
free-field plane-wave closed form; U=1 clover term vanishes; constant abelian
field strength gives a closed-form clover term; gauge covariance under a random
SU(3) transformation; Gamma5-hermiticity; Q_nu,mu = Q_mu,nu^H.
"""
from __future__ import annotations

import numpy as np

from .lattice import Lattice

I4 = np.eye(4, dtype=np.complex128)
I12 = np.eye(12, dtype=np.complex128)

# chiral representation printed in Sec. 2.2
GAMMA = np.array(
    [
        [[0, 0, 0, 1j], [0, 0, 1j, 0], [0, -1j, 0, 0], [-1j, 0, 0, 0]],
        [[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]],
        [[0, 0, 1j, 0], [0, 0, 0, -1j], [-1j, 0, 0, 0], [0, 1j, 0, 0]],
        [[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]],
    ],
    dtype=np.complex128,
)
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]


def dag(m: np.ndarray) -> np.ndarray:
    return np.conj(np.swapaxes(m, -1, -2))


def clover_leaves_sum(U: np.ndarray, lat: Lattice, mu: int, nu: int) -> np.ndarray:
    """Q_mu,nu(x): the sum of the four plaquette leaves around x (Sec. 2.2, Fig. 2)."""
    def Um(m, steps):
        # U_m(x + sum(s * e_d for d, s in steps)) as a field over x
        f = U[:, m]
        for d, s in steps:
            f = lat.shift(f, d, s)
        return f

    def prod4(a, b, c, d):
        return a @ b @ c @ d

    leaf1 = prod4(Um(mu, []), Um(nu, [(mu, +1)]), dag(Um(mu, [(nu, +1)])), dag(Um(nu, [])))
    leaf2 = prod4(Um(nu, []), dag(Um(mu, [(mu, -1), (nu, +1)])), dag(Um(nu, [(mu, -1)])), Um(mu, [(mu, -1)]))
    leaf3 = prod4(dag(Um(mu, [(mu, -1)])), dag(Um(nu, [(mu, -1), (nu, -1)])), Um(mu, [(mu, -1), (nu, -1)]), Um(nu, [(nu, -1)]))
    leaf4 = prod4(dag(Um(nu, [(nu, -1)])), Um(mu, [(nu, -1)]), Um(nu, [(nu, -1), (mu, +1)]), dag(Um(mu, [])))
    return leaf1 + leaf2 + leaf3 + leaf4


def clover_term(U: np.ndarray, lat: Lattice, c_sw: float) -> np.ndarray:
    """-c_sw/32 sum_{mu,nu=0..3} (gamma_mu gamma_nu) (x) (Q_mu,nu - Q_nu,mu), per site [V,12,12]."""
    out = np.zeros((lat.V, 12, 12), dtype=np.complex128)
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue  # Q_mu,mu - Q_mu,mu = 0
            F = clover_leaves_sum(U, lat, mu, nu) - clover_leaves_sum(U, lat, nu, mu)
            gg = GAMMA[mu] @ GAMMA[nu]
            out += np.einsum("st,xab->xsatb", gg, F).reshape(lat.V, 12, 12)
    return -(c_sw / 32.0) * out


def site_term(U: np.ndarray, lat: Lattice, m0: float, c_sw: float) -> np.ndarray:
    """(m0 + 4) I_12 + clover term, per site [V, 12, 12] (Sec. 2.2)."""
    return (m0 + 4.0) * I12[None] + clover_term(U, lat, c_sw)


class DiracOperator:
    """D(U, m0, c_sw) on a periodic lattice; fields are [V, 4, 3, ...] complex128."""

    def __init__(self, U: np.ndarray, dims, m0: float, c_sw: float):
        self.lat = Lattice(dims)
        self.U = np.asarray(U, dtype=np.complex128).reshape(self.lat.V, 4, 3, 3)
        self.m0 = float(m0)
        self.c_sw = float(c_sw)
        self.A = site_term(self.U, self.lat, self.m0, self.c_sw)
        self.Udag_back = [self.lat.shift(dag(self.U[:, mu]), mu, -1) for mu in range(4)]  # U_mu(x-mu)^H

    @property
    def V(self):
        return self.lat.V

    def apply_site(self, psi: np.ndarray) -> np.ndarray:
        p = psi.reshape((self.V, 12) + psi.shape[3:])
        return np.einsum("xij,xj...->xi...", self.A, p).reshape(psi.shape)

    def hop(self, psi: np.ndarray, mu: int, sign: int) -> np.ndarray:
        """The single hopping term of D in direction sign*mu (Sec. 2.2)."""
        nb = self.lat.shift(psi, mu, sign)
        if sign > 0:
            proj = I4 - GAMMA[mu]
            link = self.U[:, mu]
        else:
            proj = I4 + GAMMA[mu]
            link = self.Udag_back[mu]
        return -0.5 * np.einsum("st,xab,xtb...->xsa...", proj, link, nb)

    def apply(self, psi: np.ndarray, hop_mask=None, with_site=True) -> np.ndarray:
        """D psi; hop_mask(mu, sign) -> bool[V] keeps only hops from x to x+sign*mu where True."""
        out = self.apply_site(psi) if with_site else np.zeros_like(psi)
        for mu in range(4):
            for sign in (+1, -1):
                h = self.hop(psi, mu, sign)
                if hop_mask is not None:
                    m = hop_mask(mu, sign)
                    h = h * m.reshape((self.V,) + (1,) * (h.ndim - 1))
                out = out + h
        return out

    def dense(self) -> np.ndarray:
        """The n x n matrix of D, n = 12 V, in the [site, spin, colour] ordering."""
        n = 12 * self.V
        eye = np.eye(n, dtype=np.complex128).reshape(self.V, 4, 3, n)
        return self.apply(eye).reshape(n, n)


def gamma5_field(psi: np.ndarray) -> np.ndarray:
    """Gamma_5 = I (x) gamma_5 (x) I_3 applied to a spinor field [V,4,3,...]."""
    out = psi.copy()
    out[:, 2:] *= -1.0
    return out


def inner(a: np.ndarray, b: np.ndarray) -> complex:
    """<a, b> = a^H b."""
    return complex(np.vdot(a.ravel(), b.ravel()))


def apply_at_sites(U: np.ndarray, dims, m0: float, c_sw: float, psi: np.ndarray, sites: np.ndarray) -> np.ndarray:
    """(D psi)(x) for the listed sites only, by the same formulas as DiracOperator,
    gathering the needed links and neighbours instead of shifting whole fields
    (lets the full-size workloads be checked site by site)."""
    dims = tuple(int(d) for d in dims)
    sites = np.asarray(sites, dtype=np.int64)
    base = np.stack(np.unravel_index(sites, dims), axis=1)

    def idx(offsets):
        c = base.copy()
        for d, s in offsets:
            c[:, d] = (c[:, d] + s) % dims[d]
        return np.ravel_multi_index(c.T, dims)

    def Ug(m, offsets):
        return U[idx(offsets), m]

    def prod4(a, b, c, d):
        return a @ b @ c @ d

    n = len(sites)
    A = np.broadcast_to((m0 + 4.0) * I12, (n, 12, 12)).copy()

    def Q(mu, nu):
        l1 = prod4(Ug(mu, []), Ug(nu, [(mu, 1)]), dag(Ug(mu, [(nu, 1)])), dag(Ug(nu, [])))
        l2 = prod4(Ug(nu, []), dag(Ug(mu, [(mu, -1), (nu, 1)])), dag(Ug(nu, [(mu, -1)])), Ug(mu, [(mu, -1)]))
        l3 = prod4(dag(Ug(mu, [(mu, -1)])), dag(Ug(nu, [(mu, -1), (nu, -1)])), Ug(mu, [(mu, -1), (nu, -1)]), Ug(nu, [(nu, -1)]))
        l4 = prod4(dag(Ug(nu, [(nu, -1)])), Ug(mu, [(nu, -1)]), Ug(nu, [(nu, -1), (mu, 1)]), dag(Ug(mu, [])))
        return l1 + l2 + l3 + l4

    for mu in range(4):
        for nu in range(4):
            if mu != nu:
                F = Q(mu, nu) - Q(nu, mu)
                A -= (c_sw / 32.0) * np.einsum("st,xab->xsatb", GAMMA[mu] @ GAMMA[nu], F).reshape(n, 12, 12)
    out = np.einsum("xij,xj->xi", A, psi[sites].reshape(n, 12)).reshape(n, 4, 3)
    for mu in range(4):
        fwd = psi[idx([(mu, 1)])]
        out -= 0.5 * np.einsum("st,xab,xtb->xsa", I4 - GAMMA[mu], U[sites, mu], fwd)
        bi = idx([(mu, -1)])
        out -= 0.5 * np.einsum("st,xab,xtb->xsa", I4 + GAMMA[mu], dag(U[bi, mu]), psi[bi])
    return out
