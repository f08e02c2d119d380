"""Pins of the oracle's Dirac operator (Sec. 2.2) against facts the paper and mathematics fix."""
import numpy as np
import pytest

from oracle.dirac import GAMMA, GAMMA5, DiracOperator, clover_leaves_sum, gamma5_field, inner
from oracle.lattice import Lattice
from paper_1303_1377_gb300 import synth


def test_clifford_and_gamma5():
    # Eq. commutativity_rel: gamma_mu gamma_nu + gamma_nu gamma_mu = 2 delta_mu,nu I
    for mu in range(4):
        assert np.allclose(GAMMA[mu], GAMMA[mu].conj().T)  # hermitian
        for nu in range(4):
            ac = GAMMA[mu] @ GAMMA[nu] + GAMMA[nu] @ GAMMA[mu]
            assert np.allclose(ac, 2.0 * np.eye(4) * (mu == nu))
    # printed result gamma5 = diag(1, 1, -1, -1)
    assert np.allclose(GAMMA5, np.diag([1, 1, -1, -1]))


def _plane_wave(lat, k, u):
    p = 2 * np.pi * np.array(k) / np.array(lat.dims)
    phase = np.exp(1j * (lat.coords @ p))
    return phase[:, None, None] * u[None], p


@pytest.mark.parametrize("dims,k", [((4, 2, 6, 8), (1, 1, 2, 3)), ((2, 4, 4, 6), (1, 3, 1, 5)), ((6, 6, 2, 4), (0, 5, 1, 1))])
def test_free_field_plane_wave(dims, k):
    """U = 1: D e^{ipx} u = e^{ipx} [(m0 + sum(1 - cos p)) + i sum gamma_mu sin p_mu] u (derived from Sec. 2.2)."""
    m0 = -0.37
    D = DiracOperator(synth.unit_gauge(dims), dims, m0, 1.7)
    rng = np.random.default_rng(0)
    u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
    psi, p = _plane_wave(D.lat, k, u)
    Dp = (m0 + np.sum(1 - np.cos(p))) * np.eye(4) + 1j * sum(GAMMA[mu] * np.sin(p[mu]) for mu in range(4))
    expect = _plane_wave(D.lat, k, Dp @ u)[0]
    assert np.allclose(D.apply(psi), expect, atol=1e-13)


def test_free_field_spectrum_closed_form():
    """Dense spectrum at U = 1 on 2x2x2x4: m0 + sum(1-cos p) +- i sqrt(sum sin^2 p), 6-fold per momentum."""
    dims = (2, 2, 2, 4)
    m0 = 0.1
    D = DiracOperator(synth.unit_gauge(dims), dims, m0, 1.0)
    ev = np.linalg.eigvals(D.dense())
    expect = []
    for k in np.ndindex(*dims):
        p = 2 * np.pi * np.array(k) / np.array(dims)
        re = m0 + np.sum(1 - np.cos(p))
        im = np.sqrt(np.sum(np.sin(p) ** 2))
        expect += [re + 1j * im] * 6 + [re - 1j * im] * 6
    expect = np.array(expect)

    def canon(z):
        z = np.round(z.real, 8) + 1j * np.round(z.imag, 8)
        return z[np.lexsort((z.imag, z.real))]

    assert np.allclose(canon(ev), canon(expect), atol=1e-10)


def test_clover_vanishes_on_unit_gauge():
    dims = (2, 4, 2, 4)
    D = DiracOperator(synth.unit_gauge(dims), dims, 0.3, 1.0)
    assert np.allclose(D.A, (0.3 + 4.0) * np.eye(12)[None], atol=1e-15)


def test_clover_constant_abelian_field_closed_form():
    """Constant field strength Phi in the (0,1) plane: every leaf is e^{i Phi}, so
    Q_01 - Q_10 = 8 i sin(Phi) and the site term is (m0+4) - (i c_sw/2) sin(Phi) gamma_0 gamma_1,
    whose eigenvalues are (m0+4) +- (c_sw/2) sin(Phi), each six-fold."""
    dims = (6, 4, 2, 2)
    lat = Lattice(dims)
    phi = 2 * np.pi * 1 / dims[0]
    U = synth.unit_gauge(dims)
    U[:, 1] *= np.exp(1j * phi * lat.coords[:, 0])[:, None, None]
    m0, csw = -0.2, 1.9
    D = DiracOperator(U, dims, m0, csw)
    expect = (m0 + 4) * np.eye(12) - 0.5j * csw * np.sin(phi) * np.kron(GAMMA[0] @ GAMMA[1], np.eye(3))
    assert np.allclose(D.A, expect[None], atol=1e-13)
    ev = np.sort(np.linalg.eigvalsh(D.A[0]))
    s = 0.5 * csw * np.sin(phi)
    assert np.allclose(ev, np.sort([m0 + 4 - s] * 6 + [m0 + 4 + s] * 6), atol=1e-13)


def test_gauge_covariance():
    """U'_mu(x) = G(x) U_mu(x) G(x+mu)^H, psi' = G psi  =>  D' psi' = G (D psi) (Sec. 2.1-2.2)."""
    dims = (4, 2, 4, 6)
    lat = Lattice(dims)
    U = synth.gauge_field(dims, 0.6, seed=11)
    G = synth.random_su3(lat.V, seed=12)
    Up = np.empty_like(U)
    for mu in range(4):
        Gn = G[lat.neighbour(mu, +1)]
        Up[:, mu] = G @ U[:, mu] @ np.conj(np.swapaxes(Gn, -1, -2))
    psi = synth.gaussian_spinors(dims, 1, seed=13)[0]
    psip = np.einsum("xab,xsb->xsa", G, psi)
    D = DiracOperator(U, dims, -0.1, 1.3)
    Dp = DiracOperator(Up, dims, -0.1, 1.3)
    lhs = Dp.apply(psip)
    rhs = np.einsum("xab,xsb->xsa", G, D.apply(psi))
    assert np.max(np.abs(lhs - rhs)) < 1e-13 * np.max(np.abs(rhs))


def test_gamma5_hermiticity():
    """(Gamma5 D)^H = Gamma5 D (Eq. g5sym): x^H G5 D y = conj(y^H G5 D x)."""
    dims = (4, 4, 2, 4)
    D = DiracOperator(synth.gauge_field(dims, 0.5, seed=3), dims, -0.4, 1.0)
    x, y = synth.gaussian_spinors(dims, 2, seed=4)
    a = inner(x, gamma5_field(D.apply(y)))
    b = np.conj(inner(y, gamma5_field(D.apply(x))))
    assert abs(a - b) < 1e-13 * abs(a)


def test_clover_orientation_reversal_and_chiral_blocks():
    """Q_nu,mu = Q_mu,nu^H leaf by leaf; the site term is hermitian and commutes with gamma5,
    i.e. it is two hermitian 6x6 blocks (spins 0,1 and spins 2,3)."""
    dims = (2, 4, 4, 2)
    lat = Lattice(dims)
    U = synth.gauge_field(dims, 0.7, seed=5)
    for mu in range(4):
        for nu in range(4):
            if mu != nu:
                Q = clover_leaves_sum(U, lat, mu, nu)
                assert np.allclose(clover_leaves_sum(U, lat, nu, mu), np.conj(np.swapaxes(Q, -1, -2)), atol=1e-14)
    D = DiracOperator(U, dims, 0.0, 1.0)
    A = D.A
    assert np.allclose(A, np.conj(np.swapaxes(A, -1, -2)), atol=1e-14)
    g5 = np.kron(GAMMA5, np.eye(3))
    assert np.allclose(A @ g5, g5 @ A, atol=1e-14)
    assert np.allclose(A[:, :6, 6:], 0, atol=1e-14)


def test_mass_enters_diagonal_only():
    """D(m0 + d) = D(m0) + d I (Sec. 2.2: m0 appears only in (m0+4) I)."""
    dims = (2, 2, 4, 4)
    U = synth.gauge_field(dims, 0.5, seed=9)
    psi = synth.gaussian_spinors(dims, 1, seed=10)[0]
    a = DiracOperator(U, dims, 0.1, 1.0).apply(psi)
    b = DiracOperator(U, dims, 0.35, 1.0).apply(psi)
    assert np.allclose(b - a, 0.25 * psi, atol=1e-13)


def test_site_sampled_operator_equals_full_operator():
    """The gather-based evaluation at chosen sites reproduces the full-field operator."""
    from oracle.dirac import apply_at_sites

    dims = (4, 2, 6, 4)
    U = synth.gauge_field(dims, 0.5, seed=15)
    psi = synth.gaussian_spinors(dims, 1, seed=16)[0]
    D = DiracOperator(U, dims, -0.2, 1.1)
    full = D.apply(psi)
    sites = np.array([0, 5, 17, 63, 100, 191])
    assert np.allclose(apply_at_sites(U, dims, -0.2, 1.1, psi, sites), full[sites], atol=1e-13)
