"""Pins of the oracle's model layer: bond Hamiltonian, gates, Trotter layers,
duality.  Every check compares against something not computed by
oracle.model itself (closed-form spectra, the bitwise ED Hamiltonian,
the paper's printed duality pairs)."""
import os

import numpy as np
import pytest
from scipy.linalg import expm

from oracle import exact, model

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("gamma", ["x", "y", "z"])
@pytest.mark.parametrize("phi", [0.3 * np.pi, -63 / 180 * np.pi, np.pi / 2, 0.0])
def test_bond_spectrum_closed_form(gamma, phi):
    J, K = model.couplings(phi)
    w = np.linalg.eigvalsh(model.bond_hamiltonian(gamma, J, K))
    assert np.allclose(w, exact.bond_spectrum(J, K), atol=1e-14)


def test_bond_hamiltonian_matches_bitwise_two_site():
    # a 1x1 cluster has x, y, z bonds all between the same A-B pair; compare
    # the sum of the three bond terms with the bitwise ED construction.
    J, K = 0.37, -1.21
    H_ed, n = exact.honeycomb_hamiltonian(1, 1, J, K)
    H = sum(model.bond_hamiltonian(g, J, K) for g in "xyz")
    assert n == 2 and np.allclose(H, H_ed, atol=1e-15)
    H_ed, _ = exact.honeycomb_hamiltonian(1, 1, 0.0, 0.0, hA=0.3, hB=-0.8)
    assert np.allclose(model.bond_hamiltonian("z", 0, 0, hA=0.3, hB=-0.8), H_ed, atol=1e-15)


@pytest.mark.parametrize("J,K,rank", [(0.5, 1.6, 4), (0.0, 1.0, 2)])
def test_gate_properties(J, K, rank):
    for gamma in "xyz":
        g1 = model.gate(gamma, 0.013, J, K)
        g2 = model.gate(gamma, 0.029, J, K)
        assert np.allclose(g1, g1.T, atol=1e-15)
        assert np.all(np.linalg.eigvalsh(g1) > 0)
        assert np.allclose(g1 @ g2, model.gate(gamma, 0.042, J, K), atol=1e-14)
        w = np.sort(np.linalg.eigvalsh(g1))
        assert np.allclose(w, np.sort(np.exp(-0.013 * exact.bond_spectrum(J, K))), atol=1e-14)
        L, R, S = model.gate_split(g1)
        assert L.shape[2] == rank
        rec = np.einsum("Aak,Bbk->ABab", L, R).reshape(4, 4)
        assert np.allclose(rec, g1, atol=1e-15)
        U = expm(-1j * 0.3 * model.bond_hamiltonian(gamma, J, K))
        assert np.allclose(U.conj().T @ U, np.eye(4), atol=1e-14)


def _embed_two_site(g, i, j, n):
    """Dense operator of a 4x4 gate on sites (i, j) of an n-site register
    (site i = most significant factor)."""
    dim = 2 ** n
    out = np.zeros((dim, dim))
    G = g.reshape(2, 2, 2, 2)
    for col in range(dim):
        bi = (col >> (n - 1 - i)) & 1
        bj = (col >> (n - 1 - j)) & 1
        for ai in range(2):
            for aj in range(2):
                row = col & ~(1 << (n - 1 - i)) & ~(1 << (n - 1 - j))
                row |= (ai << (n - 1 - i)) | (aj << (n - 1 - j))
                out[row, col] += G[ai, aj, bi, bj]
    return out


def test_trotter_layers_second_order_against_ed():
    """The five gate layers of one step, built from model.gate and embedded on
    the 8-site cluster, equal exp(-dbeta H/2) of the bitwise Hamiltonian up to
    O(dbeta^3) (halving dbeta cuts the error ~8x)."""
    J, K, h = model.couplings(0.3 * np.pi) + (0.4,)
    H, n = exact.honeycomb_hamiltonian(2, 2, J, K, hA=h, hB=-h)
    bonds, _ = exact.honeycomb_bonds(2, 2)
    errs = []
    for db in (0.2, 0.1):
        U = np.eye(2 ** n)
        for gamma, tau in model.trotter_layers(db):
            g = model.gate(gamma, tau, J, K, hA=h, hB=-h)
            for gb, i, j in bonds:
                if gb == gamma:
                    U = _embed_two_site(g, i, j, n) @ U
        errs.append(np.abs(U - expm(-db * H / 2)).max())
    assert errs[1] < 1e-3
    assert 6.0 < errs[0] / errs[1] < 10.0


def test_duality_pairs_printed_in_paper():
    rows = np.loadtxt(os.path.join(GOLD, "duality_pairs.txt"))
    for phi_deg, dual_deg, A_dual, tol in rows:
        phi = np.deg2rad(phi_deg)
        pd = model.dual_angle(phi)
        assert abs(np.rad2deg(pd) - dual_deg) < tol
        if not np.isnan(A_dual):
            assert abs(model.dual_amplitude(phi, pd) - A_dual) < 0.005


def test_duality_is_an_involution_and_maps_the_su2_points_onto_each_other():
    """Applied twice the duality is the identity (J~~ = J, K~~ = K); the four
    SU(2)-symmetric points of Sec. II (-45, 0, 135, 180 deg) map onto each
    other, and the duals of -45 and 135 deg are pure Heisenberg (K~ = 0): the
    hidden SU(2) symmetry of those two points."""
    for phi_deg in np.linspace(-179.0, 179.0, 37):
        phi = np.deg2rad(phi_deg)
        J, K = model.couplings(phi)
        pd = model.dual_angle(phi)
        Jd, Kd = model.couplings(pd, model.dual_amplitude(phi, pd))
        assert abs(Jd + J) < 1e-12 and abs(Kd - (K + 2 * J)) < 1e-12
        pdd = model.dual_angle(pd)
        Jdd, Kdd = model.couplings(pdd, model.dual_amplitude(pd, pdd, model.dual_amplitude(phi, pd)))
        assert abs(Jdd - J) < 1e-12 and abs(Kdd - K) < 1e-12
    pairs = {-45.0: 180.0, 0.0: 135.0, 135.0: 0.0, 180.0: -45.0}
    for phi_deg, want in pairs.items():
        pd = model.dual_angle(np.deg2rad(phi_deg))
        assert abs(np.cos(pd) - np.cos(np.deg2rad(want))) < 1e-12
        assert abs(np.sin(pd) - np.sin(np.deg2rad(want))) < 1e-12
        Jd, Kd = model.couplings(pd, model.dual_amplitude(np.deg2rad(phi_deg), pd))
        if phi_deg in (-45.0, 135.0):
            assert abs(Kd) < 1e-12


@pytest.mark.parametrize("phi_deg", [-63.0, -17.0, 30.0])
def test_duality_spectrum_on_klein_cluster(phi_deg):
    """The Klein map (4-sublattice pi rotations; the 2x2 torus is compatible)
    makes H(phi, A=1) and H(phi~, A~) unitarily equivalent: equal spectra."""
    phi = np.deg2rad(phi_deg)
    pd = model.dual_angle(phi)
    Ad = model.dual_amplitude(phi, pd)
    J, K = model.couplings(phi)
    Jd, Kd = model.couplings(pd, Ad)
    w1 = np.linalg.eigvalsh(exact.honeycomb_hamiltonian(2, 2, J, K)[0])
    w2 = np.linalg.eigvalsh(exact.honeycomb_hamiltonian(2, 2, Jd, Kd)[0])
    assert np.allclose(w1, w2, atol=1e-12)
    # and it is not a trivial identity
    w3 = np.linalg.eigvalsh(exact.honeycomb_hamiltonian(2, 2, Jd, K)[0])
    assert not np.allclose(w1, w3, atol=1e-6)
