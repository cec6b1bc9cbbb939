"""Energy per site and sublattice magnetisations (oracle).

Test infrastructure only (see ``oracle/__init__``).

Expectation values of the thermal state rho ~ Tr_a |psi><psi| (Sec. III) are
<psi| O (x) 1_ancilla |psi> / <psi|psi>.  For an operator on the two sites of
one composite, that ratio is Tr(O X) / Tr(X) with X = T N T^T the composite
contracted with its converged environment metric N (Sec. III: the environment
of the gamma bond).  Readings: every bond direction is measured on the
un-gated state with its own gamma-mapped CTMRG; <S^a> of each sublattice is
taken from the z-mapped environment; E/site = (1/2) sum_gamma <H^gamma> minus
(h_A <S^z_A> + h_B <S^z_B>)/2 (N/2 sites per sublattice, 3N/2 bonds).
"""
import numpy as np

from . import model


def phys_op(O_A=None, O_B=None, O_AB=None):
    """16x16 operator on p = (sA, aA, sB, aB) from single-site operators or a
    4x4 two-site operator on (sA, sB); identity on the ancillas."""
    I2 = np.eye(2)
    if O_AB is not None:
        O = O_AB.reshape(2, 2, 2, 2)                              # [sA',sB',sA,sB]
        full = np.einsum("XYac,bB,dD->XbYdaBcD", O, I2, I2)
        return full.reshape(16, 16)
    OA = I2 if O_A is None else O_A
    OB = I2 if O_B is None else O_B
    return np.kron(np.kron(OA, I2), np.kron(OB, I2))


def expectation(X, O):
    return float(np.real(np.trace(O @ X.T)) / np.trace(X))


def site_moments(X):
    """<S^a>_A, <S^a>_B for a = x, y, z (y is identically 0 for real tensors;
    evaluated through the real antisymmetric part anyway)."""
    out = {}
    for name in "xyz":
        S = model.SPIN[name]
        OA = phys_op(O_A=S)
        OB = phys_op(O_B=S)
        out["A" + name] = float(np.real(np.trace(OA @ X.T)) / np.trace(X))
        out["B" + name] = float(np.real(np.trace(OB @ X.T)) / np.trace(X))
    return out


def order_parameters(mom):
    """Order parameters from the sublattice moments of ``site_moments`` (Sec.
    V).  Ferromagnetic (also the stripy order, measured as the ferromagnetic
    order of the dual Hamiltonian): m = 2 sqrt(sum_a <S^a>^2), <S^a> read as
    the sublattice average (<S^a_A> + <S^a_B>)/2.  Antiferromagnetic: the
    staggered m = sqrt(sum_a <S^a_A - S^a_B>^2)."""
    fm = 2.0 * np.sqrt(sum((0.5 * (mom["A" + a] + mom["B" + a])) ** 2 for a in "xyz"))
    af = np.sqrt(sum((mom["A" + a] - mom["B" + a]) ** 2 for a in "xyz"))
    return {"m_fm": float(fm), "m_af": float(af)}


def specific_heat(betas, energies):
    """C = dE/dT = -beta^2 dE/dbeta per site (the specific heat of Sec. V) by
    central differences along an imaginary-time trajectory on a uniform beta
    grid; returns (interior betas, C there)."""
    b = np.asarray(betas, dtype=np.float64)
    e = np.asarray(energies, dtype=np.float64)
    dEdb = (e[2:] - e[:-2]) / (b[2:] - b[:-2])
    return b[1:-1], -b[1:-1] ** 2 * dEdb
