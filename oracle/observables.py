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

Products of operators on the four composites of a 2 x 2 plaquette come from
the plaquette's cluster in the same environment (``ctmrg.cluster_2x2``); the
plaquette flux W of Sec. V is one such product.
"""
import numpy as np

from . import ctmrg, model, peps


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


# ---------------------------------------------------------------- 2 x 2 plaquette, flux

def plaquette_expectation(env, T, ops):
    """<O_ul O_ur O_dr O_dl> on a 2 x 2 plaquette of composite sites T
    (translation invariant): the cluster with site i's ket layer O_i T,
    divided by the plain cluster (both in the converged environment env).
    ops: four p x p operators (complex allowed) in the order upper-left,
    upper-right, lower-right, lower-left.  Returns the complex ratio."""
    p = T.shape[0]
    Tc = T.astype(np.complex128)
    plain = ctmrg.double_tensor(Tc)
    sites = [ctmrg.double_tensor((np.asarray(O) @ Tc.reshape(p, -1)).reshape(T.shape), Tc) for O in ops]
    return complex(ctmrg.cluster_2x2(env, *sites) / ctmrg.cluster_2x2(env, plain, plain, plain, plain))


PAULI = {a: 2.0 * model.SPIN[a] for a in "xyz"}


def flux_operators(gamma):
    """The plaquette flux of the hexagonal lattice, W_p = prod_{i in p}
    sigma_i^{o(i)} with o(i) the direction of the one bond at site i that
    leaves the hexagon p (Kitaev's plaquette operator; Sec. V, the flux whose
    average orders at the lower crossover), as four operators on the
    composites of a 2 x 2 plaquette of the gamma mapping.

    Geometry of the gamma mapping (``peps``): composite (i, j) holds A(i,j)
    and B(i,j) joined by gamma; its leg r = A.alpha meets the leg l = B.alpha
    of composite (i+1, j), its leg u = A.alpha' the leg d = B.alpha' of
    composite (i, j+1), the one above.  The hexagon
      A(0,0) -alpha- B(1,0) -gamma- A(1,0) -alpha'- B(1,1) -alpha- A(0,1)
             -gamma- B(0,1) -alpha'- A(0,0)
    lies in the plaquette of composites (0,1) upper-left, (1,1) upper-right,
    (1,0) lower-right, (0,0) lower-left; the leaving bonds are gamma at A(0,0)
    and B(1,1), alpha' at B(1,0) and A(0,1), alpha at A(1,0) and B(0,1).
    Returns the 16 x 16 operators on p = (sA, aA, sB, aB), upper-left first."""
    al, alp = peps.other_bonds(gamma)
    s = PAULI
    return [phys_op(O_A=s[alp], O_B=s[al]),     # (0,1): A(0,1) alpha', B(0,1) alpha
            phys_op(O_B=s[gamma]),              # (1,1): B(1,1) gamma
            phys_op(O_A=s[al], O_B=s[alp]),     # (1,0): A(1,0) alpha, B(1,0) alpha'
            phys_op(O_A=s[gamma])]              # (0,0): A(0,0) gamma


def flux(env, T, gamma):
    """<W_p> of the composite T of the gamma mapping in its converged
    environment (complex arithmetic; the value is real for a real state)."""
    return plaquette_expectation(env, T, flux_operators(gamma))
