"""Kitaev-Heisenberg bond Hamiltonians, gates and the Trotter schedule (oracle).

Test infrastructure only (see ``oracle/__init__``).

Basis convention: a spin index s=0 is S^z=+1/2, s=1 is S^z=-1/2.  A two-site
operator acting on (s_A, s_B) is a 4x4 matrix with row index 2*s_A'+s_B' and
column index 2*s_A+s_B.
"""
import numpy as np
from scipy.linalg import expm

# S = sigma/2 (Sec. II, below Eq. 2)
SX = 0.5 * np.array([[0.0, 1.0], [1.0, 0.0]], dtype=np.complex128)
SY = 0.5 * np.array([[0.0, -1.0j], [1.0j, 0.0]], dtype=np.complex128)
SZ = 0.5 * np.array([[1.0, 0.0], [0.0, -1.0]], dtype=np.complex128)
SPIN = {"x": SX, "y": SY, "z": SZ}
GAMMAS = ("x", "y", "z")


def couplings(phi, A=1.0):
    """J = A cos(phi), K = 2 A sin(phi)  (Sec. II, Eq. 3)."""
    return A * np.cos(phi), 2.0 * A * np.sin(phi)


def dual_angle(phi):
    """Klein duality tan(phi~) = -tan(phi) - 1 (Sec. II, Eq. 4); returns phi~
    on the branch of the opposite half of the phase diagram (cos phi~ < 0 when
    cos phi > 0, as in the paper's pairs -63 <-> -136.09 deg).  At the Kitaev
    points cos(phi) = 0 (J = 0, so J~ = -J = 0 and K~ = K + 2J = K) the map is
    the identity: the two self-dual points of Sec. II."""
    if abs(np.cos(phi)) < 1e-12:
        return phi
    t = -np.tan(phi) - 1.0
    base = np.arctan(t)                     # in (-pi/2, pi/2)
    cand = [base, base + np.pi, base - np.pi]
    # choose the candidate whose cosine has the opposite sign to cos(phi)
    cand = [c for c in cand if -np.pi <= c <= np.pi and np.sign(np.cos(c)) != np.sign(np.cos(phi))]
    return cand[0]


def dual_amplitude(phi, phi_dual, A=1.0):
    """A~ = -A cos(phi)/cos(phi~) so that J~ = -J (Sec. V, Eq. 14 context);
    A at the self-dual Kitaev points, where both cosines vanish."""
    if abs(np.cos(phi_dual)) < 1e-12:
        return A
    return -A * np.cos(phi) / np.cos(phi_dual)


def bond_hamiltonian(gamma, J, K, K_gamma=None, hA=0.0, hB=0.0):
    """H^(gamma)_ij = J S_i.S_j + K_gamma S_i^gamma S_j^gamma  (Sec. II, Eq. 2),
    optionally minus the bias hA S^z_A + hB S^z_B of Eq. (5).

    ``K_gamma`` (dict gamma->K) overrides K per bond direction: the
    anisotropic Kitaev couplings K_gamma of the introduction; used only as a
    test hook.  Returns a real 4x4 matrix (all terms are real because
    S^y (x) S^y is real)."""
    Kg = K if K_gamma is None else K_gamma[gamma]
    H = np.zeros((4, 4), dtype=np.complex128)
    for a in GAMMAS:
        H += J * np.kron(SPIN[a], SPIN[a])
    H += Kg * np.kron(SPIN[gamma], SPIN[gamma])
    H -= hA * np.kron(SZ, np.eye(2)) + hB * np.kron(np.eye(2), SZ)
    assert np.abs(H.imag).max() < 1e-15
    return np.ascontiguousarray(H.real)


def trotter_layers(dbeta):
    """Second-order Suzuki-Trotter step of Sec. III Eq. (6):
        e^{-dbeta H/2} ~ G_x(dbeta/2) G_y(dbeta/2) G_z(dbeta) G_y(dbeta/2) G_x(dbeta/2)
    with G_gamma(t) = prod exp(-t H^gamma / 2).  Each layer therefore applies
    exp(-tau H^gamma) with tau = dbeta/4 on x,y layers and dbeta/2 on the z layer.
    Returned in the order the gates act on the state (rightmost factor first);
    the product is palindromic so the order reads the same both ways."""
    return [("x", dbeta / 4), ("y", dbeta / 4), ("z", dbeta / 2), ("y", dbeta / 4), ("x", dbeta / 4)]


def gate(gamma, tau, J, K, K_gamma=None, hA=0.0, hB=0.0):
    """g = exp(-tau H^gamma) on (s_A, s_B); the bias of Eq. (5) enters only the
    z gate (Sec. III: H^(z)_ij includes the bias; each site has one z bond)."""
    if gamma == "z":
        H = bond_hamiltonian(gamma, J, K, K_gamma, hA, hB)
    else:
        H = bond_hamiltonian(gamma, J, K, K_gamma)
    return expm(-tau * H)


def gate_split(g, tol=1e-13):
    """Operator-Schmidt (SVD) split of a two-site gate into left/right gate
    tensors joined by an index of dimension = Schmidt rank (Fig. 3(b)):
    g[(a'b'),(ab)] = sum_k L[a',a,k] R[b',b,k]."""
    G = g.reshape(2, 2, 2, 2).transpose(0, 2, 1, 3).reshape(4, 4)   # [(a',a),(b',b)]
    U, S, Vt = np.linalg.svd(G)
    r = int(np.sum(S > tol * S[0]))
    L = (U[:, :r] * np.sqrt(S[:r])).reshape(2, 2, r)
    R = (Vt[:r].T * np.sqrt(S[:r])).reshape(2, 2, r)
    return L, R, S
