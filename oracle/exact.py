"""Independent pins for the oracle (test infrastructure only).

Nothing here shares arithmetic with the CTMRG / eeFU modules:

* ``honeycomb_ed``  -- brute-force thermal energy of periodic honeycomb
  clusters of L1 x L2 two-site cells (Sec. II Hamiltonian, Eqs. 1-5), built
  bit by bit on the S^z basis;
* ``onsager_lnZ``   -- Onsager's free energy per site of the anisotropic
  square-lattice Ising model, by quadrature of the double integral;
* ``yang_m``        -- Yang's spontaneous magnetisation (1 - sinh(2K)^-4)^(1/8);
* ``ising_peps``    -- a PEPS whose norm network is the Ising partition
  function, with optional random bond gauges (Z is gauge invariant);
* closed forms for decoupled z-dimers and a pure field.
"""
import numpy as np
from scipy.linalg import sqrtm


# ------------------------------------------------------------------ exact diagonalisation

def honeycomb_bonds(L1, L2):
    """Sites: A(i,j) = 2*(i*L2+j), B(i,j) = A+1.  Bonds: z joins A(i,j)-B(i,j);
    x joins A(i,j)-B(i-1,j); y joins A(i,j)-B(i,j-1) (periodic)."""
    bonds = []
    for i in range(L1):
        for j in range(L2):
            a = 2 * (i * L2 + j)
            bonds.append(("z", a, a + 1))
            bonds.append(("x", a, 2 * (((i - 1) % L1) * L2 + j) + 1))
            bonds.append(("y", a, 2 * (i * L2 + (j - 1) % L2) + 1))
    return bonds, 2 * L1 * L2


def honeycomb_hamiltonian(L1, L2, J, K, K_gamma=None, hA=0.0, hB=0.0):
    """Dense real H of Eqs. (1)-(2),(5) on the periodic cluster, built bit by
    bit (site i is bit n-1-i of the basis index; bit 0 = S^z = +1/2):
      S^z_i S^z_j |b> = s_i s_j / 4 |b>,  s = +1 for bit 0, -1 for bit 1;
      S^x_i S^x_j |b> = 1/4 |b with bits i,j flipped>;
      S^y_i S^y_j |b> = -s_i s_j / 4 |b with bits i,j flipped>
    (from sigma^y |b> = i (-1)^b |1-b>)."""
    bonds, n = honeycomb_bonds(L1, L2)
    dim = 2 ** n
    idx = np.arange(dim)
    spin = lambda i: 1 - 2 * ((idx >> (n - 1 - i)) & 1)          # +1 / -1
    H = np.zeros((dim, dim))
    for g, i, j in bonds:
        Kg = K if K_gamma is None else K_gamma[g]
        si, sj = spin(i), spin(j)
        cz = J + (Kg if g == "z" else 0.0)
        cx = J + (Kg if g == "x" else 0.0)
        cy = J + (Kg if g == "y" else 0.0)
        H[idx, idx] += cz * si * sj / 4.0
        flip = idx ^ (1 << (n - 1 - i)) ^ (1 << (n - 1 - j))
        H[flip, idx] += cx / 4.0 - cy * si * sj / 4.0
    for i in range(n):
        H[idx, idx] -= (hA if i % 2 == 0 else hB) * spin(i) / 2.0
    return H, n


def honeycomb_ed(L1, L2, J, K, betas, K_gamma=None, hA=0.0, hB=0.0):
    """Thermal energy per site E(beta) = Tr(H e^{-beta H}) / (n Tr e^{-beta H})."""
    H, n = honeycomb_hamiltonian(L1, L2, J, K, K_gamma, hA, hB)
    w = np.linalg.eigvalsh(H)
    out = []
    for b in np.atleast_1d(betas):
        x = np.exp(-b * (w - w.min()))
        out.append(float(np.sum(w * x) / np.sum(x) / n))
    return np.array(out)


def high_T_energy_slope(J, K, h=0.0):
    """E/site = -beta [ (3/2) <H_b^2>_0 + h^2/4 ] + O(beta^2), with
    <H_b^2>_0 = [2(J+K)^2 + (J-K)^2 + (3J+K)^2]/64 (traceless bond terms on a
    triangle-free lattice)."""
    hb2 = (2 * (J + K) ** 2 + (J - K) ** 2 + (3 * J + K) ** 2) / 64.0
    return -(1.5 * hb2 + h * h / 4.0)


def bond_spectrum(J, K):
    """Eigenvalues of J S.S + K S^z S^z: (J+K)/4 twice, (J-K)/4, -(3J+K)/4."""
    return np.sort(np.array([(J + K) / 4, (J + K) / 4, (J - K) / 4, -(3 * J + K) / 4]))


def dimer_energy(J, K, t):
    """<H_b> of one dimer in the state exp(-t H_b), from the four eigenvalues."""
    w = bond_spectrum(J, K)
    x = np.exp(-t * w)
    return float(np.sum(w * x) / np.sum(x))


def kz_only_energy(Kz, beta):
    """J=0, K_x=K_y=0: decoupled z dimers, E/site = -(Kz/8) tanh(beta Kz/4)."""
    return -(Kz / 8.0) * np.tanh(beta * Kz / 4.0)


def field_only(h, beta):
    """J=K=0, uniform field h: E/site = -(h/2) tanh(beta h/2), <S^z> = tanh(beta h/2)/2."""
    return -(h / 2.0) * np.tanh(beta * h / 2.0), 0.5 * np.tanh(beta * h / 2.0)


# ------------------------------------------------------------------ 2D Ising

def onsager_lnZ(K1, K2, n=512):
    """-beta f = ln 2 + 1/(8 pi^2) int int ln[cosh2K1 cosh2K2 - sinh2K1 cos t1
    - sinh2K2 cos t2] dt1 dt2, periodic trapezoid rule (spectrally accurate
    away from the critical coupling)."""
    t = 2 * np.pi * np.arange(n) / n
    c1, c2 = np.meshgrid(np.cos(t), np.cos(t), indexing="ij")
    f = np.log(np.cosh(2 * K1) * np.cosh(2 * K2) - np.sinh(2 * K1) * c1 - np.sinh(2 * K2) * c2)
    return np.log(2.0) + 0.5 * f.mean()


def yang_m(K):
    """Spontaneous magnetisation of the isotropic model, K > K_c."""
    return (1.0 - np.sinh(2 * K) ** -4) ** 0.125


def ising_bond_root(K):
    """V with V V^T = [[e^{K/2}, e^{-K/2}], [e^{-K/2}, e^{K/2}]], so that the
    ket-bra contraction of one bond gives (V V^T)^2 = e^{K s s'}."""
    W = np.array([[np.exp(K / 2), np.exp(-K / 2)], [np.exp(-K / 2), np.exp(K / 2)]])
    return np.real(sqrtm(W))


def ising_peps(Kh, Kv, gauge_seed=None):
    """T[s; l,u,r,d] = Vh[s,l] Vv[s,u] Vh[s,r] Vv[s,d] (p = 2, D = 2).  With a
    gauge seed, random invertible X (horizontal) and Y (vertical) bond gauges
    are inserted: T[l,u,r,d] -> X^-1[l,.] Y^-1[u,.] T X[.,r] Y[.,d]."""
    Vh, Vv = ising_bond_root(Kh), ising_bond_root(Kv)
    T = np.einsum("sl,su,sr,sd->slurd", Vh, Vv, Vh, Vv)
    if gauge_seed is not None:
        rng = np.random.default_rng(gauge_seed)
        X = np.eye(2) + 0.4 * rng.standard_normal((2, 2))
        Y = np.eye(2) + 0.4 * rng.standard_normal((2, 2))
        Xi, Yi = np.linalg.inv(X), np.linalg.inv(Y)
        T = np.einsum("lL,uU,sLURD,Rr,Dd->slurd", Xi, Yi, T, X, Y)
    return T
