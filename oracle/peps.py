"""Site tensors and the gamma-composite of the rhombic mapping (oracle).

Test infrastructure only (see ``oracle/__init__``).

Site tensors (Fig. 3(a)): A[s][a][x][y][z] and B[s][a][x][y][z], real, with
spin s, ancilla a and the three honeycomb bonds of dimension D.  Every A site
is joined to B sites by one bond of each direction gamma.

Rhombic mapping (Fig. 4(b), Sec. III): for the bond direction gamma being
updated, each A-B pair joined by a gamma bond is fused into one composite
site.  With (alpha, alpha') the two other directions in cyclic order
(gamma=x -> (y,z), y -> (z,x), z -> (x,y)), the composites form a square
lattice whose horizontal bonds are alpha bonds and vertical bonds alpha'
bonds.  The composite is stored as

    T[p; l, u, r, d],  p = (s_A, a_A, s_B, a_B)  (16 values, row-major),
    l = B.alpha, u = A.alpha', r = A.alpha, d = B.alpha'.

Applying the gate g on (s_A, s_B) before fusing gives the exact A'-B' pair of
Fig. 3(b) with its 4D-dimensional gamma bond contracted inside the composite.
"""
import numpy as np

AXIS = {"x": 2, "y": 3, "z": 4}


def other_bonds(gamma):
    """(alpha, alpha') for composite direction gamma, cyclic order."""
    order = "xyz"
    g = order.index(gamma)
    return order[(g + 1) % 3], order[(g + 2) % 3]


def product_state(D):
    """beta = 0 purification (Sec. III): every spin maximally entangled with
    its ancilla, no entanglement between sites; embedded at virtual index 0
    of bond dimension D (zero elsewhere)."""
    A = np.zeros((2, 2, D, D, D))
    A[0, 0, 0, 0, 0] = 1.0
    A[1, 1, 0, 0, 0] = 1.0
    return A, A.copy()


def composite(A, B, gamma, g=None):
    """T[p; l,u,r,d] for mapping gamma, optionally with the 4x4 gate g on
    (s_A, s_B) (ancillas untouched).  Returns shape (16, D, D, D, D)."""
    al, alp = other_bonds(gamma)
    D = A.shape[2]
    # A_g[sA, aA, u=alpha', r=alpha, k=gamma]; B_g[sB, aB, d=alpha', l=alpha, k=gamma]
    perm = (0, 1, AXIS[alp], AXIS[al], AXIS[gamma])
    Ag = A.transpose(perm)
    Bg = B.transpose(perm)
    T = np.einsum("abURk,cdDLk->abcdLURD", Ag, Bg)          # [sA,aA,sB,aB,l,u,r,d]
    if g is not None:
        G = g.reshape(2, 2, 2, 2)                           # [sA',sB',sA,sB]
        T = np.einsum("XYac,abcdLURD->XbYdLURD", G, T)
    return T.reshape(16, D, D, D, D)


def split_composite_legs(A2, B2, gamma, D):
    """Inverse of the leg assignment: given A''[sA,aA,u,r,k] and
    B''[sB,aB,d,l,k] written in the composite's frame, return site tensors
    A[s][a][x][y][z], B[s][a][x][y][z]."""
    al, alp = other_bonds(gamma)
    perm = (0, 1, AXIS[alp], AXIS[al], AXIS[gamma])
    inv = np.argsort(perm)
    return A2.transpose(inv).copy(), B2.transpose(inv).copy()


def to_composite_frame(A, B, gamma):
    """A[s][a][x][y][z] -> A_g[sA,aA,u,r,k]; B -> B_g[sB,aB,d,l,k]."""
    al, alp = other_bonds(gamma)
    perm = (0, 1, AXIS[alp], AXIS[al], AXIS[gamma])
    return A.transpose(perm).copy(), B.transpose(perm).copy()
