"""Corner-transfer-matrix renormalisation group on the rhombic lattice (oracle).

Test infrastructure only (see ``oracle/__init__``).

Follows Fig. 4 and Sec. III of the paper: the norm <psi|psi> of the
purification is a square-lattice network of quadruple tensors (a composite
ket tensor contracted with its bra over the 16 physical values, all bonds
D^2, Fig. 4(b)); CTMRG replaces the semi-infinite sectors by corners C and
edges E of dimension chi (Fig. 4(c)).  The paper defers the CTMRG details to
the square-lattice literature it cites; the readings adopted here (the same
ones the GPU library implements) are:

* directional moves left, up, right, down; each move absorbs one column;
* projectors from the half-system scheme: with the upper-left and lower-left
  enlarged corners Q_ul, Q_dl (cut index c = (chi, D^2) between them),
  M = Q_ul^T Q_dl (contracted over the cut), truncated SVD M ~ U S V^T,
  P = Q_dl V S^-1/2, P~ = S^-1/2 U^T Q_ul^T, so that P P~ is an oblique
  projector on the cut; singular values below ``cut * s_1`` are dropped;
* C and E divided by their Frobenius norm after every move;
* convergence when the top-chi projector spectra s/||s||_2 of all four moves
  of a sweep change by less than ``tol`` (max-norm) between sweeps;
* initial environment: the traced boundary (corner = 1, edge = delta over
  (ket, bra)) embedded at index 0 of chi.

Index conventions (clockwise around the centre: C1 E1 C2 E2 C3 E3 C4 E4):
  C[i][x, y]     x = leg to the previous edge, y = leg to the next edge;
  E[i][x, m, y]  x = leg to the previous corner, y = to the next corner,
                 m = the centre leg, a fused (ket, bra) pair m = k*D + b;
  a[l, u, r, d]  quadruple tensor, each leg a fused (ket, bra) pair;
  E1 attaches to u, E2 to r, E3 to d, E4 to l.
A counter-clockwise rotation of the lattice maps (C1..C4, E1..E4) to
(C2, C3, C4, C1, E2, E3, E4, E1) and a[l,u,r,d] to a[u,r,d,l]; the up, right
and down moves are the left move in the frame rotated 1, 2, 3 times.
"""
import numpy as np


def double_tensor(T, Tbra=None):
    """Quadruple tensor a = sum_p T[p;l,u,r,d] Tbra[p;l',u',r',d'] with fused
    legs (l,l') etc. (Fig. 4(a,b))."""
    if Tbra is None:
        Tbra = T
    D = T.shape[1]
    a = np.einsum("plurd,pLURD->lLuUrRdD", T, Tbra, optimize=True)
    return a.reshape(D * D, D * D, D * D, D * D)


def rotate(a, times=1):
    """Counter-clockwise lattice rotation: new (l,u,r,d) = old (u,r,d,l)."""
    for _ in range(times % 4):
        a = a.transpose(1, 2, 3, 0)
    return a


class Env:
    """Corners C[0..3] (chi x chi) and edges E[0..3] (chi x D^2 x chi)."""

    def __init__(self, C, E):
        self.C = [np.array(c, dtype=np.float64) for c in C]
        self.E = [np.array(e, dtype=np.float64) for e in E]

    @property
    def chi(self):
        return self.C[0].shape[0]

    def copy(self):
        return Env([c.copy() for c in self.C], [e.copy() for e in self.E])


def init_env(chi, D, edge_vec=None):
    """Traced boundary at index 0: C = e0 e0^T, E[0, (k,b), 0] = delta_kb
    (or the given D^2 vector, e.g. a fixed-spin boundary)."""
    if edge_vec is None:
        edge_vec = np.eye(D).reshape(D * D)
    C = np.zeros((chi, chi))
    C[0, 0] = 1.0
    E = np.zeros((chi, D * D, chi))
    E[0, :, 0] = edge_vec
    return Env([C.copy() for _ in range(4)], [E.copy() for _ in range(4)])


def enlarged_corners(C1, E1, E4, C4, E3, a):
    """Q_ul[(w,d),(z,r)] = C1 E1 E4 a   and   Q_dl[(w,u),(v,r)] = C4 E3 E4 a.
    First pair: the cut below the upper-left block; second pair: the right legs."""
    Qul = np.einsum("ab,buz,wla,lurd->wdzr", C1, E1, E4, a, optimize=True)
    Qdl = np.einsum("ab,vda,blw,lurd->wuvr", C4, E3, E4, a, optimize=True)
    return Qul, Qdl


def projectors(Qul, Qdl, chi, cut):
    """Half-system projectors (readings in the module docstring).
    Returns P (n x chi), Pt (chi x n), the kept spectrum (chi, zero-padded)
    and the discarded weight sum_{i>=chi} s_i^2 / sum_i s_i^2 of M."""
    n = Qul.shape[0] * Qul.shape[1]
    Qu = Qul.reshape(n, -1)
    Qd = Qdl.reshape(n, -1)
    M = Qu.T @ Qd
    U, S, Vt = np.linalg.svd(M)
    m = min(chi, S.size)
    s = S[:m]
    keep = s > cut * S[0] if S[0] > 0 else np.zeros(m, bool)
    isq = np.where(keep, 1.0 / np.sqrt(np.where(keep, s, 1.0)), 0.0)
    P = np.zeros((n, chi))
    Pt = np.zeros((chi, n))
    P[:, :m] = (Qd @ Vt[:m].T) * isq[None, :]
    Pt[:m, :] = isq[:, None] * (U[:, :m].T @ Qu.T)
    spec = np.zeros(chi)
    spec[:m] = np.where(keep, s, 0.0)
    tot = np.sum(S ** 2)
    trunc = float(np.sum(S[m:] ** 2) / tot) if tot > 0 else 0.0
    return P, Pt, spec, trunc


def left_move(C, E, a, chi, cut):
    """One left move in the current frame: (C1,E4,C4) absorb the column
    (E1, a, E3) through the projectors.  C, E are lists in the frame order."""
    C1, C2, C3, C4 = C
    E1, E2, E3, E4 = E
    Qul, Qdl = enlarged_corners(C1, E1, E4, C4, E3, a)
    P, Pt, spec, trunc = projectors(Qul, Qdl, chi, cut)
    d2 = a.shape[0]
    n = chi * d2
    C1E1 = np.einsum("ab,buz->auz", C1, E1).reshape(n, chi)        # [(x4,u), z]
    C4E3 = np.einsum("ab,vda->vbd", C4, E3).reshape(chi, n)        # [v, (y4,d)]
    E4a = np.einsum("wla,lurd->wdrau", E4, a).reshape(n, d2, n)    # [(w,d), r, (x4,u)]
    C1n = P.T @ C1E1                                               # [alpha, z]
    C4n = C4E3 @ Pt.T                                              # [v, alpha]
    E4n = np.einsum("ca,crC,bC->arb", P, E4a, Pt, optimize=True)   # [a_dn, r, a_up]
    C1n /= np.linalg.norm(C1n)
    C4n /= np.linalg.norm(C4n)
    E4n /= np.linalg.norm(E4n)
    return C1n, E4n, C4n, spec, trunc


def sweep(env, a, cut=1e-12):
    """One CTM sweep: left, up, right, down moves.  Updates env in place.
    Returns the four spectra (chi each) and truncation errors."""
    chi = env.chi
    specs, truncs = [], []
    for s in range(4):
        idx = [(s + i) % 4 for i in range(4)]
        C = [env.C[i] for i in idx]
        E = [env.E[i] for i in idx]
        C1n, E4n, C4n, spec, trunc = left_move(C, E, rotate(a, s), chi, cut)
        env.C[idx[0]] = C1n
        env.E[idx[3]] = E4n
        env.C[idx[3]] = C4n
        specs.append(spec)
        truncs.append(trunc)
    return specs, truncs


def normalised_spectra(specs):
    out = []
    for s in specs:
        nrm = np.linalg.norm(s)
        out.append(s / nrm if nrm > 0 else s)
    return out


def ctmrg(a, env, tol=1e-12, max_sweeps=100, min_sweeps=1, cut=1e-12):
    """Iterate sweeps until the normalised projector spectra change by less
    than tol (max-norm over the four moves), or max_sweeps.  Returns
    (env, info) with info = dict(sweeps, delta, spectra, trunc)."""
    prev = None
    delta = np.inf
    n = 0
    specs, truncs = None, None
    for n in range(1, max_sweeps + 1):
        specs, truncs = sweep(env, a, cut)
        cur = normalised_spectra(specs)
        if prev is not None:
            delta = max(float(np.max(np.abs(c - p))) for c, p in zip(cur, prev))
        prev = cur
        if n >= min_sweeps and delta < tol:
            break
    return env, dict(sweeps=n, delta=delta, spectra=specs, trunc=truncs)


# ---------------------------------------------------------------- environment metric

def metric_d2(env):
    """Ring of the 4 corners and 4 edges around one site (the environment of
    one composite, Sec. III): N[l,u,r,d] with fused (ket,bra) legs."""
    C1, C2, C3, C4 = env.C
    E1, E2, E3, E4 = env.E
    up = np.einsum("ha,aub,bc,cre->hure", C1, E1, C2, E2, optimize=True)
    dn = np.einsum("ef,fdg,gi,ilh->edlh", C3, E3, C4, E4, optimize=True)
    return np.einsum("hure,edlh->lurd", up, dn, optimize=True)


def metric(env, D):
    """Environment metric N[(l,u,r,d) ket, (l',u',r',d') bra] (D^4 x D^4),
    symmetrised (N + N^T)/2."""
    N = metric_d2(env).reshape(D, D, D, D, D, D, D, D)     # [lk,lb,uk,ub,rk,rb,dk,db]
    N = N.transpose(0, 2, 4, 6, 1, 3, 5, 7).reshape(D ** 4, D ** 4)
    return 0.5 * (N + N.T)


def expval_matrix(T, N, Tbra=None):
    """X[pk, pb] = sum T[pk; ket] N[ket, bra] Tbra[pb; bra].  <O> = Tr(O X)/Tr X."""
    if Tbra is None:
        Tbra = T
    p = T.shape[0]
    return T.reshape(p, -1) @ N @ Tbra.reshape(p, -1).T


def cluster_2x2(env, a_ul, a_ur, a_dr, a_dl):
    """The 2 x 2 cluster of double-layer sites in its environment: the
    clockwise ring C1 E1 E1 C2 E2 E2 C3 E3 E3 C4 E4 E4 (two edge tensors on
    each side, chained previous-corner leg to next-corner leg) around the
    sites a_ul, a_ur (top row) and a_dl, a_dr (bottom row), each edge on the
    outer leg of the site it faces; neighbouring sites share their facing
    legs (a_ul.r = a_ur.l, a_ur.d = a_dr.u, a_dr.l = a_dl.r, a_dl.u = a_ul.d).
    Each quarter (one corner, its two edges, one site) is contracted first;
    the four quarters close in a ring.  The cluster of the norm network of
    Fig. 4(a,b) with its semi-infinite surroundings replaced by the CTM
    environment of Fig. 4(c)."""
    C1, C2, C3, C4 = env.C
    E1, E2, E3, E4 = env.E
    # legs: chi bonds lowercase, site legs uppercase (N, U upper-left outer;
    # V, R upper-right outer; S, P lower-right outer; Q, M lower-left outer;
    # H, J, K, I the inner bonds top, right, bottom, left)
    q_ul = np.einsum("kNl,la,aUb,NUHI->kIbH", E4, C1, E1, a_ul, optimize=True)
    q_ur = np.einsum("bVc,cd,dRe,HVRJ->bHeJ", E1, C2, E2, a_ur, optimize=True)
    q_dr = np.einsum("eSf,fg,gPh,KJSP->eJhK", E2, C3, E3, a_dr, optimize=True)
    q_dl = np.einsum("hQi,ij,jMk,MIKQ->hKkI", E3, C4, E4, a_dl, optimize=True)
    return np.einsum("kIbH,bHeJ,eJhK,hKkI->", q_ul, q_ur, q_dr, q_dl, optimize=True)


def correlation_length(env, a, direction=0):
    """Correlation length in lattice constants along the horizontal
    (direction 0) or vertical (1) axis: xi = 1 / ln|lambda_1 / lambda_2| of the
    channel transfer matrix, one row of double-layer sites between the two
    boundary edges, E1 a E3; the vertical channel is the same object in the
    frame turned by a quarter (up edge E2, down edge E4, site rotate(a, 1)), as
    in the up move of a sweep.  0 when the channel has rank one."""
    if direction == 0:
        up, dn, site = env.E[0], env.E[2], a
    else:
        up, dn, site = env.E[1], env.E[3], rotate(a, 1)
    chi, d2 = up.shape[0], a.shape[0]
    T = np.einsum("auc,lurv,dvb->albcrd", up, site, dn, optimize=True).reshape(chi * d2 * chi, -1)
    w = np.sort(np.abs(np.linalg.eigvals(T)))[::-1]
    if w[1] <= 1e-14 * w[0]:
        return 0.0
    return float(1.0 / np.log(w[0] / w[1]))


# ---------------------------------------------------------------- partition-function ratios

def kappa(env, a):
    """Free energy per site of the norm network: kappa = Z11 Z00 / (Z10 Z01)
    (site, empty ring, one column of edges, one row of edges)."""
    C1, C2, C3, C4 = env.C
    E1, E2, E3, E4 = env.E
    Z11 = np.einsum("lurd,lurd->", metric_d2(env), a)
    Z00 = np.trace(C1 @ C2 @ C3 @ C4)
    Z10 = np.einsum("ha,amb,bc,cf,fmg,gh->", C1, E1, C2, C3, E3, C4, optimize=True)
    Z01 = np.einsum("ab,bc,cmd,de,ef,fma->", C1, C2, E2, C3, C4, E4, optimize=True)
    return Z11 * Z00 / (Z10 * Z01)
