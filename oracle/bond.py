"""Environment-weighted bond update A'-B' -> A''-B'' (oracle).

Test infrastructure only (see ``oracle/__init__``).

Fig. 3(b) and Sec. III: the exact pair A'-B' (gamma bond of dimension 4D,
hidden inside the composite T') is replaced by A''-B'' with bond dimension D,
chosen to minimise the error of the whole purification.  With the CTMRG
environment metric N of one composite (a D^4 x D^4 matrix on the composite's
four outer legs, identity on the physical index), the error is

    d(A'', B'') = <T'' - T'| N |T'' - T'>,
    T''[sA,aA,sB,aB; l,u,r,d] = sum_k A''[sA,aA,u,r,k] B''[sB,aB,d,l,k].

Readings (the paper is silent; the GPU library implements the same):
* start from the truncated SVD of T' as a (4D^2) x (4D^2) matrix
  [(sA,aA,u,r), (sB,aB,d,l)], keeping D values (the N = 1 optimum);
* alternating least squares: for fixed B'' the cost is quadratic in A'',
  solved from the normal equations (R_A + delta I) A'' = S_A with
  delta = reg * tr(R_A) / dim(R_A); then the same for B'';
* stop when |d_old - d_new| / <T'|N|T'> < tol, or after max_iter sweeps;
* gauge: balanced SVD split of the bond (A'' = Q_A U sqrt(S),
  B'' = Q_B V sqrt(S) from QR factors and the SVD of R_A R_B^T), sign of each
  bond vector fixed so the largest-magnitude entry of A'' in it is positive;
  then A'', B'' scaled to unit Frobenius norm.
"""
import numpy as np


def _tpp(A2, B2):
    """T''[sA,aA,sB,aB,l,u,r,d] from A''[sA,aA,u,r,k], B''[sB,aB,d,l,k]."""
    return np.einsum("abURk,cdDLk->abcdLURD", A2, B2)


def cost_terms(A2, B2, Tp, N):
    """(<T''|N|T''>, <T''|N|T'>, <T'|N|T'>) with T' given as [16, D,D,D,D]."""
    p = 16
    T2 = _tpp(A2, B2).reshape(p, -1)
    T1 = Tp.reshape(p, -1)
    NT1 = T1 @ N
    NT2 = T2 @ N
    return float(np.sum(NT2 * T2)), float(np.sum(NT2 * T1)), float(np.sum(NT1 * T1))


def cost(A2, B2, Tp, N):
    a, b, c = cost_terms(A2, B2, Tp, N)
    return a - 2.0 * b + c, c


def svd_init(Tp, D):
    """Truncated SVD of T' as [(sA,aA,u,r), (sB,aB,d,l)] keeping D values."""
    Dv = Tp.shape[1]
    T = Tp.reshape(2, 2, 2, 2, Dv, Dv, Dv, Dv)                # [sA,aA,sB,aB,l,u,r,d]
    Mt = T.transpose(0, 1, 5, 6, 2, 3, 7, 4).reshape(4 * Dv * Dv, 4 * Dv * Dv)
    U, S, Vt = np.linalg.svd(Mt)
    k = min(D, S.size)
    A2 = np.zeros((4 * Dv * Dv, D))
    B2 = np.zeros((4 * Dv * Dv, D))
    A2[:, :k] = U[:, :k] * np.sqrt(S[:k])
    B2[:, :k] = Vt[:k].T * np.sqrt(S[:k])
    return A2.reshape(2, 2, Dv, Dv, D), B2.reshape(2, 2, Dv, Dv, D), S


def _solve_reg(R, S, reg):
    n = R.shape[0]
    delta = reg * np.trace(R) / n
    return np.linalg.solve(R + delta * np.eye(n), S)


def normal_equations_A(B2, Tp, N, D):
    """R_A[(u,r,k),(u',r',k')] and S_A[(u,r,k),(sA,aA)] for fixed B''."""
    Dv = Tp.shape[1]
    N8 = N.reshape(Dv, Dv, Dv, Dv, Dv, Dv, Dv, Dv)            # [l,u,r,d,l',u',r',d']
    T = Tp.reshape(2, 2, 2, 2, Dv, Dv, Dv, Dv)
    R = np.einsum("cdDLk,LURDMVSE,cdEMj->URkVSj", B2, N8, B2, optimize=True)
    S = np.einsum("cdDLk,LURDMVSE,abcdMVSE->URkab", B2, N8, T, optimize=True)
    m = Dv * Dv * D
    return R.reshape(m, m), S.reshape(m, 4)


def normal_equations_B(A2, Tp, N, D):
    """R_B[(d,l,k),(d',l',k')] and S_B[(d,l,k),(sB,aB)] for fixed A''."""
    Dv = Tp.shape[1]
    N8 = N.reshape(Dv, Dv, Dv, Dv, Dv, Dv, Dv, Dv)
    T = Tp.reshape(2, 2, 2, 2, Dv, Dv, Dv, Dv)
    R = np.einsum("abURk,LURDMVSE,abVSj->DLkEMj", A2, N8, A2, optimize=True)
    S = np.einsum("abURk,LURDMVSE,abcdMVSE->DLkcd", A2, N8, T, optimize=True)
    m = Dv * Dv * D
    return R.reshape(m, m), S.reshape(m, 4)


def als(Tp, N, D, tol=1e-12, max_iter=50, reg=1e-12, init=None):
    """Alternating least squares for d(A'',B'').  Returns A'', B'' in the
    composite frame ([sA,aA,u,r,k], [sB,aB,d,l,k]) and info."""
    Dv = Tp.shape[1]
    if init is None:
        A2, B2, _ = svd_init(Tp, D)
    else:
        A2, B2 = init
    d_old, ref = cost(A2, B2, Tp, N)
    history = [d_old / ref if ref != 0 else 0.0]
    it = 0
    for it in range(1, max_iter + 1):
        R, S = normal_equations_A(B2, Tp, N, D)
        X = _solve_reg(R, S, reg)                             # [(u,r,k), (sA,aA)]
        A2 = X.reshape(Dv, Dv, D, 2, 2).transpose(3, 4, 0, 1, 2).copy()
        R, S = normal_equations_B(A2, Tp, N, D)
        X = _solve_reg(R, S, reg)                             # [(d,l,k), (sB,aB)]
        B2 = X.reshape(Dv, Dv, D, 2, 2).transpose(3, 4, 0, 1, 2).copy()
        d_new, ref = cost(A2, B2, Tp, N)
        history.append(d_new / ref if ref != 0 else 0.0)
        if ref == 0 or abs(d_old - d_new) / ref < tol:
            d_old = d_new
            break
        d_old = d_new
    return A2, B2, dict(iters=it, cost=d_old, ref=ref, rel_cost=d_old / ref if ref else 0.0,
                        history=history)


def cost_gradient(A2, B2, Tp, N):
    """Gradient of d = <T''-T'|N|T''-T'> with respect to A'' and B'' (same
    shapes as A'', B'').  With B'' fixed the cost is a quadratic form in
    a = A'' as [(u,r,k),(sA,aA)]: d = tr(a^T R_A a) - 2 tr(a^T S_A) + <T'|N|T'>
    (the normal-equation matrices of the bond update), so dd/da =
    (R_A + R_A^T) a - 2 S_A; likewise for B''.  The reference for gradient
    checks of the bond cost."""
    D = A2.shape[-1]
    Dv = Tp.shape[1]
    m = Dv * Dv * D
    RA, SA = normal_equations_A(B2, Tp, N, D)
    a = A2.transpose(2, 3, 4, 0, 1).reshape(m, 4)
    gA = ((RA + RA.T) @ a - 2.0 * SA).reshape(Dv, Dv, D, 2, 2).transpose(3, 4, 0, 1, 2)
    RB, SB = normal_equations_B(A2, Tp, N, D)
    b = B2.transpose(2, 3, 4, 0, 1).reshape(m, 4)
    gB = ((RB + RB.T) @ b - 2.0 * SB).reshape(Dv, Dv, D, 2, 2).transpose(3, 4, 0, 1, 2)
    return gA, gB


def balance_gauge(A2, B2):
    """Balanced SVD split of the bond; sign and scale conventions in the
    module docstring.  T'' is unchanged up to the overall scale."""
    sh_a, sh_b = A2.shape, B2.shape
    D = sh_a[-1]
    Am = A2.reshape(-1, D)
    Bm = B2.reshape(-1, D)
    Qa, Ra = np.linalg.qr(Am)
    Qb, Rb = np.linalg.qr(Bm)
    U, S, Vt = np.linalg.svd(Ra @ Rb.T)
    An = Qa @ (U * np.sqrt(S))
    Bn = Qb @ (Vt.T * np.sqrt(S))
    for j in range(D):
        i = np.argmax(np.abs(An[:, j]))
        if An[i, j] < 0:
            An[:, j] *= -1
            Bn[:, j] *= -1
    na, nb = np.linalg.norm(An), np.linalg.norm(Bn)
    if na > 0:
        An /= na
    if nb > 0:
        Bn /= nb
    return An.reshape(sh_a), Bn.reshape(sh_b), S
