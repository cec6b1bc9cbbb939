"""Kernel-level GPU tests through the self-test entry points: the contraction
GEMM (every precision built) and the Jacobi eigensolver against numpy in
float64, on ragged shapes that span several tiles."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1906_02220_gb300 as pkg
    return pkg


GEMM_TOL = {"fp64": 1e-13, "fp32": 3e-6, "tf32": 4e-3, "tf32x3": 1e-5}


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (16, 16, 16), (17, 33, 65), (128, 16, 256), (16, 128, 40),
                                   (300, 257, 129), (1024, 96, 1024), (80, 80, 1000), (64, 64, 2048)])
def test_gemm_against_numpy(g, prec, M, N, K):
    import torch
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((K, N))
    C = g.selftest_gemm(torch.as_tensor(A, device="cuda:0"), torch.as_tensor(B, device="cuda:0"), prec).cpu().numpy()
    ref = A @ B
    scale = np.sqrt(K) * np.abs(A).max() * np.abs(B).max()
    assert np.abs(C - ref).max() <= GEMM_TOL[prec] * scale


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("k", [1, 2, 7, 24, 64, 81, 112, 160])
def test_jacobi_symeig(g, prec, k):
    import torch
    if prec == "fp64" and k > 112:
        pytest.skip("beyond the FP64 Jacobi limit")
    rng = np.random.default_rng(k)
    Q, _ = np.linalg.qr(rng.standard_normal((k, k)))
    lam = np.sort(np.abs(rng.standard_normal(k)) * np.logspace(0, -6, k))[::-1]
    lam[k // 2:] = 0.0 if k > 3 else lam[k // 2:]          # a null block
    G = (Q * lam) @ Q.T
    G = 0.5 * (G + G.T)
    E, W = g.selftest_symeig(torch.as_tensor(G, device="cuda:0"), prec)
    E, W = E.cpu().numpy(), W.cpu().numpy()
    eps = 1e-15 if prec == "fp64" else 3e-7
    ref = np.sort(np.linalg.eigvalsh(G))[::-1]
    assert np.all(np.diff(E) <= 0)
    assert np.abs(E - ref).max() <= 50 * eps * k * lam.max()
    assert np.abs(W.T @ W - np.eye(k)).max() <= 50 * eps * k
    assert np.abs(W @ np.diag(E) @ W.T - G).max() <= 50 * eps * k * lam.max()


def test_jacobi_near_diagonal_relative_accuracy(g):
    """Warm-start regime: a near-diagonal Gram matrix with a 1e-10 dynamic range
    keeps every eigenvalue to high relative accuracy, even in FP32."""
    import torch
    k = 80
    rng = np.random.default_rng(3)
    d = np.logspace(0, -10, k)
    G = np.diag(d) + 1e-4 * np.sqrt(np.outer(d, d)) * rng.standard_normal((k, k))
    G = 0.5 * (G + G.T)
    ref = np.sort(np.linalg.eigvalsh(G))[::-1]
    for prec, tol in (("fp64", 1e-12), ("fp32", 2e-5)):
        E, W = g.selftest_symeig(torch.as_tensor(G, device="cuda:0"), prec)
        assert np.max(np.abs(E.cpu().numpy() - ref) / ref) < tol


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("k,decades", [(1, 0), (6, 3), (24, 9), (40, 6), (45, 6), (57, 6), (80, 12), (90, 6),
                                       (100, 8), (111, 7), (112, 6), (113, 6), (150, 6), (160, 6)])
def test_one_sided_jacobi_svd(g, prec, k, decades):
    """Singular values to absolute accuracy ~eps * s_1 (no squaring), also for
    a matrix with a null block; X Q = L S and Q orthogonal.  k = 45 in FP64
    needs 47 KB of dynamic on top of the kernel's static shared memory (the
    48 KB default covers both); k = 112 in FP64 and k = 160 in FP32 are the
    largest sizes the library accepts (about 200 KB each)."""
    import torch
    if prec == "fp64" and k > 112:
        pytest.skip("beyond the FP64 Jacobi limit")
    rng = np.random.default_rng(k + decades)
    U, _ = np.linalg.qr(rng.standard_normal((k, k)))
    V, _ = np.linalg.qr(rng.standard_normal((k, k)))
    s = np.logspace(0, -decades, k)
    s[(3 * k) // 4:] = 0.0 if k > 4 else s[(3 * k) // 4:]
    X = (U * s) @ V.T
    S, L, Q = (t.cpu().numpy() for t in g.selftest_svd(torch.as_tensor(X, device="cuda:0"), prec))
    eps = 2.3e-16 if prec == "fp64" else 1.2e-7
    ref = np.linalg.svd(X, compute_uv=False)
    assert np.abs(S - ref).max() <= 30 * eps * k * s[0]
    assert np.abs(Q.T @ Q - np.eye(k)).max() <= 30 * eps * k
    assert np.abs(X @ Q - L * S).max() <= 30 * eps * k * s[0]


@pytest.mark.parametrize("k,decades", [(1, 0), (24, 3), (80, 6), (113, 4), (160, 6)])
def test_fp32_svd_with_fp64_refinement(g, k, decades):
    """FP32 one-sided Jacobi plus three FP64 Newton steps: singular vectors
    orthonormal to FP64 rounding, X Q = L S to FP64 rounding where the FP32
    result already separated the singular values (their gap above ~1e-4 s_1,
    far beyond the FP32 error ~k 2^-24 s_1), and never worse than the FP32
    solver elsewhere (pairs whose gap is below 64 times their coupling are only
    re-orthogonalised)."""
    import torch
    rng = np.random.default_rng(3 * k + decades)
    U, _ = np.linalg.qr(rng.standard_normal((k, k)))
    V, _ = np.linalg.qr(rng.standard_normal((k, k)))
    s = np.logspace(0, -decades, k)
    X = (U * s) @ V.T
    S, L, Q = (t.cpu().numpy() for t in g.selftest_svd_refined(torch.as_tensor(X, device="cuda:0")))
    eps64, eps32 = 2.3e-16, 1.2e-7
    assert np.abs(Q.T @ Q - np.eye(k)).max() <= 1e3 * eps64 * k
    assert np.abs(L.T @ L - np.eye(k)).max() <= 1e3 * eps64 * k
    ref = np.linalg.svd(X, compute_uv=False)
    gaps = np.minimum(np.r_[np.inf, -np.diff(ref)], np.r_[-np.diff(ref), np.inf])
    sep = gaps > 1e-4 * s[0]
    assert np.abs(S - ref)[sep].max(initial=0.0) <= 1e3 * eps64 * k * s[0]
    assert np.abs(S - ref).max() <= 30 * eps32 * k * s[0]
    resid = np.abs(X @ Q - L * S).max(axis=0)
    assert resid[sep].max(initial=0.0) <= 1e3 * eps64 * k * s[0]


def test_fp64_newton_reciprocals_match_ieee(g):
    """The FP64 reciprocal / reciprocal square root / square root used by the
    latency-bound FP64 kernels (Newton-Raphson from FP32 estimates) agree with
    the correctly rounded IEEE results to 2 ulp, also at the edges of the FP32
    range where they fall back to the IEEE operations."""
    import torch
    rng = np.random.default_rng(5)
    x = np.concatenate([10.0 ** rng.uniform(-29, 29, 4000), rng.uniform(0.5, 2.0, 1000),
                        [1.0, 2.0, 3.0, 1e-31, 1e31, 1e-300, 1e300, 5e-324, 2.0 ** -1022]])
    xs = np.concatenate([x, -x[:100]])
    r, rs, sq = (t.cpu().numpy() for t in g.selftest_fp64_newton(torch.as_tensor(xs, device="cuda:0")))
    ulp = 2.3e-16
    with np.errstate(over="ignore", divide="ignore"):
        ref = 1.0 / xs
    fin = np.isfinite(ref)
    assert np.all(np.abs(r[fin] / ref[fin] - 1.0) <= 2 * ulp)
    assert np.all(r[~fin] == ref[~fin])
    pos = xs > 0
    assert np.all(np.abs(rs[pos] / (1.0 / np.sqrt(xs[pos])) - 1.0) <= 2 * ulp)
    assert np.all(np.abs(sq[pos] / np.sqrt(xs[pos]) - 1.0) <= 2 * ulp)
    assert np.all(rs[~pos] == 0.0) and np.all(sq[~pos] == 0.0)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n,k,decades", [(1, 1, 0), (37, 5, 2), (200, 33, 8), (300, 76, 5),
                                         (400, 54, 5), (700, 90, 7), (1024, 80, 6), (300, 160, 4)])
def test_cholqr2_orthonormal_basis(g, prec, n, k, decades):
    """Ordered CholQR2 on graded columns with an exactly dependent and a zero
    column: the kept columns are orthonormal, the dropped ones exactly zero,
    their number equals the rank, span(Q) holds every column of Y, and the
    first column lies along the largest column of Y.  At (400, 54, 5) and
    (700, 90, 7) the dependent column is nearly parallel to column 0 (residual
    ~1e-5 of its norm) and sorts right after it: without deferring that pivot
    the FP64 span error grows to ~eps ||Y|| / 1e-5 and breaks the bound."""
    import torch
    if prec == "fp64" and k > 112:
        pytest.skip("beyond the FP64 Jacobi limit")
    rng = np.random.default_rng(n + k)
    Y = rng.standard_normal((n, k)) * np.logspace(0, -decades, k)[rng.permutation(k)]
    rank = min(n, k)
    if k > 4 and n > k:
        Y[:, k - 1] = Y[:, 0] + 0.5 * Y[:, 1]
        Y[:, k - 2] = 0.0
        rank = k - 2
    Q = g.selftest_orth(torch.as_tensor(Y, device="cuda:0"), prec).cpu().numpy()
    eps = 2.3e-16 if prec == "fp64" else 1.2e-7
    norms = np.linalg.norm(Q, axis=0)
    live = norms > 0.5
    assert np.all(norms[~live] == 0.0)
    assert live.sum() == rank
    Ql = Q[:, live]
    assert np.abs(Ql.T @ Ql - np.eye(rank)).max() <= 50 * eps * k
    assert np.abs(Y - Ql @ (Ql.T @ Y)).max() <= 1e3 * eps * np.abs(Y).max()
    j0 = np.argmax(np.linalg.norm(Y, axis=0))
    assert abs(Q[:, 0] @ Y[:, j0]) / np.linalg.norm(Y[:, j0]) > 1 - 1e3 * eps


@pytest.mark.parametrize("prec", ["tf32", "tf32x3"])
@pytest.mark.parametrize("M,N,K", [(128, 128, 32), (256, 256, 16), (200, 300, 96), (512, 16, 256),
                                   (130, 40, 1028), (1024, 1024, 1024)])
def test_tensor_core_gemm(g, prec, M, N, K):
    """tcgen05 GEMM (TMA + TMEM) against numpy: ragged M/N tiles, K below one
    32-wide K block (zero-filled by TMA), N = 16 tiles, K spanning many stages.
    TF32 bound: operand truncation 2^-10 each, random-sign accumulation."""
    import torch
    rng = np.random.default_rng(M + 3 * N + 7 * K)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((K, N))
    C = g.selftest_gemm(torch.as_tensor(A, device="cuda:0"), torch.as_tensor(B, device="cuda:0"), prec).cpu().numpy()
    ref = A @ B
    scale = np.sqrt(K) * np.abs(A).max() * np.abs(B).max()
    err = np.abs(C - ref).max()
    assert err <= GEMM_TOL[prec] * scale, (err, scale)


def _frame_tensor(T, f):
    """Site tensor [p][l][u][r][d] seen from frame f: each quarter turn makes
    the new legs (l, u, r, d) the old (d, l, u, r)."""
    for _ in range(f):
        T = T.transpose(0, 2, 3, 4, 1)
    return T


def _layer_operand(T, kind, f):
    """TL[in][p][out]: corner (kind 0) in = (l, u), out = (r, d); edge (kind 1)
    in = (l, d), out = (u, r)."""
    Tf = _frame_tensor(T, f)
    p, D = T.shape[0], T.shape[1]
    axes = (1, 2, 0, 3, 4) if kind == 0 else (1, 4, 0, 2, 3)
    return np.ascontiguousarray(Tf.transpose(axes)).reshape(D * D, p, D * D)


# (npass, D, p, kind, frame, nb): several tiles per CTA with a ragged last
# tile (128 // D^2 blocks per tile), streamed and resident operand images,
# chunks of the physical index that p does not fill
LAYERED_CASES = [
    (3, 4, 16, 0, 0, 8 * 300 + 5), (3, 4, 16, 1, 1, 37), (3, 2, 16, 0, 2, 32 * 200 + 7),
    (3, 3, 16, 1, 3, 14 * 160 + 3), (3, 5, 16, 0, 1, 5 * 170 + 2), (3, 6, 16, 1, 0, 3 * 170 + 1),
    (3, 7, 16, 0, 3, 2 * 160 + 1), (3, 8, 16, 1, 2, 2 * 160 + 1), (1, 4, 16, 0, 0, 8 * 200 + 3),
    (1, 6, 16, 0, 1, 3 * 100 + 2), (3, 4, 3, 0, 1, 100), (3, 6, 5, 0, 0, 200), (3, 1, 2, 1, 0, 300),
    # BF16 (npass 16): one pass of kind::f16
    (16, 4, 16, 0, 0, 8 * 300 + 5), (16, 6, 16, 1, 2, 3 * 170 + 1), (16, 3, 5, 0, 3, 14 * 20 + 3),
    (16, 8, 16, 1, 1, 2 * 160 + 1), (16, 2, 16, 0, 0, 32 * 30 + 7),
]


@pytest.mark.parametrize("npass,D,p,kind,frame,nb", LAYERED_CASES)
def test_layered_site_contraction(g, npass, D, p, kind, frame, nb):
    """The layered tensor-core contraction against an FP64 einsum of the same
    ket-then-bra network (Fig. 4), elementwise within the TF32, 3xTF32 or
    BF16 error bound relative to the contraction of absolute values."""
    import torch
    rng = np.random.default_rng(1000 * D + 10 * p + nb)
    T = rng.standard_normal((p, D, D, D, D))
    Y = rng.standard_normal((nb, D * D, D * D))
    out = g.selftest_site_layered(torch.as_tensor(T, device="cuda:0"), torch.as_tensor(Y, device="cuda:0"),
                                  kind=kind, frame=frame, npass=npass).cpu().numpy()
    TL = _layer_operand(T, kind, frame)
    ref = np.einsum("ipo,bji,jpq->boq", TL, Y, TL, optimize=True)
    scale = np.einsum("ipo,bji,jpq->boq", np.abs(TL), np.abs(Y), np.abs(TL), optimize=True)
    # 3xTF32: FP32-level; TF32: 2^-11 per rounded factor; BF16: the operands Y,
    # T and the intermediate Z each rounded to 8 bits (u = 2^-9), so about 4u
    tol = {3: 1e-5, 1: 3e-3, 16: 8e-3}[npass]
    assert np.all(np.abs(out - ref) <= tol * scale + 1e-30)
