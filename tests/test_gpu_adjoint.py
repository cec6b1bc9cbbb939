"""The hand-written adjoint of the eeFU bond cost (Fig. 3(b)):
d(A'', B'') = <T''-T'|N|T''-T'> and its gradient from eefu_cost_gradient,
against the oracle's FP64 gradient (``bond.cost_gradient``), against central
differences of the library's own cost with the environment fixed, through
torch.autograd, and driving a gradient-based bond optimisation."""
import numpy as np
import pytest

import kh_inputs
from oracle import bond, ctmrg, model, peps

pytestmark = pytest.mark.gpu

GAMMA = {"x": 0, "y": 1, "z": 2}


@pytest.fixture(scope="module")
def g():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1906_02220_gb300 as pkg
    return pkg


def _t(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda:0")


# projector cut-off of each precision, the same on both sides (the library's
# single-precision default)
CUT = {"fp64": 1e-12, "tf32x3": 1e-4}


def _setup(D, chi, gamma, seed, prec="fp64"):
    """A random state, the gate of gamma at phi = 0.3 pi, the oracle's T' and
    converged N (at the precision's cut-off), and trial factors: the truncated
    SVD start of T' plus 20 % noise (so the gradient is far from zero)."""
    J, K = model.couplings(0.3 * np.pi)
    A, B = kh_inputs.random_site_tensors(D, seed)
    gt = model.gate(gamma, 0.01, J, K)
    Tp = peps.composite(A, B, gamma, gt)
    env, _ = ctmrg.ctmrg(ctmrg.double_tensor(Tp), ctmrg.init_env(chi, D), 1e-12, 400, 1, CUT[prec])
    N = ctmrg.metric(env, D)
    A2, B2, _ = bond.svd_init(Tp, D)
    rng = np.random.default_rng(seed + 100)
    A2 = A2 + 0.2 * np.abs(A2).max() * rng.standard_normal(A2.shape)
    B2 = B2 + 0.2 * np.abs(B2).max() * rng.standard_normal(B2.shape)
    return A, B, gt, Tp, N, A2, B2


@pytest.mark.parametrize("gamma", ["x", "z"])
@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_cost_gradient_matches_oracle(g, gamma, prec):
    """dd/dA'' and dd/dB'' of the library against the oracle's FP64 gradient
    (same state, gate and trial factors; each side converges its own
    environment at the same cut-off): FP64 to 1e-8 of the gradient's scale,
    3xTF32 (metric from single-precision contractions) to 2e-4, the metric's
    own single-precision parity bound."""
    D, chi = 2, 8
    A, B, gt, Tp, N, A2, B2 = _setup(D, chi, gamma, seed=11, prec=prec)
    gA_ref, gB_ref = bond.cost_gradient(A2, B2, Tp, N)
    d_ref, c_ref = bond.cost(A2, B2, Tp, N)
    ctx = g.Context(D, chi, prec, svd_cut=CUT[prec])
    ctx.set_state(_t(A), _t(B))
    gA, gB, d, c = ctx.cost_gradient(GAMMA[gamma], gt, _t(A2), _t(B2), ctm_max_sweeps=400, ctm_tol=1e-12
                                     if prec == "fp64" else 1e-7)
    tol = 1e-8 if prec == "fp64" else 2e-4
    scale = max(np.abs(gA_ref).max(), np.abs(gB_ref).max())
    assert np.abs(gA.cpu().numpy() - gA_ref).max() < tol * scale
    assert np.abs(gB.cpu().numpy() - gB_ref).max() < tol * scale
    assert abs(d - d_ref) < tol * c_ref
    assert abs(c - c_ref) < tol * c_ref
    ctx.close()


def test_cost_gradient_central_differences(g):
    """With the environment fixed (ctm_max_sweeps = 0 after one converged
    call) d is a quadratic form in each factor, so the central difference
    along any direction equals the directional derivative up to rounding."""
    D, chi = 3, 12
    A, B, gt, Tp, N, A2, B2 = _setup(D, chi, "y", seed=4)
    ctx = g.Context(D, chi, "fp64")
    ctx.set_state(_t(A), _t(B))
    gA, gB, d0, c = ctx.cost_gradient(1, gt, _t(A2), _t(B2), ctm_max_sweeps=400, ctm_tol=1e-12)
    rng = np.random.default_rng(0)
    h = 1e-6
    for _ in range(4):
        eA = rng.standard_normal(A2.shape)
        eA /= np.linalg.norm(eA)
        eB = rng.standard_normal(B2.shape)
        eB /= np.linalg.norm(eB)
        _, _, dp, _ = ctx.cost_gradient(1, gt, _t(A2 + h * eA), _t(B2 + h * eB), ctm_max_sweeps=0)
        _, _, dm, _ = ctx.cost_gradient(1, gt, _t(A2 - h * eA), _t(B2 - h * eB), ctm_max_sweeps=0)
        fd = (dp - dm) / (2 * h)
        an = float((gA.cpu().numpy() * eA).sum() + (gB.cpu().numpy() * eB).sum())
        assert abs(fd - an) < 1e-6 * max(1.0, abs(an)) * c, (fd, an)
    ctx.close()


def test_bond_cost_autograd_and_gradient_descent(g):
    """The cost as a torch.autograd.Function: backward returns the library's
    gradient, and plain gradient descent with a backtracking step (N fixed)
    lowers the cost monotonically, most of the way to the cost the ALS
    update reaches."""
    import torch
    D, chi = 2, 8
    A, B, gt, Tp, N, A2, B2 = _setup(D, chi, "x", seed=3)
    ctx = g.Context(D, chi, "fp64")
    ctx.set_state(_t(A), _t(B))
    gA_lib, gB_lib, d0, c = ctx.cost_gradient(0, gt, _t(A2), _t(B2), ctm_max_sweeps=400, ctm_tol=1e-12)
    a = _t(A2).requires_grad_(True)
    b = _t(B2).requires_grad_(True)
    d = g.bond_cost(ctx, 0, gt, a, b)
    d.backward()
    assert abs(float(d.detach()) - d0) < 1e-12 * c
    assert torch.allclose(a.grad, gA_lib, rtol=0, atol=1e-14 * float(gA_lib.abs().max()))
    assert torch.allclose(b.grad, gB_lib, rtol=0, atol=1e-14 * float(gB_lib.abs().max()))
    # gradient descent on (A'', B'') with backtracking (Armijo)
    x = [_t(A2), _t(B2)]
    cur = float(g.bond_cost(ctx, 0, gt, *x))
    step = 1.0 / c
    hist = [cur]
    for _ in range(60):
        xa = x[0].clone().requires_grad_(True)
        xb = x[1].clone().requires_grad_(True)
        dd = g.bond_cost(ctx, 0, gt, xa, xb)
        dd.backward()
        gn2 = float((xa.grad ** 2).sum() + (xb.grad ** 2).sum())
        while True:
            ya = x[0] - step * xa.grad
            yb = x[1] - step * xb.grad
            new = float(g.bond_cost(ctx, 0, gt, ya, yb))
            if new <= cur - 0.25 * step * gn2 or step < 1e-30:
                break
            step *= 0.5
        x = [ya, yb]
        cur = new
        hist.append(cur)
        step *= 2.0
    assert all(h1 <= h0 for h0, h1 in zip(hist, hist[1:]))
    # most of the way from the start to the cost the ALS reaches (oracle)
    A_opt, B_opt, _ = bond.als(Tp, N, D, 1e-14, 200, 1e-12)
    d_opt, _ = bond.cost(A_opt, B_opt, Tp, N)
    assert hist[-1] - d_opt < 0.5 * (hist[0] - d_opt), (hist[0], hist[-1], d_opt)
    ctx.close()
