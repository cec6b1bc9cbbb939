"""Batched trajectories (many coupling angles advanced concurrently,
eefu_evolve_batch): every problem of a batch agrees with the oracle's
trajectory for its own couplings (Sec. III, Eq. 6), and with the same problem
run alone."""
import numpy as np
import pytest

import kh_inputs
from oracle import eefu, model

pytestmark = pytest.mark.gpu


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


def _contexts(g, n, D, chi, prec, A, B, **kw):
    out = []
    for _ in range(n):
        c = g.Context(D, chi, prec, **kw)
        c.set_state(_t(A), _t(B))
        out.append(c)
    return out


PHIS = [0.1 * np.pi, 0.3 * np.pi, 0.75 * np.pi, 1.5 * np.pi]


def test_batch_matches_oracle_per_problem(g):
    """Four coupling angles phi (J = cos phi, K = 2 sin phi) with a bias, D = 2,
    chi = 8, FP64: each problem's rows match the oracle's evolution of the
    same start state under its own couplings."""
    A, B = kh_inputs.perturbed_product_state(2, seed=7, eps=0.05)
    dbeta, n, hA, hB = 0.02, 4, 0.1, -0.05
    ctxs = _contexts(g, len(PHIS), 2, 8, "fp64", A, B)
    Js, Ks = zip(*[model.couplings(phi) for phi in PHIS])
    trajs = g.evolve_batch(ctxs, Js, [[k, k, k] for k in Ks], dbeta, n, 1, hA=[hA] * len(PHIS), hB=[hB] * len(PHIS),
                           ctm_max_sweeps=300, ctm_tol=1e-12)
    for J, K, traj in zip(Js, Ks, trajs):
        prm = eefu.Params(D=2, chi=8, J=J, K=K, hA=hA, hB=hB, ctm_tol=1e-12, ctm_max_sweeps=300)
        ref = eefu.evolve(eefu.State(A, B, prm), dbeta, n, measure_every=1)
        assert len(traj) == n
        for r, o in zip(traj, ref):
            assert abs(r["beta"] - o["beta"]) < 1e-12
            for key in ("E_site", "Hx", "Hy", "Hz", "Ax", "Az", "Bx", "Bz"):
                assert abs(r[key] - o[key]) < 1e-9 * max(1.0, abs(o[key])), (J, K, key, r[key], o[key])
    for c in ctxs:
        c.close()


@pytest.mark.parametrize("prec", ["tf32x3"])
def test_batch_matches_single_runs(g, prec):
    """The bench-sized problem (D = 4, chi = 32) at four angles: the batch
    gives each problem the trajectory it has when run alone (the FP64
    atomics of the Gram accumulation differ in order only: 1e-6 relative)."""
    A, B = kh_inputs.perturbed_product_state(4, seed=3, eps=0.05)
    dbeta, n = 0.01, 2
    Js, Ks = zip(*[model.couplings(phi) for phi in PHIS])
    Kx = [[k, k, k] for k in Ks]
    ctxs = _contexts(g, len(PHIS), 4, 32, prec, A, B)
    batch = g.evolve_batch(ctxs, Js, Kx, dbeta, n, 1, ctm_max_sweeps=6, ctm_min_sweeps=6, ctm_tol=-1.0)
    for c in ctxs:
        c.close()
    for J, Kv, traj in zip(Js, Kx, batch):
        c = _contexts(g, 1, 4, 32, prec, A, B)[0]
        alone = c.evolve(J, Kv, dbeta, n, 1, ctm_max_sweeps=6, ctm_min_sweeps=6, ctm_tol=-1.0)
        c.close()
        for r, o in zip(traj, alone):
            for key in ("E_site", "Hx", "Hy", "Hz", "Ax", "Az", "Bx", "Bz"):
                assert abs(r[key] - o[key]) < 1e-6 * max(1.0, abs(o[key])), (J, key, r[key], o[key])


def test_batch_refuses_a_context_twice(g):
    """One host thread per context: a batch naming a context twice is refused
    (KH_EINVAL, nothing runs); the same contexts once each run to the end."""
    A, B = kh_inputs.perturbed_product_state(2, seed=1, eps=0.05)
    ctxs = _contexts(g, 2, 2, 8, "fp64", A, B)
    with pytest.raises(g.KhError):
        g.evolve_batch([ctxs[0], ctxs[0]], [0.0, 0.0], [[1, 1, 1]] * 2, 0.01, 1)   # same context twice
    trajs = g.evolve_batch(ctxs, [0.0, 0.0], [[1, 1, 1]] * 2, 0.01, 2, ctm_max_sweeps=50, ctm_tol=1e-10)
    assert len(trajs) == 2 and all(len(t) == 2 for t in trajs)
    for c in ctxs:
        c.close()
