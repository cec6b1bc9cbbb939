"""The 2 x 2 plaquette cluster and the plaquette flux W (Sec. V) on the GPU
(ctm_plaquette, ctm_flux through the C ABI) against the oracle's explicit
cluster contraction (``ctmrg.cluster_2x2``, ``observables.flux``).

The library's contraction is compared on the library's own converged
environment (its FP64 masters read back), so the test isolates the cluster:
the four enlarged corners with operators on their ket layers, closed in a
ring.  Error model: a cluster is a sum of products whose rounding errors are
bounded relative to the same sum taken over absolute values, so the
tolerance of a cluster value is U x cond with cond = |cluster| of the
absolute values / |cluster| (computed by the oracle on the same
environment) and U per arithmetic: FP64 1e-13; FP32 and 3xTF32 1e-5
(2^-24 times sqrt(K) for the longest sums, K = chi D^2 <= 256, and a
safety factor); one TF32 pass 3e-3 (operands rounded to 2^-11); BF16 2.5e-2
(operands and the layer intermediate rounded to 2^-8).  The operators are
the identity plus N(0, 1/4p) noise: each position's operator shows, and
cond stays below ~10."""
import numpy as np
import pytest

import kh_inputs
from oracle import ctmrg, observables, peps

pytestmark = pytest.mark.gpu

U = {"fp64": 1e-13, "fp32": 1e-5, "tf32x3": 1e-5, "tf32": 3e-3, "bf16": 2.5e-2}
CTM_TOL = {"fp64": 1e-12, "fp32": 1e-7, "tf32x3": 1e-7, "tf32": 1e-5, "bf16": 1e-4}


@pytest.fixture(scope="module")
def g():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1906_02220_gb300 as pkg
    return pkg


def _t(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda:0")


def _gpu_env(ctx, slot, D, chi):
    C, E = ctx.ctm_get_env(slot)
    return ctmrg.Env(list(C.cpu().numpy().reshape(4, chi, chi)), list(E.cpu().numpy().reshape(4, chi, D * D, chi)))


def _ops(p, seed):
    rng = np.random.default_rng(seed)
    return np.stack([np.eye(p) + 0.5 / np.sqrt(p) * rng.standard_normal((p, p)) for _ in range(4)])


def _cond(env, T, ops):
    """(cluster, cond) of the cluster with ket layers ops_f T: cond = the
    cluster of absolute values over |cluster|."""
    p = T.shape[0]
    Tc = T.astype(np.complex128)
    sites = [ctmrg.double_tensor((np.asarray(O) @ Tc.reshape(p, -1)).reshape(T.shape), Tc) for O in ops]
    z = ctmrg.cluster_2x2(env, *sites)
    ae = ctmrg.Env([np.abs(c) for c in env.C], [np.abs(e) for e in env.E])
    return z, ctmrg.cluster_2x2(ae, *[np.abs(x) for x in sites]) / abs(z)


@pytest.mark.parametrize("prec,D,chi,p", [("fp64", 2, 12, 4), ("fp64", 3, 8, 16), ("fp32", 2, 12, 4),
                                          ("tf32x3", 2, 12, 16), ("tf32x3", 4, 16, 16), ("tf32", 4, 16, 16),
                                          ("bf16", 4, 16, 16), ("tf32x3", 4, 64, 16)])
def test_plaquette_matches_oracle_on_the_library_environment(g, prec, D, chi, p):
    """Generic composite: <O_0 O_1 O_2 O_3> and the plain cluster against the
    oracle's cluster in the same environment.  The tensor-core precisions run
    the layered site contraction with a dressed ket image and a plain bra
    image; (4, 16) spans two 128-row tiles of chi^2 = 256 blocks, (4, 64) is
    the timed workload's size (n = chi D^2 = 1024, 32 tiles)."""
    T = kh_inputs.random_composite(D, 40 + D, p=p)
    ctx = g.Context(D, chi, prec, n_slots=1)
    ctx.ctm_set_tensor(0, _t(T))
    ctx.ctm_sweep(0, 200, 3, CTM_TOL[prec], allow_noconv=True)
    env = _gpu_env(ctx, 0, D, chi)
    ops = _ops(p, 5)
    val, z = ctx.ctm_plaquette(0, ops)
    ref = observables.plaquette_expectation(env, T, ops)
    zref, c1 = _cond(env, T, np.stack([np.eye(p)] * 4))
    _, cO = _cond(env, T, ops)
    assert cO < 20 and c1 < 20
    assert abs(ref.imag) < 1e-14
    assert abs(val - ref.real) < U[prec] * (cO + c1) * abs(ref.real), (val, ref, cO, c1)
    assert abs(z - zref.real) < U[prec] * c1 * abs(zref), (z, zref, c1)
    # identity operators give exactly one (same kernels for both clusters)
    one, _ = ctx.ctm_plaquette(0, np.stack([np.eye(p)] * 4))
    assert abs(one - 1.0) < 1e-12
    ctx.close()


def test_plaquette_single_operator_and_pairs_on_the_ising_network(g):
    """The Ising PEPS (p = 2): a sigma^z pair on the horizontal neighbours of
    the plaquette is the horizontal nearest-neighbour correlator, on the
    vertical neighbours the vertical one, and the two differ (anisotropic
    couplings) -- the library's positions are the oracle's."""
    from oracle import exact
    Kh, Kv = 0.3, 0.2
    h = 1e-5
    dh = (exact.onsager_lnZ(Kh + h, Kv) - exact.onsager_lnZ(Kh - h, Kv)) / (2 * h)
    dv = (exact.onsager_lnZ(Kh, Kv + h) - exact.onsager_lnZ(Kh, Kv - h)) / (2 * h)
    T = exact.ising_peps(Kh, Kv, gauge_seed=7)
    ctx = g.Context(2, 24, "fp64", n_slots=1, p_max=2)
    ctx.ctm_set_tensor(0, _t(T))
    ctx.ctm_sweep(0, 400, 3, 1e-13, allow_noconv=True)
    sz = np.diag([1.0, -1.0])
    for (i, j), want in (((0, 1), dh), ((3, 2), dh), ((0, 3), dv), ((1, 2), dv)):
        ops = np.stack([np.eye(2)] * 4)
        ops[i] = sz
        ops[j] = sz
        val, _ = ctx.ctm_plaquette(0, ops)
        assert abs(val - want) < 1e-9, (i, j, val, want)
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_flux_matches_oracle_in_every_mapping(g, prec):
    """<W_p> of a random D = 2 state (|W| ~ 7e-3, cond ~ 30) from the
    composite of each mapping (slots 3 + gamma, as observables() leaves
    them): against the oracle's flux on the same environment (tolerance
    U x cond), and the three mappings against each other (three placements
    of the hexagon, three networks; FP64 1e-6 relative, the environments'
    own convergence)."""
    D, chi = 2, 16
    A, B = kh_inputs.random_site_tensors(D, 36)
    ctx = g.Context(D, chi, prec)
    ctx.set_state(_t(A), _t(B))
    w = []
    for gi, gamma in enumerate("xyz"):
        ctx.ctm_build_composite(3 + gi, gamma)
        ctx.ctm_init(3 + gi)
        ctx.ctm_sweep(3 + gi, 300, 3, CTM_TOL[prec], allow_noconv=True)
        val = ctx.flux(gamma)
        env = _gpu_env(ctx, 3 + gi, D, chi)
        T = peps.composite(A, B, gamma)
        ref = observables.flux(env, T, gamma)
        _, cW = _cond(env, T, observables.flux_operators(gamma))
        _, c1 = _cond(env, T, [np.eye(16)] * 4)
        assert abs(ref.imag) < 1e-15
        assert abs(val - ref.real) < U[prec] * (cW + c1) * abs(ref.real), (gamma, val, ref, cW)
        w.append(val)
    assert min(abs(x) for x in w) > 1e-3
    rel = 1e-6 if prec == "fp64" else 2e-4
    assert max(w) - min(w) < rel * max(abs(x) for x in w), w
    ctx.close()


def test_flux_after_observables_and_argument_checks(g):
    """After observables() the flux of each mapping is read from slot
    3 + gamma; a slot without a composite tensor (p != 16) and a gamma outside
    0..2 are rejected with KH_EINVAL."""
    D, chi = 2, 12
    A, B = kh_inputs.random_site_tensors(D, 6)
    ctx = g.Context(D, chi, "fp64")
    ctx.set_state(_t(A), _t(B))
    Hs = [g.bond_hamiltonian(gm, 0.0, 1.0) for gm in "xyz"]
    ctx.observables(Hs, ctm_max_sweeps=400, ctm_tol=1e-10)
    w = [ctx.flux(gm) for gm in "xyz"]
    ref = observables.flux(_gpu_env(ctx, 5, D, chi), peps.composite(A, B, "z"), "z").real
    assert abs(w[2] - ref) < 1e-10 * abs(ref)
    assert max(w) - min(w) < 1e-6 * max(abs(x) for x in w), w
    with pytest.raises(g.KhError) as e:
        ctx.flux(3, slot=3)
    assert e.value.status == g.KH_EINVAL
    T = kh_inputs.random_composite(D, 3, p=4)
    ctx.ctm_set_tensor(0, _t(T))
    ctx.ctm_init(0)
    with pytest.raises(g.KhError) as e:
        ctx.flux("x", slot=0)
    assert e.value.status == g.KH_EINVAL
    ctx.close()


def test_trajectory_with_flux(g):
    """eefu_evolve_flux: the same rows as eefu_evolve (the flux reads the
    environments and changes nothing), and in every row the flux of the z
    mapping's observables environment at that point: the last one equal to
    ctm_flux afterwards and to the oracle's cluster on the library's
    environment and state."""
    from oracle import model
    J, K = model.couplings(0.3 * np.pi)
    D, chi = 2, 8
    A, B = kh_inputs.random_site_tensors(D, 36)
    kw = dict(ctm_max_sweeps=300, ctm_tol=1e-12)
    c1 = g.Context(D, chi, "fp64")
    c1.set_state(_t(A), _t(B))
    t1 = c1.evolve(J, [K, K, K], 0.02, 4, 2, flux=True, **kw)
    c2 = g.Context(D, chi, "fp64")
    c2.set_state(_t(A), _t(B))
    t2 = c2.evolve(J, [K, K, K], 0.02, 4, 2, **kw)
    assert len(t1) == 2 and all("W" in r for r in t1)
    for r1, r2 in zip(t1, t2):
        for key in ("beta", "E_site", "Hx", "Hy", "Hz", "Ax", "Az", "Bx", "Bz"):
            assert abs(r1[key] - r2[key]) < 1e-10 * max(1.0, abs(r2[key])), (key, r1[key], r2[key])
    w_last = c1.flux("z")
    assert abs(t1[-1]["W"] - w_last) < 1e-12 * abs(w_last) + 1e-18
    As, Bs = c1.get_state()
    ref = observables.flux(_gpu_env(c1, 5, D, chi), peps.composite(As.cpu().numpy(), Bs.cpu().numpy(), "z"), "z")
    assert abs(t1[-1]["W"] - ref.real) < 1e-10 * abs(ref.real), (t1[-1]["W"], ref)
    assert abs(ref.real) > 1e-6
    c1.close()
    c2.close()
