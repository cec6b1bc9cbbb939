"""GPU parity: the CUDA library (through the C ABI) against the CPU oracle on
the same seeded inputs.  Gauge-invariant quantities only: free energies,
the normalised environment metric N / ||N||, projector spectra s / ||s||,
energies and magnetisations, bond costs.

Tolerances: FP64 path 1e-9 (accumulated rounding of CTM iterations plus the
subspace-iteration vs full-SVD difference at convergence); FP32 path 2e-5
relative on normalised quantities (single-precision contractions with K up
to chi^2 terms; bound = 2^-23 * sqrt(K) * a safety factor of ~30).  Energies
per site in the single-precision modes within |dE| / max(|E|, 1) <= 1e-6 and
normalised projector spectra within 1e-5 of the FP64 oracle: an energy is a
ratio Tr(H X) / Tr(X) of two contractions of the same FP32 metric, so the
rounding common to both cancels to first order, and a converged spectrum
carries the FP32 rounding of M (~2^-24 sqrt(n) relative to s_1)."""
import numpy as np
import pytest

import kh_inputs
from oracle import ctmrg, eefu, exact, model, peps

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "fp32": 2e-5, "tf32x3": 2e-5, "tf32": 2e-3}
# Targets of the single-precision contraction modes against the FP64 oracle:
# energy per site |dE| / max(|E|, 1) and normalised projector spectra.
E_TOL = 1e-6
SPEC_TOL = 1e-5
# The cut-off of the projectors' S^-1/2 (singular values below cut * s_1
# dropped): FP64 1e-12; the single-precision modes use the library's default,
# 1e-4, above the ~2e-5 s_1 below which their subspace iteration does not
# resolve the spectrum (kept noise directions, weighted by S^-1/2, would
# otherwise enter the environment).
CUT = {"fp64": 1e-12, "fp32": 1e-4, "tf32x3": 1e-4, "tf32": 1e-4}


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


def _nrm(x):
    x = np.asarray(x, dtype=np.float64)
    return x / np.linalg.norm(x)


def _oracle_ctm(T, chi, sweeps, edge=None):
    a = ctmrg.double_tensor(T)
    env = ctmrg.init_env(chi, T.shape[1], edge)
    specs, truncs = None, None
    for _ in range(sweeps):
        specs, truncs = ctmrg.sweep(env, a)
    return env, specs, truncs


# ----------------------------------------------------------------- CTMRG alone

@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "tf32"])
@pytest.mark.parametrize("Kh,Kv,seed,chi", [(0.3, 0.2, 7, 16), (0.25, 0.25, None, 24), (0.15, 0.36, 11, 13)])
def test_ising_free_energy(g, prec, Kh, Kv, seed, chi):
    T = exact.ising_peps(Kh, Kv, gauge_seed=seed)
    ctx = g.Context(2, chi, prec, p_max=2, n_slots=1, svd_cut=CUT[prec])
    ctx.ctm_set_tensor(0, _t(T))
    ctx.ctm_sweep(0, 300, 3, 1e-11 if prec == "fp64" else 10 * TOL[prec], allow_noconv=prec == "tf32")
    lnk = np.log(ctx.ctm_kappa(0))
    ref = exact.onsager_lnZ(Kh, Kv)
    assert abs(lnk - ref) < (1e-9 if prec == "fp64" else TOL[prec])


@pytest.mark.parametrize("chi", [28, 96])
def test_fp64_projectors_at_the_jacobi_size_limit(g, chi):
    """FP64 projector SVD at k = 112, the largest FP64 size the library
    accepts: the dense path at chi = 28 (n = chi D^2 = 112) and the subspace
    path at chi = 96 (chi + 16 oversampling = 112), against Onsager."""
    Kh, Kv = 0.3, 0.2
    T = exact.ising_peps(Kh, Kv, gauge_seed=7)
    ctx = g.Context(2, chi, "fp64", p_max=2, n_slots=1, svd_cut=CUT["fp64"])
    ctx.ctm_set_tensor(0, _t(T))
    ctx.ctm_sweep(0, 300, 3, 1e-11)
    assert abs(np.log(ctx.ctm_kappa(0)) - exact.onsager_lnZ(Kh, Kv)) < 1e-9


def test_contexts_on_two_host_threads(g):
    """Two contexts driven concurrently from two host threads (FP64 at
    chi = 16 and FP32 at chi = 24: the same kernels with different
    shared-memory grants) give the free energies each gives alone."""
    import threading
    import torch
    Kh, Kv = 0.3, 0.2
    T = exact.ising_peps(Kh, Kv, gauge_seed=7)
    cases = [("fp64", 16), ("fp32", 24)]

    def run(prec, chi, out, i):
        try:
            with torch.cuda.stream(torch.cuda.Stream()):
                ctx = g.Context(2, chi, prec, p_max=2, n_slots=1, svd_cut=CUT[prec])
                ctx.ctm_set_tensor(0, _t(T))
                ctx.ctm_sweep(0, 300, 3, 1e-11 if prec == "fp64" else 10 * TOL[prec])
                out[i] = np.log(ctx.ctm_kappa(0))
                torch.cuda.current_stream().synchronize()
        except Exception as e:          # surfaced below
            out[i] = e

    alone = [None, None]
    for i, (prec, chi) in enumerate(cases):
        run(prec, chi, alone, i)
    both = [None, None]
    ths = [threading.Thread(target=run, args=(prec, chi, both, i)) for i, (prec, chi) in enumerate(cases)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    for i, (prec, _) in enumerate(cases):
        assert not isinstance(both[i], Exception), both[i]
        assert abs(both[i] - alone[i]) < (1e-12 if prec == "fp64" else 1e-6)
        assert abs(both[i] - exact.onsager_lnZ(Kh, Kv)) < (1e-9 if prec == "fp64" else TOL[prec])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_yang_magnetisation(g, prec):
    K = 0.5
    T = exact.ising_peps(K, K)
    V = exact.ising_bond_root(K)
    ctx = g.Context(2, 20, prec, p_max=2, n_slots=1, svd_cut=CUT[prec])
    ctx.ctm_set_tensor(0, _t(T))
    ctx.ctm_init(0, np.outer(V[0], V[0]).reshape(4))
    ctx.ctm_sweep(0, 300, 3, 1e-11 if prec == "fp64" else 1e-6)
    m = ctx.ctm_expval(0, np.diag([1.0, -1.0]))[0]
    assert abs(m - exact.yang_m(K)) < (1e-9 if prec == "fp64" else 2e-5)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3"])
@pytest.mark.parametrize("D,chi", [(2, 8), (3, 20), (3, 14)])
def test_ctm_metric_and_spectra_match_oracle(g, prec, D, chi):
    """Converged CTMRG of a seeded composite: metric N/||N|| and the four
    projector spectra agree with the oracle's converged values, the spectra
    s/||s|| within 1e-5 in the single-precision modes (1e-8 in FP64).  (3,20)
    and (3,14) exercise the subspace-iteration path (n = chi D^2 > Jacobi
    limit in FP64) and ragged tile edges."""
    A, B = kh_inputs.perturbed_product_state(D, seed=3, eps=0.2)
    T = peps.composite(A, B, "z")
    env, specs, _ = _oracle_ctm(T, chi, 0)
    env, info = ctmrg.ctmrg(ctmrg.double_tensor(T), env, tol=1e-13, max_sweeps=300, cut=CUT[prec])
    N_ref = ctmrg.metric(env, D)
    ctx = g.Context(D, chi, prec, svd_cut=CUT[prec])
    ctx.ctm_set_tensor(0, _t(T))
    ctx.ctm_sweep(0, 300, 3, 1e-12 if prec == "fp64" else 1e-7, allow_noconv=True)
    N = ctx.ctm_metric(0).cpu().numpy()
    tol = TOL[prec]
    assert np.abs(_nrm(N) - _nrm(N_ref)).max() < tol * 10
    for d in range(4):
        s, tr = ctx.ctm_projectors(0, d)
        s = s.cpu().numpy()
        ref = info["spectra"][d]
        assert np.abs(_nrm(s) - _nrm(ref)).max() < (1e-8 if prec == "fp64" else SPEC_TOL)
        # the discarded weight is (|M|^2 - sum_kept s^2)/|M|^2: resolvable down to
        # ~k eps of the arithmetic (FP64 1e-12, FP32 ~1e-5)
        assert abs(tr - info["trunc"][d]) < max(1e-12, 1e-3 * info["trunc"][d]) + (0 if prec == "fp64" else 1e-5)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3"])
@pytest.mark.parametrize("D,p,chi", [(2, 1, 8), (3, 2, 12), (3, 2, 13), (4, 2, 12)])
def test_ctm_layered_path_matches_oracle(g, prec, D, p, chi):
    """Tensors with D^2 > 2p take the layer-by-layer site contraction (the
    double-layer operand would cost more there); converged metric and
    projector spectra agree with the oracle.  (4, 2, 12) runs the subspace
    iteration (n = 192); (3, 2, 13) has n = 117, not a multiple of 4, so the
    tensor-core precisions fall back to CUDA cores for the half-system product
    (TMA rows must be 16-byte multiples)."""
    T = kh_inputs.random_composite(D, 17 + D, p=p)
    env, specs, _ = _oracle_ctm(T, chi, 0)
    env, info = ctmrg.ctmrg(ctmrg.double_tensor(T), env, tol=1e-13, max_sweeps=300, cut=CUT[prec])
    N_ref = ctmrg.metric(env, D)
    ctx = g.Context(D, chi, prec, p_max=p, n_slots=1, svd_cut=CUT[prec])
    ctx.ctm_set_tensor(0, _t(T))
    ctx.ctm_sweep(0, 300, 3, 1e-12 if prec == "fp64" else 1e-7, allow_noconv=True)
    N = ctx.ctm_metric(0).cpu().numpy()
    tol = TOL[prec]
    assert np.abs(_nrm(N) - _nrm(N_ref)).max() < tol * 10
    for d in range(4):
        s, _ = ctx.ctm_projectors(0, d)
        assert np.abs(_nrm(s.cpu().numpy()) - _nrm(info["spectra"][d])).max() < tol * 10


def test_ctm_single_sweep_is_deterministic_and_exact_for_small_n(g):
    """With n = chi D^2 within the Jacobi limit the projector SVD is exact, so
    ONE sweep from the traced boundary matches the oracle's single sweep."""
    D, chi = 2, 6
    T = kh_inputs.random_composite(D, 5)
    env, specs, truncs = _oracle_ctm(T, chi, 1)
    ctx = g.Context(D, chi, "fp64")
    ctx.ctm_set_tensor(0, _t(T))
    ctx.ctm_sweep(0, 1)
    N = ctx.ctm_metric(0).cpu().numpy()
    assert np.abs(_nrm(N) - _nrm(ctmrg.metric(env, D))).max() < 1e-12
    got = [ctx.ctm_projectors(0, d) for d in range(4)]
    errs = [np.abs(s.cpu().numpy() - specs[d]).max() for d, (s, tr) in enumerate(got)]
    terrs = [abs(tr - truncs[d]) for d, (s, tr) in enumerate(got)]
    assert max(errs) < 1e-12 * max(1.0, specs[0][0]), errs
    assert max(terrs) < 1e-12, terrs


def test_edge_cases(g):
    # chi = 1, D = 1 product tensor (exact), p = 1
    T = np.array([0.7]).reshape(1, 1, 1, 1, 1)
    ctx = g.Context(1, 1, "fp64", p_max=1, n_slots=1)
    ctx.ctm_set_tensor(0, _t(T))
    ctx.ctm_sweep(0, 3)
    s, tr = ctx.ctm_projectors(0, 0)
    assert tr < 1e-28
    assert abs(ctx.ctm_kappa(0) - 0.49) < 1e-14
    # invalid configuration / arguments return status codes, not crashes
    with pytest.raises(g.KhError):
        g.Context(0, 4, "fp64")
    with pytest.raises(g.KhError):
        ctx.ctm_sweep(3, 1)
    # zero sweeps requested is rejected
    with pytest.raises(g.KhError):
        ctx.ctm_sweep(0, 0)


# ----------------------------------------------------------------- eeFU pipeline

def _oracle_state(D, chi, J, K, A=None, B=None, **kw):
    prm = eefu.Params(D=D, chi=chi, J=J, K=K, **kw)
    if A is None:
        A, B = peps.product_state(D)
    return eefu.State(A, B, prm)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_single_layer_dimer_exact(g, prec):
    J, K = model.couplings(0.3 * np.pi)
    D = 4
    ctx = g.Context(D, 8, prec, svd_cut=CUT[prec])
    A, B = peps.product_state(D)
    ctx.set_state(_t(A), _t(B))
    db = 0.2
    H = g.bond_hamiltonian("x", J, K)
    info = ctx.eefu_apply_gate("x", g.gate(H, db / 4))
    Hs = [g.bond_hamiltonian(gm, J, K) for gm in "xyz"]
    r = ctx.observables(Hs)
    want = exact.dimer_energy(J, K, db / 2)
    assert abs(r["Hx"] - want) < TOL[prec]
    assert abs(r["Hy"]) < TOL[prec] and abs(r["Hz"]) < TOL[prec]
    assert abs(r["E_site"] - 0.5 * want) < TOL[prec]
    assert info["rel_cost"] < 1e-10


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_kz_only_closed_form(g, prec):
    Kz = 1.3
    ctx = g.Context(2, 6, prec, svd_cut=CUT[prec])
    for n in range(8):
        ctx.eefu_trotter_step(0.0, [0.0, 0.0, Kz], 0.05)
    Hs = [g.bond_hamiltonian(gm, 0.0, k) for gm, k in zip("xyz", [0.0, 0.0, Kz])]
    r = ctx.observables(Hs)
    assert abs(r["E_site"] - exact.kz_only_energy(Kz, 0.4)) < TOL[prec]


@pytest.mark.parametrize("prec,D", [("fp64", 7), ("fp64", 8), ("tf32x3", 8)])
def test_wide_bonds_closed_forms(g, prec, D):
    """D = 7, 8: the bond matrix T' has 4 D^2 = 196, 256 rows, past the
    one-CTA Jacobi, so the bond update starts from the subspace-iteration
    triplets.  One x layer from the beta = 0 state is the exact dimer (the
    gated bond has Schmidt rank 4 <= D: no truncation, zero cost); K_z-only
    Trotter steps (decoupled z dimers) follow the closed form."""
    J, K = model.couplings(0.3 * np.pi)
    chi = 8
    ctx = g.Context(D, chi, prec, svd_cut=CUT[prec])
    db = 0.2
    info = ctx.eefu_apply_gate("x", g.gate(g.bond_hamiltonian("x", J, K), db / 4),
                               ctm_tol=1e-12 if prec == "fp64" else 1e-7)
    r = ctx.observables([g.bond_hamiltonian(gm, J, K) for gm in "xyz"], ctm_tol=1e-12 if prec == "fp64" else 1e-7)
    want = exact.dimer_energy(J, K, db / 2)
    tol = TOL[prec]
    assert abs(r["Hx"] - want) < tol
    assert abs(r["Hy"]) < tol and abs(r["Hz"]) < tol
    assert info["rel_cost"] < (1e-10 if prec == "fp64" else 1e-6)
    ctx.close()
    Kz = 1.3
    ctx = g.Context(D, chi, prec, svd_cut=CUT[prec])
    for _ in range(2):
        ctx.eefu_trotter_step(0.0, [0.0, 0.0, Kz], 0.05)
    r = ctx.observables([g.bond_hamiltonian(gm, 0.0, k) for gm, k in zip("xyz", [0.0, 0.0, Kz])])
    assert abs(r["E_site"] - exact.kz_only_energy(Kz, 0.1)) < tol
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_wide_bond_gate_layer_matches_oracle(g, prec):
    """D = 8 (the bond matrix 256 x 256, the subspace-iteration start): one z
    layer of a Kitaev-Heisenberg step on a random state with its CTMRG
    converged, the bond update, then the observables, against the oracle's
    stored values (tests/golden/wide_bond_parity_D8_chi8.json, written by
    make_wide_bond_parity.py from oracle/ only).  All eight kept singular
    values lie above 1e-3 s_1, so the single-precision cut-off (1e-4) and the
    FP64 one truncate alike.  FP64: energies and moments within 1e-8, spectra
    1e-7 (the kept tail is flat, s_8 / s_2 ~ 0.6, so the fixed point converges
    slowly in the tail), relative cost 1e-6 relative; 3xTF32 with the FP64
    projector SVD: the single-precision targets."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "wide_bond_parity_D8_chi8.json")))
    c = gold["case"]
    D, chi = c["D"], c["chi"]
    gl = gold["gate_layer"]
    assert min(min(s) for s in gl["spectra"]) > 1e-3 * max(max(s) for s in gl["spectra"])
    A, B = kh_inputs.random_site_tensors(D, c["seed"])
    fp64 = prec == "fp64"
    ctx = g.Context(D, chi, prec, svd_cut=CUT[prec], proj_fp64=0 if fp64 else 1)
    ctx.set_state(_t(A), _t(B))
    gate = g.gate(g.bond_hamiltonian("z", c["J"], c["K"]), c["dbeta"] / 2)
    ctm_tol = 1e-10 if fp64 else 1e-7
    info = ctx.eefu_apply_gate("z", gate, ctm_max_sweeps=400, ctm_min_sweeps=3, ctm_tol=ctm_tol)
    assert abs(info["rel_cost"] - gl["rel_cost"]) < (1e-6 if fp64 else 1e-4) * gl["rel_cost"], \
        (info["rel_cost"], gl["rel_cost"])
    for d in range(4):
        s, _ = ctx.ctm_projectors(2, d)
        err = np.abs(_nrm(s.cpu().numpy()) - _nrm(gl["spectra"][d])).max()
        assert err < (1e-7 if fp64 else SPEC_TOL), (d, err)
    Hs = [g.bond_hamiltonian(gm, c["J"], c["K"]) for gm in "xyz"]
    r = ctx.observables(Hs, ctm_max_sweeps=400, ctm_min_sweeps=3, ctm_tol=ctm_tol)
    ro = gold["observables"]
    tol = 1e-8 if fp64 else E_TOL
    for key in ("E_site", "Hx", "Hy", "Hz", "Ax", "Az", "Bx", "Bz"):
        assert abs(r[key] - ro[key]) < tol * max(1.0, abs(ro[key])), (key, r[key], ro[key])
    ctx.close()


@pytest.mark.parametrize("D,chi,steps", [(2, 16, 4), (3, 12, 2)])
def test_bf16_trotter_steps_near_oracle(g, D, chi, steps):
    """BF16 contractions (the layered site contraction on kind::f16, one
    pass, FP32 accumulation): after the same Trotter steps as the FP64 and
    3xTF32 parity test, E/site, <H^gamma> and the magnetisations agree with
    the oracle run at the same projector cut-off (1e-3 s_1, above the BF16
    noise of the projector spectrum) within 1e-4 of max(1, |x|).  A single
    BF16 contraction is good to its unit roundoff 2^-9 ~ 2e-3 (the kernel
    test); the converged environment and the ALS do not accumulate it (1.7e-5
    measured at (3, 12))."""
    J, K = model.couplings(0.3 * np.pi)
    hA, hB = 0.3, -0.1
    A, B = kh_inputs.perturbed_product_state(D, seed=11, eps=0.05)
    st = _oracle_state(D, chi, J, K, A, B, hA=hA, hB=hB, svd_cut=1e-3, ctm_tol=1e-12)
    ctx = g.Context(D, chi, "bf16", svd_cut=1e-3)
    ctx.set_state(_t(A), _t(B))
    for n in range(steps):
        eefu.trotter_step(st, 0.02)
        ctx.eefu_trotter_step(J, [K, K, K], 0.02, hA, hB, ctm_max_sweeps=60, ctm_tol=1e-5)
    ro = eefu.measure(st)
    Hs = [g.bond_hamiltonian(gm, J, K) for gm in "xyz"]
    r = ctx.observables(Hs, hA, hB, ctm_max_sweeps=60, ctm_tol=1e-5)
    for key in ("E_site", "Hx", "Hy", "Hz", "Ax", "Az", "Bx", "Bz"):
        assert abs(r[key] - ro[key]) < 1e-4 * max(1.0, abs(ro[key])), (key, r[key], ro[key])
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3"])
@pytest.mark.parametrize("D,chi,steps", [(2, 16, 4), (3, 12, 2)])
def test_trotter_steps_match_oracle(g, prec, D, chi, steps):
    """KH model at phi = 0.3 pi from a seeded perturbed product state (bias on):
    per-layer relative costs, and after the steps E/site, <H^gamma> and the
    sublattice magnetisations agree with the oracle."""
    J, K = model.couplings(0.3 * np.pi)
    hA, hB = 0.3, -0.1
    A, B = kh_inputs.perturbed_product_state(D, seed=11, eps=0.05)
    cut = CUT[prec]
    st = _oracle_state(D, chi, J, K, A, B, hA=hA, hB=hB, svd_cut=cut, ctm_tol=1e-12)
    ctx = g.Context(D, chi, prec, svd_cut=cut)
    ctx.set_state(_t(A), _t(B))
    ctol = 1e-12 if prec == "fp64" else 1e-7
    dbeta = 0.02
    for n in range(steps):
        oinf = eefu.trotter_step(st, dbeta)
        ginf = ctx.eefu_trotter_step(J, [K, K, K], dbeta, hA, hB, ctm_max_sweeps=200, ctm_tol=ctol)
        worst = max(i["rel_cost"] for i in oinf)
        assert abs(ginf["rel_cost"] - worst) < 1e-6 * max(worst, 1e-12) + (1e-12 if prec == "fp64" else 1e-7)
    ro = eefu.measure(st)
    Hs = [g.bond_hamiltonian(gm, J, K) for gm in "xyz"]
    r = ctx.observables(Hs, hA, hB, ctm_max_sweeps=200, ctm_tol=ctol)
    tol = 1e-9 if prec == "fp64" else E_TOL
    for key in ("E_site", "Hx", "Hy", "Hz", "Ax", "Az", "Bx", "Bz"):
        assert abs(r[key] - ro[key]) < tol * max(1.0, abs(ro[key])), (key, r[key], ro[key])
    # site tensors agree up to the bond gauge: compare gauge-invariant T
    Ag, Bg = ctx.get_state()
    for gm in "xyz":
        To = peps.composite(st.A, st.B, gm)
        Tg = peps.composite(Ag.cpu().numpy(), Bg.cpu().numpy(), gm)
        # gauge-covariant (fixed by the balanced-SVD convention), hence looser
        # than the invariants above
        assert np.abs(_nrm(Tg) - _nrm(To)).max() < (1e-7 if prec == "fp64" else 1e-4)


def test_bench_configuration_full_size_against_fp64_path(g):
    """The bench workload at full size (Kitaev K=1, J=0, D=4, chi=64, dbeta=0.01,
    4 CTM sweeps per layer, 2 per observables mapping) in the launch
    configuration bench.py times (3xTF32, three lanes): one Trotter step plus
    observables agrees with the library's FP64 path on the same start to the
    FP32-level tolerance, and the properties that hold at any size hold: E/site
    is half the sum of the bond energies (no field), real tensors give <S^y> = 0,
    truncation errors lie in [0, 1)."""
    import torch
    D, chi = 4, 64
    A0, B0 = kh_inputs.perturbed_product_state(D, seed=0, eps=0.05)
    Hs = [g.bond_hamiltonian(gm, 0.0, 1.0) for gm in "xyz"]
    res = {}
    for prec in ("tf32x3", "fp64"):
        ctx = g.Context(D, chi, prec, svd_cut=CUT[prec])
        ctx.set_state(_t(A0), _t(B0))
        ctx.eefu_trotter_step(0.0, [1.0, 1.0, 1.0], 0.01, ctm_max_sweeps=4, ctm_min_sweeps=4, ctm_tol=-1.0,
                              info=False)
        res[prec] = ctx.observables(Hs, ctm_max_sweeps=2, ctm_min_sweeps=2, ctm_tol=-1.0)
        torch.cuda.synchronize()
    a, b = res["tf32x3"], res["fp64"]
    for r in (a, b):
        assert all(np.isfinite(v) for v in r.values())
        assert abs(r["E_site"] - 0.5 * (r["Hx"] + r["Hy"] + r["Hz"])) < 1e-12
        assert r["Ay"] == 0.0 and r["By"] == 0.0
        assert 0.0 <= r["trunc"] < 1.0
    scale = max(abs(b["E_site"]), 1e-3)
    assert abs(a["E_site"] - b["E_site"]) < 2e-5 * scale
    for k in ("Hx", "Hy", "Hz", "Ax", "Az", "Bx", "Bz"):
        assert abs(a[k] - b[k]) < 2e-5 * max(abs(b[k]), 1e-3), k


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("tf32x3", 2e-5)])
def test_lanes_match_single_stream(g, prec, tol):
    """A context with six slots runs the independent pieces of a CTM move
    (corner s+3, P, the corner updates) on a second stream with its own
    scratch; one with three slots runs every move on its one stream.  Both
    give the same converged metric and projector spectra."""
    D, chi = 3, 14
    A, B = kh_inputs.perturbed_product_state(D, seed=9, eps=0.2)
    T = peps.composite(A, B, "y")
    out = []
    for n_slots in (3, 6):
        ctx = g.Context(D, chi, prec, n_slots=n_slots, svd_cut=CUT[prec])
        ctx.ctm_set_tensor(0, _t(T))
        ctx.ctm_sweep(0, 200, 3, 1e-12 if prec == "fp64" else 1e-7, allow_noconv=True)
        N = _nrm(ctx.ctm_metric(0).cpu().numpy())
        specs = [_nrm(ctx.ctm_projectors(0, d)[0].cpu().numpy()) for d in range(4)]
        out.append((N, specs))
    (N3, s3), (N6, s6) = out
    assert np.abs(N3 - N6).max() < tol
    for d in range(4):
        assert np.abs(s3[d] - s6[d]).max() < tol


def _gpu_env(ctx, slot, D, chi):
    """The FP64 environment masters of a slot as an oracle Env."""
    C, E = ctx.ctm_get_env(slot)
    C = C.cpu().numpy().reshape(4, chi, chi)
    E = E.cpu().numpy().reshape(4, chi, D * D, chi)
    return ctmrg.Env(list(C), list(E))


@pytest.mark.parametrize("D,chi,seed", [(5, 100, 4), (6, 144, 6)])
def test_large_configurations_against_oracle_samples(g, D, chi, seed):
    """The larger configurations at full size, (D, chi) = (5, 100)
    (double-layer site contraction on CUDA cores: D^4 = 625 rows are not
    16-byte multiples) and (6, 144) (layer-by-layer site contraction, k = chi
    + 16 = 160 at the Jacobi limit, the 216 x 216 ALS solve in global memory),
    in 3xTF32 with three lanes: one z gate layer on a seeded random state with
    its CTMRG converged, then the oracle recomputes, one by one from the
    library's own FP64 environment masters, (i) the environment metric N
    (element by element, normalised) and (ii) the left move's half-system
    product M and its singular values (the projector spectrum s/||s|| -- the
    values above the cut-off, zeros after them -- within 1e-5, the discarded
    weight within the FP32 resolution); the observables satisfy the
    properties that hold at any size."""
    import torch
    J, K, dbeta = 0.0, 1.0, 0.01
    A, B = kh_inputs.random_site_tensors(D, seed)
    gate_np = model.gate("z", dbeta / 2, J, K)
    ctx = g.Context(D, chi, "tf32x3")            # the single-precision defaults (cut 1e-4 s_1)
    cut = ctx.cfg.svd_cut
    ctx.set_state(_t(A), _t(B))
    info = ctx.eefu_apply_gate("z", g.gate(g.bond_hamiltonian("z", J, K), dbeta / 2), ctm_max_sweeps=200,
                               ctm_min_sweeps=3, ctm_tol=1e-7)
    assert np.isfinite(info["rel_cost"]) and 0.0 <= info["trunc"] < 1.0
    # the state was updated: the environment of slot 2 belongs to the gated
    # composite of the input state
    env = _gpu_env(ctx, 2, D, chi)
    Tp = peps.composite(A, B, "z", gate_np)
    a = ctmrg.double_tensor(Tp)
    N = ctx.ctm_metric(2).cpu().numpy()
    assert np.abs(_nrm(N) - _nrm(ctmrg.metric(env, D))).max() < 10 * TOL["tf32x3"]
    s_gpu, tr_gpu = ctx.ctm_projectors(2, 0)
    Qul, Qdl = ctmrg.enlarged_corners(env.C[0], env.E[0], env.E[3], env.C[3], env.E[2], a)
    n = chi * D * D
    M = Qul.reshape(n, n).T @ Qdl.reshape(n, n)
    del Qul, Qdl
    sv = np.linalg.svd(M, compute_uv=False)
    del M
    s_ref = np.where(sv[:chi] > cut * sv[0], sv[:chi], 0.0)     # the reported spectrum: kept values only
    assert np.abs(_nrm(s_gpu.cpu().numpy()) - _nrm(s_ref)).max() < SPEC_TOL
    tr_ref = float(np.sum(sv[chi:] ** 2) / np.sum(sv ** 2))
    assert abs(tr_gpu - tr_ref) < 1e-3 * tr_ref + 1e-5
    Hs = [g.bond_hamiltonian(gm, J, K) for gm in "xyz"]
    r = ctx.observables(Hs, ctm_max_sweeps=40, ctm_min_sweeps=3, ctm_tol=1e-7)
    assert all(np.isfinite(v) for v in r.values())
    assert abs(r["E_site"] - 0.5 * (r["Hx"] + r["Hy"] + r["Hz"])) < 1e-12
    assert r["Ay"] == 0.0 and r["By"] == 0.0
    assert 0.0 <= r["trunc"] < 1.0
    del ctx
    torch.cuda.synchronize()


@pytest.mark.parametrize("D,chi", [(2, 2), (3, 5), (2, 13)])
def test_small_and_odd_shapes_with_lanes(g, D, chi):
    """Tiny and odd shapes through a whole Trotter step and the observables on a
    six-slot context (three lanes), every CTMRG converged, against the oracle
    with the same cut-off: chi = 2 (n = 8), n = 45 and n = 52 (the
    half-system product on CUDA cores when n is not a multiple of 4 in the
    tensor-core precisions).  E/site and the bond energies within
    |dE| / max(|E|, 1) <= 1e-6 (3xTF32) and 1e-9 (FP64)."""
    import torch
    J, K, hA, hB, dbeta = 0.3, 1.0, 0.2, -0.1, 0.02
    A, B = kh_inputs.perturbed_product_state(D, seed=2, eps=0.1)
    Hs = [g.bond_hamiltonian(gm, J, K) for gm in "xyz"]
    for prec in ("tf32x3", "fp64"):
        cut = CUT[prec]
        st = _oracle_state(D, chi, J, K, A, B, hA=hA, hB=hB, svd_cut=cut, ctm_tol=1e-12, ctm_max_sweeps=300)
        eefu.trotter_step(st, dbeta)
        ro = eefu.measure(st)
        ctol = 1e-12 if prec == "fp64" else 1e-7
        ctx = g.Context(D, chi, prec, svd_cut=cut)
        ctx.set_state(_t(A), _t(B))
        ctx.eefu_trotter_step(J, [K, K, K], dbeta, hA, hB, ctm_max_sweeps=300, ctm_tol=ctol, info=False)
        r = ctx.observables(Hs, hA, hB, ctm_max_sweeps=300, ctm_tol=ctol)
        torch.cuda.synchronize()
        assert all(np.isfinite(v) for v in r.values())
        assert 0.0 <= r["trunc"] < 1.0
        tol = 1e-9 if prec == "fp64" else E_TOL
        for key in ("E_site", "Hx", "Hy", "Hz", "Ax", "Az", "Bx", "Bz"):
            assert abs(r[key] - ro[key]) < tol * max(1.0, abs(ro[key])), (prec, key, r[key], ro[key])


@pytest.mark.parametrize("proj_fp64", [0, 1])
def test_bench_configuration_matches_oracle(g, proj_fp64):
    """The bench's full size and launch configuration (D = 4, chi = 64, p = 16,
    3xTF32 contractions, six slots on three lanes; the projector
    factorisations in FP32 or, proj_fp64 = 1, in FP64) against the oracle's stored
    values (tests/golden/bench_parity_D4_chi64.json, written by
    make_bench_parity.py from oracle/ only): a seeded random state, the z gate
    of a Kitaev step (K = 1, J = 0, dbeta = 0.01) with its CTMRG converged,
    the environment-weighted bond update, then the observables with the three
    mappings converged.  E/site and <H^gamma> within |dE| / max(|E|, 1) <= 1e-6,
    <S^a> too with the FP64 projector SVD (3e-6 with the FP32 one); the four
    projector spectra s/||s|| within 1e-5; their largest
    discarded weight within the FP32 resolution; the bond update's relative
    cost within 1e-4 relative."""
    import json
    import os
    import torch
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "bench_parity_D4_chi64.json")))
    c = gold["case"]
    D, chi = c["D"], c["chi"]
    A, B = kh_inputs.random_site_tensors(D, c["seed"])
    ctx = g.Context(D, chi, "tf32x3", svd_cut=c["svd_cut"], proj_fp64=proj_fp64)
    ctx.set_state(_t(A), _t(B))
    gate = g.gate(g.bond_hamiltonian("z", c["J"], c["K"]), c["dbeta"] / 2)
    info = ctx.eefu_apply_gate("z", gate, ctm_max_sweeps=400, ctm_min_sweeps=3, ctm_tol=1e-7)
    gl = gold["gate_layer"]
    assert abs(info["rel_cost"] - gl["rel_cost"]) < 1e-4 * gl["rel_cost"], (info["rel_cost"], gl["rel_cost"])
    trs = []
    for d in range(4):
        s, tr = ctx.ctm_projectors(2, d)
        trs.append(tr)
        err = np.abs(_nrm(s.cpu().numpy()) - _nrm(gl["spectra"][d])).max()
        assert err < SPEC_TOL, (d, err)
    assert abs(max(trs) - gl["trunc"]) < 1e-3 * gl["trunc"] + 1e-5
    Hs = [g.bond_hamiltonian(gm, c["J"], c["K"]) for gm in "xyz"]
    r = ctx.observables(Hs, ctm_max_sweeps=400, ctm_min_sweeps=3, ctm_tol=1e-7)
    ro = gold["observables"]
    # the sublattice moments with the FP32 projector SVD: within 3e-6 (measured
    # up to 1.4e-6; its spectra move by ~1e-6 from sweep to sweep)
    mtol = E_TOL if proj_fp64 else 3e-6
    for key in ("E_site", "Hx", "Hy", "Hz"):
        assert abs(r[key] - ro[key]) < E_TOL * max(1.0, abs(ro[key])), (key, r[key], ro[key])
    for key in ("Ax", "Az", "Bx", "Bz"):
        assert abs(r[key] - ro[key]) < mtol * max(1.0, abs(ro[key])), (key, r[key], ro[key])
    assert abs(r["trunc"] - ro["trunc"]) < 1e-3 * ro["trunc"] + 1e-5
    del ctx
    torch.cuda.synchronize()


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_trajectory_specific_heat_of_decoupled_z_dimers(g, prec):
    """eefu_evolve on the K_z-only model (decoupled z dimers: no Trotter error,
    D = 2 exact): the energies along the trajectory follow the closed form
    E(beta) = -(K_z/8) tanh(beta K_z/4), and the library's specific heat is the
    oracle's central difference of the closed-form energies on the same grid
    (the finite-difference formula is the same; within 1e-9 relative for FP64,
    the single-precision energy error over the grid spacing for 3xTF32)."""
    from oracle import observables
    Kz, dbeta, n, every = 1.3, 0.05, 12, 2
    ctx = g.Context(2, 6, prec, svd_cut=CUT[prec])
    traj = ctx.evolve(0.0, [0.0, 0.0, Kz], dbeta, n, every, ctm_max_sweeps=100,
                      ctm_tol=1e-12 if prec == "fp64" else 1e-7)
    assert len(traj) == n // every
    beta = np.array([r["beta"] for r in traj])
    assert np.abs(beta - dbeta * every * np.arange(1, n // every + 1)).max() < 1e-12
    E = np.array([r["E_site"] for r in traj])
    Eref = exact.kz_only_energy(Kz, beta)
    etol = 1e-10 if prec == "fp64" else E_TOL
    assert np.abs(E - Eref).max() < etol
    b, Cref = observables.specific_heat(beta, Eref)
    C = np.array([r["C"] for r in traj])
    assert np.isnan(C[0]) and np.isnan(C[-1])
    ctol = 2 * etol * beta.max() ** 2 / (2 * dbeta * every)
    assert np.abs(C[1:-1] - Cref).max() < ctol + 1e-12


def test_trajectory_matches_oracle_evolution(g):
    """eefu_evolve on the Kitaev-Heisenberg model with a bias (D = 2, chi = 8,
    FP64 path): every measured row (beta, E/site, bond energies, moments) and
    the specific heat agree with the oracle's trajectory and its central
    differences."""
    from oracle import observables
    J, K = model.couplings(0.3 * np.pi)
    hA, hB, dbeta, n = 0.2, -0.1, 0.02, 6
    A, B = kh_inputs.perturbed_product_state(2, seed=5, eps=0.05)
    st = _oracle_state(2, 8, J, K, A, B, hA=hA, hB=hB, ctm_tol=1e-12, ctm_max_sweeps=300)
    ref = eefu.evolve(st, dbeta, n, measure_every=1)
    ctx = g.Context(2, 8, "fp64")
    ctx.set_state(_t(A), _t(B))
    traj = ctx.evolve(J, [K, K, K], dbeta, n, 1, hA=hA, hB=hB, ctm_max_sweeps=300, ctm_tol=1e-12)
    for r, o in zip(traj, ref):
        assert abs(r["beta"] - o["beta"]) < 1e-12
        for key in ("E_site", "Hx", "Hy", "Hz", "Ax", "Az", "Bx", "Bz"):
            assert abs(r[key] - o[key]) < 1e-9 * max(1.0, abs(o[key])), (key, r[key], o[key])
    _, Cref = observables.specific_heat([o["beta"] for o in ref], [o["E_site"] for o in ref])
    C = np.array([r["C"] for r in traj])[1:-1]
    assert np.abs(C - Cref).max() < 1e-9 * 2 * ref[-1]["beta"] ** 2 / (2 * dbeta) + 1e-12


@pytest.mark.parametrize("prec,D,chi,dbeta,n", [("fp64", 2, 8, 0.05, 10), ("fp64", 4, 12, 0.02, 10),
                                                 ("tf32x3", 4, 16, 0.05, 6)])
def test_klein_duality_of_trajectories(g, prec, D, chi, dbeta, n):
    """Eq. (4): the library's trajectories at (J, K) and at the dual couplings
    (-J, K + 2J), both from the beta = 0 state in the 2-site cell, give the
    same E/site and bond energies (exactly in exact arithmetic: the duality
    is a product of single-site rotations that the symmetric iterates absorb
    as a virtual gauge; see the oracle pin).  FP64 within 1e-9; 3xTF32 within
    twice the single-precision energy target (two independent runs)."""
    J, K = model.couplings(0.3 * np.pi)
    rows = []
    for j, k in ((J, K), (-J, K + 2 * J)):
        ctx = g.Context(D, chi, prec, svd_cut=CUT[prec])
        traj = ctx.evolve(j, [k, k, k], dbeta, n, n // 2, ctm_max_sweeps=200,
                          ctm_tol=1e-12 if prec == "fp64" else 1e-7)
        rows.append(np.array([[r["E_site"], r["Hx"], r["Hy"], r["Hz"]] for r in traj]))
        ctx.close()
    tol = 1e-9 if prec == "fp64" else 2 * E_TOL
    assert np.abs(rows[0]).min() > 1e-3
    assert np.abs(rows[0] - rows[1]).max() < tol, rows[0] - rows[1]


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
@pytest.mark.parametrize("Kh", [0.3, 0.6])
def test_correlation_length_of_decoupled_chains(g, prec, Kh):
    """K_v = 0: the rows are independent 1D Ising chains, the environment is
    exact and the channel transfer matrix reduces to the chain's, whose
    eigenvalue ratio is tanh K_h: xi_x = -1 / ln tanh K_h (closed form);
    nothing is correlated along y."""
    T = exact.ising_peps(Kh, 0.0)
    ctx = g.Context(2, 8, prec, p_max=2, n_slots=1, svd_cut=CUT[prec])
    ctx.ctm_set_tensor(0, _t(T))
    ctx.ctm_sweep(0, 300, 3, 1e-12 if prec == "fp64" else 1e-7, allow_noconv=prec != "fp64")
    xi, ratio, its = ctx.ctm_correlation_length(0, 0, max_iter=400, tol=1e-10 if prec == "fp64" else 1e-6)
    want = -1.0 / np.log(np.tanh(Kh))
    assert abs(xi - want) < (1e-8 if prec == "fp64" else 1e-4) * want, (xi, want, its)
    xi_y, _, _ = ctx.ctm_correlation_length(0, 1, max_iter=400)
    # nothing correlates along y: |l2|/|l1| is zero up to rounding (~1e-7 in
    # single precision, i.e. xi ~ 0.06)
    assert xi_y < (0.05 if prec == "fp64" else 0.1)


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
@pytest.mark.parametrize("D,chi,direction", [(2, 8, 0), (2, 12, 1), (3, 6, 0)])
def test_correlation_length_matches_oracle_on_the_library_environment(g, prec, D, chi, direction):
    """A generic composite (a perturbed product state's z composite): the
    library's block power iteration on the channel transfer matrix against the
    oracle's dense eigenvalues of the same matrix, built from the library's own
    converged environment (so only the eigen-solve is compared)."""
    A, B = kh_inputs.perturbed_product_state(D, seed=8, eps=0.3)
    T = peps.composite(A, B, "z")
    ctx = g.Context(D, chi, prec, n_slots=1, svd_cut=CUT[prec])
    ctx.ctm_set_tensor(0, _t(T))
    ctx.ctm_sweep(0, 300, 3, 1e-12 if prec == "fp64" else 1e-7, allow_noconv=True)
    xi, ratio, its = ctx.ctm_correlation_length(0, direction, max_iter=800, tol=1e-10 if prec == "fp64" else 1e-7)
    env = _gpu_env(ctx, 0, D, chi)
    ref = ctmrg.correlation_length(env, ctmrg.double_tensor(T), direction)
    assert abs(xi - ref) < (1e-7 if prec == "fp64" else 1e-4) * max(ref, 1e-3), (xi, ref, its)
