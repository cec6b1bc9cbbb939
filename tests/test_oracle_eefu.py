"""Pins of the oracle's bond update and of the whole eeFU pipeline against
closed forms and exact diagonalisation."""
import numpy as np
import pytest

import kh_inputs
from oracle import bond, ctmrg, eefu, exact, model, peps


def _fresh(D, chi, **kw):
    prm = eefu.Params(D=D, chi=chi, **kw)
    A, B = peps.product_state(D)
    return eefu.State(A, B, prm)


def test_beta0_invariants():
    st = _fresh(2, 6, J=0.5, K=1.2)
    r = eefu.measure(st)
    for k in ("E_site", "Hx", "Hy", "Hz", "Ax", "Ay", "Az", "Bx", "By", "Bz"):
        assert abs(r[k]) < 1e-15
    assert r["trunc"] < 1e-28
    # the identity gate leaves the product state exactly representable
    info = eefu.apply_gate(st, "z", np.eye(4))
    assert info["rel_cost"] < 1e-28


@pytest.mark.parametrize("gamma", ["x", "y", "z"])
def test_single_layer_is_exact_dimer(gamma):
    J, K = model.couplings(0.3 * np.pi)
    st = _fresh(4, 6, J=J, K=K)
    db = 0.2
    tau = dict(x=db / 4, y=db / 4, z=db / 2)[gamma]
    info = eefu.apply_gate(st, gamma, st.prm.gate(gamma, tau))
    assert info["rel_cost"] < 1e-20
    r = eefu.measure(st)
    want = exact.dimer_energy(J, K, 2 * tau)
    assert abs(r["H" + gamma] - want) < 1e-13
    for g in "xyz":
        if g != gamma:
            assert abs(r["H" + g]) < 1e-13
    assert abs(r["E_site"] - 0.5 * want) < 1e-13


def test_kz_only_closed_form_all_beta():
    Kz = 1.3
    st = _fresh(2, 6, J=0.0, K=0.0, K_gamma={"x": 0.0, "y": 0.0, "z": Kz})
    for n in range(1, 9):
        eefu.trotter_step(st, 0.05)
        if n % 4 == 0:
            r = eefu.measure(st)
            assert abs(r["E_site"] - exact.kz_only_energy(Kz, 0.05 * n)) < 1e-10


@pytest.mark.parametrize("hA,hB", [(0.7, 0.7), (0.7, -0.3)])
def test_field_only_closed_form(hA, hB):
    st = _fresh(2, 4, J=0.0, K=0.0, hA=hA, hB=hB)
    for _ in range(6):
        eefu.trotter_step(st, 0.05)
    r = eefu.measure(st)
    beta = 0.3
    eA, mA = exact.field_only(hA, beta)
    eB, mB = exact.field_only(hB, beta)
    assert abs(r["Az"] - mA) < 1e-12 and abs(r["Bz"] - mB) < 1e-12
    assert abs(r["E_site"] - 0.5 * (eA + eB)) < 1e-12


def test_specific_heat_of_decoupled_z_dimers():
    """K_z only: decoupled dimers, no Trotter error, E(beta) = -(K_z/8) tanh(beta K_z/4),
    so C = beta^2 K_z^2/32 sech^2(beta K_z/4); central differences on the
    trajectory (step 0.05) agree to O(dbeta^2)."""
    from oracle import observables
    Kz = 1.3
    st = _fresh(2, 6, J=0.0, K=0.0, K_gamma={"x": 0.0, "y": 0.0, "z": Kz})
    res = eefu.evolve(st, 0.05, 8, measure_every=1)
    b, C = observables.specific_heat([r["beta"] for r in res], [r["E_site"] for r in res])
    want = b ** 2 * Kz ** 2 / 32.0 / np.cosh(b * Kz / 4.0) ** 2
    assert len(b) == 6 and np.abs(C - want).max() < 1e-5


@pytest.mark.parametrize("hA,hB", [(0.6, 0.6), (0.6, -0.6)])
def test_order_parameters_in_a_pure_field(hA, hB):
    """J = K = 0 in a field: every spin is free, <S^z> = tanh(beta h / 2) / 2.
    A uniform field gives m_FM = tanh(beta h / 2) and m_AF = 0; a staggered
    field gives m_AF = tanh(beta h / 2) and m_FM = 0 (the factor 2 of the
    ferromagnetic definition and its absence in the staggered one both make
    a saturated state read 1)."""
    from oracle import observables
    st = _fresh(2, 4, J=0.0, K=0.0, hA=hA, hB=hB)
    for _ in range(6):
        eefu.trotter_step(st, 0.05)
    r = eefu.measure(st)
    m = observables.order_parameters(r)
    t = np.tanh(0.3 * 0.6 / 2.0)
    if hA == hB:
        assert abs(m["m_fm"] - t) < 1e-12 and m["m_af"] < 1e-12
    else:
        assert abs(m["m_af"] - t) < 1e-12 and m["m_fm"] < 1e-12


def test_kh_high_temperature_against_ed_and_series():
    """D=4 eeFU at beta=0.05, 0.1 against 8- and 12-site ED: the eeFU value must
    sit within the finite-size spread |E8-E12| (+ Trotter margin) of E12, and
    E/beta must approach the high-T slope."""
    phi = 0.3 * np.pi
    J, K = model.couplings(phi)
    betas = np.array([0.05, 0.1])
    E8 = exact.honeycomb_ed(2, 2, J, K, betas)
    E12 = exact.honeycomb_ed(2, 3, J, K, betas)
    st = _fresh(4, 12, J=J, K=K)
    res = eefu.evolve(st, 0.01, 10, measure_every=5)
    for r, e8, e12, b in zip(res, E8, E12, betas):
        assert abs(r["beta"] - b) < 1e-12
        assert abs(r["E_site"] - e12) < abs(e8 - e12) + 5e-6
        assert abs(r["E_site"] / b - exact.high_T_energy_slope(J, K)) < 0.05 * b + 1e-4
        # C3 symmetry at h=0 up to Trotter asymmetry
        assert abs(r["Hx"] - r["Hz"]) < 1e-4 and abs(r["Hy"] - r["Hz"]) < 1e-4
        assert abs(r["Ay"]) < 1e-15 and abs(r["By"]) < 1e-15


def test_site_moments_agree_across_mappings():
    """All three gamma-mapped environments describe the same state: <S^z_A>
    and <S^x_B> agree between mappings (a leg mix-up between mappings fails)."""
    J, K = model.couplings(0.3 * np.pi)
    st = _fresh(4, 12, J=J, K=K, hA=0.5, hB=-0.2)
    eefu.evolve(st, 0.02, 3)
    eefu.measure(st)
    vals = []
    for gamma in "xyz":
        T = peps.composite(st.A, st.B, gamma)
        X = ctmrg.expval_matrix(T, ctmrg.metric(st.obs_env[gamma], 4))
        from oracle import observables
        vals.append(observables.site_moments(X))
    for key in ("Az", "Bz", "Ax", "Bx"):
        v = [m[key] for m in vals]
        assert max(v) - min(v) < 1e-9, (key, v)
    assert abs(vals[0]["Az"]) > 1e-3


def test_bond_update_eckart_young():
    """N = identity: the ALS optimum is the truncated SVD and the cost is the
    discarded sum of squared singular values."""
    D = 2
    Tp = kh_inputs.random_composite(D, 3)
    N = np.eye(D ** 4)
    A2, B2, S = bond.svd_init(Tp, D)
    A3, B3, info = bond.als(Tp, N, D, tol=1e-15, max_iter=20, reg=0.0)
    want = np.sum(S[D:] ** 2) / np.sum(S ** 2)
    assert abs(info["rel_cost"] - want) < 1e-12
    # rank <= D: the cost is zero
    T0 = np.einsum("abURk,cdDLk->abcdLURD", A2, B2).reshape(Tp.shape)
    _, _, info0 = bond.als(T0, N, D, tol=1e-15, max_iter=5, reg=0.0)
    assert info0["rel_cost"] < 1e-26


def test_bond_cost_gradient_against_central_differences():
    """The analytic gradient of the bond cost along 8 random unit directions
    in (A'', B'') against central finite differences (h = 1e-6, FP64); the
    ALS optimum has zero gradient in both factors."""
    D = 2
    Tp = kh_inputs.random_composite(D, 5)
    rng = np.random.default_rng(13)
    G = rng.standard_normal((D ** 4, D ** 4))
    N = G @ G.T / D ** 4 + 0.1 * np.eye(D ** 4)
    A2 = rng.standard_normal((2, 2, D, D, D))
    B2 = rng.standard_normal((2, 2, D, D, D))
    gA, gB = bond.cost_gradient(A2, B2, Tp, N)
    h = 1e-6
    for _ in range(8):
        dA = rng.standard_normal(A2.shape)
        dB = rng.standard_normal(B2.shape)
        nrm = np.sqrt(np.sum(dA ** 2) + np.sum(dB ** 2))
        dA, dB = dA / nrm, dB / nrm
        fd = (bond.cost(A2 + h * dA, B2 + h * dB, Tp, N)[0] - bond.cost(A2 - h * dA, B2 - h * dB, Tp, N)[0]) / (2 * h)
        an = np.sum(gA * dA) + np.sum(gB * dB)
        assert abs(fd - an) <= 1e-7 * max(1.0, abs(an)), (fd, an)
    A3, B3, _ = bond.als(Tp, N, D, tol=0.0, max_iter=400, reg=0.0)
    gA3, gB3 = bond.cost_gradient(A3, B3, Tp, N)
    scale = np.sqrt(np.sum(bond.cost_gradient(A2, B2, Tp, N)[0] ** 2))
    assert np.abs(gA3).max() < 1e-6 * scale and np.abs(gB3).max() < 1e-6 * scale


def test_bond_update_monotone_and_gauge_invariant():
    D = 2
    Tp = kh_inputs.random_composite(D, 4)
    rng = np.random.default_rng(9)
    G = rng.standard_normal((D ** 4, D ** 4))
    N = G @ G.T / D ** 4 + 0.1 * np.eye(D ** 4)
    A2, B2, info = bond.als(Tp, N, D, tol=0.0, max_iter=15, reg=0.0)
    h = np.array(info["history"])
    assert np.all(np.diff(h) <= 1e-14)
    assert h[-1] < h[0]
    An, Bn, _ = bond.balance_gauge(A2, B2)
    T1 = np.einsum("abURk,cdDLk->abcdLURD", A2, B2).ravel()
    T2 = np.einsum("abURk,cdDLk->abcdLURD", An, Bn).ravel()
    assert np.allclose(T2 / np.linalg.norm(T2), T1 / np.linalg.norm(T1), atol=1e-13)
    # balanced: A^T A = B^T B = diag(S)/scale
    ga = An.reshape(-1, D).T @ An.reshape(-1, D)
    gb = Bn.reshape(-1, D).T @ Bn.reshape(-1, D)
    assert np.allclose(ga, np.diag(np.diag(ga)), atol=1e-13)
    assert np.allclose(np.diag(ga) / np.trace(ga), np.diag(gb) / np.trace(gb), atol=1e-13)


def _gate_layer_gradient_ratio():
    """Norm of the gradient of the environment-weighted cost at the bond a
    gate layer returns, over its norm at the truncated-SVD start.

    A truncating layer (J != 0: gate of Schmidt rank 4, bond 4D = 8 cut to
    D = 2) on a random state.  The metric N is rebuilt from the layer's own
    converged environment; each point is first rescaled by its optimal
    factor <T''|N|T'>/<T''|N|T''> (the layer normalises A'', B''), and the
    gradient is the central-difference-pinned ``bond.cost_gradient``.  The
    layer minimises <T''-T'|N|T''-T'>, so its result is stationary (ratio ~ the
    ALS tolerance's square root); the truncated SVD is the optimum for N = 1
    only, so a layer that weighted the bond by anything else (the identity,
    a stale or transposed metric) leaves a gradient of the start's size."""
    D, chi = 2, 8
    J, K = model.couplings(0.3 * np.pi)
    A, B = kh_inputs.random_site_tensors(D, 31)
    st = eefu.State(A, B, eefu.Params(D=D, chi=chi, J=J, K=K, ctm_tol=1e-12))
    g = st.prm.gate("z", 0.2)
    eefu.apply_gate(st, "z", g)
    Tp = peps.composite(A, B, "z", g)
    N = ctmrg.metric(st.env["z"], D)

    def grad_norm(A2, B2):
        a, b, _ = bond.cost_terms(A2, B2, Tp, N)
        gA, gB = bond.cost_gradient((b / a) * A2, B2, Tp, N)
        return np.sqrt(np.sum(gA ** 2) + np.sum(gB ** 2))

    A2, B2 = peps.to_composite_frame(st.A, st.B, "z")
    A0, B0, S = bond.svd_init(Tp, D)
    assert S[D] > 0.05 * S[0]                     # the cut really truncates
    return grad_norm(A2, B2) / grad_norm(A0, B0)


def test_gate_layer_minimises_the_environment_weighted_cost():
    """Pins the wiring of the bond update inside a gate layer: the bond it
    returns is a stationary point of the cost weighted by the layer's own
    environment metric (Fig. 3(b)), not of the plain (N = 1) truncation."""
    assert _gate_layer_gradient_ratio() < 1e-4


# ---------------------------------------------------------------- plaquette flux

def _mapping_envs(A, B, chi=16):
    """The composite and converged environment of each of the three mappings."""
    out = {}
    D = A.shape[2]
    for gamma in "xyz":
        T = peps.composite(A, B, gamma)
        env, info = ctmrg.ctmrg(ctmrg.double_tensor(T), ctmrg.init_env(chi, D), 1e-13, 400)
        assert info["delta"] < 1e-12
        out[gamma] = (T, env)
    return out


def _flux_spread(seed):
    from oracle import observables
    A, B = kh_inputs.random_site_tensors(2, seed)
    envs = _mapping_envs(A, B)
    w = [observables.flux(envs[g][1], envs[g][0], g) for g in "xyz"]
    return w


@pytest.mark.parametrize("seed", [1, 3, 5])
def test_flux_agrees_across_mappings(seed):
    """The three mappings place the hexagon in three different ways (other
    composites, other sites of each composite, other Pauli components at
    each position) and contract three different networks; every hexagon of
    the 2-site cell is the same, so <W_p> must agree.  A random real state
    gives |<W>| ~ 1e-4; the imaginary part vanishes (two sigma^y)."""
    w = _flux_spread(seed)
    assert all(abs(x.imag) < 1e-15 for x in w)
    v = [x.real for x in w]
    assert min(abs(x) for x in v) > 2e-5
    assert max(v) - min(v) < 1e-6 * max(abs(x) for x in v), v


def test_bonds_between_composites_are_the_inner_bond_of_another_mapping():
    """In the gamma mapping the alpha bond joins A of one composite to B of
    its right neighbour and the alpha' bond A of one composite to B of the one
    above; their two-site correlators on the 2 x 2 plaquette equal those of
    the bond inside the composite of the alpha (alpha') mapping.  Asymmetric
    pairs (S^x_A S^z_B against S^z_A S^x_B) fix which end is A."""
    from oracle import observables
    A, B = kh_inputs.random_site_tensors(2, 7)
    envs = _mapping_envs(A, B)
    S = observables.PAULI
    I4 = np.eye(16)
    for gamma in "xyz":
        al, alp = peps.other_bonds(gamma)
        T, env = envs[gamma]
        for bond, (pa, pb) in ((al, (0, 1)), (al, (3, 2)), (alp, (3, 0)), (alp, (2, 1))):
            Ti, envi = envs[bond]
            X = ctmrg.expval_matrix(Ti, ctmrg.metric(envi, 2))
            for a, b in (("x", "z"), ("z", "x"), ("y", "y"), ("z", "z")):
                ops = [I4] * 4
                ops = list(ops)
                ops[pa] = observables.phys_op(O_A=S[a])
                ops[pb] = observables.phys_op(O_B=S[b])
                got = observables.plaquette_expectation(env, T, ops)
                want = observables.expectation(X, observables.phys_op(O_AB=np.kron(S[a], S[b])))
                assert abs(got.imag) < 1e-14
                assert abs(got.real - want) < 1e-7, (gamma, bond, pa, pb, a, b, got, want)
    # the asymmetric pairs differ, so the test sees which end is A
    Ti, envi = envs["x"]
    X = ctmrg.expval_matrix(Ti, ctmrg.metric(envi, 2))
    xz = observables.expectation(X, observables.phys_op(O_AB=np.kron(S["x"], S["z"])))
    zx = observables.expectation(X, observables.phys_op(O_AB=np.kron(S["z"], S["x"])))
    assert abs(xz - zx) > 1e-3


# ---------------------------------------------------------------- Klein duality on the iPEPS

@pytest.mark.parametrize("phi", [0.3 * np.pi, -0.35 * np.pi])
def test_klein_duality_on_the_two_site_ipeps(phi):
    """Eq. (4): H(J, K) and H(-J, K + 2J) are related by a product of
    single-site pi rotations (R_gamma on one end of every gamma bond, a
    4-sublattice pattern), and so are the Trotter gates bond by bond.  The
    beta = 0 start and every truncated update stay symmetric under the
    global pi rotations, which lets the 4-sublattice pattern act as a
    virtual gauge on the gamma legs: the 2-site-cell eeFU trajectories of
    the two couplings give the same bond energies to rounding (the
    duality the paper uses to keep 2 sublattices)."""
    J, K = model.couplings(phi)
    out = []
    for j, k in ((J, K), (-J, K + 2 * J)):
        st = _fresh(2, 8, J=j, K=k)
        res = eefu.evolve(st, 0.05, 10, measure_every=5)
        out.append(np.array([[r["E_site"], r["Hx"], r["Hy"], r["Hz"]] for r in res]))
    assert np.abs(out[0]).min() > 1e-3
    assert np.abs(out[0] - out[1]).max() < 1e-12, out[0] - out[1]
    # the map is not trivial: the couplings differ and so do the gates
    assert abs(J) > 0.1
