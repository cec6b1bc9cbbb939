"""The pins catch plausible mistakes: each test plants one mistake in the
oracle (a dropped term, a wrong sign, a transposed leg or operand, a wrong
time step) with monkeypatch, on the CPU, and checks that the pin meant to
guard that part now fails.  Each pin is restated here as a function that
returns its worst deviation in units of its tolerance (< 1 = the pin
passes); `test_pins_pass_unmutated` checks the restatements themselves.

Transformations that leave every result unchanged are not planted:
transposing the expectation matrix (X = T N T^T is symmetric for real
tensors), exchanging ket and bra legs inside the metric (the layers are
identical), or reversing the two chi legs of the new edge of a move (the
same projector pair serves both cuts, so this only relabels the fixed
point; it reproduces Onsager's free energy even with reflection-asymmetric
bond weights)."""
import numpy as np
import pytest
from scipy.linalg import expm

import kh_inputs
from oracle import bond, ctmrg, eefu, exact, model, observables, peps


def _fresh(D, chi, **kw):
    A, B = peps.product_state(D)
    return eefu.State(A, B, eefu.Params(D=D, chi=chi, **kw))


# ------------------------------------------------------------------ pins

def pin_bond_spectrum():
    J, K = model.couplings(0.3 * np.pi)
    return max(np.abs(np.linalg.eigvalsh(model.bond_hamiltonian(g, J, K)) - exact.bond_spectrum(J, K)).max()
               for g in "xyz") / 1e-14


def pin_beta0():
    r = eefu.measure(_fresh(2, 6, J=0.5, K=1.2))
    return max(abs(r[k]) for k in ("E_site", "Hx", "Hy", "Hz", "Ax", "Az", "Bx", "Bz")) / 1e-15


def pin_dimer(gamma="x"):
    J, K = model.couplings(0.3 * np.pi)
    st = _fresh(4, 6, J=J, K=K)
    tau = 0.05
    eefu.apply_gate(st, gamma, st.prm.gate(gamma, tau))
    r = eefu.measure(st)
    want = exact.dimer_energy(J, K, 2 * tau)
    dev = [abs(r["H" + gamma] - want), abs(r["E_site"] - 0.5 * want)]
    dev += [abs(r["H" + g]) for g in "xyz" if g != gamma]
    return max(dev) / 1e-13


def pin_kz_only():
    Kz = 1.3
    st = _fresh(2, 6, J=0.0, K=0.0, K_gamma={"x": 0.0, "y": 0.0, "z": Kz})
    for _ in range(4):
        eefu.trotter_step(st, 0.05)
    return abs(eefu.measure(st)["E_site"] - exact.kz_only_energy(Kz, 0.2)) / 1e-10


def pin_field_only(hA=0.7, hB=-0.3):
    st = _fresh(2, 4, J=0.0, K=0.0, hA=hA, hB=hB)
    for _ in range(6):
        eefu.trotter_step(st, 0.05)
    r = eefu.measure(st)
    eA, mA = exact.field_only(hA, 0.3)
    eB, mB = exact.field_only(hB, 0.3)
    return max(abs(r["Az"] - mA), abs(r["Bz"] - mB), abs(r["E_site"] - 0.5 * (eA + eB))) / 1e-12


def pin_mappings(D=3, chi=9):
    """After two Trotter steps with a staggered field (every bond type
    entangled), the three gamma-mapped environments give the same site
    moments."""
    J, K = model.couplings(0.3 * np.pi)
    st = _fresh(D, chi, J=J, K=K, hA=0.5, hB=-0.2)
    eefu.evolve(st, 0.02, 2)
    eefu.measure(st)
    vals = []
    for gamma in "xyz":
        T = peps.composite(st.A, st.B, gamma)
        X = ctmrg.expval_matrix(T, ctmrg.metric(st.obs_env[gamma], D))
        vals.append(observables.site_moments(X))
    return max(max(m[k] for m in vals) - min(m[k] for m in vals) for k in ("Az", "Bz", "Ax", "Bx")) / 1e-9


def pin_onsager(Kh=0.3, Kv=0.2, seed=7, chi=16):
    T = exact.ising_peps(Kh, Kv, gauge_seed=seed)
    a = ctmrg.double_tensor(T)
    env, _ = ctmrg.ctmrg(a, ctmrg.init_env(chi, 2), tol=1e-13, max_sweeps=300)
    return abs(np.log(ctmrg.kappa(env, a)) - exact.onsager_lnZ(Kh, Kv)) / 1e-10


def pin_bond_correlations(Kh=0.3, Kv=0.2):
    """<s s> on a horizontal (leg r) and a vertical (leg d) bond, as one-site
    impurities, against the coupling derivatives of the free energy."""
    T = exact.ising_peps(Kh, Kv)
    a = ctmrg.double_tensor(T)
    env, _ = ctmrg.ctmrg(a, ctmrg.init_env(16, 2), tol=1e-13, max_sweeps=300)
    N = ctmrg.metric(env, 2)
    h = 1e-5
    dev = []
    for leg, Kb in (("r", Kh), ("d", Kv)):
        Vi = np.linalg.inv(exact.ising_bond_root(Kb))
        W = np.array([[np.exp(Kb / 2), np.exp(-Kb / 2)], [np.exp(-Kb / 2), np.exp(Kb / 2)]])
        M = Vi @ (W * np.array([[1.0, -1.0], [-1.0, 1.0]])) @ Vi.T
        Ti = np.einsum("slurd,rR->sluRd", T, M) if leg == "r" else np.einsum("slurd,dD->slurD", T, M)
        c = np.trace(ctmrg.expval_matrix(Ti, N, T)) / np.trace(ctmrg.expval_matrix(T, N))
        if leg == "r":
            ref = (exact.onsager_lnZ(Kh + h, Kv) - exact.onsager_lnZ(Kh - h, Kv)) / (2 * h)
        else:
            ref = (exact.onsager_lnZ(Kh, Kv + h) - exact.onsager_lnZ(Kh, Kv - h)) / (2 * h)
        dev.append(abs(c - ref))
    return max(dev) / 1e-9


def pin_eckart_young():
    D = 2
    Tp = kh_inputs.random_composite(D, 3)
    _, _, S = bond.svd_init(Tp, D)
    _, _, info = bond.als(Tp, np.eye(D ** 4), D, tol=1e-15, max_iter=20, reg=0.0)
    return abs(info["rel_cost"] - np.sum(S[D:] ** 2) / np.sum(S ** 2)) / 1e-12


def pin_balanced_gauge():
    D = 2
    Tp = kh_inputs.random_composite(D, 4)
    rng = np.random.default_rng(9)
    G = rng.standard_normal((D ** 4, D ** 4))
    N = G @ G.T / D ** 4 + 0.1 * np.eye(D ** 4)
    A2, B2, _ = bond.als(Tp, N, D, tol=0.0, max_iter=5, reg=0.0)
    An, Bn, _ = bond.balance_gauge(A2, B2)
    T1 = np.einsum("abURk,cdDLk->abcdLURD", A2, B2).ravel()
    T2 = np.einsum("abURk,cdDLk->abcdLURD", An, Bn).ravel()
    ga = An.reshape(-1, D).T @ An.reshape(-1, D)
    gb = Bn.reshape(-1, D).T @ Bn.reshape(-1, D)
    dev = [np.abs(T2 / np.linalg.norm(T2) - T1 / np.linalg.norm(T1)).max(),
           np.abs(ga - np.diag(np.diag(ga))).max(),
           np.abs(np.diag(ga) / np.trace(ga) - np.diag(gb) / np.trace(gb)).max()]
    return max(dev) / 1e-13


def pin_environment_weighted_layer():
    """The bond a truncating gate layer returns is stationary for the cost
    weighted by the layer's own environment metric (gradient ratio against
    the truncated-SVD start, see test_oracle_eefu)."""
    from test_oracle_eefu import _gate_layer_gradient_ratio
    return _gate_layer_gradient_ratio() / 1e-4


def pin_plaquette_pairs(Kh=0.3, Kv=0.2, seed=7):
    """Horizontal and vertical <s s> of the 2 x 2 cluster against the Onsager
    derivatives (see test_oracle_ctmrg)."""
    h = 1e-5
    dh = (exact.onsager_lnZ(Kh + h, Kv) - exact.onsager_lnZ(Kh - h, Kv)) / (2 * h)
    dv = (exact.onsager_lnZ(Kh, Kv + h) - exact.onsager_lnZ(Kh, Kv - h)) / (2 * h)
    T = exact.ising_peps(Kh, Kv, gauge_seed=seed)
    env, _ = ctmrg.ctmrg(ctmrg.double_tensor(T), ctmrg.init_env(24, 2), 1e-13, 400)
    sz = np.diag([1.0, -1.0])
    dev = []
    for (i, j), want in (((0, 1), dh), ((3, 2), dh), ((0, 3), dv), ((1, 2), dv)):
        ops = [np.eye(2)] * 4
        ops = list(ops)
        ops[i] = sz
        ops[j] = sz
        dev.append(abs(observables.plaquette_expectation(env, T, ops) - want))
    return max(dev) / 1e-9


def pin_flux_mappings(seed=3):
    """<W_p> agrees between the three mappings (see test_oracle_eefu)."""
    A, B = kh_inputs.random_site_tensors(2, seed)
    w = []
    for gamma in "xyz":
        T = peps.composite(A, B, gamma)
        env, _ = ctmrg.ctmrg(ctmrg.double_tensor(T), ctmrg.init_env(16, 2), 1e-13, 400)
        w.append(observables.flux(env, T, gamma).real)
    return (max(w) - min(w)) / (1e-6 * max(abs(x) for x in w))


PINS = [pin_bond_spectrum, pin_beta0, pin_dimer, pin_kz_only, pin_field_only, pin_mappings, pin_onsager,
        pin_bond_correlations, pin_eckart_young, pin_balanced_gauge, pin_environment_weighted_layer,
        pin_plaquette_pairs, pin_flux_mappings]


@pytest.mark.parametrize("pin", PINS, ids=lambda p: p.__name__)
def test_pins_pass_unmutated(pin):
    assert pin() < 1.0


# ------------------------------------------------------------------ planted mistakes

def _fails(pin):
    v = pin()
    return not (v < 1.0)          # NaN counts as a failure too


def test_z_layer_with_the_xy_time_step_is_caught(monkeypatch):
    monkeypatch.setattr(model, "trotter_layers", lambda db: [("x", db / 4), ("y", db / 4), ("z", db / 4),
                                                             ("y", db / 4), ("x", db / 4)])
    assert _fails(pin_kz_only)


def test_bias_with_the_wrong_sign_is_caught(monkeypatch):
    orig = model.bond_hamiltonian
    monkeypatch.setattr(model, "bond_hamiltonian",
                        lambda g, J, K, Kg=None, hA=0.0, hB=0.0: orig(g, J, K, Kg, -hA, -hB))
    assert _fails(pin_field_only)


def test_bias_in_every_layer_is_caught(monkeypatch):
    def gate(gamma, tau, J, K, K_gamma=None, hA=0.0, hB=0.0):
        return expm(-tau * model.bond_hamiltonian(gamma, J, K, K_gamma, hA, hB))
    monkeypatch.setattr(model, "gate", gate)
    assert _fails(pin_field_only)


def test_dropped_heisenberg_component_is_caught(monkeypatch):
    orig = model.bond_hamiltonian
    SYSY = np.real(np.kron(model.SY, model.SY))
    monkeypatch.setattr(model, "bond_hamiltonian",
                        lambda g, J, K, Kg=None, hA=0.0, hB=0.0: orig(g, J, K, Kg, hA, hB) - J * SYSY)
    assert _fails(pin_bond_spectrum)


def test_unentangled_ancilla_at_beta0_is_caught(monkeypatch):
    def product_state(D):
        A = np.zeros((2, 2, D, D, D))
        A[0, 0, 0, 0, 0] = 1.0
        A[1, 0, 0, 0, 0] = 1.0
        return A, A.copy()
    monkeypatch.setattr(peps, "product_state", product_state)
    assert _fails(pin_beta0)


def test_composite_with_swapped_b_legs_is_caught(monkeypatch):
    # B's l and d legs exchanged in the composite (not in the inverse split);
    # invisible after a single layer, where only the gated bond is nontrivial
    orig = peps.composite
    monkeypatch.setattr(peps, "composite", lambda A, B, gamma, g=None: orig(A, B, gamma, g).transpose(0, 4, 2, 3, 1))
    assert not _fails(pin_dimer)
    assert _fails(pin_mappings)


def test_projectors_without_inverse_square_root_are_caught(monkeypatch):
    orig = ctmrg.projectors

    def projectors(Qul, Qdl, chi, cut):
        P, Pt, spec, trunc = orig(Qul, Qdl, chi, cut)
        r = np.sqrt(spec)
        return P * r[None, :], r[:, None] * Pt, spec, trunc
    monkeypatch.setattr(ctmrg, "projectors", projectors)
    assert _fails(pin_onsager)


def test_clockwise_frame_rotation_is_caught(monkeypatch):
    orig = ctmrg.rotate
    monkeypatch.setattr(ctmrg, "rotate", lambda a, times=1: orig(a, -times))
    assert _fails(pin_onsager)


def test_transposed_edge_in_the_enlarged_corner_is_caught(monkeypatch):
    orig = ctmrg.enlarged_corners
    monkeypatch.setattr(ctmrg, "enlarged_corners",
                        lambda C1, E1, E4, C4, E3, a: orig(C1, E1, E4.transpose(2, 1, 0), C4, E3, a))
    assert _fails(pin_onsager)


def test_kappa_without_the_empty_ring_is_caught(monkeypatch):
    orig = ctmrg.kappa

    def kappa(env, a):
        C1, C2, C3, C4 = env.C
        return orig(env, a) / np.trace(C1 @ C2 @ C3 @ C4)
    monkeypatch.setattr(ctmrg, "kappa", kappa)
    assert _fails(pin_onsager)


def test_metric_with_horizontal_and_vertical_legs_swapped_is_caught(monkeypatch):
    orig = ctmrg.metric_d2
    monkeypatch.setattr(ctmrg, "metric_d2", lambda env: orig(env).transpose(0, 2, 1, 3))
    assert _fails(pin_bond_correlations)


def test_normal_equations_with_the_physical_legs_transposed_are_caught(monkeypatch):
    # S_A built from T' with the (sA, aA) and (sB, aB) pairs exchanged.  (A
    # negated S_A is no mistake: A'' flips sign, B'' follows, T'' is unchanged.)
    orig = bond.normal_equations_A

    def normal_equations_A(B2, Tp, N, D):
        Tt = Tp.reshape((2, 2, 2, 2) + Tp.shape[1:]).transpose(2, 3, 0, 1, 4, 5, 6, 7).reshape(Tp.shape)
        return orig(B2, Tt, N, D)
    monkeypatch.setattr(bond, "normal_equations_A", normal_equations_A)
    assert _fails(pin_eckart_young)


def test_one_sided_gauge_split_is_caught(monkeypatch):
    def balance_gauge(A2, B2):
        D = A2.shape[-1]
        Qa, Ra = np.linalg.qr(A2.reshape(-1, D))
        Qb, Rb = np.linalg.qr(B2.reshape(-1, D))
        U, S, Vt = np.linalg.svd(Ra @ Rb.T)
        return (Qa @ (U * S)).reshape(A2.shape), (Qb @ Vt.T).reshape(B2.shape), S
    monkeypatch.setattr(bond, "balance_gauge", balance_gauge)
    assert _fails(pin_balanced_gauge)


def test_energy_without_the_half_per_site_is_caught(monkeypatch):
    orig = eefu.measure

    def measure(st):
        r = orig(st)
        r["E_site"] *= 2.0
        return r
    monkeypatch.setattr(eefu, "measure", measure)
    assert _fails(pin_dimer)


def test_sublattice_moments_swapped_are_caught(monkeypatch):
    orig = observables.site_moments

    def site_moments(X):
        m = orig(X)
        return {("B" if k[0] == "A" else "A") + k[1:]: v for k, v in m.items()}
    monkeypatch.setattr(observables, "site_moments", site_moments)
    assert _fails(pin_field_only)


def test_bond_update_without_the_environment_metric_is_caught(monkeypatch):
    """The gate layer hands the identity instead of N to the bond update: the
    update degenerates to the plain truncated SVD."""
    orig = bond.als
    monkeypatch.setattr(bond, "als", lambda Tp, N, D, *a, **k: orig(Tp, np.eye(N.shape[0]), D, *a, **k))
    assert _fails(pin_environment_weighted_layer)


def test_cluster_with_two_sites_exchanged_is_caught(monkeypatch):
    """The upper-right and lower-left sites trade places: a horizontal pair
    becomes a vertical one."""
    orig = ctmrg.cluster_2x2
    monkeypatch.setattr(ctmrg, "cluster_2x2", lambda env, a, b, c, d: orig(env, a, d, c, b))
    assert _fails(pin_plaquette_pairs)


def test_cluster_with_a_transposed_corner_is_caught(monkeypatch):
    orig = ctmrg.cluster_2x2

    def cluster_2x2(env, *a):
        e = env.copy()
        e.C[1] = e.C[1].T
        return orig(e, *a)
    monkeypatch.setattr(ctmrg, "cluster_2x2", cluster_2x2)
    assert _fails(pin_plaquette_pairs)


@pytest.mark.parametrize("mistake", ["alpha_swapped_upper_left", "mirrored", "rotated", "sublattices_swapped"])
def test_flux_with_misplaced_operators_is_caught(monkeypatch, mistake):
    orig = observables.flux_operators

    def flux_operators(gamma):
        ops = orig(gamma)
        al, alp = peps.other_bonds(gamma)
        s = observables.PAULI
        if mistake == "alpha_swapped_upper_left":
            ops[0] = observables.phys_op(O_A=s[al], O_B=s[alp])
        elif mistake == "mirrored":
            ops = [ops[1], ops[0], ops[3], ops[2]]
        elif mistake == "rotated":
            ops = ops[1:] + ops[:1]
        else:
            ops = [observables.phys_op(O_A=s[al], O_B=s[alp]), observables.phys_op(O_A=s[gamma]),
                   observables.phys_op(O_A=s[alp], O_B=s[al]), observables.phys_op(O_B=s[gamma])]
        return ops
    monkeypatch.setattr(observables, "flux_operators", flux_operators)
    assert _fails(pin_flux_mappings)
