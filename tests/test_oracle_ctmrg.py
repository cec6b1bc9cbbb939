"""Pins of the oracle CTMRG: the norm network of a PEPS whose double layer is
the 2D Ising partition function (Onsager, Yang), with anisotropic couplings
and random bond gauges so that a transposed or swapped leg fails."""
import numpy as np
import pytest

from oracle import ctmrg, exact


def _run(T, chi, edge_vec=None, tol=1e-13, max_sweeps=400):
    a = ctmrg.double_tensor(T)
    env = ctmrg.init_env(chi, T.shape[1], edge_vec)
    env, info = ctmrg.ctmrg(a, env, tol=tol, max_sweeps=max_sweeps)
    return a, env, info


@pytest.mark.parametrize("Kh,Kv,seed", [(0.30, 0.30, None), (0.30, 0.20, 7), (0.15, 0.36, 11), (0.25, 0.25, 3)])
def test_onsager_disordered(Kh, Kv, seed):
    T = exact.ising_peps(Kh, Kv, gauge_seed=seed)
    a, env, info = _run(T, 24)
    assert info["delta"] < 1e-12
    assert abs(np.log(ctmrg.kappa(env, a)) - exact.onsager_lnZ(Kh, Kv)) < 1e-10


def test_onsager_ordered_with_broken_boundary():
    Kh, Kv = 0.6, 0.5
    T = exact.ising_peps(Kh, Kv)
    V = exact.ising_bond_root(Kh)
    a, env, info = _run(T, 24, edge_vec=np.outer(V[0], V[0]).reshape(4))
    assert abs(np.log(ctmrg.kappa(env, a)) - exact.onsager_lnZ(Kh, Kv)) < 1e-10


@pytest.mark.parametrize("K", [0.5, 0.7])
def test_yang_magnetisation(K):
    T = exact.ising_peps(K, K)
    V = exact.ising_bond_root(K)
    a, env, info = _run(T, 24, edge_vec=np.outer(V[0], V[0]).reshape(4))
    X = ctmrg.expval_matrix(T, ctmrg.metric(env, 2))
    m = np.trace(np.diag([1.0, -1.0]) @ X.T) / np.trace(X)
    assert abs(m - exact.yang_m(K)) < 1e-9


def test_rotation_is_a_4_cycle_and_moves_are_gauge_covariant():
    T = exact.ising_peps(0.3, 0.2, gauge_seed=5)
    a = ctmrg.double_tensor(T)
    assert np.array_equal(ctmrg.rotate(a, 4), a)
    # rotating the lattice by 90 degrees swaps the couplings: same free energy
    # as the transposed anisotropy
    T2 = exact.ising_peps(0.2, 0.3, gauge_seed=None)
    a2, env2, _ = _run(T2, 20)
    a1, env1, _ = _run(T, 20)
    assert abs(np.log(ctmrg.kappa(env1, a1)) - np.log(ctmrg.kappa(env2, a2))) < 1e-10


def test_product_state_is_exact_at_chi_1_and_truncation_zero():
    rng = np.random.default_rng(0)
    v = rng.standard_normal(3)
    # a D=1 product PEPS with a random 3-dim physical vector: rank-1 everything
    T = v.reshape(3, 1, 1, 1, 1)
    a, env, info = _run(T, 4)
    assert max(info["trunc"]) < 1e-28
    X = ctmrg.expval_matrix(T, ctmrg.metric(env, 1))
    assert np.allclose(X / np.trace(X), np.outer(v, v) / (v @ v), atol=1e-14)


def test_projector_is_oblique_identity_when_untruncated():
    """With chi >= rank, P P~ acts as the identity between the two halves."""
    rng = np.random.default_rng(1)
    chi, d2 = 3, 4
    Qul = rng.standard_normal((chi, d2, chi, d2))
    Qdl = rng.standard_normal((chi, d2, chi, d2))
    P, Pt, spec, trunc = ctmrg.projectors(Qul, Qdl, chi * d2, 1e-14)
    n = chi * d2
    M = Qul.reshape(n, n).T @ Qdl.reshape(n, n)
    assert np.allclose(Qul.reshape(n, n).T @ P @ Pt @ Qdl.reshape(n, n), M, atol=1e-10)
    assert trunc < 1e-28
    assert np.allclose(np.sort(spec)[::-1], np.linalg.svd(M, compute_uv=False), atol=1e-12)


def _bond_correlator(Kh, Kv, leg, broken=False, chi=24):
    """<s_i s_j> on the bond leaving a site through leg r (horizontal) or d
    (vertical), as a one-site impurity: a ket-only bond matrix
    M = V^-1 (W o s s^T) V^-T absorbed into that leg turns the bond weight
    W(s_i, s_j) of psi into s_i s_j W(s_i, s_j), so <T'|N|T> / <T|N|T> is the
    correlator (metric and mixed ket/bra expectation of the oracle)."""
    T = exact.ising_peps(Kh, Kv)
    Kb = Kh if leg == "r" else Kv
    Vi = np.linalg.inv(exact.ising_bond_root(Kb))
    W = np.array([[np.exp(Kb / 2), np.exp(-Kb / 2)], [np.exp(-Kb / 2), np.exp(Kb / 2)]])
    M = Vi @ (W * np.array([[1.0, -1.0], [-1.0, 1.0]])) @ Vi.T
    Ti = np.einsum("slurd,rR->sluRd", T, M) if leg == "r" else np.einsum("slurd,dD->slurD", T, M)
    edge = None
    if broken:
        V = exact.ising_bond_root(Kh)
        edge = np.outer(V[0], V[0]).reshape(4)
    a, env, info = _run(T, chi, edge_vec=edge)
    N = ctmrg.metric(env, 2)
    return np.trace(ctmrg.expval_matrix(Ti, N, T)) / np.trace(ctmrg.expval_matrix(T, N))


@pytest.mark.parametrize("K,broken", [(0.2, False), (0.3, False), (0.6, True)])
def test_nearest_neighbour_correlation_closed_form(K, broken):
    """Isotropic square-lattice Ising internal energy (Onsager): per site
    u/J = -coth 2K [1 + (2/pi)(2 tanh^2 2K - 1) K1(k)], k = 2 sinh 2K / cosh^2 2K,
    K1 the complete elliptic integral of the first kind; two bonds per site, so
    <s s> = -u / 2J.  Independent of the free-energy integral used above."""
    from scipy.special import ellipk
    k = 2 * np.sinh(2 * K) / np.cosh(2 * K) ** 2
    ref = 0.5 / np.tanh(2 * K) * (1 + (2 / np.pi) * (2 * np.tanh(2 * K) ** 2 - 1) * ellipk(k * k))
    for leg in ("r", "d"):
        assert abs(_bond_correlator(K, K, leg, broken) - ref) < 1e-10


@pytest.mark.parametrize("Kh,Kv", [(0.3, 0.2), (0.15, 0.36)])
def test_anisotropic_correlations_are_free_energy_derivatives(Kh, Kv):
    """d(-beta f)/dK_h = <s s>_horizontal and d(-beta f)/dK_v = <s s>_vertical
    (central differences of the Onsager integral, step 1e-5): a swap of the
    horizontal and vertical legs of the metric fails."""
    h = 1e-5
    dh = (exact.onsager_lnZ(Kh + h, Kv) - exact.onsager_lnZ(Kh - h, Kv)) / (2 * h)
    dv = (exact.onsager_lnZ(Kh, Kv + h) - exact.onsager_lnZ(Kh, Kv - h)) / (2 * h)
    assert abs(dh - dv) > 0.05
    assert abs(_bond_correlator(Kh, Kv, "r") - dh) < 1e-9
    assert abs(_bond_correlator(Kh, Kv, "d") - dv) < 1e-9


def _directed_ising(Kh, Kv, hh, hv):
    """Ising PEPS with directed bond weights: the ket bond between a site's
    leg r (d) and its neighbour's leg l (u) is W(s_i, s_j) with
    W^2 = exp(K s s' + h (s - s')).  W is not symmetric, so neither are the
    corners and edges; on the infinite lattice the h terms telescope (each
    site is the left end of one horizontal bond and the right end of another),
    so the free energy per site is Onsager's for every h."""
    s = np.array([1.0, -1.0])

    def W(K, h):
        return np.exp(0.5 * (K * np.outer(s, s) + h * (s[:, None] - s[None, :])))
    I = np.eye(2)
    return np.einsum("sl,su,sr,sd->slurd", W(Kh, hh).T, W(Kv, hv).T, I, I)


@pytest.mark.parametrize("hh,hv", [(0.4, 0.0), (0.4, -0.7)])
def test_onsager_with_reflection_asymmetric_bond_weights(hh, hv):
    Kh, Kv = 0.3, 0.2
    T = _directed_ising(Kh, Kv, hh, hv)
    a, env, info = _run(T, 16)
    assert info["delta"] < 1e-12
    assert abs(np.log(ctmrg.kappa(env, a)) - exact.onsager_lnZ(Kh, Kv)) < 1e-10


@pytest.mark.filterwarnings("ignore::scipy.linalg.LinAlgWarning")
@pytest.mark.parametrize("Kh", [0.3, 0.6, 1.0])
def test_correlation_length_of_decoupled_chains(Kh):
    """K_v = 0: the rows are independent 1D Ising chains, the environment is
    exact, and the channel transfer matrix reduces to the chain's, whose
    eigenvalue ratio is tanh K_h: xi_x = -1 / ln tanh K_h; nothing is
    correlated along y."""
    T = exact.ising_peps(Kh, 0.0)
    a, env, info = _run(T, 8)
    assert abs(ctmrg.correlation_length(env, a, 0) - (-1.0 / np.log(np.tanh(Kh)))) < 1e-12
    assert ctmrg.correlation_length(env, a, 1) < 0.05


def test_correlation_length_vertical_channel_is_the_rotated_horizontal_one():
    """On a network without reflection symmetry (directed bond weights), xi
    along y of T equals xi along x of T turned by a quarter (its own CTMRG)."""
    T = _directed_ising(0.3, 0.2, 0.4, -0.7)
    a, env, _ = _run(T, 16, tol=1e-14)
    Tr = T.transpose(0, 2, 3, 4, 1)            # new (l,u,r,d) = old (u,r,d,l)
    ar, envr, _ = _run(Tr, 16, tol=1e-14)
    assert abs(ctmrg.correlation_length(env, a, 1) - ctmrg.correlation_length(envr, ar, 0)) < 1e-9
    assert abs(ctmrg.correlation_length(env, a, 0) - ctmrg.correlation_length(envr, ar, 1)) < 1e-9


# ---------------------------------------------------------------- 2 x 2 cluster

SZ2 = np.diag([1.0, -1.0])
I2 = np.eye(2)
# plaquette positions: 0 upper-left, 1 upper-right, 2 lower-right, 3 lower-left
PAIRS = {"h": [(0, 1), (3, 2)], "v": [(0, 3), (1, 2)], "diag": [(0, 2), (1, 3)]}


def _pair_ops(i, j, O=SZ2, p=2):
    ops = [np.eye(p) for _ in range(4)]
    ops[i] = O
    ops[j] = O
    return ops


@pytest.mark.parametrize("Kh,Kv,seed", [(0.3, 0.2, 7), (0.15, 0.36, 11)])
def test_plaquette_neighbour_pairs_are_free_energy_derivatives(Kh, Kv, seed):
    """<s s> of the two horizontal pairs of the 2 x 2 cluster is d(-beta f)/dK_h
    and of the two vertical pairs d(-beta f)/dK_v (central differences of the
    Onsager integral); with anisotropic couplings and random bond gauges, a
    cluster that joins the wrong legs or places the sites wrongly fails."""
    from oracle import observables
    h = 1e-5
    dh = (exact.onsager_lnZ(Kh + h, Kv) - exact.onsager_lnZ(Kh - h, Kv)) / (2 * h)
    dv = (exact.onsager_lnZ(Kh, Kv + h) - exact.onsager_lnZ(Kh, Kv - h)) / (2 * h)
    T = exact.ising_peps(Kh, Kv, gauge_seed=seed)
    a, env, _ = _run(T, 24)
    for kind, want in (("h", dh), ("v", dv)):
        for i, j in PAIRS[kind]:
            got = observables.plaquette_expectation(env, T, _pair_ops(i, j))
            assert abs(got - want) < 1e-9, (kind, i, j, got, want)


@pytest.mark.parametrize("hh,hv", [(0.4, -0.7)])
def test_plaquette_pairs_without_reflection_symmetry(hh, hv):
    """Directed bond weights (no reflection symmetry of the network, the
    same Boltzmann weights on the infinite lattice): the pairs still give the
    plain model's derivatives, and the two diagonals agree."""
    from oracle import observables
    Kh, Kv = 0.3, 0.2
    h = 1e-5
    dh = (exact.onsager_lnZ(Kh + h, Kv) - exact.onsager_lnZ(Kh - h, Kv)) / (2 * h)
    dv = (exact.onsager_lnZ(Kh, Kv + h) - exact.onsager_lnZ(Kh, Kv - h)) / (2 * h)
    T = _directed_ising(Kh, Kv, hh, hv)
    a, env, _ = _run(T, 16, tol=1e-14)
    for kind, want in (("h", dh), ("v", dv)):
        for i, j in PAIRS[kind]:
            assert abs(observables.plaquette_expectation(env, T, _pair_ops(i, j)) - want) < 1e-9
    d = [observables.plaquette_expectation(env, T, _pair_ops(i, j)) for i, j in PAIRS["diag"]]
    assert abs(d[0] - d[1]) < 1e-9
    assert dv < abs(d[0]) < dh or dh < abs(d[0]) < dv or abs(d[0]) < min(dh, dv)


def test_plaquette_single_operator_is_the_site_expectation():
    """One operator at any of the four positions (identity elsewhere) is the
    one-site expectation Tr(O X) / Tr(X) of the environment metric, up to the
    finite-chi difference of the two environments (3e-8 at chi = 16)."""
    from oracle import observables
    import kh_inputs
    T = kh_inputs.random_composite(2, 3, p=4)
    a, env, info = _run(T, 16)
    rng = np.random.default_rng(2)
    O = rng.standard_normal((4, 4))
    O = O + O.T
    X = ctmrg.expval_matrix(T, ctmrg.metric(env, 2))
    want = np.trace(O @ X.T) / np.trace(X)
    assert abs(want) > 1e-2
    for pos in range(4):
        ops = [np.eye(4) for _ in range(4)]
        ops[pos] = O
        got = observables.plaquette_expectation(env, T, ops)
        assert abs(got - want) < 1e-6 * max(1.0, abs(want)), (pos, got, want)
