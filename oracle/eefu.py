"""Exact-environment full update driver (oracle).

Test infrastructure only (see ``oracle/__init__``).

Sec. III: |psi(beta)> = (e^{-dbeta H/2})^N |psi(0)>, each factor the
second-order Trotter product of Eq. (6).  Each gate layer gamma:
  1. builds the gated composite T' (exact A'-B', gamma bond hidden inside);
  2. converges the CTMRG of T' (warm start from this gamma's last
     environment) -- the exact environment of the gamma bond;
  3. forms the metric N and updates the bond A''-B'' (``bond.als``);
  4. fixes the bond gauge and normalises.
"""
import numpy as np

from . import bond, ctmrg, model, observables, peps


class Params:
    def __init__(self, D, chi, J=0.0, K=1.0, K_gamma=None, hA=0.0, hB=0.0,
                 ctm_tol=1e-12, ctm_max_sweeps=100, ctm_min_sweeps=1, svd_cut=1e-12,
                 als_tol=1e-12, als_max_iter=50, als_reg=1e-12):
        self.D, self.chi = D, chi
        self.J, self.K, self.K_gamma, self.hA, self.hB = J, K, K_gamma, hA, hB
        self.ctm_tol, self.ctm_max_sweeps, self.ctm_min_sweeps = ctm_tol, ctm_max_sweeps, ctm_min_sweeps
        self.svd_cut = svd_cut
        self.als_tol, self.als_max_iter, self.als_reg = als_tol, als_max_iter, als_reg

    def gate(self, gamma, tau):
        return model.gate(gamma, tau, self.J, self.K, self.K_gamma, self.hA, self.hB)


class State:
    """Site tensors plus one CTM environment per mapping (eeFU) and per
    mapping for measurements."""

    def __init__(self, A, B, prm):
        self.A = np.array(A, dtype=np.float64)
        self.B = np.array(B, dtype=np.float64)
        self.prm = prm
        self.env = {g: None for g in model.GAMMAS}
        self.obs_env = {g: None for g in model.GAMMAS}
        self.log = []

    def _env(self, store, gamma):
        e = store[gamma]
        if e is None:
            e = ctmrg.init_env(self.prm.chi, self.prm.D)
        return e


def apply_gate(st, gamma, g):
    """One eeFU gate layer on bond direction gamma.  Returns info dict."""
    prm = st.prm
    D = prm.D
    Tp = peps.composite(st.A, st.B, gamma, g)
    a = ctmrg.double_tensor(Tp)
    env, cinfo = ctmrg.ctmrg(a, st._env(st.env, gamma), prm.ctm_tol, prm.ctm_max_sweeps,
                             prm.ctm_min_sweeps, prm.svd_cut)
    st.env[gamma] = env
    N = ctmrg.metric(env, D)
    A2, B2, binfo = bond.als(Tp, N, D, prm.als_tol, prm.als_max_iter, prm.als_reg)
    A2, B2, _ = bond.balance_gauge(A2, B2)
    st.A, st.B = peps.split_composite_legs(A2, B2, gamma, D)
    info = dict(gamma=gamma, ctm_sweeps=cinfo["sweeps"], ctm_delta=cinfo["delta"],
                trunc=max(cinfo["trunc"]), spectra=cinfo["spectra"],
                als_iters=binfo["iters"], rel_cost=binfo["rel_cost"])
    st.log.append(info)
    return info


def trotter_step(st, dbeta):
    infos = []
    for gamma, tau in model.trotter_layers(dbeta):
        infos.append(apply_gate(st, gamma, st.prm.gate(gamma, tau)))
    return infos


def measure(st):
    """E/site, <S^a>_{A,B} and the largest truncation error, from three
    gamma-mapped CTMRGs of the un-gated state (warm start from the last
    measurement environment, else from the eeFU environment)."""
    prm = st.prm
    D = prm.D
    res = {}
    Eb = {}
    trunc = 0.0
    X_z = None
    for gamma in model.GAMMAS:
        T = peps.composite(st.A, st.B, gamma)
        a = ctmrg.double_tensor(T)
        start = st.obs_env[gamma]
        if start is None:
            start = st.env[gamma].copy() if st.env[gamma] is not None else ctmrg.init_env(prm.chi, D)
        env, cinfo = ctmrg.ctmrg(a, start, prm.ctm_tol, prm.ctm_max_sweeps, prm.ctm_min_sweeps,
                                 prm.svd_cut)
        st.obs_env[gamma] = env
        trunc = max(trunc, max(cinfo["trunc"]))
        N = ctmrg.metric(env, D)
        X = ctmrg.expval_matrix(T, N)
        H = model.bond_hamiltonian(gamma, prm.J, prm.K, prm.K_gamma)
        Eb[gamma] = observables.expectation(X, observables.phys_op(O_AB=H))
        if gamma == "z":
            X_z = X
    mom = observables.site_moments(X_z)
    res.update({"H" + g: Eb[g] for g in model.GAMMAS})
    res.update(mom)
    res["E_site"] = 0.5 * sum(Eb.values()) - 0.5 * (prm.hA * mom["Az"] + prm.hB * mom["Bz"])
    res["trunc"] = trunc
    return res


def evolve(st, dbeta, n_steps, measure_every=0):
    out = []
    for n in range(1, n_steps + 1):
        trotter_step(st, dbeta)
        if measure_every and n % measure_every == 0:
            r = measure(st)
            r["beta"] = n * dbeta
            out.append(r)
    return out
