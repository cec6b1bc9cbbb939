"""Writes tests/golden/wide_bond_parity_D8_chi8.json: the oracle's converged
values for one eeFU gate layer plus the observables at bond dimension D = 8,
where the bond matrix of the update, T' as (4 D^2) x (4 D^2) = 256 x 256, is
wider than the GPU library's one-CTA Jacobi and its truncated-SVD start comes
from a subspace iteration instead.

Calls only the CPU oracle (``oracle/``) on the seeded inputs of
``kh_inputs``; nothing here touches the CUDA library.  Run from the repo
root (a few minutes on eight cores):

    python tests/golden/make_wide_bond_parity.py

Workload: site tensors A, B ~ N(0,1), unit Frobenius norm (seed 31), a
generic state; the z layer of a Kitaev-Heisenberg Trotter step at
phi = 0.3 pi (J = cos phi, K = 2 sin phi), g = exp(-(dbeta/2) H^z) with
dbeta = 0.02 (Sec. III, Eq. 6); CTMRG at chi = 8 converged to 1e-10 in the
normalised spectra, FP64 cut-off 1e-12; the metric, ALS and gauge of the bond
update (Fig. 3(b)); then the three gamma-mapped CTMRGs of the un-gated state
and the observables of Sec. V.
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import kh_inputs  # noqa: E402
from oracle import eefu, model  # noqa: E402

PHI = 0.3 * np.pi
CASE = dict(D=8, chi=8, phi=PHI, J=float(model.couplings(PHI)[0]), K=float(model.couplings(PHI)[1]), dbeta=0.02,
            seed=31, svd_cut=1e-12, ctm_tol=1e-10, ctm_max_sweeps=400)
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "wide_bond_parity_D8_chi8.json")


def main():
    c = CASE
    A, B = kh_inputs.random_site_tensors(c["D"], c["seed"])
    prm = eefu.Params(D=c["D"], chi=c["chi"], J=c["J"], K=c["K"], ctm_tol=c["ctm_tol"],
                      ctm_max_sweeps=c["ctm_max_sweeps"], svd_cut=c["svd_cut"])
    st = eefu.State(A, B, prm)
    t0 = time.time()
    info = eefu.apply_gate(st, "z", prm.gate("z", c["dbeta"] / 2))
    t1 = time.time()
    obs = eefu.measure(st)
    t2 = time.time()
    out = {
        "case": c,
        "gate_layer": {"gamma": "z", "rel_cost": info["rel_cost"], "als_iters": info["als_iters"],
                       "ctm_sweeps": info["ctm_sweeps"], "ctm_delta": info["ctm_delta"], "trunc": info["trunc"],
                       "spectra": [list(map(float, s)) for s in info["spectra"]]},
        "observables": {k: float(v) for k, v in obs.items()},
        "seconds": {"gate_layer": t1 - t0, "observables": t2 - t1},
    }
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote %s (gate layer %.0f s, %d sweeps; observables %.0f s)" % (OUT, t1 - t0, info["ctm_sweeps"],
                                                                            t2 - t1))


if __name__ == "__main__":
    main()
