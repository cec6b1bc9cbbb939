"""Writes tests/golden/bench_parity_D4_chi64.json: the oracle's converged
values for one eeFU gate layer plus the observables at the benchmark's full
size (D = 4, chi = 64, p = 16, Kitaev point K = 1, J = 0, dbeta = 0.01).

Calls only the CPU oracle (``oracle/``) on the seeded inputs of
``kh_inputs``; nothing here touches the CUDA library.  Run from the repo
root (about ten minutes on eight cores):

    python tests/golden/make_bench_parity.py

Workload: site tensors A, B ~ N(0,1), unit Frobenius norm (seed 21) -- a
generic state whose environments have no exact degeneracies and a slowly
decaying projector spectrum, so all chi kept singular values lie above the
single-precision cut-off; the z layer of a Trotter step, g = exp(-(dbeta/2)
H^z) (Sec. III, Eq. 6); CTMRG of the gated composite converged to 1e-10 in
the normalised spectra; the metric, ALS and gauge of the bond update
(Fig. 3(b)); then the three gamma-mapped CTMRGs of the un-gated state and the
observables of Sec. V.  The cut-off is the single-precision path's (1e-4,
above the resolution floor of its projector spectra), so both sides apply the
same truncation rule.
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
from oracle import eefu  # noqa: E402

CASE = dict(D=4, chi=64, J=0.0, K=1.0, dbeta=0.01, seed=21, svd_cut=1e-4, ctm_tol=1e-10, ctm_max_sweeps=400)
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "bench_parity_D4_chi64.json")
if len(sys.argv) > 2:                  # python make_bench_parity.py <svd_cut> <output>
    CASE["svd_cut"] = float(sys.argv[1])
    OUT = sys.argv[2]


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
