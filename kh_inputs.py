"""Seeded synthetic inputs shared by the oracle tests and the GPU library tests.

This module holds no arithmetic of the method: only random draws and fixed
workload descriptions.  Both the CPU oracle and the CUDA path receive the
same arrays from here.

Workloads (imaginary-time eeFU for the Kitaev-Heisenberg model on the
honeycomb lattice; the paper gives (phi, D, chi, dbeta) ranges but no data
set, so inputs are synthetic):
  * site tensors A, B of shape [2 spin][2 ancilla][D][D][D], entries
    N(0,1) from ``numpy.random.default_rng(seed)``, each scaled to unit
    Frobenius norm;
  * couplings J = cos(phi), K = 2 sin(phi) at the stated angle.
"""
import numpy as np

WORKLOADS = {
    # small case: D=2, chi=16, phi=0.3 pi, dbeta=0.01, beta 0 -> 0.5
    "kh_D2_chi16": dict(D=2, chi=16, phi=0.3 * np.pi, dbeta=0.01, n_steps=50),
    # timed case: pure Kitaev K=1, J=0 (phi=pi/2 with A=1/2), D=4, chi=64, dbeta=0.01
    "kitaev_D4_chi64": dict(D=4, chi=64, J=0.0, K=1.0, dbeta=0.01, n_steps=500),
}


def random_site_tensors(D, seed):
    """A, B ~ N(0,1), each normalised to unit Frobenius norm."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((2, 2, D, D, D))
    B = rng.standard_normal((2, 2, D, D, D))
    return A / np.linalg.norm(A), B / np.linalg.norm(B)


def random_composite(D, seed, p=16):
    """A generic composite site tensor T[p][D][D][D][D], N(0,1), unit norm."""
    rng = np.random.default_rng(seed)
    T = rng.standard_normal((p, D, D, D, D))
    return T / np.linalg.norm(T)


def perturbed_product_state(D, seed, eps=0.05):
    """beta=0 product state (spin maximally entangled with ancilla at virtual
    index 0) plus eps * N(0,1) noise, normalised: a well-conditioned start
    with generic, non-degenerate environments."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(2):
        X = eps * rng.standard_normal((2, 2, D, D, D))
        X[0, 0, 0, 0, 0] += 1.0
        X[1, 1, 0, 0, 0] += 1.0
        out.append(X / np.linalg.norm(X))
    return out[0], out[1]
