/*
 * eefu.h -- C ABI of the GB300 exact-environment full update (eeFU) library.
 *
 * Method: Czarnik, Francuz, Dziarmaga, "Tensor network simulation of the
 * Kitaev-Heisenberg model at finite temperature" (arXiv:1906.02220), Sec. III
 * with Figs. 3 and 4: an iPEPS purification of exp(-beta H) on the honeycomb
 * lattice is evolved in imaginary time by Trotter gates (Eq. 6); for each gate
 * layer on bond direction gamma, every A-B pair joined by a gamma bond is
 * fused into one composite site so that the lattice becomes a square
 * (rhombic) lattice, CTMRG on the double-layer norm network of the gated
 * composite gives the exact environment of the gamma bond, and the bond
 * A'-B' (dimension 4D) is replaced by A''-B'' (dimension D) minimising the
 * environment-weighted error.
 *
 * Conventions shared by every call
 *   - All pointers named dev_* are device pointers on the context's device;
 *     host_* are host pointers.  The caller owns every buffer passed in,
 *     including the workspace; the library never allocates device memory.
 *   - All work is issued on the stream given to kh_create.  Calls that return
 *     host values synchronise that stream before returning.
 *   - Site tensors are real FP64, row-major A[s][a][x][y][z] (spin, ancilla,
 *     the three bonds), shape [2][2][D][D][D] (Fig. 3(a)).
 *   - Composite (rhombic) site tensors are row-major T[p][l][u][r][d] with
 *     p = (s_A, a_A, s_B, a_B) for composites (p = 16) and bonds of dimension
 *     D (Fig. 4(b)).  For mapping gamma with (alpha, alpha') the other two
 *     directions in cyclic order: r = A.alpha, u = A.alpha', l = B.alpha,
 *     d = B.alpha'.
 *   - Two-site operators (gates, bond Hamiltonians) are 4x4 row-major on
 *     (s_A, s_B): row 2*s_A'+s_B', column 2*s_A+s_B; s = 0 is S^z = +1/2.
 *   - Environments (Fig. 4(c)), clockwise C1 E1 C2 E2 C3 E3 C4 E4:
 *     C[i][x][y] (chi x chi), x = leg to the previous edge, y = to the next;
 *     E[i][x][k][b][y] (chi x D x D x chi), k = ket leg, b = bra leg.
 *     E1 attaches to u, E2 to r, E3 to d, E4 to l.
 *   - Errors: every call returns a kh_status; nothing aborts or traps.
 *     On failure kh_last_error() gives a one-line reason.
 *   - Threads: one host thread at a time per context; different contexts
 *     may be driven from different host threads concurrently (the state
 *     they share -- per-kernel shared-memory grants, the tensor-map encoder,
 *     the launch counter -- is synchronised).
 */
#ifndef EEFU_H
#define EEFU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    KH_OK = 0,
    KH_EINVAL = 1,      /* bad argument or size beyond a stated limit */
    KH_ENOMEM = 2,      /* workspace smaller than kh_workspace_bytes() */
    KH_ENOCONV = 3,     /* CTM or ALS did not converge within its limit */
    KH_ENUMERIC = 4,    /* NaN/Inf or a breakdown in a solve */
    KH_ETIMEOUT = 5,    /* a bounded device wait gave up */
    KH_ECUDA = 6        /* a CUDA runtime call failed */
} kh_status;

/* Arithmetic of the dense contractions (enlarged corners, half-system
 * product, absorption, metric).  Masters of C, E, T and everything in the
 * projector solve, metric solve and normalisation stay FP64 / FP32 as
 * documented per call. */
typedef enum {
    KH_FP64 = 0,        /* CUDA-core FP64 throughout (plain FP64 GPU form)      */
    KH_FP32 = 1,        /* CUDA-core FP32 contractions, FP32 accumulate         */
    KH_TF32 = 2,        /* tcgen05 kind::tf32, FP32 accumulate in TMEM          */
    KH_TF32X3 = 3,      /* tcgen05 kind::tf32 with hi/lo operand split (3 MMAs) */
    KH_BF16 = 4         /* the layered site contraction on tcgen05 kind::f16 with
                           BF16 operands (one pass), FP32 accumulate; the
                           half-system product TF32 (one pass)                  */
} kh_prec;

typedef struct kh_config {
    int D;                   /* bond dimension, 1 <= D <= 8                           */
    int chi;                 /* environment dimension, 1 <= chi <= 256                */
    int prec;                /* kh_prec                                              */
    int n_slots;             /* environment slots, >= 1 (eeFU uses 0..2, measure 3..5) */
    int p_max;               /* largest physical dimension of a slot tensor (<= 16)    */
    int svd_oversample;      /* subspace vectors beyond chi in the projector SVD      */
    int svd_iters_cold;      /* subspace iterations on a cold start                   */
    int svd_iters_warm;      /* subspace iterations when warm-started                 */
    int jacobi_max_sweeps;   /* cap on Jacobi sweeps per small eigenproblem           */
    double svd_cut;          /* drop singular values below svd_cut * s_1 (S^-1/2)    */
    double als_tol;          /* ALS stop: |d_old - d_new| / <T'|N|T'> < als_tol       */
    int als_max_iter;        /* ALS iteration cap                                    */
    double als_reg;          /* Tikhonov shift reg * tr(R)/dim(R) in the normal eqns  */
    uint64_t seed;           /* seed of the counter-based start vectors              */
    int proj_fp64;           /* 1: in the single-precision modes, the projector
                                SVD is FP64: the Rayleigh-Ritz matrix accumulated
                                in FP64, its SVD refined to FP64 by Newton steps
                                from the FP32 Jacobi, S^-1/2 and the cut-off in
                                FP64; the products with the contraction data stay
                                in the contraction precision.  The FP64 mode
                                always computes in FP64.                        */
    int site_form;           /* two-layer site contraction of the corners and
                                edges: 0 = automatic (layered, ket then bra, on
                                the tensor cores in the TF32 precisions; on the
                                CUDA cores the double-layer operand where
                                D^2 <= 2p, which halves the flops), 1 = layered
                                always, 2 = the double-layer operand wherever
                                D^2 <= 2p.  The layered tensor-core form keeps
                                the chi^2 D^4 p intermediate on chip; the
                                layered CUDA-core form writes it to scratch.   */
} kh_config;

typedef struct kh_ctx kh_ctx;   /* opaque; host memory owned by the library */

/* Fills cfg with the defaults used by the tests (D, chi must then be set). */
void kh_config_defaults(kh_config* cfg);

/* Device workspace the context needs for cfg, in bytes (0 on invalid cfg). */
size_t kh_workspace_bytes(const kh_config* cfg);

/* Creates a context on the current device.  dev_workspace: caller-owned,
 * 256-byte aligned, at least kh_workspace_bytes(cfg) bytes, not touched by
 * the caller while the context lives.  stream: a cudaStream_t (0 = legacy
 * default stream).  All environments start at the traced boundary; the
 * state starts at the beta = 0 purification (Sec. III).  A context with
 * n_slots >= 6 also creates two non-blocking streams of its own (freed by
 * kh_destroy), with their own scratch in the workspace, on which independent
 * parts of a CTM move and the three mappings of the observables run
 * concurrently; every call forks them from `stream` and joins them back
 * before it returns or synchronises, so callers only order work on `stream`. */
kh_status kh_create(kh_ctx** ctx, const kh_config* cfg, void* dev_workspace,
                    size_t workspace_bytes, void* stream);
void kh_destroy(kh_ctx* ctx);
const char* kh_last_error(const kh_ctx* ctx);

/* Copy the FP64 site tensors A, B ([2][2][D][D][D] each) in / out. */
kh_status kh_set_state(kh_ctx* ctx, const double* dev_A, const double* dev_B);
kh_status kh_get_state(kh_ctx* ctx, double* dev_A, double* dev_B);

/* --- checkpoint / resume (the paper has no counterpart) ------------------- */

/* kh_save writes the context's persistent state to the file at path: the
 * configuration, the site tensors A, B, and for every slot its FP64 master
 * site tensor, environment (C, E), warm projector subspaces with their
 * live-column masks, last spectra, discarded weights and flags, plus the
 * random-stream counter.  Scratch is not saved; the operands derived from a
 * slot's site tensor are rebuilt on load.  The file is binary in native
 * byte order (read back on the same kind of machine).  Synchronises the
 * context's stream.  Errors: KH_EINVAL (null path, the file cannot be
 * written), KH_ECUDA.
 * kh_load_config reads a checkpoint's configuration (host only, no GPU),
 * so that the caller can allocate kh_workspace_bytes(cfg) bytes of
 * workspace.  KH_EINVAL if the file is missing or not a checkpoint.
 * kh_load creates a context from a checkpoint on the given workspace and
 * stream (as kh_create with the file's configuration) and restores its
 * state: continuing from it computes what the saved context would have.
 * On a failure after the context was created (a truncated file) *ctx is
 * still returned and must be destroyed; kh_last_error(*ctx) says why. */
kh_status kh_save(kh_ctx* ctx, const char* path);
kh_status kh_load_config(const char* path, kh_config* cfg);
kh_status kh_load(kh_ctx** ctx, const char* path, void* dev_workspace, size_t workspace_bytes, void* stream);

/* --- CTMRG (Fig. 4(c), Sec. III) ------------------------------------------ */

/* Load an arbitrary site tensor T[p][D][D][D][D] (FP64, device) into slot;
 * p <= p_max.  Used for generic square-lattice tensors (e.g. the Ising PEPS). */
kh_status ctm_set_tensor(kh_ctx* ctx, int slot, const double* dev_T, int p);

/* Build the gamma-composite of the current A, B into slot (Fig. 4(b)),
 * applying the 4x4 gate host_gate on (s_A, s_B) if non-NULL (the exact
 * A'-B' pair of Fig. 3(b), its 4D bond contracted inside the composite). */
kh_status ctm_build_composite(kh_ctx* ctx, int slot, int gamma, const double* host_gate);

/* Reset slot's environment to the traced boundary: every corner e0 e0^T and
 * every edge E[0][k][b][0] = host_edge[k*D+b] (delta_kb if host_edge is
 * NULL).  Also marks the projector subspaces cold. */
kh_status ctm_init(kh_ctx* ctx, int slot, const double* host_edge);

/* Copy the environment (and warm subspaces with their live-column masks) of
 * src_slot into dst_slot. */
kh_status ctm_copy_env(kh_ctx* ctx, int dst_slot, int src_slot);

/* CTM sweeps (left, up, right, down moves) on slot.  Runs until the
 * normalised top-chi projector spectra of all four moves change by less than
 * tol between sweeps (at least min_sweeps), or max_sweeps.  tol < 0 runs
 * exactly max_sweeps with no host synchronisation; then host outputs may be
 * NULL.  Returns KH_ENOCONV if tol >= 0 and max_sweeps was reached. */
kh_status ctm_sweep(kh_ctx* ctx, int slot, int max_sweeps, int min_sweeps, double tol,
                    int* host_sweeps_done, double* host_delta);

/* Spectrum (chi values, descending, zeros past the kept ones) of the last
 * half-system product M = Q_ul^T Q_dl of move dir (0 left, 1 up, 2 right,
 * 3 down) and its discarded weight sum_{i>=chi} s_i^2 / sum_i s_i^2. */
kh_status ctm_projectors(kh_ctx* ctx, int slot, int dir, double* dev_spectrum,
                         double* host_trunc_err);

/* Copy out the FP64 environment: dev_C [4][chi][chi], dev_E [4][chi][D][D][chi]. */
kh_status ctm_get_env(kh_ctx* ctx, int slot, double* dev_C, double* dev_E);

/* Environment metric of one site (ring of C1..C4, E1..E4), reshaped to
 * N[(l,u,r,d) ket][(l,u,r,d) bra] (D^4 x D^4, FP64) and symmetrised. */
kh_status ctm_metric(kh_ctx* ctx, int slot, double* dev_N);

/* Free energy per site of slot's norm network, kappa = Z11 Z00 / (Z10 Z01). */
kh_status ctm_kappa(kh_ctx* ctx, int slot, double* host_kappa);

/* <O_i> = Tr(O_i X) / Tr(X), X = T N T^T, for n_ops p x p operators. */
kh_status ctm_expval(kh_ctx* ctx, int slot, const double* host_ops, int n_ops,
                     double* host_vals);

/* Correlation length of slot's network along direction 0 (horizontal: the
 * column transfer matrix E1 (site) E3) or 1 (vertical: E2 (site) E4), the
 * length of the paper's scaling analysis (Sec. IV): xi = 1 / ln(|l1| / |l2|)
 * from the two largest eigenvalues in modulus of the channel transfer matrix
 * (dimension chi^2 D^2, never formed), by a block power iteration on up to 4
 * vectors with Rayleigh-Ritz steps every 4 iterations, stopped when
 * |l2| / |l1| changes by less than tol (relative) or after max_iter.
 * host_out[3]: xi (0 when |l2| / |l1| < 1e-14), |l2| / |l1|, iterations.
 * The environment should be converged (ctm_sweep); uses the slot's scratch.
 * Errors: KH_EINVAL (no environment, direction not 0 or 1), KH_ENUMERIC. */
kh_status ctm_correlation_length(kh_ctx* ctx, int slot, int direction, int max_iter, double tol,
                                 double* host_out);

/* Product of four operators on a 2 x 2 plaquette of slot's square lattice
 * (the plaquette flux of Sec. V is one such product).  host_ops holds four
 * p x p real operators, row-major, acting on the physical index of slot's
 * tensor, for the positions upper-left, upper-right, lower-right, lower-left.
 * The cluster of the four sites in slot's environment -- the enlarged
 * corners of the four frames closed in a ring, Tr(Q_0 Q_1 Q_2 Q_3) -- is
 * evaluated with operator f applied to the ket layer of site f and divided
 * by the plain cluster: host_out[0] = <O_0 O_1 O_2 O_3>, host_out[1] = the
 * plain cluster (a normalisation diagnostic).  The environment should be
 * converged (ctm_sweep).  Uses the context's scratch and synchronises the
 * stream.  Errors: KH_EINVAL (bad slot, no tensor or environment, NULL
 * pointers), KH_ENUMERIC (plain cluster zero or not finite). */
kh_status ctm_plaquette(kh_ctx* ctx, int slot, const double* host_ops, double* host_out);

/* Plaquette flux <W_p> (Sec. V): W_p = prod of sigma_i^{o(i)} over the six
 * sites i of a hexagon, o(i) the direction of the one bond at i that leaves
 * the hexagon (Kitaev's plaquette operator, +1 in the flux-free ground
 * state).  slot holds the gamma composite (p = 16) of the un-gated state and
 * its converged environment (after observables(): slot 3 + gamma).  In the
 * gamma mapping, with (alpha, alpha') the other two directions in cyclic
 * order, the hexagon's sites and operators are: upper-left composite A
 * sigma^alpha', B sigma^alpha; upper-right B sigma^gamma; lower-right A
 * sigma^alpha, B sigma^alpha'; lower-left A sigma^gamma.  Evaluated by
 * ctm_plaquette with sigma^y = i [[0,-1],[1,0]] (W_p holds two of them).
 * host_out[0] = <W_p>, host_out[1] = the plain cluster.  Errors as
 * ctm_plaquette; KH_EINVAL also for gamma outside 0..2 or p != 16. */
kh_status ctm_flux(kh_ctx* ctx, int slot, int gamma, double* host_out);

/* --- eeFU bond update (Fig. 3(b), Sec. III) -------------------------------- */

/* One gate layer on direction gamma (0 x, 1 y, 2 z): build the gated
 * composite T' into slot gamma, converge its CTMRG (warm start from that
 * slot; ctm_* arguments as in ctm_sweep), form the metric N, minimise
 * <T''-T'|N|T''-T'> by ALS from the truncated SVD of T', fix the balanced
 * gauge and normalise, and store A'', B'' as the new state.
 * host_info (may be NULL when ctm_tol < 0): [0] relative cost d/<T'|N|T'>,
 * [1] CTM sweeps, [2] ALS iterations, [3] largest discarded weight. */
kh_status eefu_apply_gate(kh_ctx* ctx, int gamma, const double* host_gate,
                          int ctm_max_sweeps, int ctm_min_sweeps, double ctm_tol,
                          double* host_info);

/* Gradient of the bond cost of Fig. 3(b), d = <T''-T'|N|T''-T'>, with respect
 * to trial factors A'' and B'' (the hand-written adjoint of the eeFU cost):
 * builds the gated composite T' of the current state into slot gamma and its
 * metric N as eefu_apply_gate does (ctm_max_sweeps = 0 reuses the slot's
 * environment as it stands instead of sweeping), then for the caller's
 * dev_A2 [sA][aA][u][r][k] and dev_B2 [sB][aB][d][l][k] (device, FP64,
 * 4 D^3 each; u, r the legs of A other than gamma, d, l those of B) writes
 *   dev_gA = dd/dA'' = (R_A + R_A^T) a - 2 S_A,  dev_gB = dd/dB'' likewise,
 * where R, S are the normal-equation matrices of that side with the other
 * factor fixed (same layouts as A'', B''), and host_cost[0] = d, [1] =
 * <T'|N|T'>, [2] = d evaluated from the B side (equal to [0] up to
 * rounding).  The state A, B is not changed; the slot's environment is
 * (warm-started sweeps).  Synchronises the stream. */
kh_status eefu_cost_gradient(kh_ctx* ctx, int gamma, const double* host_gate,
                             const double* dev_A2, const double* dev_B2, int ctm_max_sweeps,
                             int ctm_min_sweeps, double ctm_tol, double* dev_gA, double* dev_gB,
                             double* host_cost);

/* Observables of the current (un-gated) state: for each gamma a CTMRG of the
 * composite in slot 3+gamma (warm start from its last run, else from slot
 * gamma), then <H^gamma> with host_H = three 4x4 bond Hamiltonians (x, y, z,
 * without bias), <S^a> of both sublattices from the z mapping, and
 * E/site = 1/2 sum_gamma <H^gamma> - (hA <S^z_A> + hB <S^z_B>)/2.
 * host_out[12]: E_site, Hx, Hy, Hz, SxA, SyA, SzA, SxB, SyB, SzB, trunc, sweeps. */
kh_status observables(kh_ctx* ctx, const double* host_H, double hA, double hB,
                      int ctm_max_sweeps, int ctm_min_sweeps, double ctm_tol,
                      double* host_out);

/* --- gates (Sec. II Eqs. 2-5, Sec. III Eq. 6); host FP64 -------------------- */

/* H^gamma = J S_A.S_B + K_gamma S_A^gamma S_B^gamma - hA S^z_A - hB S^z_B as a
 * 4x4 row-major matrix on (s_A, s_B) (pass hA = hB = 0 except for the z
 * bond, which carries the bias of Eq. 5). */
kh_status kh_bond_hamiltonian(int gamma, double J, double K_gamma, double hA, double hB,
                              double* host_H);

/* g = exp(-tau H) for a real symmetric 4x4 H (eigendecomposition by Jacobi). */
kh_status kh_gate(const double* host_H, double tau, double* host_g);

/* The four 16 x 16 composite-site operators that ctm_flux places on the 2 x 2
 * plaquette of the gamma mapping (Sec. V flux; layout and geometry as in
 * ctm_flux), in real form: sigma^y entered as [[0,-1],[1,0]], so W_p is
 * minus the product of these four.  host_ops[4][16][16], row-major on
 * p = (sA, aA, sB, aB), upper-left first.  Host only.  KH_EINVAL for gamma
 * outside 0..2 or a NULL pointer. */
kh_status kh_flux_operators(int gamma, double* host_ops);

/* One second-order Trotter step (Eq. 6): gate layers x, y, z, y, x with
 * exp(-tau H^gamma), tau = dbeta/4, dbeta/4, dbeta/2, dbeta/4, dbeta/4, the
 * bias (hA, hB) in the z gate, couplings J and K_gamma = K_xyz[gamma].  Each
 * layer is eefu_apply_gate with the given CTM arguments.  host_info (may be
 * NULL when ctm_tol < 0): [0] largest relative cost, [1] total CTM sweeps,
 * [2] total ALS iterations, [3] largest discarded weight. */
kh_status eefu_trotter_step(kh_ctx* ctx, double J, const double* host_K_xyz, double hA, double hB,
                            double dbeta, int ctm_max_sweeps, int ctm_min_sweeps, double ctm_tol,
                            double* host_info);

/* An imaginary-time trajectory (Sec. III, Eq. 6) with its thermodynamics
 * (Sec. V): n_steps Trotter steps of dbeta as eefu_trotter_step (CTM
 * arguments mx, mn, tol per gate layer), and after every measure_every-th
 * step the observables (CTM arguments obs_*).  host_traj receives
 * n_steps / measure_every rows of 13 doubles: beta (counted from the first
 * call on this context, which starts at the initial state's beta = 0), E_site,
 * Hx, Hy, Hz, SxA, SyA, SzA, SxB, SyB, SzB, the largest discarded weight, and
 * the specific heat per site C = dE/dT = -beta^2 dE/dbeta by central
 * differences over the measurement grid (NaN in the first and last row).
 * The couplings and the bias are those of eefu_trotter_step; the bond
 * energies are measured without the bias, E_site includes it. */
kh_status eefu_evolve(kh_ctx* ctx, double J, const double* host_K_xyz, double hA, double hB, double dbeta,
                      int n_steps, int measure_every, int ctm_max_sweeps, int ctm_min_sweeps, double ctm_tol,
                      int obs_max_sweeps, int obs_min_sweeps, double obs_tol, double* host_traj);

/* eefu_evolve plus the plaquette flux <W_p> (Sec. V: its ordering marks
 * the lower crossover of the pure Kitaev model) after every measurement, as
 * ctm_flux computes it from the z mapping's observables environment (slot 5):
 * host_flux[n_steps / measure_every] (host, not NULL).  host_traj as in
 * eefu_evolve.  Needs the six slots of the observables (KH_EINVAL
 * otherwise). */
kh_status eefu_evolve_flux(kh_ctx* ctx, double J, const double* host_K_xyz, double hA, double hB, double dbeta,
                           int n_steps, int measure_every, int ctm_max_sweeps, int ctm_min_sweeps, double ctm_tol,
                           int obs_max_sweeps, int obs_min_sweeps, double obs_tol, double* host_traj,
                           double* host_flux);

/* Batched trajectories: n independent problems (different couplings, or
 * different D / chi / precision per context) advanced concurrently, one host
 * thread per context, each context's kernels on its own streams, so that the
 * problems' latency-bound launches overlap on the GPU.  Problem i runs
 * eefu_evolve on ctxs[i] with couplings J[i], K_xyz[3i..3i+2], hA[i], hB[i]
 * (hA, hB may be null: no field) and the shared step settings; its trajectory
 * goes to host_traj + i (n_steps / measure_every) 13 doubles in the layout of
 * eefu_evolve.  The contexts must be distinct.  status (host, n entries, may
 * be null) receives each problem's status; the return value is the first
 * non-OK one (each context's message in its kh_last_error).  Returns after
 * every context's work has completed. */
kh_status eefu_evolve_batch(kh_ctx* const* ctxs, int n, const double* J, const double* K_xyz,
                            const double* hA, const double* hB, double dbeta, int n_steps,
                            int measure_every, int ctm_max_sweeps, int ctm_min_sweeps, double ctm_tol,
                            int obs_max_sweeps, int obs_min_sweeps, double obs_tol, double* host_traj,
                            kh_status* status);

/* --- instrumentation (no counterpart in the paper; used by the benchmark) -- */

/* Number of kernels this library has launched since it was loaded. */
unsigned long long kh_launch_count(void);

/* enable != 0: reset and start CUDA-event timing of ten categories on the
 * context's stream; enable == 0: synchronise, stop, and write host_out[30] =
 * {launches, milliseconds, algorithmic flops} per category: 0 half-system
 * product Mt = Q_{s+3} Q_s (2 n^3 flops, n = chi D^2), 1 two-layer site
 * contractions (4 nb p D^6 flops per call), 2 the two enlarged corners of a
 * move (2 (2 chi^3 D^2 + 2 chi^3 D^4 + 4 p chi^2 D^6) flops), 3 projector
 * SVD without Mt, 4 absorption (6 chi^3 D^2 + 4 chi^3 D^4 + 4 p chi^2 D^6
 * flops), 5 environment metric, 6 ALS and gauge,
 * 7 one-sided Jacobi SVD, 8 CholQR orthonormalisation, 9 subspace products
 * M V and M^T U (2 n^2 k flops).  Categories without a flop model report 0,
 * except 7, whose third entry is the total number of Jacobi sweeps;
 * nested categories overlap (2 and 4 contain 1; 3 contains 7, 8, 9). */
kh_status kh_profile(kh_ctx* ctx, int enable, double* host_out);

/* --- kernel self-tests (test hooks; no counterpart in the paper) ----------- */

/* Scratch bytes the self-tests below need for an M x K by K x N product. */
size_t kh_selftest_bytes(int M, int N, int K);

/* dev_C (M x N) = dev_A (M x K) dev_B (K x N), all row-major FP64 device
 * arrays, computed by the library's contraction GEMM for precision prec
 * (operands converted to its input type, result converted back).  dev_scratch
 * holds at least kh_selftest_bytes(M, N, K) bytes.  Synchronises stream. */
kh_status kh_selftest_gemm(int prec, int M, int N, int K, const double* dev_A, const double* dev_B,
                           double* dev_C, void* dev_scratch, size_t scratch_bytes, void* stream);

/* Eigen-decomposition of a symmetric k x k FP64 matrix by the library's
 * Jacobi kernel in FP64 (prec = KH_FP64) or FP32 (otherwise): dev_evals
 * descending, column j of dev_W its eigenvector.  Scratch as above with
 * M = N = K = k.  Synchronises stream. */
kh_status kh_selftest_symeig(int prec, int k, const double* dev_G, double* dev_W, double* dev_evals,
                             void* dev_scratch, size_t scratch_bytes, void* stream);

/* One-sided Jacobi SVD of a k x k FP64 matrix X (row-major) by the library
 * kernel used in the projector Rayleigh-Ritz step, in FP64 or FP32:
 * X Q = L S with dev_S descending (k), dev_L, dev_Q k x k (columns = vectors). */
kh_status kh_selftest_svd(int prec, int k, const double* dev_X, double* dev_S, double* dev_L, double* dev_Q,
                          void* dev_scratch, size_t scratch_bytes, void* stream);

/* The projector SVD of the FP64-projector option (kh_config.proj_fp64) on a
 * k x k FP64 matrix X (k <= 160): the FP32 one-sided Jacobi SVD followed by
 * three FP64 Newton refinement steps and a re-orthogonalisation (first-order corrections L' = L (I + F),
 * Q' = Q (I + H) from R = I - L^T L, P = I - Q^T Q and T = L^T X Q, pairs
 * whose gap is below 64 times their coupling only re-orthogonalised).  X Q = L S with dev_S
 * (k, in the Jacobi's descending order), dev_L, dev_Q k x k (columns =
 * vectors).  Scratch as for kh_selftest_svd.  Synchronises stream. */
kh_status kh_selftest_svd_refined(int k, const double* dev_X, double* dev_S, double* dev_L, double* dev_Q,
                                  void* dev_scratch, size_t scratch_bytes, void* stream);

/* Orthonormal basis of the columns of an n x k FP64 matrix Y (row-major) by
 * the library's ordered CholQR2 (two Cholesky-QR passes, columns taken in
 * order of decreasing norm), the orthonormalisation step of the projector's
 * subspace iteration, in FP64 (k <= 112) or FP32 (k <= 160).  Columns of norm
 * <= cut * (largest norm), and directions whose Cholesky pivot falls below
 * the rounding floor, come out as zero columns of dev_Q (n x k, row-major);
 * the others are orthonormal, the first one along the largest column of Y.
 * Scratch as above with M = n, N = K = k.  KH_EINVAL for k beyond the limit.
 * Synchronises stream. */
kh_status kh_selftest_orth(int prec, int n, int k, double cut, const double* dev_Y, double* dev_Q,
                           void* dev_scratch, size_t scratch_bytes, void* stream);

/* Layered two-layer site contraction on the tensor cores (Fig. 4 and Sec. III:
 * the enlarged-corner and edge contractions with ket and bra layers applied
 * one after the other, the chi^2 D^4 p intermediate kept on chip):
 *   dev_out[b][ok][ob] = sum_p sum_{ik,ib} TL[ik][p][ok] dev_Y[b][ib][ik] TL[ib][p][ob]
 * for b < nb, all row-major FP64 (computed from FP32 copies), where ik, ib, ok,
 * ob index D^2 leg pairs and TL is the site tensor dev_T[p][l][u][r][d] seen
 * from frame `frame` (0..3, each a quarter turn (l,u,r,d) <- (d,l,u,r) of the
 * previous): kind 0 (corner) TL[(l,u)][p][(r,d)], kind 1 (edge)
 * TL[(l,d)][p][(u,r)].  npass 1 = TF32, 3 = 3xTF32, 16 = BF16.  dev_scratch holds at
 * least kh_selftest_site_layered_bytes(npass, D, p, nb) bytes (0 = invalid
 * arguments).  KH_ETIMEOUT if a wait in the kernel timed out.  Synchronises
 * stream. */
size_t kh_selftest_site_layered_bytes(int npass, int D, int p, long long nb);
kh_status kh_selftest_site_layered(int npass, int D, int p, int kind, int frame, long long nb,
                                   const double* dev_T, const double* dev_Y, double* dev_out,
                                   void* dev_scratch, size_t scratch_bytes, void* stream);

/* FP64 reciprocal, reciprocal square root and square root as the library's
 * latency-bound FP64 kernels form them (Newton-Raphson iteration from the FP32
 * hardware estimates, IEEE operations outside the FP32 normal range): for the
 * n device values x, dev_out[3i] = 1/x_i, dev_out[3i+1] = 1/sqrt(x_i) (0 for
 * x_i <= 0), dev_out[3i+2] = sqrt(x_i) (0 for x_i < 0).  Synchronises stream. */
kh_status kh_selftest_fp64_newton(int n, const double* dev_x, double* dev_out, void* stream);

/* --- allocation-free variant (the paper has no counterpart) ---------------- */

/* Same result as kh_selftest_gemm (dev_C = dev_A dev_B, row-major FP64 device
 * arrays, computed by the library's contraction GEMM for precision prec), for
 * callers that cannot allocate device memory -- code whose device memory is
 * owned by another allocator, or loops that cannot afford an allocation's
 * implicit synchronisation.  Scratch is a static device array of
 * kh_gemm_noalloc_max_bytes() bytes (16 MiB) that every GPU loading the
 * library holds until exit; sizes needing more (kh_selftest_bytes(M, N, K))
 * return KH_EINVAL.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current and keeps it for
 * later calls on that device (the lookup is safe when several host threads
 * make their first calls at once); make that first call before any stream
 * capture.  A device reset (cudaDeviceReset) discards the array, so the
 * entry point must not be called on that device afterwards.  All calls
 * share the array: calls that overlap on the GPU race.  Every call ends by
 * synchronising stream; no cudaMalloc or cudaFree. */
size_t kh_gemm_noalloc_max_bytes(void);
kh_status kh_gemm_noalloc(int prec, int M, int N, int K, const double* dev_A, const double* dev_B, double* dev_C,
                          void* stream);

/* Library build information (static string). */
const char* kh_version(void);

#ifdef __cplusplus
}
#endif
#endif /* EEFU_H */
