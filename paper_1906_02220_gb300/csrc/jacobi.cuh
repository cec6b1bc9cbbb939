// Symmetric eigensolver for small dense matrices (k <= 160 in FP32, <= 112 in
// FP64): cyclic two-sided Jacobi with the parallel round-robin ordering, one
// CTA per matrix, matrix and rotation accumulator in shared memory.
//
// Jacobi is used because it is accurate in the sense that matters here: on
// the near-diagonal Gram matrices of a warm-started subspace iteration it
// converges in one or two sweeps and keeps every eigenvalue to high relative
// accuracy (Demmel-Veselic), with no tridiagonal reduction.  Rotation
// formula: Golub & Van Loan, "Matrix Computations", the symmetric 2x2 Schur
// decomposition used by the classical Jacobi method.
#pragma once
#include "common.cuh"

namespace kh {

constexpr int kJacobiThreads = 512;

template <typename T>
__device__ __forceinline__ void round_robin_pair(int r, int i, int kp, int& p, int& q) {
    // circle method: player 0 fixed, players 1..kp-1 rotate with the round
    int m = kp - 1;
    if (i == 0) {
        p = 0;
        q = 1 + (r % m);
    } else {
        p = 1 + ((r + i) % m);
        q = 1 + ((r - i + m) % m);
    }
    if (p > q) { int t = p; p = q; q = t; }
}

// In: G (k x k, leading dimension ldg, symmetric; batch stride sG).
// Out: evals (k, descending), W (k x k, column j = eigenvector of evals[j],
// leading dimension ldw, batch stride sW).  The padded index (k odd) carries
// eigenvalue -1 (after scaling) and is dropped.  sweeps_out[b] (nullable)
// records the sweeps used.  skip (nullable device flag): if *skip != 0 the
// kernel returns immediately (used to freeze converged iterations on device).
#ifdef KH_JACOBI_KERNEL
template <typename T>
__global__ void __launch_bounds__(kJacobiThreads)
jacobi_eig_kernel(const T* __restrict__ G, int k, int ldg, long long sG, T* __restrict__ W, int ldw,
                  long long sW, T* __restrict__ evals, long long sE, int max_sweeps, double tol,
                  int* sweeps_out, const int* skip) {
    if (skip && *skip) return;
    extern __shared__ unsigned char smem_raw[];
    const int kp = (k + 1) & ~1;
    T* A = reinterpret_cast<T*>(smem_raw);
    T* V = A + kp * kp;
    __shared__ T rc[80], rs[80];
    __shared__ int rp[80], rq[80];
    __shared__ double red[kJacobiThreads / 32];
    __shared__ double s_scale, s_off, s_diag;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int b = blockIdx.x;
    G += b * sG;
    W += b * sW;
    evals += b * sE;

    // scale by the largest |diagonal| so the padding value -1 sits below a PSD spectrum
    double mx = 0.0;
    for (int i = tid; i < k; i += nt) mx = fmax(mx, fabs((double)G[(long long)i * ldg + i]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((tid & 31) == 0) red[tid >> 5] = mx;
    __syncthreads();
    if (tid == 0) {
        double m = 0.0;
        for (int w = 0; w < nt / 32; ++w) m = fmax(m, red[w]);
        s_scale = (m > 0.0) ? m : 1.0;
    }
    __syncthreads();
    const T inv = (T)(1.0 / s_scale);
    for (int e = tid; e < kp * kp; e += nt) {
        int i = e / kp, j = e % kp;
        T v;
        if (i < k && j < k) v = T(0.5) * (G[(long long)i * ldg + j] + G[(long long)j * ldg + i]) * inv;
        else v = (i == j) ? T(-1) : T(0);
        A[e] = v;
        V[e] = (i == j) ? T(1) : T(0);
    }
    __syncthreads();

    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        // convergence: off-diagonal Frobenius vs diagonal
        T offT = T(0), dgT = T(0);
        for (int e = tid; e < kp * kp; e += nt) {
            int i = e / kp, j = e % kp;
            T v = A[e];
            if (i == j) dgT = fma(v, v, dgT); else offT = fma(v, v, offT);
        }
        for (int o = 16; o > 0; o >>= 1) {
            offT += __shfl_xor_sync(0xffffffffu, offT, o);
            dgT += __shfl_xor_sync(0xffffffffu, dgT, o);
        }
        double off = (double)offT, dg = (double)dgT;
        if ((tid & 31) == 0) red[tid >> 5] = off;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int w = 0; w < nt / 32; ++w) s += red[w];
            s_off = s;
        }
        __syncthreads();
        if ((tid & 31) == 0) red[tid >> 5] = dg;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int w = 0; w < nt / 32; ++w) s += red[w];
            s_diag = s;
        }
        __syncthreads();
        if (s_off <= tol * tol * s_diag) break;

        for (int r = 0; r < kp - 1; ++r) {
            for (int i = tid; i < kp / 2; i += nt) {
                int p, q;
                round_robin_pair<T>(r, i, kp, p, q);
                T app = A[p * kp + p], aqq = A[q * kp + q], apq = A[p * kp + q];
                T c = T(1), s = T(0);
                if (apq != T(0)) {
                    T tau = (aqq - app) / (T(2) * apq);
                    T t = (tau >= T(0)) ? T(1) / (tau + sqrt(T(1) + tau * tau))
                                        : T(-1) / (-tau + sqrt(T(1) + tau * tau));
                    c = T(1) / sqrt(T(1) + t * t);
                    s = t * c;
                }
                rc[i] = c; rs[i] = s; rp[i] = p; rq[i] = q;
            }
            __syncthreads();
            // columns: A <- A J, V <- V J
            for (int e = tid; e < (kp / 2) * kp; e += nt) {
                int i = e / kp, row = e % kp;
                T c = rc[i], s = rs[i];
                if (s == T(0)) continue;
                int p = rp[i], q = rq[i];
                T ap = A[row * kp + p], aq = A[row * kp + q];
                A[row * kp + p] = c * ap - s * aq;
                A[row * kp + q] = s * ap + c * aq;
                T vp = V[row * kp + p], vq = V[row * kp + q];
                V[row * kp + p] = c * vp - s * vq;
                V[row * kp + q] = s * vp + c * vq;
            }
            __syncthreads();
            // rows: A <- J^T A
            for (int e = tid; e < (kp / 2) * kp; e += nt) {
                int i = e / kp, col = e % kp;
                T c = rc[i], s = rs[i];
                if (s == T(0)) continue;
                int p = rp[i], q = rq[i];
                T ap = A[p * kp + col], aq = A[q * kp + col];
                A[p * kp + col] = c * ap - s * aq;
                A[q * kp + col] = s * ap + c * aq;
            }
            __syncthreads();
        }
    }
    if (sweeps_out && tid == 0) sweeps_out[b] = sweep;
    // sort descending by rank; the pad (value -1) ranks last
    for (int i = tid; i < kp; i += nt) {
        T di = A[i * kp + i];
        int rank = 0;
        for (int j = 0; j < kp; ++j) {
            T dj = A[j * kp + j];
            rank += (dj > di) || (dj == di && j < i);
        }
        if (rank < k) {
            evals[rank] = (T)((double)di * s_scale);
            for (int row = 0; row < k; ++row) W[(long long)row * ldw + rank] = V[row * kp + i];
        }
    }
}

#endif  // KH_JACOBI_KERNEL

template <typename T>
inline size_t jacobi_smem(int k) {
    int kp = (k + 1) & ~1;
    return (size_t)2 * kp * kp * sizeof(T);
}

template <typename T>
inline int jacobi_kmax() { return sizeof(T) == 8 ? 112 : 160; }

// Launch wrapper, defined once (ctm.cu) for T = float, double.
template <typename T>
void jacobi_eig(const T* G, int k, int ldg, long long sG, T* W, int ldw, long long sW, T* evals, long long sE,
                int batch, int max_sweeps, double tol, int* sweeps, const int* skip, cudaStream_t st);


// One-sided (Hestenes) Jacobi SVD of a small dense k x k matrix X, one CTA:
// columns of X are rotated pairwise (round-robin ordering, one warp per pair)
// until mutually orthogonal; then X Q = L S with s_j = |column j|.  Singular
// values come out with absolute error ~ eps |X| (no squaring of the condition
// number, unlike a Gram-matrix eigensolve).  Outputs sorted descending:
// s (k), L (k x k, column j = X q_j / s_j, zero when s_j <= cut s_0), Q (k x k).
template <typename T>
void svd_jacobi(const T* X, int k, T* s, T* L, T* Q, int max_sweeps, double tol, double cut, cudaStream_t st,
                int* sweep_count = nullptr, int nrel = 0);

#ifdef KH_JACOBI_KERNEL
// 8-lane groups, one column pair per group (64 groups = every pair of a
// round in flight for k <= 128); columns stored contiguously with an odd
// stride.  A sweep ends the iteration when no pair needed a rotation, or when
// the largest pair cosine stops falling quadratically while already below
// 1e3 * eps (the rounding floor of the column dot products).
template <typename T>
__global__ void __launch_bounds__(kJacobiThreads)
svd_jacobi_kernel(const T* __restrict__ Xin, int k, T* __restrict__ s_out, T* __restrict__ L_out,
                  T* __restrict__ Q_out, int max_sweeps, double tol, double cut, int* sweep_count, int nrel) {
    extern __shared__ unsigned char smem_raw[];
    const int kp = (k + 1) & ~1;
    const int ld = kp + 1;                     // odd column stride
    T* Xc = reinterpret_cast<T*>(smem_raw);   // Xc[c * ld + r]
    T* Qc = Xc + kp * ld;
    __shared__ int s_rot;
    __shared__ float s_cmax;
    __shared__ double s_norm[160];
    __shared__ T s_cn[160];
    __shared__ unsigned char s_top[160];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int grp = tid >> 3, gl = tid & 7, ngrp = nt >> 3;
    const unsigned gmask = 0xFFu << (tid & 24);
    const double eps = sizeof(T) == 8 ? 1.1e-16 : 6e-8;
    for (int e = tid; e < kp * kp; e += nt) {
        int c = e / kp, r = e % kp;
        Xc[c * ld + r] = (r < k && c < k) ? Xin[(long long)r * k + c] : T(0);
        Qc[c * ld + r] = (r == c) ? T(1) : T(0);
    }
    // the cosine of two columns is only known to ~k eps (dot-product rounding)
    const T tol_eff = (T)fmax(tol, 2.0 * k * eps);
    float prev_cmax = 1e30f;
    int sw = 0;
    if (nrel <= 0 || nrel > kp) nrel = kp;
    for (; sw < max_sweeps; ++sw) {
        if (tid == 0) { s_rot = 0; s_cmax = 0.f; }
        if (nrel < kp) {
            // columns among the nrel largest must converge; tail-tail pairs are
            // still rotated but do not keep the sweep loop alive
            const int w0 = tid >> 5, l0 = tid & 31, nw0 = nt >> 5;
            for (int c = w0; c < kp; c += nw0) {
                T a = T(0);
                for (int row = l0; row < kp; row += 32) { T u = Xc[c * ld + row]; a = fma(u, u, a); }
                for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
                if (l0 == 0) s_cn[c] = a;
            }
            __syncthreads();
            for (int c = tid; c < kp; c += nt) {
                int rank = 0;
                for (int j = 0; j < kp; ++j) rank += (s_cn[j] > s_cn[c]) || (s_cn[j] == s_cn[c] && j < c);
                s_top[c] = rank < nrel;
            }
        } else {
            for (int c = tid; c < kp; c += nt) s_top[c] = 1;
        }
        __syncthreads();
        for (int r = 0; r < kp - 1; ++r) {
            for (int i = grp; i < kp / 2; i += ngrp) {
                int p, q;
                round_robin_pair<T>(r, i, kp, p, q);
                T* xp = Xc + p * ld;
                T* xq = Xc + q * ld;
                T a = T(0), b = T(0), g = T(0);
                for (int row = gl; row < kp; row += 8) {
                    T u = xp[row], v = xq[row];
                    a = fma(u, u, a); b = fma(v, v, b); g = fma(u, v, g);
                }
                for (int o = 4; o > 0; o >>= 1) {
                    a += __shfl_xor_sync(gmask, a, o);
                    b += __shfl_xor_sync(gmask, b, o);
                    g += __shfl_xor_sync(gmask, g, o);
                }
                T den = sqrt(a) * sqrt(b);
                if (g == T(0) || den == T(0)) continue;            // group-uniform
                const bool rel = s_top[p] || s_top[q];
                float cosv = (float)(fabs(g) / den);
                if (gl == 0 && rel) atomicMax((int*)&s_cmax, __float_as_int(cosv));
                if (fabs(g) <= tol_eff * den) continue;
                T zeta = (b - a) / (T(2) * g);
                T t = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
                T cT = T(1) / sqrt(T(1) + t * t), sT = cT * t;
                T* qp = Qc + p * ld;
                T* qq = Qc + q * ld;
                for (int row = gl; row < kp; row += 8) {
                    T u = xp[row], v = xq[row];
                    xp[row] = cT * u - sT * v;
                    xq[row] = sT * u + cT * v;
                    T qu = qp[row], qv = qq[row];
                    qp[row] = cT * qu - sT * qv;
                    qq[row] = sT * qu + cT * qv;
                }
                if (gl == 0 && rel) atomicAdd(&s_rot, 1);
            }
            __syncthreads();
        }
        const float cmax = s_cmax;
        const int rot = s_rot;
        __syncthreads();
        if (rot == 0) break;
        if (cmax < 1e3f * (float)eps && cmax > 0.25f * prev_cmax) break;   // stagnated at the floor
        prev_cmax = cmax;
    }
    if (sweep_count && tid == 0) atomicAdd(sweep_count, sw + 1);
    const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
    for (int c = warp; c < kp; c += nw) {
        T a = T(0);
        for (int row = lane; row < kp; row += 32) { T u = Xc[c * ld + row]; a = fma(u, u, a); }
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) s_norm[c] = (c < k) ? (double)sqrt(a) : -1.0;
    }
    __syncthreads();
    double smax = 0.0;
    for (int c = 0; c < k; ++c) smax = fmax(smax, s_norm[c]);
    for (int c = warp; c < k; c += nw) {
        double sc = s_norm[c];
        int rank = 0;
        for (int j = 0; j < k; ++j) rank += (s_norm[j] > sc) || (s_norm[j] == sc && j < c);
        T inv = (smax > 0.0 && sc > cut * smax) ? (T)(1.0 / sc) : T(0);
        for (int row = lane; row < k; row += 32) {
            L_out[(long long)row * k + rank] = Xc[c * ld + row] * inv;
            Q_out[(long long)row * k + rank] = Qc[c * ld + row];
        }
        if (lane == 0) s_out[rank] = (T)sc;
    }
}
#endif  // KH_JACOBI_KERNEL


// Ordered Cholesky-QR factor for orthonormalising the columns of Y (n x k)
// from its FP64 Gram dG: columns sorted by norm (largest, most trusted,
// first), scaled to unit norm, dead columns (norm <= cut_abs max) and
// pivots <= tau dropped; X (k x k) such that Q = Y X has orthonormal columns
// (in sorted order, dropped ones zero).  Unlike a symmetric (Loewdin)
// orthogonalisation, a weak column nearly parallel to a strong one never
// rotates the strong one.
template <typename T>
void cholqr_factor(const double* dG, int k, double cut_abs, double tau, T* X, cudaStream_t st);

#ifdef KH_JACOBI_KERNEL
template <typename T>
__global__ void __launch_bounds__(kJacobiThreads)
cholqr_kernel(const double* __restrict__ G, int k, double cut_abs, double tau, T* __restrict__ X) {
    extern __shared__ unsigned char smem_raw[];
    const int ld = k | 1;                          // odd row stride: conflict-free column walks
    T* Lm = reinterpret_cast<T*>(smem_raw);       // k x ld, row-major
    T* Li = Lm + k * ld;
    __shared__ T s_inv[160];
    __shared__ int s_perm[160];
    __shared__ int s_keep[160];
    __shared__ double s_diag[160];
    __shared__ double s_max;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    for (int j = tid; j < k; j += nt) s_diag[j] = G[(long long)j * k + j];
    __syncthreads();
    if (tid == 0) {
        double m = 0.0;
        for (int j = 0; j < k; ++j) m = fmax(m, s_diag[j]);
        s_max = sqrt(fmax(m, 0.0));
    }
    __syncthreads();
    for (int j = tid; j < k; j += nt) {
        double nj = sqrt(fmax(s_diag[j], 0.0));
        s_inv[j] = (s_max > 0.0 && nj > cut_abs * s_max) ? (T)(1.0 / nj) : T(0);
        int rank = 0;
        for (int i = 0; i < k; ++i) rank += (s_diag[i] > s_diag[j]) || (s_diag[i] == s_diag[j] && i < j);
        s_perm[rank] = j;
    }
    __syncthreads();
    for (int e = tid; e < k * k; e += nt) {
        int a = e / k, b = e % k;
        int pa = s_perm[a], pb = s_perm[b];
        Lm[a * ld + b] = (T)G[(long long)pa * k + pb] * s_inv[pa] * s_inv[pb];
        Li[a * ld + b] = T(0);
    }
    __syncthreads();
    for (int j = 0; j < k; ++j) {
        const T d = Lm[j * ld + j];
        const bool keep = (double)d > tau;        // same value in every thread
        if (keep) {
            const T ljj = sqrt(d);
            for (int i = j + 1 + tid; i < k; i += nt) Lm[i * ld + j] /= ljj;
            __syncthreads();
            if (tid == 0) { Lm[j * ld + j] = ljj; s_keep[j] = 1; }
            for (int i = j + 1 + warp; i < k; i += nw) {           // rows by warps, columns by lanes
                const T lij = Lm[i * ld + j];
                for (int c = j + 1 + lane; c <= i; c += 32) Lm[i * ld + c] -= lij * Lm[c * ld + j];
            }
        } else {
            __syncthreads();
            for (int i = j + tid; i < k; i += nt) Lm[i * ld + j] = T(0);
            if (tid == 0) s_keep[j] = 0;
        }
        __syncthreads();
    }
    // Li = L^-1 on the kept index set, one warp per column
    for (int j = warp; j < k; j += nw) {
        if (!s_keep[j]) continue;
        if (lane == 0) Li[j * ld + j] = T(1) / Lm[j * ld + j];
        __syncwarp();
        for (int i = j + 1; i < k; ++i) {
            if (!s_keep[i]) continue;
            T sum = T(0);
            for (int m = j + lane; m < i; m += 32) sum = fma(Lm[i * ld + m], Li[m * ld + j], sum);
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
            if (lane == 0) Li[i * ld + j] = -sum / Lm[i * ld + i];
            __syncwarp();
        }
    }
    __syncthreads();
    // X[perm a][b] = inv[perm a] * Li[b][a]   (Q = Y_s L^-T)
    for (int e = tid; e < k * k; e += nt) {
        int a = e / k, b = e % k;
        int pa = s_perm[a];
        X[(long long)pa * k + b] = s_inv[pa] * Li[b * ld + a];
    }
}
#endif  // KH_JACOBI_KERNEL

}  // namespace kh
