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
        double off = 0.0, dg = 0.0;
        for (int e = tid; e < kp * kp; e += nt) {
            int i = e / kp, j = e % kp;
            double v = (double)A[e];
            if (i == j) dg += v * v; else off += v * v;
        }
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            dg += __shfl_xor_sync(0xffffffffu, dg, o);
        }
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

template <typename T>
inline size_t jacobi_smem(int k) {
    int kp = (k + 1) & ~1;
    return (size_t)2 * kp * kp * sizeof(T);
}

template <typename T>
inline int jacobi_kmax() { return sizeof(T) == 8 ? 112 : 160; }

template <typename T>
inline void jacobi_eig(const T* G, int k, int ldg, long long sG, T* W, int ldw, long long sW,
                       T* evals, long long sE, int batch, int max_sweeps, double tol, int* sweeps,
                       const int* skip, cudaStream_t st) {
    if (k > jacobi_kmax<T>()) fail(KH_EINVAL, "jacobi: k beyond limit");
    size_t sm = jacobi_smem<T>(k);
    static bool attr_set[2] = {false, false};
    int ti = sizeof(T) == 8 ? 1 : 0;
    if (!attr_set[ti]) {
        KH_CUDA(cudaFuncSetAttribute(jacobi_eig_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(227 * 1024)));
        attr_set[ti] = true;
    }
    jacobi_eig_kernel<T><<<batch, kJacobiThreads, sm, st>>>(G, k, ldg, sG, W, ldw, sW, evals, sE,
                                                           max_sweeps, tol, sweeps, skip);
    KH_LAUNCHED();
}

}  // namespace kh
