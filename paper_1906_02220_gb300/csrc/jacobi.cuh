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
#include <type_traits>

#include "common.cuh"

namespace kh {

constexpr int kJacobiThreads = 512;

template <typename T>
__device__ __forceinline__ void round_robin_pair(int r, int i, int kp, int& p, int& q) {
    // circle method: player 0 fixed, players 1..kp-1 rotate with the round
    // (r < m = kp - 1 and i < kp / 2, so each index wraps at most once)
    const int m = kp - 1;
    if (i == 0) {
        p = 0;
        q = 1 + r;
    } else {
        int x = r + i;
        if (x >= m) x -= m;
        int y = r - i + m;
        if (y >= m) y -= m;
        p = 1 + x;
        q = 1 + y;
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

// Column stride of the one-sided Jacobi's shared-memory matrices: the RL =
// LP R rows a group touches, rounded up to whole 128-byte bank rows (32 FP32
// or 16 FP64 elements).  FP64 at kp = 112 then needs 2 kp ld 8 = 200,704 bytes
// for X and Q instead of the 229,376 that a 32-element rounding would take
// (over the 227 KB per-CTA limit together with the static arrays).
template <typename T>
__host__ __device__ constexpr int svdj_ld(int rl) {
    return (rl + (int)(128 / sizeof(T)) - 1) / (int)(128 / sizeof(T)) * (int)(128 / sizeof(T));
}

#ifdef KH_JACOBI_KERNEL
// Rotation (c, s) that orthogonalises two columns with squared norms a, b and
// inner product g (the symmetric 2x2 Schur rotation of [[a, g], [g, b]]).
// FP32 uses the hardware reciprocal / reciprocal-square-root approximations:
// c and s stay a rotation to a few ulps, and an inexact angle only leaves a
// residual that the next sweep removes.
__device__ __forceinline__ void jacobi_rotation(float a, float b, float g, float& c, float& s) {
    const float zeta = __fdividef(b - a, 2.f * g);
    const float az = fabsf(zeta);
    float t;
    if (az > 1e15f) {
        t = __fdividef(0.5f, az);
    } else {
        const float r = fmaf(az, az, 1.f);
        t = __fdividef(1.f, az + r * rsqrtf(r));
    }
    t = copysignf(t, zeta);
    c = rsqrtf(fmaf(t, t, 1.f));
    s = c * t;
}
__device__ __forceinline__ void jacobi_rotation(double a, double b, double g, double& c, double& s) {
    const double zeta = (b - a) / (2.0 * g);
    const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
    c = 1.0 / sqrt(1.0 + t * t);
    s = c * t;
}

// LP-lane groups (LP = 8), one column pair per group and every pair of a
// round in flight (kp/2 groups); lane l of a group owns R rows (R/2 pairs of
// adjacent rows, each loaded and stored as one vector), so all row loops are
// unrolled at compile time.  The matrix is
// scaled by a power of two so that its largest entry is O(1) (exact), which
// lets the convergence test use squared cosines g^2 <= tol^2 a b without
// square roots.  Columns are stored contiguously with a stride of whole
// 128-byte bank rows (svdj_ld), zero below row k; the four groups of a warp walk the
// 16-row blocks of their columns in orders shifted by their slot, so that the
// two 64-byte halves a warp's vector access touches fall in alternate bank
// halves (two wavefronts, the minimum for 256 bytes) except where the
// shifted order wraps.  A sweep ends the iteration when no pair
// needed a rotation, when its largest pair cosine c had c^2 < tol / 10 (the
// cosines left are ~c^2, so the next sweep would rotate nothing), or when the
// largest pair cosine stops falling quadratically while already below
// 1e3 eps (the rounding floor of the column dot products).
template <typename T, int LP, int R>
__global__ void __launch_bounds__(LP * R / 2 * LP)
svd_jacobi_kernel(const T* __restrict__ Xin, int k, T* __restrict__ s_out, T* __restrict__ L_out,
                  T* __restrict__ Q_out, int max_sweeps, double tol, double cut, int* sweep_count, int nrel) {
    extern __shared__ unsigned char smem_raw[];
    constexpr int RL = LP * R;
    constexpr bool kPrefetchQ = sizeof(T) * R <= 48;   // keep the Q column pair in registers too
    const int kp = (k + 1) & ~1;
    const int ld = svdj_ld<T>(RL);             // column stride: whole bank rows
    T* Xc = reinterpret_cast<T*>(smem_raw);   // Xc[c * ld + r]
    T* Qc = Xc + kp * ld;
    __shared__ T s_wmax[32];
    __shared__ int s_wrot[32];
    __shared__ T s_norm[160];
    __shared__ T s_cn[160];
    __shared__ unsigned char s_top[160];
    __shared__ T s_scale;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int grp = tid / LP, gl = tid % LP;
    const int lane = tid & 31, warp = tid >> 5, nw = (nt + 31) >> 5;
    const unsigned gmask = (LP >= 32) ? 0xffffffffu : (((1u << LP) - 1u) << (lane & ~(LP - 1)));
    const double eps = sizeof(T) == 8 ? 1.1e-16 : 6e-8;
    // exact power-of-two scaling: largest |entry| in [1, 2)
    T mx = T(0);
    for (int e = tid; e < k * k; e += nt) mx = fmax(mx, fabs(Xin[e]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) s_wmax[warp] = mx;
    __syncthreads();
    if (tid == 0) {
        T m = T(0);
        for (int w = 0; w < nw; ++w) m = fmax(m, s_wmax[w]);
        int ex = 0;
        if (m > T(0)) frexp(m, &ex);
        s_scale = (m > T(0)) ? (T)ldexp(1.0, 1 - ex) : T(1);
    }
    __syncthreads();
    const T scale = s_scale;
    for (int e = tid; e < kp * ld; e += nt) {
        int c = e / ld, r = e % ld;
        Xc[e] = (r < k && c < k) ? Xin[(long long)r * k + c] * scale : T(0);
        Qc[e] = (r == c) ? T(1) : T(0);
    }
    // the cosine of two columns is only known to ~k eps (dot-product rounding)
    const T tol_eff = (T)fmax(tol, 2.0 * k * eps);
    const T tol2 = tol_eff * tol_eff;
    const T floor2 = (T)(1e6 * eps * eps);
    T prev2 = T(1e30);
    int sw = 0;
    if (nrel <= 0 || nrel > kp) nrel = kp;
    const bool active = grp < kp / 2;
    // lane gl owns the row pairs (2 gl, 2 gl + 1) + 2 LP jb, jb < R/2, accessed
    // as one 2-element vector; the row-pair blocks are visited in an order
    // shifted by the group's slot in its warp
    static_assert(R % 2 == 0, "R even");
    using V2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
    int offs[R / 2];
    {
        int jb = (grp % (32 / LP)) % (R / 2);
#pragma unroll
        for (int j = 0; j < R / 2; ++j) {
            offs[j] = 2 * LP * jb;
            if (++jb == R / 2) jb = 0;
        }
    }
    for (; sw < max_sweeps; ++sw) {
        __syncthreads();
        if (nrel < kp) {
            // columns among the nrel largest must converge; tail-tail pairs are
            // still rotated but do not keep the sweep loop alive
            for (int c = warp; c < kp; c += nw) {
                T a = T(0);
                for (int row = lane; row < kp; row += 32) { T u = Xc[c * ld + row]; a = fma(u, u, a); }
                for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
                if (lane == 0) s_cn[c] = a;
            }
            __syncthreads();
            for (int c = tid; c < kp; c += nt) {
                int rank = 0;
                const T cc = s_cn[c];
                for (int j = 0; j < kp; ++j) rank += (s_cn[j] > cc) || (s_cn[j] == cc && j < c);
                s_top[c] = rank < nrel;
            }
        } else {
            for (int c = tid; c < kp; c += nt) s_top[c] = 1;
        }
        __syncthreads();
        T c2max = T(0);
        int rot = 0;
        for (int r = 0; r < kp - 1; ++r) {
            if (active) {
                int p, q;
                round_robin_pair<T>(r, grp, kp, p, q);
                T* xp = Xc + p * ld + 2 * gl;
                T* xq = Xc + q * ld + 2 * gl;
                T* qp = Qc + p * ld + 2 * gl;
                T* qq = Qc + q * ld + 2 * gl;
                T u[R], v[R], qu[R], qv[R];
                auto ld2 = [&](const T* base, T* dst) {
#pragma unroll
                    for (int j = 0; j < R / 2; ++j) {
                        const V2 w = *reinterpret_cast<const V2*>(base + offs[j]);
                        dst[2 * j] = w.x;
                        dst[2 * j + 1] = w.y;
                    }
                };
                auto st2 = [&](T* base, const T* src) {
#pragma unroll
                    for (int j = 0; j < R / 2; ++j) {
                        V2 w;
                        w.x = src[2 * j];
                        w.y = src[2 * j + 1];
                        *reinterpret_cast<V2*>(base + offs[j]) = w;
                    }
                };
                ld2(xp, u);
                ld2(xq, v);
                if (kPrefetchQ) {
                    ld2(qp, qu);
                    ld2(qq, qv);
                }
                T a = T(0), b = T(0), g = T(0);
#pragma unroll
                for (int j = 0; j < R; ++j) { a = fma(u[j], u[j], a); b = fma(v[j], v[j], b); g = fma(u[j], v[j], g); }
#pragma unroll
                for (int o = LP / 2; o > 0; o >>= 1) {
                    a += __shfl_xor_sync(gmask, a, o);
                    b += __shfl_xor_sync(gmask, b, o);
                    g += __shfl_xor_sync(gmask, g, o);
                }
                // a, b, g are bitwise equal in all lanes of the group: the
                // branches below are group-uniform
                const T ab = a * b, g2 = g * g;
                if (g != T(0) && ab > T(0)) {
                    const bool rel = s_top[p] | s_top[q];
                    if (rel) c2max = fmax(c2max, g2 / ab);
                    if (g2 > tol2 * ab) {
                        T cT, sT;
                        jacobi_rotation(a, b, g, cT, sT);
                        T nu[R], nv[R];
#pragma unroll
                        for (int j = 0; j < R; ++j) {
                            nu[j] = cT * u[j] - sT * v[j];
                            nv[j] = sT * u[j] + cT * v[j];
                        }
                        st2(xp, nu);
                        st2(xq, nv);
                        if (!kPrefetchQ) {
                            ld2(qp, qu);
                            ld2(qq, qv);
                        }
#pragma unroll
                        for (int j = 0; j < R; ++j) {
                            nu[j] = cT * qu[j] - sT * qv[j];
                            nv[j] = sT * qu[j] + cT * qv[j];
                        }
                        st2(qp, nu);
                        st2(qq, nv);
                        rot |= rel;
                    }
                }
            }
            __syncthreads();
        }
        // block-wide max squared cosine and rotation flag, once per sweep
        for (int o = 16; o > 0; o >>= 1) {
            c2max = fmax(c2max, __shfl_xor_sync(0xffffffffu, c2max, o));
            rot |= __shfl_xor_sync(0xffffffffu, rot, o);
        }
        if (lane == 0) { s_wmax[warp] = c2max; s_wrot[warp] = rot; }
        __syncthreads();
        T bmax = T(0);
        int brot = 0;
        for (int w = 0; w < nw; ++w) { bmax = fmax(bmax, s_wmax[w]); brot |= s_wrot[w]; }
        if (brot == 0) break;
        // quadratic convergence: the cosines left after a sweep whose largest
        // was c are ~c^2, so c^2 < tol / 10 needs no confirming sweep
        if (bmax < T(0.1) * tol_eff) break;
        if (bmax < floor2 && bmax > T(0.0625) * prev2) break;   // stagnated at the floor
        prev2 = bmax;
    }
    __syncthreads();
    if (sweep_count && tid == 0) atomicAdd(sweep_count, sw + 1);
    for (int c = warp; c < kp; c += nw) {
        T a = T(0);
        for (int row = lane; row < kp; row += 32) { T u = Xc[c * ld + row]; a = fma(u, u, a); }
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) s_norm[c] = (c < k) ? sqrt(a) : T(-1);
    }
    __syncthreads();
    T smax = T(0);
    for (int c = lane; c < k; c += 32) smax = fmax(smax, s_norm[c]);
    for (int o = 16; o > 0; o >>= 1) smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
    const T cutT = (T)cut, rscale = T(1) / scale;
    for (int c = warp; c < k; c += nw) {
        const T sc = s_norm[c];
        int rank = 0;
        for (int j = lane; j < k; j += 32) rank += (s_norm[j] > sc) || (s_norm[j] == sc && j < c);
        for (int o = 16; o > 0; o >>= 1) rank += __shfl_xor_sync(0xffffffffu, rank, o);
        const T inv = (smax > T(0) && sc > cutT * smax) ? T(1) / sc : T(0);
        for (int row = lane; row < k; row += 32) {
            L_out[(long long)row * k + rank] = Xc[c * ld + row] * inv;
            Q_out[(long long)row * k + rank] = Qc[c * ld + row];
        }
        if (lane == 0) s_out[rank] = sc * rscale;
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
// sorted = false keeps the given column order (a second pass over columns that
// are already orthonormal: their norms carry no information).  ns_tol > 0:
// when the Gram matrix of the nonzero columns deviates from the identity by
// less than ns_tol (max entry), X is one Newton-Schulz step (3I - G)/2
// instead (orthogonality error ~ (3/4) ns_tol^2), zero for zero columns.
// defer > tau: a column whose pivot lies in (tau, defer) is moved, once, to the
// end of the order.  Accepting a pivot d multiplies the rounding error of every
// later pivot by about 1/d, and Q = Y X inherits an error ~ eps ||Y|| / sqrt(d)
// outside span(Y); a column nearly parallel to the ones before it is therefore
// taken after the well-conditioned ones, by which time its residual has
// usually become exactly zero (a rank-revealing order, as in column pivoting).
template <typename T>
void cholqr_factor(const double* dG, int k, double cut_abs, double tau, T* X, cudaStream_t st, bool sorted = true,
                   double ns_tol = 0.0, double defer = 0.0);

#ifdef KH_JACOBI_KERNEL
__device__ __forceinline__ float chol_recip(float x) { return __fdividef(1.f, x); }
__device__ __forceinline__ double chol_recip(double x) { return 1.0 / x; }

// Shared state of the two CholQR factor kernels (shared memory).
template <typename T>
struct CholShared {
    static constexpr int KM = sizeof(T) == 8 ? 112 : 160;   // largest k
    T inv[KM], diag[KM], rs[KM];
    int perm[KM];
    int keep[KM];
    T mx;
};

// Prologue of the factor kernels: column norms, the Newton-Schulz shortcut
// (returns true when X was written that way), the order (by norm when
// sorted), and the scaled, permuted Gram matrix into Lm (k x ld); Li zeroed.
template <typename T>
__device__ bool cholqr_prologue(const double* __restrict__ G, int k, double cut_abs, T* __restrict__ X, int sorted,
                                double ns_tol, T* Lm, T* Li, int ld, CholShared<T>& sh) {
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    for (int j = tid; j < k; j += nt) sh.diag[j] = (T)fmax(G[(long long)j * k + j], 0.0);
    __syncthreads();
    if (ns_tol > 0.0) {
        // Gram of the nonzero columns close to the identity: one Newton-Schulz step
        T dev = T(0);
        for (int e = tid; e < k * k; e += nt) {
            const int i = e / k, j = e % k;
            if (sh.diag[i] > T(0) && sh.diag[j] > T(0)) dev = fmax(dev, fabs((T)G[e] - (i == j ? T(1) : T(0))));
        }
        for (int o = 16; o > 0; o >>= 1) dev = fmax(dev, __shfl_xor_sync(0xffffffffu, dev, o));
        if (lane == 0) sh.inv[warp] = dev;          // inv reused as the reduction buffer (nw <= 32)
        __syncthreads();
        if (tid == 0) {
            T m = T(0);
            for (int w = 0; w < nw; ++w) m = fmax(m, sh.inv[w]);
            sh.mx = m;
        }
        __syncthreads();
        if (sh.mx < (T)ns_tol) {
            for (int e = tid; e < k * k; e += nt) {
                const int i = e / k, j = e % k;
                const bool live = sh.diag[i] > T(0) && sh.diag[j] > T(0);
                X[e] = live ? ((i == j ? T(1.5) : T(0)) - T(0.5) * (T)G[e]) : T(0);
            }
            return true;
        }
        __syncthreads();
    }
    if (warp == 0) {
        T m = T(0);
        for (int j = lane; j < k; j += 32) m = fmax(m, sh.diag[j]);
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) sh.mx = sqrt(m);
    }
    __syncthreads();
    const T cutT = (T)cut_abs;
    for (int j = tid; j < k; j += nt) {
        const T dj = sh.diag[j];
        const T nj = sqrt(dj);
        sh.inv[j] = (sh.mx > T(0) && nj > cutT * sh.mx) ? T(1) / nj : T(0);
        int rank = j;
        if (sorted) {
            rank = 0;
            for (int i = 0; i < k; ++i) rank += (sh.diag[i] > dj) || (sh.diag[i] == dj && i < j);
        }
        sh.perm[rank] = j;
    }
    __syncthreads();
    for (int e = tid; e < k * k; e += nt) {
        int a = e / k, b = e % k;
        int pa = sh.perm[a], pb = sh.perm[b];
        Lm[a * ld + b] = (T)G[(long long)pa * k + pb] * sh.inv[pa] * sh.inv[pb];
        Li[a * ld + b] = T(0);
    }
    __syncthreads();
    return false;
}

// Epilogue: Lm holds the Schur-complement entries a_ij (i > j) and pivots
// d_j = a_jj; pivots <= tau are dropped directions.  Scales the factor,
// inverts it (8 x 8 diagonal blocks in parallel, then recursive doubling:
// pairs of inverted diagonal blocks A (above) and C (below) are joined by
// Li_CA = -Li_CC (L_CA Li_AA), two parallel products per level, the
// intermediate kept in the unused upper triangle of L) and writes X.
template <typename T>
__device__ void cholqr_epilogue(int k, double tau, T* __restrict__ X, T* Lm, T* Li, int ld, CholShared<T>& sh) {
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const T tauT = (T)tau;
    for (int j = tid; j < k; j += nt) {
        const T d = Lm[j * ld + j];
        const bool keep = d > tauT;
        sh.keep[j] = keep;
        sh.rs[j] = keep ? T(1) / sqrt(d) : T(0);
    }
    __syncthreads();
    for (int e = tid; e < k * k; e += nt) {       // L_ij = a_ij / sqrt(d_j); unit diagonal for dropped j
        int i = e / k, j = e % k;
        if (i > j) Lm[i * ld + j] *= sh.rs[j];
        else if (i == j) Lm[i * ld + i] = sh.keep[i] ? sqrt(Lm[i * ld + i]) : T(1);
    }
    __syncthreads();
    // diagonal 8 x 8 blocks of L^-1: lane c < 8 of warp w inverts column c of block w
    const int nb = (k + 7) / 8;
    for (int blk = warp; blk < nb; blk += nw) {
        const int j0 = blk * 8, bs = min(8, k - j0);
        if (lane < bs) {
            const int c = lane;
            T x[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const int rr = r < bs ? r : bs - 1;        // in-bounds address for padded rows
                T v = (r == c) ? T(1) : T(0);
#pragma unroll
                for (int m = 0; m < 8; ++m)
                    if (m < r) v -= Lm[(j0 + rr) * ld + j0 + m] * x[m];
                x[r] = v / Lm[(j0 + rr) * ld + j0 + rr];
            }
#pragma unroll
            for (int r = 0; r < 8; ++r)
                if (r < bs) Li[(j0 + r) * ld + j0 + c] = x[r];
        }
    }
    __syncthreads();
    // recursive doubling over spans s = 8, 16, 32, ...: A = rows [a0, a0+s),
    // C = rows [a0+s, min(a0+2s, k)); Tm[c][a] = sum_m L[c][m] Li[m][a] stored
    // at Lm[a][c] (upper triangle), then Li[c][a] = -sum_m Li[c][m] Tm[m][a]
    // Each thread computes a 2 x 2 tile (rows ci, ci+1; columns aj, aj+1): the
    // sums run over the pair's common range, the extra terms being products
    // with zeros of the upper triangles of Li (zero from the prologue and the
    // diagonal-block inversion).
    for (int sp = 8; sp < k; sp *= 2) {
        const int npair = (k + 2 * sp - 1) / (2 * sp);
        const int hs = sp / 2;
        const int items = npair * hs * hs;          // pair p, C row pair, A column pair
        for (int e = tid; e < items; e += nt) {
            const int p = e / (hs * hs), rem = e % (hs * hs);
            const int a0 = p * 2 * sp, ci = a0 + sp + 2 * (rem / hs), aj = a0 + 2 * (rem % hs);
            if (ci >= k) continue;
            const bool r1 = ci + 1 < k;
            T s00 = T(0), s01 = T(0), s10 = T(0), s11 = T(0);
            for (int m = aj; m < a0 + sp; ++m) {
                const T l0 = Lm[ci * ld + m], l1 = r1 ? Lm[(ci + 1) * ld + m] : T(0);
                const T i0 = Li[m * ld + aj], i1 = Li[m * ld + aj + 1];
                s00 = fma(l0, i0, s00);
                s01 = fma(l0, i1, s01);
                s10 = fma(l1, i0, s10);
                s11 = fma(l1, i1, s11);
            }
            Lm[aj * ld + ci] = s00;                 // Tm[c][a] at Lm[a][c] (upper triangle)
            Lm[(aj + 1) * ld + ci] = s01;
            if (r1) {
                Lm[aj * ld + ci + 1] = s10;
                Lm[(aj + 1) * ld + ci + 1] = s11;
            }
        }
        __syncthreads();
        for (int e = tid; e < items; e += nt) {
            const int p = e / (hs * hs), rem = e % (hs * hs);
            const int a0 = p * 2 * sp, ci = a0 + sp + 2 * (rem / hs), aj = a0 + 2 * (rem % hs);
            if (ci >= k) continue;
            const bool r1 = ci + 1 < k;
            const int mend = r1 ? ci + 1 : ci;      // row ci's term at m = ci + 1 is Li[ci][ci+1] = 0
            T s00 = T(0), s01 = T(0), s10 = T(0), s11 = T(0);
            for (int m = a0 + sp; m <= mend; ++m) {
                const T l0 = Li[ci * ld + m], l1 = r1 ? Li[(ci + 1) * ld + m] : T(0);
                const T t0 = Lm[aj * ld + m], t1 = Lm[(aj + 1) * ld + m];
                s00 = fma(l0, t0, s00);
                s01 = fma(l0, t1, s01);
                s10 = fma(l1, t0, s10);
                s11 = fma(l1, t1, s11);
            }
            Li[ci * ld + aj] = -s00;
            Li[ci * ld + aj + 1] = -s01;
            if (r1) {
                Li[(ci + 1) * ld + aj] = -s10;
                Li[(ci + 1) * ld + aj + 1] = -s11;
            }
        }
        __syncthreads();
    }
    // X[perm a][b] = inv[perm a] * Li[b][a]   (Q = Y_s L^-T; dropped b give zero columns)
    for (int e = tid; e < k * k; e += nt) {
        int a = e / k, b = e % k;
        int pa = sh.perm[a];
        X[(long long)pa * k + b] = sh.keep[b] ? sh.inv[pa] * Li[b * ld + a] : T(0);
    }
}

// Right-looking Cholesky with one barrier per column (unscaled columns, the
// scaling applied at the end) and pivot deferral (see cholqr_factor).
template <typename T>
__global__ void __launch_bounds__(1024)
cholqr_kernel(const double* __restrict__ G, int k, double cut_abs, double tau, T* __restrict__ X, int sorted,
              double ns_tol, double defer) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ CholShared<T> sh;
    const int ld = k | 1;                          // odd row stride: conflict-free column walks
    T* Lm = reinterpret_cast<T*>(smem_raw);       // k x ld, row-major (lower triangle: L)
    T* Li = Lm + k * ld;                           // k x ld: L^-1
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    if (cholqr_prologue<T>(G, k, cut_abs, X, sorted, ns_tol, Lm, Li, ld, sh)) return;
    const T tauT = (T)tau;
    // Cholesky: step j leaves the Schur-complement entries a_ij (i > j) in
    // column j and subtracts a_ij a_cj / d_j from the trailing block; a pivot
    // d_j <= tau drops direction j (no update, zero column).  A pivot in
    // (tau, defer) is first rotated to the end of the order (positions
    // j+1, ..., k-1 move up by one), each column at most once: the nd deferred
    // columns occupy the last nd positions.
    const T deferT = (T)defer;
    int nd = 0;
    for (int j = 0; j < k;) {
        const T d = Lm[j * ld + j];              // same value in every thread
        if (d > tauT && d < deferT && j < k - nd) {
            // new position a holds old position src(a): a (a < j), a + 1 (j <= a < k-1), j (a = k-1).
            // Rows j.. of the lower triangle are gathered into Li, then copied back.
            const int rows = k - j;
            int pnew = 0;
            if (tid < rows) pnew = sh.perm[tid + 1 < rows ? j + tid + 1 : j];
            for (int e = tid; e < rows * k; e += nt) {
                const int a = j + e / k, b = e % k;
                if (b > a) continue;
                const int pa = a < k - 1 ? a + 1 : j;
                const int pb = b < j ? b : (b < k - 1 ? b + 1 : j);
                Li[a * ld + b] = pa >= pb ? Lm[pa * ld + pb] : Lm[pb * ld + pa];
            }
            __syncthreads();
            for (int e = tid; e < rows * k; e += nt) {
                const int a = j + e / k, b = e % k;
                if (b > a) continue;
                Lm[a * ld + b] = Li[a * ld + b];
                Li[a * ld + b] = T(0);
            }
            if (tid < rows) sh.perm[j + tid] = pnew;
            __syncthreads();
            ++nd;
            continue;
        }
        if (d > tauT) {
            // trailing update a_ic -= a_ij a_cj / d_j (c <= i): rows
            // i = j + 1 + warp + nw a, columns c = j + 1 + lane + 32 b; the pivot
            // column's entries of a thread's rows and columns are loaded first
            // (independent loads), then only the tile entries below the
            // diagonal are visited
            constexpr int RT = (CholShared<T>::KM + 31) / 32;   // rows per warp / columns per lane at nw = 32
            const T rd = chol_recip(d);
            T li[RT], lc[RT];
#pragma unroll
            for (int a = 0; a < RT; ++a) {
                const int i = j + 1 + warp + nw * a, c = j + 1 + lane + 32 * a;
                li[a] = i < k ? Lm[i * ld + j] : T(0);
                lc[a] = c < k ? Lm[c * ld + j] : T(0);
            }
#pragma unroll
            for (int a = 0; a < RT; ++a) {
                const int i = j + 1 + warp + nw * a;
                if (i >= k) break;
                const T lia = li[a] * rd;
#pragma unroll
                for (int b = 0; b < RT; ++b) {
                    const int c = j + 1 + lane + 32 * b;
                    if (c > i) break;
                    Lm[i * ld + c] -= lia * lc[b];
                }
            }
            // rows beyond the tile (fewer than 32 warps)
            for (int i = j + 1 + warp + nw * RT; i < k; i += nw) {
                const T lij = Lm[i * ld + j] * rd;
                for (int c = j + 1 + lane; c <= i; c += 32) Lm[i * ld + c] -= lij * Lm[c * ld + j];
            }
        }
        __syncthreads();
        ++j;
    }
    cholqr_epilogue<T>(k, tau, X, Lm, Li, ld, sh);
}

#endif  // KH_JACOBI_KERNEL

}  // namespace kh
