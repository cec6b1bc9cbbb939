// FP64 refinement of a small SVD computed in single precision.
//
// The projector's Rayleigh-Ritz step needs the SVD of a k x k matrix G
// (k <= 160).  The one-sided Jacobi kernel computes it in FP32 in one CTA;
// an FP64 Jacobi in one CTA would run on the SM's FP64 pipe, a small fraction
// of its FP32 rate on this GPU, and cost a millisecond per call.  Instead one
// Newton step in FP64 squares the FP32 factors' errors, further steps take
// them to FP64 rounding: every piece is a k x k product or an elementwise
// formula, spread over many CTAs.
//
// With G Q ~ L S from single precision, write the exact factors as
// L' = L (I + F), Q' = Q (I + H).  To first order in the small quantities
//   R = I - L^T L,  P = I - Q^T Q,  T = L^T G Q (~ diagonal),
// orthogonality of L' and Q' asks F + F^T = R and H + H^T = P, and a diagonal
// L'^T G Q' asks, for i != j,
//   t_ij + f_ji s_j + s_i h_ij = 0   and   t_ji + f_ij s_i + s_j h_ji = 0.
// Eliminating f_ji = r_ij - f_ij and h_ji = p_ij - h_ij leaves a 2 x 2 system
// per pair with determinant s_j^2 - s_i^2:
//   f_ij = (s_j a + s_i b) / (s_j^2 - s_i^2),  h_ij = (s_i a + s_j b) / (s_j^2 - s_i^2),
//   a = t_ij + s_j r_ij,  b = t_ji + s_j p_ij;
// the diagonal gives f_ii = r_ii / 2, h_ii = p_ii / 2 and the refined
// singular value s_i' = t_ii (1 + (r_ii + p_ii) / 2).  The step is Newton's
// method for the SVD equations (quadratic convergence; the same iteration as
// the refinement of Ogita and Aishima, J. Comput. Appl. Math. 2020, derived
// here from first-order perturbation theory).  For a pair whose singular
// values agree to within the single-precision error the 2 x 2 system is
// ill-conditioned and only the orthogonality part (f_ij = r_ij / 2,
// h_ij = p_ij / 2) is applied: the pair's common subspace, which is all the
// projectors depend on, is kept.
#include <cooperative_groups.h>

#include "engine.cuh"

namespace kh {

namespace {

constexpr int kRefineThreads = 64;   // one output entry per thread; k^2 / 64 CTAs

// R = I - L^T L, P = I - Q^T Q, W = L^T G (all k x k, row-major; L, Q hold
// vectors as columns).
__global__ void __launch_bounds__(kRefineThreads)
refine_products_kernel(const double* __restrict__ G, const double* __restrict__ L, const double* __restrict__ Q,
                       int k, double* __restrict__ R, double* __restrict__ P, double* __restrict__ W) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= k * k) return;
    const int i = e / k, j = e % k;
    double r = 0.0, p = 0.0, w = 0.0;
    for (int m = 0; m < k; ++m) {
        const double lmi = L[m * k + i];
        r = fma(lmi, L[m * k + j], r);
        p = fma(Q[m * k + i], Q[m * k + j], p);
        w = fma(lmi, G[m * k + j], w);
    }
    const double d = (i == j) ? 1.0 : 0.0;
    R[e] = d - r;
    P[e] = d - p;
    W[e] = w;
}

// T = W Q
__global__ void __launch_bounds__(kRefineThreads)
refine_t_kernel(const double* __restrict__ W, const double* __restrict__ Q, int k, double* __restrict__ T) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= k * k) return;
    const int i = e / k, j = e % k;
    double t = 0.0;
    for (int m = 0; m < k; ++m) t = fma(W[i * k + m], Q[m * k + j], t);
    T[e] = t;
}

// F, H (the corrections) and the refined singular values (diagonal threads).
// A pair is treated as clustered when its singular values differ by no more
// than rel_gap times the larger one, or by no more than 64 times its coupling
// |t_ij|, |t_ji| (or both vanish): the correction of a pair it does rotate is
// then below 1/64, whose square the next step removes.
__global__ void __launch_bounds__(kRefineThreads)
refine_corrections_kernel(const double* __restrict__ R, const double* __restrict__ P, const double* __restrict__ T,
                          int k, double rel_gap, double* __restrict__ F, double* __restrict__ H,
                          double* __restrict__ s_out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= k * k) return;
    const int i = e / k, j = e % k;
    const double rij = R[e], pij = P[e];
    if (i == j) {
        F[e] = 0.5 * rij;
        H[e] = 0.5 * pij;
        s_out[i] = T[e] * (1.0 + 0.5 * (rij + pij));
        return;
    }
    // Newton's correction is valid while the pair's coupling is small against
    // the gap of its singular values
    const double si = T[i * k + i], sj = T[j * k + j];
    const double big = fmax(fabs(si), fabs(sj));
    const double coupling = fmax(fabs(T[e]), fabs(T[j * k + i]));
    if (!(fabs(sj - si) > fmax(rel_gap * big, 64.0 * coupling)) || big == 0.0) {
        F[e] = 0.5 * rij;
        H[e] = 0.5 * pij;
        return;
    }
    const double a = T[e] + sj * rij;
    const double b = T[j * k + i] + sj * pij;
    const double inv = 1.0 / ((sj - si) * (sj + si));
    F[e] = (sj * a + si * b) * inv;
    H[e] = (si * a + sj * b) * inv;
}

// L' = L + L F and Q' = Q + Q H (blockIdx.y selects the factor).
__global__ void __launch_bounds__(kRefineThreads)
refine_apply_kernel(const double* __restrict__ L, const double* __restrict__ Q, const double* __restrict__ F,
                    const double* __restrict__ H, int k, double* __restrict__ Lo, double* __restrict__ Qo) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= k * k) return;
    const int i = e / k, j = e % k;
    const double* X = blockIdx.y == 0 ? L : Q;
    const double* C = blockIdx.y == 0 ? F : H;
    double acc = X[e];
    for (int m = 0; m < k; ++m) acc = fma(X[i * k + m], C[m * k + j], acc);
    (blockIdx.y == 0 ? Lo : Qo)[e] = acc;
}

// Newton correction (f_ij, h_ij) of entry (i, j) from R, P, T (see above).
__device__ __forceinline__ void newton_entry(const double* __restrict__ R, const double* __restrict__ P,
                                             const double* __restrict__ T, int k, double gap, int i, int j,
                                             double& f, double& h) {
    const long long e = (long long)i * k + j;
    const double rij = R[e], pij = P[e];
    if (i == j) {
        f = 0.5 * rij;
        h = 0.5 * pij;
        return;
    }
    const double si = T[(long long)i * k + i], sj = T[(long long)j * k + j];
    const double tij = T[e], tji = T[(long long)j * k + i];
    const double big = fmax(fabs(si), fabs(sj));
    const double coupling = fmax(fabs(tij), fabs(tji));
    if (!(fabs(sj - si) > fmax(gap * big, 64.0 * coupling)) || big == 0.0) {
        f = 0.5 * rij;
        h = 0.5 * pij;
        return;
    }
    const double a = tij + sj * rij;
    const double b = tji + sj * pij;
    const double inv = 1.0 / ((sj - si) * (sj + si));
    f = (sj * a + si * b) * inv;
    h = (si * a + sj * b) * inv;
}

// All refinement steps in one cooperative launch.  Every CTA owns 8 x 8
// output tiles (grid-stride over the (k/8)^2 tiles) with 256 threads: four
// groups of 64 split each k-long FP64 dot product into quarters (shorter
// dependent chains, all four SM sub-partitions busy), the partial sums joined
// in shared memory in a fixed order.  Three phases per step, separated by
// grid barriers: R, P, W = L^T G; T = W Q; L' = L + L F and Q' = Q + Q H with
// the corrections F, H formed on the fly from R, P, T for the tile's column
// slab.  Operands are staged as 8-wide slabs in shared memory (the FP64 pipe
// then runs from shared memory).  The factors ping-pong between (L1, Q1) and
// (Lo, Qo).
constexpr int kRT = 8;                                     // tile edge
constexpr int kRQ = 4;                                     // K split
constexpr int kRThreads = kRT * kRT * kRQ;
__global__ void __launch_bounds__(kRThreads)
refine_coop_kernel(const double* __restrict__ G, int k, const double* L0, const double* Q0, double* s_out,
                   double* Lo, double* Qo, double* work, double rel_gap, int newton_steps) {
    namespace cg = cooperative_groups;
    cg::grid_group grid = cg::this_grid();
    extern __shared__ double slab[];                       // 5 slabs of 8 x k, then 3 x kRQ x 64 partial sums
    const long long kk = (long long)k * k;
    double *R = work, *P = work + kk, *W = work + 2 * kk, *T = work + 3 * kk, *L1 = work + 6 * kk,
           *Q1 = work + 7 * kk;
    const int nt = (k + kRT - 1) / kRT, ntiles = nt * nt;
    const int tid = threadIdx.x, q = tid / (kRT * kRT), e64 = tid % (kRT * kRT), ti = e64 / kRT, tj = e64 % kRT;
    const int mq0 = q * k / kRQ, mq1 = (q + 1) * k / kRQ;  // this group's part of the sum
    double* s0 = slab;
    double* s1 = slab + kRT * k;
    double* s2 = slab + 2 * kRT * k;
    double* s3 = slab + 3 * kRT * k;
    double* s4 = slab + 4 * kRT * k;
    double* red = slab + 5 * kRT * k;                      // red[(c * kRQ + q) * 64 + e64]
    // slab of columns [c0, c0+8) of X (k x k): sl[m * 8 + c] = X[m][c0 + c]
    auto load_cols = [&](double* sl, const double* X, int c0) {
        for (int e = tid; e < kRT * k; e += kRThreads) {
            const int m = e / kRT, c = e % kRT;
            sl[e] = (c0 + c < k) ? X[m * k + c0 + c] : 0.0;
        }
    };
    // slab of rows [r0, r0+8) of X: sl[m * 8 + r] = X[r0 + r][m] (same indexing as a column slab of X^T)
    auto load_rows = [&](double* sl, const double* X, int r0) {
        for (int e = tid; e < kRT * k; e += kRThreads) {
            const int r = e / k, m = e % k;
            sl[m * kRT + r] = (r0 + r < k) ? X[(r0 + r) * k + m] : 0.0;
        }
    };
    // sum over this group's m of a[m][ti] b[m][tj] (two chains)
    auto dot = [&](const double* a, const double* b) {
        double x0 = 0.0, x1 = 0.0;
        int m = mq0;
        for (; m + 1 < mq1; m += 2) {
            x0 = fma(a[m * kRT + ti], b[m * kRT + tj], x0);
            x1 = fma(a[(m + 1) * kRT + ti], b[(m + 1) * kRT + tj], x1);
        }
        if (m < mq1) x0 = fma(a[m * kRT + ti], b[m * kRT + tj], x0);
        return x0 + x1;
    };
    // joins the kRQ partial sums of quantity c (group 0 reads them in order)
    auto joined = [&](int c) {
        double x = 0.0;
#pragma unroll
        for (int g = 0; g < kRQ; ++g) x += red[(c * kRQ + g) * 64 + e64];
        return x;
    };
    const int nsteps = newton_steps + 1;
    for (int step = 0; step < nsteps; ++step) {
        const int rem = nsteps - 1 - step;                 // steps after this one; the last writes (Lo, Qo)
        const double* Li = step == 0 ? L0 : ((rem % 2 == 0) ? L1 : Lo);
        const double* Qi = step == 0 ? Q0 : ((rem % 2 == 0) ? Q1 : Qo);
        double* Ln = (rem % 2 == 0) ? Lo : L1;
        double* Qn = (rem % 2 == 0) ? Qo : Q1;
        const double gap = step < newton_steps ? rel_gap : INFINITY;
        // phase 1: R = I - L^T L, P = I - Q^T Q, W = L^T G on tile (I, J)
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            const int i0 = (t / nt) * kRT, j0 = (t % nt) * kRT;
            __syncthreads();
            load_cols(s0, Li, i0);
            load_cols(s1, Li, j0);
            load_cols(s2, Qi, i0);
            load_cols(s3, Qi, j0);
            load_cols(s4, G, j0);
            __syncthreads();
            red[(0 * kRQ + q) * 64 + e64] = dot(s0, s1);
            red[(1 * kRQ + q) * 64 + e64] = dot(s2, s3);
            red[(2 * kRQ + q) * 64 + e64] = dot(s0, s4);
            __syncthreads();
            const int i = i0 + ti, j = j0 + tj;
            if (q == 0 && i < k && j < k) {
                const double d = (i == j) ? 1.0 : 0.0;
                R[i * k + j] = d - joined(0);
                P[i * k + j] = d - joined(1);
                W[i * k + j] = joined(2);
            }
        }
        grid.sync();
        // phase 2: T = W Q
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            const int i0 = (t / nt) * kRT, j0 = (t % nt) * kRT;
            __syncthreads();
            load_rows(s0, W, i0);
            load_cols(s1, Qi, j0);
            __syncthreads();
            red[q * 64 + e64] = dot(s0, s1);
            __syncthreads();
            const int i = i0 + ti, j = j0 + tj;
            if (q == 0 && i < k && j < k) T[i * k + j] = joined(0);
        }
        grid.sync();
        // refined singular values (one CTA)
        if (blockIdx.x == 0)
            for (int i = tid; i < k; i += kRThreads) {
                const long long e = (long long)i * k + i;
                s_out[i] = T[e] * (1.0 + 0.5 * (R[e] + P[e]));
            }
        // phase 3: L' = L + L F, Q' = Q + Q H, the corrections of the tile's
        // column slab formed from R, P, T
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            const int i0 = (t / nt) * kRT, j0 = (t % nt) * kRT;
            __syncthreads();
            load_rows(s0, Li, i0);
            load_rows(s2, Qi, i0);
            for (int e = tid; e < kRT * k; e += kRThreads) {
                const int m = e / kRT, j = j0 + e % kRT;
                double f = 0.0, h = 0.0;
                if (j < k) newton_entry(R, P, T, k, gap, m, j, f, h);
                s1[e] = f;
                s3[e] = h;
            }
            __syncthreads();
            red[(0 * kRQ + q) * 64 + e64] = dot(s0, s1);
            red[(1 * kRQ + q) * 64 + e64] = dot(s2, s3);
            __syncthreads();
            const int i = i0 + ti, j = j0 + tj;
            if (q == 0 && i < k && j < k) {
                Ln[i * k + j] = Li[i * k + j] + joined(0);
                Qn[i * k + j] = Qi[i * k + j] + joined(1);
            }
        }
        if (step + 1 < nsteps) grid.sync();
    }
}

}  // namespace

size_t svd_refine_scratch(int k) { return (size_t)8 * k * k; }

// G (k x k, FP64), L and Q (k x k FP64, columns = the single-precision left
// and right singular vectors, G Q ~ L diag(s)): three Newton steps and a
// re-orthogonalisation, the refined
// factors to Lo, Qo and the refined singular values to s (k).  work:
// svd_refine_scratch(k) doubles.
void svd_refine_fp64(const double* G, int k, const double* L, const double* Q, double* s, double* Lo, double* Qo,
                     double* work, double rel_gap, cudaStream_t st) {
    const long long kk = (long long)k * k;
    double *R = work, *P = work + kk, *W = work + 2 * kk, *T = work + 3 * kk, *F = work + 4 * kk, *H = work + 5 * kk;
    const int blocks = (int)((kk + kRefineThreads - 1) / kRefineThreads);
    {
        // one cooperative launch when the device allows it and the grid fits
        int dev = 0, coop = 0, sms = 0, per_sm = 0;
        KH_CUDA(cudaGetDevice(&dev));
        KH_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
        KH_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const size_t smem = ((size_t)5 * kRT * k + 3 * kRQ * kRT * kRT) * sizeof(double);
        static std::atomic<size_t> granted[kMaxDevices] = {};
        smem_opt_in(refine_coop_kernel, smem, granted);
        KH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, refine_coop_kernel, kRThreads, smem));
        const int ntiles = ((k + kRT - 1) / kRT) * ((k + kRT - 1) / kRT);
        const int cblocks = std::min(ntiles, per_sm * sms);
        if (coop && cblocks >= 1) {
            int newton = 3;
            void* args[] = {(void*)&G, (void*)&k, (void*)&L, (void*)&Q, (void*)&s, (void*)&Lo, (void*)&Qo,
                            (void*)&work, (void*)&rel_gap, (void*)&newton};
            KH_CUDA(cudaLaunchCooperativeKernel((const void*)refine_coop_kernel, dim3(cblocks), dim3(kRThreads),
                                                args, smem, st));
            KH_LAUNCHED();
            return;
        }
    }
    // three Newton steps: each squares the residuals of the pairs it rotates
    // (the FP32 ones, ~k 2^-24, reach FP64 rounding after two; a pair whose
    // correction was near the 1/64 limit needs the third) and re-orthogonalises
    // the clustered ones; a fourth step only re-orthogonalises (every pair
    // treated as clustered), squaring what the last rotation left of R and P
    for (int step = 0; step < 4; ++step) {
        const double* Li = step == 0 ? L : Lo;
        const double* Qi = step == 0 ? Q : Qo;
        refine_products_kernel<<<blocks, kRefineThreads, 0, st>>>(G, Li, Qi, k, R, P, W);
        KH_LAUNCHED();
        refine_t_kernel<<<blocks, kRefineThreads, 0, st>>>(W, Qi, k, T);
        KH_LAUNCHED();
        refine_corrections_kernel<<<blocks, kRefineThreads, 0, st>>>(R, P, T, k, step < 3 ? rel_gap : INFINITY, F,
                                                                      H, s);
        KH_LAUNCHED();
        // in place after the first step: each output entry reads its row of the
        // old factor, so the update goes through W and T (free by now) first
        double* Lt = step == 0 ? Lo : W;
        double* Qt = step == 0 ? Qo : T;
        refine_apply_kernel<<<dim3(blocks, 2), kRefineThreads, 0, st>>>(Li, Qi, F, H, k, Lt, Qt);
        KH_LAUNCHED();
        if (step > 0) {
            KH_CUDA(cudaMemcpyAsync(Lo, Lt, sizeof(double) * kk, cudaMemcpyDeviceToDevice, st));
            KH_CUDA(cudaMemcpyAsync(Qo, Qt, sizeof(double) * kk, cudaMemcpyDeviceToDevice, st));
        }
    }
}

}  // namespace kh
