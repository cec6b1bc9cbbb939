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

}  // namespace

size_t svd_refine_scratch(int k) { return (size_t)6 * k * k; }

// G (k x k, FP64), L and Q (k x k FP64, columns = the single-precision left
// and right singular vectors, G Q ~ L diag(s)): three Newton steps, the refined
// factors to Lo, Qo and the refined singular values to s (k).  work:
// svd_refine_scratch(k) doubles.
void svd_refine_fp64(const double* G, int k, const double* L, const double* Q, double* s, double* Lo, double* Qo,
                     double* work, double rel_gap, cudaStream_t st) {
    const long long kk = (long long)k * k;
    double *R = work, *P = work + kk, *W = work + 2 * kk, *T = work + 3 * kk, *F = work + 4 * kk, *H = work + 5 * kk;
    const int blocks = (int)((kk + kRefineThreads - 1) / kRefineThreads);
    // three steps: each squares the residuals of the pairs it rotates (the
    // FP32 ones, ~k 2^-24, reach FP64 rounding after two; a pair whose
    // correction was near the 1/64 limit needs the third) and re-orthogonalises
    // the clustered ones
    for (int step = 0; step < 3; ++step) {
        const double* Li = step == 0 ? L : Lo;
        const double* Qi = step == 0 ? Q : Qo;
        refine_products_kernel<<<blocks, kRefineThreads, 0, st>>>(G, Li, Qi, k, R, P, W);
        KH_LAUNCHED();
        refine_t_kernel<<<blocks, kRefineThreads, 0, st>>>(W, Qi, k, T);
        KH_LAUNCHED();
        refine_corrections_kernel<<<blocks, kRefineThreads, 0, st>>>(R, P, T, k, rel_gap, F, H, s);
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
