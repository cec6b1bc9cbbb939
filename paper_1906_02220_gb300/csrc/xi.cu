// Correlation length from the CTM environment (Sec. IV: the length the
// paper's scaling analysis uses, read off the channel transfer matrix).
//
// The channel transfer matrix of a direction is one column of double-layer
// sites between the two boundary edges across it: for the horizontal
// direction T[(a,l,b),(c,r,d)] = sum_{u,v} E1[a,u,c] site[l,u,r,v] E3[d,v,b],
// the vertical one the same in the frame turned by a quarter (edges E2, E4).
// xi = 1 / ln(|lambda_1| / |lambda_2|) from its two largest eigenvalues in
// modulus.  T (dimension chi^2 D^2) is never formed: it is applied to a block
// of b <= 4 vectors by the same contractions as an edge absorption (the
// edge GEMMs and the two-layer site contraction), and its leading eigenvalues
// come from a block power iteration with Rayleigh-Ritz steps: V <- orth(T V),
// H = V^T T V (b x b), eigenvalues of H by the shifted QR algorithm on the
// host (4 x 4).  A complex pair lambda_2 = conj(lambda_3) is captured by the
// block (its invariant subspace is real and two-dimensional).
#include <algorithm>
#include <complex>

#include "engine.cuh"

namespace kh {

namespace {

// x <- x - (d / s) y with d, s device scalars (s = 1 when null)
template <typename T>
__global__ void axpy_dev_kernel(const T* __restrict__ y, T* __restrict__ x, long long n, const double* d,
                                const double* s) {
    const double c = s ? *d / *s : *d;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] -= (T)(c * (double)y[i]);
}

// x <- x / sqrt(s), zero when s == 0
template <typename T>
__global__ void scale_rsqrt_kernel(T* __restrict__ x, long long n, const double* s) {
    const double v = *s;
    const double f = v > 0.0 ? 1.0 / sqrt(v) : 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] = (T)(f * (double)x[i]);
}

// out += sum_i a_i b_i (FP64 accumulation, one atomic per block)
template <typename T>
__global__ void dot_acc_kernel(const T* __restrict__ a, const T* __restrict__ b, long long n, double* out) {
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        s += (double)a[i] * (double)b[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double red[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = s;
    __syncthreads();
    if (w == 0) {
        s = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) atomicAdd(out, s);
    }
}

// x <- fresh random vector when its squared norm after the projections (post)
// is below rel2 times the one before them (pre): the column was dependent on
// the earlier ones, and what is left of it is rounding correlated with them
template <typename T>
__global__ void refill_if_dependent_kernel(T* __restrict__ x, long long n, const double* post, const double* pre,
                                           double rel2, uint64_t seed, uint64_t stream) {
    if (*post > rel2 * *pre) return;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] = (T)rnd_uniform(seed, stream, (uint64_t)i);
}

template <typename T>
__global__ void fill_random_kernel(T* V, long long n, uint64_t seed, uint64_t stream) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        V[i] = (T)rnd_uniform(seed, stream, (uint64_t)i);
}

// Eigenvalues of a small real matrix (m <= 4, row-major) by the shifted QR
// algorithm in complex arithmetic: A - mu I = Q R by Givens rotations,
// A <- R Q + mu I with the Wilkinson shift mu of the trailing 2 x 2 block,
// deflating the last row once its subdiagonal part is negligible.
std::vector<std::complex<double>> small_eigenvalues(const double* H, int m) {
    using C = std::complex<double>;
    C A[4][4];
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) A[i][j] = H[i * m + j];
    std::vector<C> ev;
    int hi = m - 1;
    for (int iter = 0; iter < 1000 && hi >= 0; ++iter) {
        if (hi == 0) {
            ev.push_back(A[0][0]);
            break;
        }
        double off = 0.0, scale = 0.0;
        for (int j = 0; j < hi; ++j) off = std::max(off, std::abs(A[hi][j]));
        for (int i = 0; i <= hi; ++i) scale = std::max(scale, std::abs(A[i][i]));
        if (off <= 1e-15 * (scale > 0.0 ? scale : 1.0)) {
            ev.push_back(A[hi][hi]);
            --hi;
            continue;
        }
        const int n = hi + 1;
        const C a = A[hi - 1][hi - 1], b = A[hi - 1][hi], c = A[hi][hi - 1], d = A[hi][hi];
        const C half = (a + d) / 2.0, disc = std::sqrt(half * half - (a * d - b * c));
        C mu = std::abs(half + disc - d) < std::abs(half - disc - d) ? half + disc : half - disc;
        if (iter % 16 == 15) mu += C(0.0, 1e-3 * (scale > 0.0 ? scale : 1.0));   // exceptional shift
        C Q[4][4];
        for (int i = 0; i < n; ++i) {
            A[i][i] -= mu;
            for (int j = 0; j < n; ++j) Q[i][j] = (i == j) ? C(1.0) : C(0.0);
        }
        for (int k = 0; k < n - 1; ++k)
            for (int i = k + 1; i < n; ++i) {
                const C x = A[k][k], y = A[i][k];
                const double r = std::sqrt(std::norm(x) + std::norm(y));
                if (r == 0.0 || std::abs(y) == 0.0) continue;
                const C cc = x / r, ss = y / r;
                for (int j = 0; j < n; ++j) {          // rows k, i of A and of Q
                    const C u = A[k][j], v = A[i][j];
                    A[k][j] = std::conj(cc) * u + std::conj(ss) * v;
                    A[i][j] = -ss * u + cc * v;
                    const C qu = Q[k][j], qv = Q[i][j];
                    Q[k][j] = std::conj(cc) * qu + std::conj(ss) * qv;
                    Q[i][j] = -ss * qu + cc * qv;
                }
            }
        // A = R, Q = Q_total with Q_total (A - mu I) = R: A <- R Q_total^H + mu I
        C R[4][4];
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) R[i][j] = A[i][j];
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                C s = 0.0;
                for (int p = 0; p < n; ++p) s += R[i][p] * std::conj(Q[j][p]);
                A[i][j] = s + (i == j ? mu : C(0.0));
            }
    }
    return ev;
}

}  // namespace

template <typename T>
void Engine<T>::correlation_length(int slot, int dir, int max_iter, double tol, double* out) {
    Slot<T>& sl = slots[slot];
    if (sl.p <= 0 || !sl.env_valid) fail(KH_EINVAL, "slot has no converged environment");
    if (dir < 0 || dir > 1) fail(KH_EINVAL, "direction must be 0 (horizontal) or 1 (vertical)");
    const int chi = dm.chi, d2 = dm.d2, D = dm.D, n = dm.n;
    const long long nt = (long long)chi * d2 * chi, chi2 = (long long)chi * chi, E1 = nt;
    const int b = (int)std::min<long long>(std::min(4, d2), nt);
    refresh_operands(sl);
    const int f = dir + 1;                         // frame whose corner operand contracts (u, r)
    const T* up = Eop + (long long)dir * E1;
    const T* dn = Eop + (long long)(dir + 2) * E1;
    T* V = Mt;                                     // b vectors, nt each (b <= D^2: b nt <= n^2)
    T* W = mupp;
    double* sc = dscr + DscrOff::kStage;           // FP64 scalars: 16 Gram / Ritz entries
    const int grid = grid_for(nt);
    auto apply_T = [&](const T* v, T* w) {
        // X[a,(uk,ub),(rk,rb),d] = sum_c up[a,u,c] v[c,r,d]
        gemm_rm<T>(chi * d2, d2 * chi, chi, up, false, v, false, Y1, st);
        // blocks (a, d) of [(ub, rb)][(uk, rk)]: the frame-f corner layout (L, U) = (u, r)
        site_operand(sl, Y1, Yp, {chi, D, D, D, D, chi}, {0, 5, 2, 4, 1, 3});
        const long long w4 = (long long)f * dm.D4 * dm.D4;
        site_layer(Yp, chi2, sl.Tcor + (long long)f * dm.pmax * dm.D4, lay_img(sl, 1, 0, f), lay_img(sl, 2, 0, f),
                   sl.p, Qt, sl.dl ? sl.Wcor + w4 : nullptr,
                   sl.dl && sl.Wcor_lo ? sl.Wcor_lo + w4 : nullptr, site_presplit(sl));
        // Qt[a][d][(vk, lk)][(vb, lb)] -> Y1[a][(lk, lb)][(d, vk, vb)]
        permute<T, T>(Qt, Y1, {chi, chi, D, D, D, D}, {0, 3, 5, 1, 2, 4}, st);
        // w[a,(lk,lb),b] = sum_{d,v} Y1[(a,l)][(d,v)] dn[(d,v)][b]
        gemm_rm<T>(chi * d2, chi, chi * d2, Y1, false, dn, false, w, st);
    };
    // Gram-Schmidt on the b columns with FP64 scalars, the projections applied
    // twice (one pass leaves the residual of a nearly dependent column with
    // components along the earlier ones of its own size).  The transfer matrix
    // may have fewer than b nonzero eigenvalues, so T V can be rank deficient:
    // a column whose residual falls below the rounding floor of its own norm
    // is what is left of a dependent column -- rounding correlated with the
    // earlier columns, which normalising would turn into one of them -- and is
    // replaced by a random vector, projected twice in turn.
    const double rel2 = sizeof(T) == 8 ? 1e-20 : 1e-8;
    uint64_t refills = 0;
    auto project = [&](T* X, int j) {
        T* xj = X + j * nt;
        for (int pass = 0; pass < 2; ++pass)
            for (int i = 0; i < j; ++i) {
                double* r = sc + 2 * b + i * b + j;
                KH_CUDA(cudaMemsetAsync(r, 0, sizeof(double), st));
                dot_acc_kernel<T><<<sumsq_grid(nt), 256, 0, st>>>(X + i * nt, xj, nt, r);
                KH_LAUNCHED();
                axpy_dev_kernel<T><<<grid, 256, 0, st>>>(X + i * nt, xj, nt, r, nullptr);
                KH_LAUNCHED();
            }
    };
    auto orthonormalise = [&](T* X) {
        KH_CUDA(cudaMemsetAsync(sc, 0, sizeof(double) * 2 * b, st));
        for (int j = 0; j < b; ++j) {
            T* xj = X + j * nt;
            dot_acc_kernel<T><<<sumsq_grid(nt), 256, 0, st>>>(xj, xj, nt, sc + b + j);
            KH_LAUNCHED();
            project(X, j);
            if (j > 0) {
                dot_acc_kernel<T><<<sumsq_grid(nt), 256, 0, st>>>(xj, xj, nt, sc + j);
                KH_LAUNCHED();
                refill_if_dependent_kernel<T><<<grid, 256, 0, st>>>(xj, nt, sc + j, sc + b + j, rel2, cfg.seed,
                                                                    0x5eedULL + (refills++));
                KH_LAUNCHED();
                project(X, j);
                KH_CUDA(cudaMemsetAsync(sc + j, 0, sizeof(double), st));
            }
            dot_acc_kernel<T><<<sumsq_grid(nt), 256, 0, st>>>(xj, xj, nt, sc + j);
            KH_LAUNCHED();
            scale_rsqrt_kernel<T><<<grid, 256, 0, st>>>(xj, nt, sc + j);
            KH_LAUNCHED();
        }
    };
    fill_random_kernel<T><<<grid, 256, 0, st>>>(V, b * nt, cfg.seed, 0x7e11ULL + (uint64_t)slot * 2 + dir);
    KH_LAUNCHED();
    orthonormalise(V);
    double ratio = 0.0, prev = -1.0, l1 = 0.0, l2 = 0.0;
    int it = 0;
    for (it = 1; it <= max_iter; ++it) {
        for (int j = 0; j < b; ++j) apply_T(V + j * nt, W + j * nt);
        if (it % 4 == 0 || it == max_iter) {
            // Ritz matrix H = V^T (T V), then V <- orth(T V)
            double* Hd_ = sc + 2 * b + b * b;
            KH_CUDA(cudaMemsetAsync(Hd_, 0, sizeof(double) * b * b, st));
            for (int i = 0; i < b; ++i)
                for (int j = 0; j < b; ++j) {
                    dot_acc_kernel<T><<<sumsq_grid(nt), 256, 0, st>>>(V + i * nt, W + j * nt, nt, Hd_ + i * b + j);
                    KH_LAUNCHED();
                }
            double H[16];
            KH_CUDA(cudaMemcpyAsync(H, Hd_, sizeof(double) * b * b, cudaMemcpyDeviceToHost, st));
            KH_CUDA(cudaStreamSynchronize(st));
            for (int i = 0; i < b * b; ++i)
                if (!(H[i] == H[i])) fail(KH_ENUMERIC, "NaN in the transfer-matrix iteration");
            auto ev = small_eigenvalues(H, b);
            std::vector<double> mag;
            for (auto& z : ev) mag.push_back(std::abs(z));
            std::sort(mag.begin(), mag.end(), [](double x, double y) { return x > y; });
            l1 = mag.size() > 0 ? mag[0] : 0.0;
            l2 = mag.size() > 1 ? mag[1] : 0.0;
            ratio = l1 > 0.0 ? l2 / l1 : 0.0;
            if (prev >= 0.0 && std::fabs(ratio - prev) <= tol * std::fmax(ratio, 1e-300)) {
                std::swap(V, W);
                break;
            }
            prev = ratio;
        }
        std::swap(V, W);
        orthonormalise(V);
    }
    out[0] = (ratio > 1e-14 && ratio < 1.0) ? -1.0 / std::log(ratio) : 0.0;
    out[1] = ratio;
    out[2] = std::min(it, max_iter);
}

template struct Engine<double>;
template struct Engine<float>;

}  // namespace kh
