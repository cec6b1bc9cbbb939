// Kernel self-test entry points (test hooks; the paper has no counterpart):
// run one library kernel on caller-provided device data so that tests can
// pin it directly against a host reference.
#include "engine.cuh"
#include "layered.cuh"

namespace {

template <typename T>
void run_gemm(int M, int N, int K, const double* A, const double* B, double* C, void* scratch, size_t bytes,
              cudaStream_t st) {
    kh::Carver cv(scratch, bytes);
    T* a = cv.take<T>((size_t)M * K);
    T* b = cv.take<T>((size_t)K * N);
    T* c = cv.take<T>((size_t)M * N);
    const long long skn = 8LL * M * N;                 // split-K scratch (up to 8 partial products)
    T* sk = (cv.off + skn * sizeof(T) + 256 <= bytes) ? cv.take<T>((size_t)skn) : nullptr;
    kh::cast<double, T>(A, a, (long long)M * K, st);
    kh::cast<double, T>(B, b, (long long)K * N, st);
    kh::gemm_rm<T>(M, N, K, a, false, b, false, c, st, T(1), T(0), nullptr, sk, sk ? skn : 0);
    kh::cast<T, double>(c, C, (long long)M * N, st);
}

// tensor-core path: B^T made K-major by a permutation, optional hi/lo split
void run_tc_gemm(int npass, int M, int N, int K, const double* A, const double* B, double* C, void* scratch,
                 size_t bytes, cudaStream_t st) {
    kh::Carver cv(scratch, bytes);
    float* a = cv.take<float>((size_t)M * K);
    float* bt = cv.take<float>((size_t)K * N);
    float* c = cv.take<float>((size_t)M * N);
    float* ah = cv.take<float>((size_t)M * K);
    float* al = cv.take<float>((size_t)M * K);
    float* bh = cv.take<float>((size_t)K * N);
    float* bl = cv.take<float>((size_t)K * N);
    int* err = cv.take<int>(64);
    KH_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    kh::cast<double, float>(A, a, (long long)M * K, st);
    kh::permute<double, float>(B, bt, {K, N}, {1, 0}, st);
    kh::TcOperand oa{a, nullptr, K}, ob{bt, nullptr, K};
    if (npass == 3) {
        kh::tc_split(a, ah, al, (long long)M * K, st);
        kh::tc_split(bt, bh, bl, (long long)K * N, st);
        oa = kh::TcOperand{ah, al, K};
        ob = kh::TcOperand{bh, bl, K};
    }
    kh::tc_gemm(oa, ob, c, M, N, K, N, 1.f, 0.f, nullptr, npass, err, st);
    kh::cast<float, double>(c, C, (long long)M * N, st);
    int h = 0;
    KH_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    KH_CUDA(cudaStreamSynchronize(st));
    if (h) kh::fail(KH_ETIMEOUT, "tensor-core GEMM wait timed out");
}

template <typename T>
void run_eig(int k, const double* G, double* W, double* E, void* scratch, size_t bytes, cudaStream_t st) {
    kh::Carver cv(scratch, bytes);
    T* g = cv.take<T>((size_t)k * k);
    T* w = cv.take<T>((size_t)k * k);
    T* e = cv.take<T>((size_t)k);
    kh::cast<double, T>(G, g, (long long)k * k, st);
    kh::jacobi_eig<T>(g, k, k, 0, w, k, 0, e, 0, 1, 60, sizeof(T) == 8 ? 1e-14 : 2e-6, nullptr, nullptr, st);
    kh::cast<T, double>(w, W, (long long)k * k, st);
    kh::cast<T, double>(e, E, (long long)k, st);
}

template <typename T>
void run_svd(int k, const double* X, double* S, double* L, double* Qm, void* scratch, size_t bytes, cudaStream_t st) {
    kh::Carver cv(scratch, bytes);
    T* x = cv.take<T>((size_t)k * k);
    T* l = cv.take<T>((size_t)k * k);
    T* q = cv.take<T>((size_t)k * k);
    T* sv = cv.take<T>((size_t)k);
    kh::cast<double, T>(X, x, (long long)k * k, st);
    kh::svd_jacobi<T>(x, k, sv, l, q, 60, sizeof(T) == 8 ? 1e-15 : 1e-6, 0.0, st);
    kh::cast<T, double>(sv, S, (long long)k, st);
    kh::cast<T, double>(l, L, (long long)k * k, st);
    kh::cast<T, double>(q, Qm, (long long)k * k, st);
}

template <typename T>
void run_orth(int n, int k, double cut, const double* Y, double* Q, void* scratch, size_t bytes, cudaStream_t st) {
    kh::Carver cv(scratch, bytes);
    T* y = cv.take<T>((size_t)n * k);
    T* tmp = cv.take<T>((size_t)n * k);
    T* u = cv.take<T>((size_t)n * k);
    T* xk = cv.take<T>((size_t)k * k);
    double* dg = cv.take<double>((size_t)k * k);
    kh::cast<double, T>(Y, y, (long long)n * k, st);
    kh::cholqr2<T>(y, n, k, cut, tmp, xk, dg, u, st);
    kh::cast<T, double>(u, Q, (long long)n * k, st);
}

// Layered tensor-core site contraction of one (kind, frame): operand images
// from the FP64 site tensor, Y cast to FP32, out cast back to FP64.
struct LayeredScratch {
    float *img1, *img2, *y, *out;
    int* err;
    long long per1, per2;
};

// npass: 1 = TF32, 3 = 3xTF32, 16 = BF16 (one pass)
LayeredScratch carve_layered(kh::Carver& cv, int npass, int D, int p, long long nb) {
    LayeredScratch L;
    const bool bf = npass == 16;
    const int np = bf ? 1 : npass;
    L.per1 = kh::layered_img1_floats(D, p, np, bf);
    L.per2 = kh::layered_img2_floats(D, p, np, bf);
    const long long d4 = (long long)D * D * D * D;
    L.img1 = cv.take<float>((size_t)(8 * L.per1));
    L.img2 = cv.take<float>((size_t)(8 * L.per2));
    L.y = cv.take<float>((size_t)(nb * d4));
    L.out = cv.take<float>((size_t)(nb * d4));
    L.err = cv.take<int>(64);
    return L;
}

void run_site_layered(int npass, int D, int p, int kind, int frame, long long nb, const double* T, const double* Y,
                      double* out, void* scratch, size_t bytes, cudaStream_t st) {
    kh::Carver cv(scratch, bytes);
    LayeredScratch L = carve_layered(cv, npass, D, p, nb);
    const long long d4 = (long long)D * D * D * D;
    KH_CUDA(cudaMemsetAsync(L.err, 0, sizeof(int), st));
    const bool bf = npass == 16;
    const int np = bf ? 1 : npass;
    kh::build_layered_images(T, p, D, np, bf, L.img1, L.img2, L.per1, L.per2, st);
    kh::cast<double, float>(Y, L.y, nb * d4, st);
    const int kf = kind * 4 + frame;
    kh::site_layered_tc(L.y, nb, D, p, L.img1 + kf * L.per1, L.img2 + kf * L.per2, L.out, np, bf, L.err, st);
    kh::cast<float, double>(L.out, out, nb * d4, st);
    int h = 0;
    KH_CUDA(cudaMemcpyAsync(&h, L.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    KH_CUDA(cudaStreamSynchronize(st));
    if (h) kh::fail(KH_ETIMEOUT, "layered site contraction wait timed out");
}

// FP32 one-sided Jacobi, then one FP64 Newton refinement step (the projector
// SVD of the FP64-projector option).
void run_svd_refined(int k, const double* X, double* S, double* L, double* Qm, void* scratch, size_t bytes,
                     cudaStream_t st) {
    kh::Carver cv(scratch, bytes);
    float* x = cv.take<float>((size_t)k * k);
    float* l = cv.take<float>((size_t)k * k);
    float* q = cv.take<float>((size_t)k * k);
    float* sv = cv.take<float>((size_t)k);
    double* ld = cv.take<double>((size_t)k * k);
    double* qd = cv.take<double>((size_t)k * k);
    double* work = cv.take<double>(kh::svd_refine_scratch(k));
    kh::cast<double, float>(X, x, (long long)k * k, st);
    kh::svd_jacobi<float>(x, k, sv, l, q, 60, 1e-6, 0.0, st);
    kh::cast<float, double>(l, ld, (long long)k * k, st);
    kh::cast<float, double>(q, qd, (long long)k * k, st);
    kh::svd_refine_fp64(X, k, ld, qd, S, L, Qm, work, 1e-5, st);
}

__global__ void newton_kernel(const double* __restrict__ x, int n, double* __restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        out[3 * i] = kh::rcp_nr(x[i]);
        out[3 * i + 1] = x[i] > 0.0 ? kh::rsqrt_nr(x[i]) : 0.0;
        out[3 * i + 2] = x[i] >= 0.0 ? kh::sqrt_nr(x[i]) : 0.0;
    }
}

template <typename F>
kh_status run(F&& f) {
    try {
        f();
        return KH_OK;
    } catch (const kh::Error& e) {
        fprintf(stderr, "eefu selftest: %s\n", e.msg.c_str());
        return e.st;
    }
}

}  // namespace

namespace kh {
// The self-test GEMM body on a given scratch buffer (shared with noalloc.cu).
kh_status selftest_gemm_on(int prec, int M, int N, int K, const double* A, const double* B, double* C,
                           void* scratch, size_t bytes, cudaStream_t st) {
    return run([&] {
        if (prec == KH_FP64) run_gemm<double>(M, N, K, A, B, C, scratch, bytes, st);
        else if (prec == KH_FP32) run_gemm<float>(M, N, K, A, B, C, scratch, bytes, st);
        else if (prec == KH_TF32) run_tc_gemm(1, M, N, K, A, B, C, scratch, bytes, st);
        else if (prec == KH_TF32X3) run_tc_gemm(3, M, N, K, A, B, C, scratch, bytes, st);
        else kh::fail(KH_EINVAL, "precision not built");
        KH_CUDA(cudaStreamSynchronize(st));
    });
}
}  // namespace kh

extern "C" {

size_t kh_selftest_bytes(int M, int N, int K) {
    return 8 * ((size_t)M * K + (size_t)K * N + (size_t)M * N) * 3 + 8 * 8 * (size_t)M * N + 8192;
}

kh_status kh_selftest_gemm(int prec, int M, int N, int K, const double* A, const double* B, double* C,
                           void* scratch, size_t bytes, void* stream) {
    if (M < 1 || N < 1 || K < 1 || !A || !B || !C || !scratch) return KH_EINVAL;
    if (bytes < kh_selftest_bytes(M, N, K)) return KH_ENOMEM;
    cudaStream_t st = (cudaStream_t)stream;
    return run([&] {
        if (prec == KH_FP64) run_gemm<double>(M, N, K, A, B, C, scratch, bytes, st);
        else if (prec == KH_FP32) run_gemm<float>(M, N, K, A, B, C, scratch, bytes, st);
        else if (prec == KH_TF32) run_tc_gemm(1, M, N, K, A, B, C, scratch, bytes, st);
        else if (prec == KH_TF32X3) run_tc_gemm(3, M, N, K, A, B, C, scratch, bytes, st);
        else kh::fail(KH_EINVAL, "precision not built");
        KH_CUDA(cudaStreamSynchronize(st));
    });
}

kh_status kh_selftest_symeig(int prec, int k, const double* G, double* W, double* E, void* scratch, size_t bytes,
                             void* stream) {
    if (k < 1 || !G || !W || !E || !scratch) return KH_EINVAL;
    if (bytes < kh_selftest_bytes(k, k, k)) return KH_ENOMEM;
    cudaStream_t st = (cudaStream_t)stream;
    return run([&] {
        if (prec == KH_FP64) run_eig<double>(k, G, W, E, scratch, bytes, st);
        else run_eig<float>(k, G, W, E, scratch, bytes, st);
        KH_CUDA(cudaStreamSynchronize(st));
    });
}

kh_status kh_selftest_svd(int prec, int k, const double* X, double* S, double* L, double* Qm, void* scratch,
                          size_t bytes, void* stream) {
    if (k < 1 || !X || !S || !L || !Qm || !scratch) return KH_EINVAL;
    if (bytes < kh_selftest_bytes(k, k, k)) return KH_ENOMEM;
    cudaStream_t st = (cudaStream_t)stream;
    return run([&] {
        if (prec == KH_FP64) run_svd<double>(k, X, S, L, Qm, scratch, bytes, st);
        else run_svd<float>(k, X, S, L, Qm, scratch, bytes, st);
        KH_CUDA(cudaStreamSynchronize(st));
    });
}

kh_status kh_selftest_svd_refined(int k, const double* X, double* S, double* L, double* Qm, void* scratch,
                                  size_t bytes, void* stream) {
    if (k < 1 || k > 160 || !X || !S || !L || !Qm || !scratch) return KH_EINVAL;
    if (bytes < kh_selftest_bytes(k, k, k)) return KH_ENOMEM;
    cudaStream_t st = (cudaStream_t)stream;
    return run([&] {
        run_svd_refined(k, X, S, L, Qm, scratch, bytes, st);
        KH_CUDA(cudaStreamSynchronize(st));
    });
}

size_t kh_selftest_site_layered_bytes(int npass, int D, int p, long long nb) {
    if ((npass != 1 && npass != 3 && npass != 16) || D < 1 || D > 8 || p < 1 || p > 16 || nb < 0) return 0;
    kh::Carver cv;
    carve_layered(cv, npass, D, p, nb);
    return cv.off;
}

kh_status kh_selftest_site_layered(int npass, int D, int p, int kind, int frame, long long nb, const double* T,
                                   const double* Y, double* out, void* scratch, size_t bytes, void* stream) {
    if ((npass != 1 && npass != 3 && npass != 16) || D < 1 || D > 8 || p < 1 || p > 16 || kind < 0 || kind > 1 ||
        frame < 0 ||
        frame > 3 || nb < 1 || !T || !Y || !out || !scratch)
        return KH_EINVAL;
    if (bytes < kh_selftest_site_layered_bytes(npass, D, p, nb)) return KH_ENOMEM;
    cudaStream_t st = (cudaStream_t)stream;
    return run([&] { run_site_layered(npass, D, p, kind, frame, nb, T, Y, out, scratch, bytes, st); });
}

kh_status kh_selftest_fp64_newton(int n, const double* x, double* out, void* stream) {
    if (n < 1 || !x || !out) return KH_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    return run([&] {
        newton_kernel<<<kh::grid_for(n), 256, 0, st>>>(x, n, out);
        KH_LAUNCHED();
        KH_CUDA(cudaStreamSynchronize(st));
    });
}

kh_status kh_selftest_orth(int prec, int n, int k, double cut, const double* Y, double* Qm, void* scratch,
                           size_t bytes, void* stream) {
    if (n < 1 || k < 1 || !Y || !Qm || !scratch || !(cut >= 0.0)) return KH_EINVAL;
    if (k > (prec == KH_FP64 ? 112 : 160)) return KH_EINVAL;
    if (bytes < kh_selftest_bytes(n, k, k)) return KH_ENOMEM;
    cudaStream_t st = (cudaStream_t)stream;
    return run([&] {
        if (prec == KH_FP64) run_orth<double>(n, k, cut, Y, Qm, scratch, bytes, st);
        else run_orth<float>(n, k, cut, Y, Qm, scratch, bytes, st);
        KH_CUDA(cudaStreamSynchronize(st));
    });
}

}  // extern "C"
