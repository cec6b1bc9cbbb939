// Internal header of the eeFU GB300 library: context layout, workspace
// carving, error handling and the small generic kernels (permutation,
// strided batched GEMM on CUDA cores, reductions, casts).
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <atomic>
#include <cstdio>
#include <mutex>
#include <stdio.h>
#include <string.h>
#include <string>
#include <vector>

#include "../../include/eefu.h"

namespace kh {

// ------------------------------------------------------------------ errors

struct Error {
    kh_status st;
    std::string msg;
};

#define KH_CUDA(call)                                                                 \
    do {                                                                              \
        cudaError_t _e = (call);                                                      \
        if (_e != cudaSuccess) {                                                      \
            throw ::kh::Error{KH_ECUDA, std::string(#call) + ": " + cudaGetErrorString(_e) + " at " + \
                              __FILE__ + ":" + std::to_string(__LINE__)};                        \
        }                                                                             \
    } while (0)

#define KH_CHECK_LAUNCH() KH_CUDA(cudaGetLastError())
#define KH_LAUNCHED() do { KH_CUDA(cudaGetLastError()); ::kh::count_launch(); } while (0)

inline void fail(kh_status st, const std::string& m) { throw Error{st, m}; }

// number of kernels this library has launched (read by kh_launch_count);
// atomic because contexts may be driven from several host threads
extern std::atomic<unsigned long long> g_launches;
inline void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// ------------------------------------------------------------------ workspace

// Bump allocator over the caller's workspace; every block 256-byte aligned.
struct Carver {
    char* base;
    size_t cap, off;
    explicit Carver(void* b = nullptr, size_t c = 0) : base((char*)b), cap(c), off(0) {}
    template <typename T>
    T* take(size_t n) {
        size_t bytes = ((n * sizeof(T) + 255) / 256) * 256;
        size_t at = off;
        off += bytes;
        if (base == nullptr) return nullptr;          // sizing pass
        if (off > cap) fail(KH_ENOMEM, "workspace too small");
        return (T*)(base + at);
    }
};

// ------------------------------------------------------------------ permutation

constexpr int kMaxRank = 8;

// Division of 32-bit n < 2^31 by a divisor d fixed on the host: with
// l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1, q = (umulhi(n, m) + n) >> l
// (Granlund & Montgomery, "Division by invariant integers using multiplication").
struct FastDiv {
    uint32_t d, m, l;
};
inline FastDiv make_fastdiv(uint32_t d) {
    FastDiv f;
    f.d = d;
    uint32_t l = 0;
    while ((1ull << l) < d) ++l;
    f.l = l;
    f.m = (uint32_t)((((1ull << l) - d) << 32) / d + 1);
    return f;
}
__device__ __forceinline__ uint32_t fast_div(uint32_t n, const FastDiv& f) {
    return (__umulhi(n, f.m) + n) >> f.l;
}

struct PermArgs {
    int rank;
    long long total;
    long long out_dims[kMaxRank];   // output shape (row-major)
    long long in_strides[kMaxRank]; // input stride of each output axis
    FastDiv div[kMaxRank];          // output dims as fast divisors (32-bit path)
};

// out[i_0..i_{r-1}] = in[sum_j i_j * in_strides[j]]
template <typename Ti, typename To>
__global__ void permute_kernel(const Ti* __restrict__ in, To* __restrict__ out, PermArgs a) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long step = (long long)gridDim.x * blockDim.x;
    for (; idx < a.total; idx += step) {
        long long rem = idx, src = 0;
        for (int j = a.rank - 1; j >= 0; --j) {
            long long d = a.out_dims[j];
            long long i = rem % d;
            rem /= d;
            src += i * a.in_strides[j];
        }
        out[idx] = (To)in[src];
    }
}

// Same with 32-bit index arithmetic (total < 2^31): multiply-shift divisions.
template <typename Ti, typename To>
__global__ void permute32_kernel(const Ti* __restrict__ in, To* __restrict__ out, PermArgs a) {
    const uint32_t total = (uint32_t)a.total;
    const uint32_t step = gridDim.x * blockDim.x;
    for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += step) {
        uint32_t rem = idx, src = 0;
#pragma unroll
        for (int j = kMaxRank - 1; j >= 0; --j) {
            if (j < a.rank) {
                const uint32_t q = fast_div(rem, a.div[j]);
                src += (rem - q * a.div[j].d) * (uint32_t)a.in_strides[j];
                rem = q;
            }
        }
        out[idx] = (To)in[src];
    }
}

// Permutation fused with the 3xTF32 operand split: hi = the value with its 13
// low mantissa bits cleared (exactly TF32), lo = value - hi (32-bit path);
// the permuted value itself also goes to out when out is not null.
static __global__ void permute_split32_kernel(const float* __restrict__ in, float* __restrict__ hi,
                                              float* __restrict__ lo, float* __restrict__ out, PermArgs a) {
    const uint32_t total = (uint32_t)a.total;
    const uint32_t step = gridDim.x * blockDim.x;
    for (uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += step) {
        uint32_t rem = idx, src = 0;
#pragma unroll
        for (int j = kMaxRank - 1; j >= 0; --j) {
            if (j < a.rank) {
                const uint32_t q = fast_div(rem, a.div[j]);
                src += (rem - q * a.div[j].d) * (uint32_t)a.in_strides[j];
                rem = q;
            }
        }
        const float v = in[src];
        const float h = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
        hi[idx] = h;
        lo[idx] = v - h;
        if (out) out[idx] = v;
    }
}

// Build PermArgs from an input shape and the axis order of the output:
// out axis j is input axis order[j].
inline PermArgs make_perm(const std::vector<long long>& in_shape, const std::vector<int>& order) {
    PermArgs a;
    memset(&a, 0, sizeof(a));
    int r = (int)in_shape.size();
    if (r > kMaxRank || (int)order.size() != r) fail(KH_EINVAL, "permute rank");
    std::vector<long long> in_str(r);
    long long s = 1;
    for (int j = r - 1; j >= 0; --j) { in_str[j] = s; s *= in_shape[j]; }
    a.rank = r;
    a.total = s;
    for (int j = 0; j < r; ++j) {
        a.out_dims[j] = in_shape[order[j]];
        a.in_strides[j] = in_str[order[j]];
        if (a.out_dims[j] >= 1 && a.out_dims[j] < (1LL << 31)) a.div[j] = make_fastdiv((uint32_t)a.out_dims[j]);
    }
    return a;
}

// Let a kernel launch with `bytes` of dynamic shared memory on the current
// device: the 48 KB default covers static plus dynamic shared memory, so the
// opt-in is made when the kernel's static size plus `bytes` exceeds it; once
// per (kernel, device) and size, cache being the call site's table of the
// sizes already settled, indexed by device ordinal (the attribute is per
// device, so a context on a second GPU needs its own opt-in).  Contexts may
// live on several host threads: the settled size is read lock-free, and a
// raise is made under one lock, so the attribute only ever grows (a smaller
// request arriving second never lowers a larger grant another thread is
// about to launch with).
constexpr int kMaxDevices = 64;
inline std::mutex& smem_opt_in_mutex() {
    static std::mutex m;
    return m;
}
template <typename K>
inline void smem_opt_in(K kernel, size_t bytes, std::atomic<size_t> (&cache)[kMaxDevices]) {
    int dev = 0;
    KH_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) fail(KH_EINVAL, "device ordinal beyond 63");
    if (cache[dev].load(std::memory_order_acquire) >= bytes) return;
    std::lock_guard<std::mutex> lock(smem_opt_in_mutex());
    if (cache[dev].load(std::memory_order_relaxed) >= bytes) return;
    cudaFuncAttributes fa;
    KH_CUDA(cudaFuncGetAttributes(&fa, kernel));
    if (fa.sharedSizeBytes + bytes > 48 * 1024)
        KH_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    cache[dev].store(bytes, std::memory_order_release);
}

inline int grid_for(long long n, int block = 256) {
    long long g = (n + block - 1) / block;
    if (g > 152LL * 64) g = 152LL * 64;
    if (g < 1) g = 1;
    return (int)g;
}

inline void permute_split(const float* in, float* hi, float* lo, const std::vector<long long>& in_shape,
                          const std::vector<int>& order, cudaStream_t st, float* out = nullptr) {
    PermArgs a = make_perm(in_shape, order);
    if (a.total <= 0) return;
    if (a.total >= (1LL << 31)) fail(KH_EINVAL, "permute_split: tensor too large");
    permute_split32_kernel<<<grid_for(a.total), 256, 0, st>>>(in, hi, lo, out, a);
    KH_LAUNCHED();
}

template <typename Ti, typename To>
inline void permute(const Ti* in, To* out, const std::vector<long long>& in_shape,
                    const std::vector<int>& order, cudaStream_t st) {
    PermArgs a = make_perm(in_shape, order);
    if (a.total <= 0) return;
    if (a.total < (1LL << 31))
        permute32_kernel<Ti, To><<<grid_for(a.total), 256, 0, st>>>(in, out, a);
    else
        permute_kernel<Ti, To><<<grid_for(a.total), 256, 0, st>>>(in, out, a);
    KH_LAUNCHED();
}

template <typename Ti, typename To>
__global__ void cast_kernel(const Ti* __restrict__ in, To* __restrict__ out, long long n) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long step = (long long)gridDim.x * blockDim.x;
    for (; i < n; i += step) out[i] = (To)in[i];
}

template <typename Ti, typename To>
inline void cast(const Ti* in, To* out, long long n, cudaStream_t st) {
    cast_kernel<Ti, To><<<grid_for(n), 256, 0, st>>>(in, out, n);
    KH_LAUNCHED();
}

// ------------------------------------------------------------------ SIMT GEMM

// C[b](m,n) = alpha * colscale[n] * sum_k A[b](m,k) B[b](k,n) + beta * C[b](m,n)
// with arbitrary element strides.  CUDA-core FMA in T.
template <typename T>
struct GemmArgs {
    int M, N, K, batch;
    const T* A; long long sAm, sAk, sAb;
    const T* B; long long sBk, sBn, sBb;
    T* C; long long sCm, sCn, sCb;
    T alpha, beta;
    const T* colscale;   // nullable, length N
    T* sk = nullptr;     // optional split-K scratch (for few output tiles and long K)
    long long sk_elems = 0;
};

constexpr int GT_K = 16;

// Tile BM x BN per CTA, each of the 256 threads computes TM x TN outputs
// strided by (BM/TM, BN/TN) so that shared-memory reads are conflict-free.
template <typename T, int BM, int BN, int TM, int TN>
__global__ void __launch_bounds__(256) gemm_simt_kernel(GemmArgs<T> g) {
    static_assert((BM / TM) * (BN / TN) == 256, "256 threads");
    constexpr int RX = BN / TN;                    // threads along N
    __shared__ T As[GT_K][BM + 1];
    __shared__ T Bs[GT_K][BN + 1];
    const int tid = threadIdx.x;
    const int tx = tid % RX, ty = tid / RX;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const long long b = blockIdx.z;
    const T* A = g.A + b * g.sAb;
    const T* B = g.B + b * g.sBb;
    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
    const bool a_kfast = (g.sAk == 1);
    const bool b_nfast = (g.sBn == 1);
    // register double buffering: the next K tile's global loads are issued
    // before the current tile's FMAs
    constexpr int NA = BM * GT_K / 256, NB = BN * GT_K / 256;
    static_assert(NA * 256 == BM * GT_K && NB * 256 == BN * GT_K, "tile/thread mismatch");
    T ra[NA], rb[NB];
    auto load_tiles = [&](int k0) {
#pragma unroll
        for (int t = 0; t < NA; ++t) {
            const int e = tid + 256 * t;
            int mm, kk;
            if (a_kfast) { mm = e / GT_K; kk = e % GT_K; } else { mm = e % BM; kk = e / BM; }
            const int gm = m0 + mm, gk = k0 + kk;
            ra[t] = (gm < g.M && gk < g.K) ? A[gm * g.sAm + gk * g.sAk] : T(0);
        }
#pragma unroll
        for (int t = 0; t < NB; ++t) {
            const int e = tid + 256 * t;
            int nn, kb;
            if (b_nfast) { nn = e % BN; kb = e / BN; } else { nn = e / GT_K; kb = e % GT_K; }
            const int gn = n0 + nn, gkb = k0 + kb;
            rb[t] = (gn < g.N && gkb < g.K) ? B[gkb * g.sBk + gn * g.sBn] : T(0);
        }
    };
    load_tiles(0);
    for (int k0 = 0; k0 < g.K; k0 += GT_K) {
#pragma unroll
        for (int t = 0; t < NA; ++t) {
            const int e = tid + 256 * t;
            int mm, kk;
            if (a_kfast) { mm = e / GT_K; kk = e % GT_K; } else { mm = e % BM; kk = e / BM; }
            As[kk][mm] = ra[t];
        }
#pragma unroll
        for (int t = 0; t < NB; ++t) {
            const int e = tid + 256 * t;
            int nn, kb;
            if (b_nfast) { nn = e % BN; kb = e / BN; } else { nn = e / GT_K; kb = e % GT_K; }
            Bs[kb][nn] = rb[t];
        }
        __syncthreads();
        if (k0 + GT_K < g.K) load_tiles(k0 + GT_K);
#pragma unroll
        for (int kk = 0; kk < GT_K; ++kk) {
            T a[TM], bb[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + (BM / TM) * i];
#pragma unroll
            for (int j = 0; j < TN; ++j) bb[j] = Bs[kk][tx + RX * j];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
        }
        __syncthreads();
    }
    T* C = g.C + b * g.sCb;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        int gm = m0 + ty + (BM / TM) * i;
        if (gm >= g.M) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            int gn = n0 + tx + RX * j;
            if (gn >= g.N) continue;
            T v = g.alpha * acc[i][j];
            if (g.colscale) v *= g.colscale[gn];
            T* dst = C + gm * g.sCm + gn * g.sCn;
            if (g.beta != T(0)) v += g.beta * (*dst);
            *dst = v;
        }
    }
}

template <typename T, int BM, int BN, int TM, int TN>
inline void gemm_launch(const GemmArgs<T>& g, cudaStream_t st) {
    dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, g.batch);
    if (grid.y > 65535) fail(KH_EINVAL, "gemm M too large");
    gemm_simt_kernel<T, BM, BN, TM, TN><<<grid, 256, 0, st>>>(g);
    KH_LAUNCHED();
}

// out[i] = alpha * colscale[col] * sum_s part[s][i] + beta * out   (split-K reduction)
template <typename T>
__global__ void splitk_reduce_kernel(const T* __restrict__ part, int splits, int M, int N, T* C, long long sCm,
                                     long long sCn, T alpha, T beta, const T* colscale) {
    long long tot = (long long)M * N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
         i += (long long)gridDim.x * blockDim.x) {
        T acc = T(0);
        for (int s = 0; s < splits; ++s) acc += part[s * tot + i];
        int m = (int)(i / N), n = (int)(i % N);
        T v = alpha * acc;
        if (colscale) v *= colscale[n];
        T* dst = C + m * sCm + n * sCn;
        if (beta != T(0)) v += beta * (*dst);
        *dst = v;
    }
}

template <typename T>
inline void gemm_dispatch(const GemmArgs<T>& g, cudaStream_t st) {
    const long long tiles64 = (long long)((g.M + 63) / 64) * ((g.N + 63) / 64) * g.batch;
    if (g.M <= 16 && g.N <= 16) gemm_launch<T, 16, 16, 1, 1>(g, st);
    else if (g.N <= 16) gemm_launch<T, 128, 16, 2, 4>(g, st);
    else if (g.M <= 16) gemm_launch<T, 16, 128, 4, 2>(g, st);
    else if (g.N <= 128 && tiles64 < 76) gemm_launch<T, 16, 128, 4, 2>(g, st);   // few 64x64 tiles: more, thinner CTAs
    else gemm_launch<T, 64, 64, 4, 4>(g, st);
}

template <typename T>
inline void gemm(const GemmArgs<T>& g, cudaStream_t st) {
    if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return;
    if (g.batch > 65535) fail(KH_EINVAL, "gemm batch > 65535");
    // few output tiles and a long K: split K over CTAs into the scratch,
    // then reduce in a fixed order (deterministic)
    const long long tiles = (long long)((g.M + 63) / 64) * ((g.N + 63) / 64);
    if (g.batch == 1 && g.sk && tiles < 76 && g.K >= 256) {
        int splits = (int)((304 + tiles - 1) / tiles);   // about two CTAs per SM
        int maxs = g.K / 128;
        if (splits > maxs) splits = maxs;
        if (splits > 32) splits = 32;
        const long long mn = (long long)g.M * g.N;
        if (splits >= 2 && splits * mn <= g.sk_elems) {
            const int kchunk = ((g.K + splits - 1) / splits + GT_K - 1) / GT_K * GT_K;
            splits = (g.K + kchunk - 1) / kchunk;
            GemmArgs<T> p = g;
            p.K = kchunk;
            p.batch = splits;
            p.sAb = kchunk * g.sAk;            // batch b = K range [b*kchunk, ...)
            p.sBb = kchunk * g.sBk;
            p.C = g.sk; p.sCm = g.N; p.sCn = 1; p.sCb = mn;
            p.alpha = T(1); p.beta = T(0); p.colscale = nullptr; p.sk = nullptr;
            // the last chunk may overrun K: handled by a separate launch with the remainder
            const int last = g.K - (splits - 1) * kchunk;
            if (last == kchunk) {
                gemm_dispatch<T>(p, st);
            } else {
                p.batch = splits - 1;
                gemm_dispatch<T>(p, st);
                GemmArgs<T> r = p;
                r.batch = 1; r.K = last;
                r.A = g.A + (long long)(splits - 1) * kchunk * g.sAk;
                r.B = g.B + (long long)(splits - 1) * kchunk * g.sBk;
                r.C = g.sk + (long long)(splits - 1) * mn;
                gemm_dispatch<T>(r, st);
            }
            splitk_reduce_kernel<T><<<grid_for(mn), 256, 0, st>>>(g.sk, splits, g.M, g.N, g.C, g.sCm, g.sCn, g.alpha,
                                                                  g.beta, g.colscale);
            KH_LAUNCHED();
            return;
        }
    }
    gemm_dispatch<T>(g, st);
}

// Plain row-major C(MxN) = A(MxK) B(KxN) [+beta C]; transposes by flags.
template <typename T>
inline void gemm_rm(int M, int N, int K, const T* A, bool tA, const T* B, bool tB, T* C,
                    cudaStream_t st, T alpha = T(1), T beta = T(0), const T* colscale = nullptr,
                    T* sk = nullptr, long long sk_elems = 0) {
    GemmArgs<T> g;
    g.sk = sk;
    g.sk_elems = sk_elems;
    g.M = M; g.N = N; g.K = K; g.batch = 1;
    g.A = A; g.sAm = tA ? 1 : K; g.sAk = tA ? M : 1; g.sAb = 0;
    g.B = B; g.sBk = tB ? 1 : N; g.sBn = tB ? K : 1; g.sBb = 0;
    g.C = C; g.sCm = N; g.sCn = 1; g.sCb = 0;
    g.alpha = alpha; g.beta = beta; g.colscale = colscale;
    gemm(g, st);
}

// ------------------------------------------------------------------ reductions

// out[0] = sum x^2 (FP64 accumulate), one atomic per block; launch it on a
// grid of a few blocks per SM (sumsq_grid): one atomic per element block
// would serialise thousands of FP64 atomics on one address
template <typename T>
__global__ void sumsq_kernel(const T* __restrict__ x, long long n, double* out) {
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        double v = (double)x[i];
        s += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double red[32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = s;
    __syncthreads();
    if (w == 0) {
        s = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) atomicAdd(out, s);
    }
}

// FP64 reciprocal, reciprocal square root and square root by Newton-Raphson
// iteration from the FP32 hardware estimates: each step squares the relative
// error (reciprocal: y <- y + y (1 - x y); reciprocal square root:
// y <- y (3/2 - (x/2) y^2)), so two steps take the ~2^-23 estimate below FP64
// rounding (a few ulp).  FP64 division and square root issue as long
// dependent sequences on GB300's narrow FP64 pipe; these take four or five
// FP64 FMAs.  Arguments outside the FP32 normal range use the IEEE operation.
__device__ __forceinline__ double rcp_nr(double x) {
    const float ax = fabsf((float)x);
    if (!(ax > 1e-30f && ax < 1e30f)) return 1.0 / x;
    double y = (double)__frcp_rn((float)x);
    double e = fma(-x, y, 1.0);
    y = fma(y, e, y);
    e = fma(-x, y, 1.0);
    return fma(y, e, y);
}
__device__ __forceinline__ double rsqrt_nr(double x) {      // x > 0
    const float xf = (float)x;
    if (!(xf > 1e-30f && xf < 1e30f)) return 1.0 / sqrt(x);
    double y = (double)rsqrtf(xf);
    const double h = 0.5 * x;
    y = y * fma(-h * y, y, 1.5);
    return y * fma(-h * y, y, 1.5);
}
__device__ __forceinline__ double sqrt_nr(double x) {       // x >= 0
    const float xf = (float)x;
    if (!(xf > 1e-30f && xf < 1e30f)) return sqrt(x);
    const double r = rsqrt_nr(x);
    const double s = x * r;
    return fma(fma(-s, s, x), 0.5 * r, s);                   // s + (x - s^2) / (2 sqrt x)
}

inline int sumsq_grid(long long n) {
    long long g = (n + 255) / 256;
    return (int)(g < 304 ? (g < 1 ? 1 : g) : 304);
}

}  // namespace kh
