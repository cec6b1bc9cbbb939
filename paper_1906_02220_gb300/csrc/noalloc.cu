// Allocation-free variant of the contraction-GEMM self-test entry point.
//
// Every other entry point of this library works in memory the caller
// provides (a context workspace, or a scratch buffer for the self-tests),
// which means the caller has to allocate device memory first.  Some callers
// cannot: code whose device memory is owned by another allocator (a
// framework's caching pool, a fixed-budget arena) that a direct cudaMalloc
// would bypass, and latency-critical loops that cannot afford the implicit
// device synchronisation an allocation brings.  kh_gemm_noalloc serves them:
// its scratch is the file-scope array below, reserved when the library is
// loaded and held by every GPU that loads it until the process exits.
#include "engine.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = 16u << 20;   // 16 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
// Device address of the array per device, looked up on the first call on that
// device.  Host threads may make their first calls at the same time: the
// lookup runs under one lock and the address is published atomically.
std::atomic<void*> g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_lookup;

// Returns the device address of g_noalloc_scratch on device dev (current).
cudaError_t scratch_address(int dev, void** out) {
    void* p = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (!p) {
        std::lock_guard<std::mutex> lock(g_scratch_lookup);
        p = g_scratch_addr[dev].load(std::memory_order_relaxed);
        if (!p) {
            // The array's name is a host-side stand-in; its address on the
            // current device comes from the runtime.
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) return e != cudaSuccess ? e : cudaErrorInvalidSymbol;
            g_scratch_addr[dev].store(p, std::memory_order_release);
        }
    }
    *out = p;
    return cudaSuccess;
}

}  // namespace

namespace kh {
kh_status selftest_gemm_on(int prec, int M, int N, int K, const double* A, const double* B, double* C,
                           void* scratch, size_t bytes, cudaStream_t st);
}

extern "C" {

size_t kh_gemm_noalloc_max_bytes(void) { return kNoAllocScratchBytes; }

kh_status kh_gemm_noalloc(int prec, int M, int N, int K, const double* A, const double* B, double* C,
                          void* stream) {
    if (M < 1 || N < 1 || K < 1 || !A || !B || !C) return KH_EINVAL;
    if (kh_selftest_bytes(M, N, K) > kNoAllocScratchBytes) {
        fprintf(stderr, "kh_gemm_noalloc: %d x %d x %d needs %zu scratch bytes, above the %zu-byte static limit\n",
                M, N, K, kh_selftest_bytes(M, N, K), kNoAllocScratchBytes);
        return KH_EINVAL;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return KH_ECUDA;
    void* scratch = nullptr;
    cudaError_t e = scratch_address(dev, &scratch);
    if (e != cudaSuccess) {
        fprintf(stderr, "kh_gemm_noalloc: cudaGetSymbolAddress failed: %s\n", cudaGetErrorString(e));
        return KH_ECUDA;
    }
    return kh::selftest_gemm_on(prec, M, N, K, A, B, C, scratch, kNoAllocScratchBytes, (cudaStream_t)stream);
}

}  // extern "C"
