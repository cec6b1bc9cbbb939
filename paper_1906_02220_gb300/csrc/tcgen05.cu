// Tensor-core GEMM for sm_103a (5th-generation tensor cores):
//   C[m][n] = alpha * colscale[n] * sum_k A[m][k] B[n][k] + beta * C[m][n]
// A (M x K) and B (N x K) row-major ("K-major"), FP32 storage read as TF32;
// C FP32 row-major.  NPASS = 3 runs the error-compensated split
// A = A_hi + A_lo, B = B_hi + B_lo (hi = the TF32-representable part) as
// A_hi B_hi + A_hi B_lo + A_lo B_hi, which restores FP32-level accuracy.
//
// One 128 x BN output tile per CTA, 6 warps:
//   warp 0     TMA producer: 128B-swizzled K-major tiles into a STAGES-deep
//              ring of shared-memory buffers (mbarrier full/empty pairs);
//   warp 1     allocates the TMEM accumulator; one elected lane issues
//              tcgen05.mma (M=128, N=BN, K=8 per instruction) and commits
//              to the empty barriers;
//   warps 2-5  epilogue: tcgen05.ld of their TMEM lane quadrant, scaling,
//              predicated stores.
// Every mbarrier wait is bounded; on time-out the kernel raises an error
// flag, lets the other roles drain, frees TMEM and returns.
#include "engine.cuh"
#include "tc_ptx.cuh"

namespace kh {

namespace tc {

constexpr int BM = 128;
constexpr int BK = 32;               // 32 FP32 = one 128-byte swizzle row
constexpr int THREADS = 192;


template <int BN, int NPASS>
struct Cfg {
    static constexpr int A_BYTES = BM * BK * 4;
    static constexpr int B_BYTES = BN * BK * 4;
    static constexpr int STAGE_BYTES = (NPASS == 3 ? 2 : 1) * (A_BYTES + B_BYTES);
    static constexpr int STAGES = (NPASS == 3 ? 3 : 4);
    static constexpr int SMEM = STAGES * STAGE_BYTES + 1024;
    // consecutive MMAs into one accumulator form a dependent chain whose
    // latency exceeds a narrow tile's MMA time: narrow tiles spread their
    // MMAs round-robin over NACC accumulators (32-column aligned), summed in
    // the epilogue
    static constexpr int NACC = BN <= 32 ? 4 : (BN <= 64 ? 2 : 1);
    static constexpr int ACC_COLS = BN < 32 ? 32 : BN;
    static constexpr int TMEM_COLS = NACC * ACC_COLS;
    static constexpr uint32_t IDESC = (1u << 4)                     // D: FP32
                                      | (2u << 7) | (2u << 10)      // A, B: TF32
                                      | ((uint32_t)(BN >> 3) << 17) // N / 8
                                      | ((uint32_t)(BM >> 4) << 24);// M / 16
};

template <int BN, int NPASS>
__global__ void __launch_bounds__(THREADS, 1)
gemm_kernel(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB,
            const __grid_constant__ CUtensorMap mA2, const __grid_constant__ CUtensorMap mB2, float* __restrict__ C,
            int M, int N, int K, long long ldc, float alpha, float beta, const float* __restrict__ colscale,
            int* err) {
    using G = Cfg<BN, NPASS>;
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[G::STAGES], empty_bar[G::STAGES], acc_bar;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int KT = (K + BK - 1) / BK;
    uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);

    if (threadIdx.x == 0) {
        for (int s = 0; s < G::STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&acc_bar, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"((uint32_t)G::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = s_tmem;
    volatile int* abort_flag = &s_abort;

    if (warp == 0) {
        if (lane == 0) {
            for (int kt = 0; kt < KT; ++kt) {
                const int s = kt % G::STAGES;
                const uint32_t ph = (kt / G::STAGES) & 1;
                if (!mbar_wait(&empty_bar[s], ph ^ 1, abort_flag)) { s_abort = 1; atomicOr(err, 1); break; }
                uint8_t* st = base + s * G::STAGE_BYTES;
                mbar_expect_tx(&full_bar[s], G::STAGE_BYTES);
                tma_load_2d(st, &mA, &full_bar[s], kt * BK, m0);
                tma_load_2d(st + G::A_BYTES, &mB, &full_bar[s], kt * BK, n0);
                if (NPASS == 3) {
                    tma_load_2d(st + G::A_BYTES + G::B_BYTES, &mA2, &full_bar[s], kt * BK, m0);
                    tma_load_2d(st + 2 * G::A_BYTES + G::B_BYTES, &mB2, &full_bar[s], kt * BK, n0);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            bool ok = true;
            for (int kt = 0; kt < KT; ++kt) {
                const int s = kt % G::STAGES;
                const uint32_t ph = (kt / G::STAGES) & 1;
                if (!mbar_wait(&full_bar[s], ph, abort_flag)) { s_abort = 1; atomicOr(err, 2); ok = false; break; }
                fence_after();
                const uint32_t a0 = smem_u32(base + s * G::STAGE_BYTES);
                const uint32_t b0 = a0 + G::A_BYTES;
                const uint32_t a1 = b0 + G::B_BYTES;           // A_lo
                const uint32_t b1 = a1 + G::A_BYTES;           // B_lo
#pragma unroll
                for (int kk = 0; kk < BK / 8; ++kk) {
                    const uint32_t off = kk * 32;               // 8 TF32 = 32 bytes along K
                    const uint64_t da = smem_desc(a0 + off), db = smem_desc(b0 + off);
                    // accumulator of this k-step; its first use (first k-steps of the tile) overwrites
                    const int i = kt * (BK / 8) + kk;
                    const uint32_t d = tmem + (uint32_t)((i % G::NACC) * G::ACC_COLS);
                    umma_tf32(d, da, db, G::IDESC, i >= G::NACC ? 1u : 0u);
                    if (NPASS == 3) {
                        umma_tf32(d, da, smem_desc(b1 + off), G::IDESC, 1u);
                        umma_tf32(d, smem_desc(a1 + off), db, G::IDESC, 1u);
                    }
                }
                umma_commit(&empty_bar[s]);
            }
            (void)ok;
            umma_commit(&acc_bar);   // also after an abort: lets the epilogue wait for MMAs in flight
        }
    } else {
        // epilogue: warp w reads TMEM lanes [32 (w % 4), +32)
        const int q = warp & 3;
        const int row = m0 + 32 * q + lane;
        if (mbar_wait(&acc_bar, 0, abort_flag) && !*abort_flag) {
            fence_after();
            // accumulators a written by the first min(NACC, K steps) k-steps
            const int nacc = (KT * (BK / 8)) < G::NACC ? KT * (BK / 8) : G::NACC;
            for (int c0 = 0; c0 < BN; c0 += 16) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, v);
                for (int a = 1; a < nacc; ++a) {
                    float w[16];
                    tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(a * G::ACC_COLS + c0), w);
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] += w[j];
                }
                if (row < M) {
                    float* crow = C + (long long)row * ldc;
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int col = n0 + c0 + j;
                        if (col < N) {
                            float x = alpha * v[j];
                            if (colscale) x *= colscale[col];
                            if (beta != 0.f) x += beta * crow[col];
                            crow[col] = x;
                        }
                    }
                }
            }
        } else if (lane == 0) {
            atomicOr(err, 4);
            s_abort = 1;
        }
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"((uint32_t)G::TMEM_COLS)
                     : "memory");
    }
}

// hi = value with the 13 low mantissa bits cleared (exactly TF32), lo = x - hi
__global__ void split_kernel(const float* __restrict__ x, float* __restrict__ hi, float* __restrict__ lo,
                             long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        float v = x[i];
        float h = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
        hi[i] = h;
        lo[i] = v - h;
    }
}

}  // namespace tc

// ------------------------------------------------------------------ host side

// The driver's tensor-map encoder, looked up once (a function-local static:
// initialised once even when contexts run on several host threads; a failed
// lookup throws and is retried by the next call).
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        cudaDriverEntryPointQueryResult q;
        void* f = nullptr;
        KH_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q));
        if (!f || q != cudaDriverEntryPointSuccess) fail(KH_ECUDA, "cuTensorMapEncodeTiled unavailable");
        return (PFN_cuTensorMapEncodeTiled_v12000)f;
    }();
    return fn;
}

// Row-major FP32 matrix rows x K (leading dimension ld) as a 2-D tensor map
// with box {32, box_rows} and 128-byte swizzle.
static CUtensorMap make_map(const float* p, long long rows, long long K, long long ld, int box_rows) {
    const PFN_cuTensorMapEncodeTiled_v12000 encode = encode_fn();
    if (((uintptr_t)p & 15) != 0) fail(KH_EINVAL, "tensor-core operand not 16-byte aligned");
    if ((ld * 4) % 16 != 0) fail(KH_EINVAL, "tensor-core operand leading dimension not a multiple of 4");
    CUtensorMap m;
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * 4)};
    cuuint32_t box[2] = {(cuuint32_t)tc::BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)p, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) fail(KH_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return m;
}

template <int BN, int NPASS>
static void launch_tc(const TcOperand& A, const TcOperand& B, float* C, int M, int N, int K, long long ldc,
                      float alpha, float beta, const float* colscale, int* err, cudaStream_t st) {
    using G = tc::Cfg<BN, NPASS>;
    static std::atomic<size_t> granted[kMaxDevices] = {};
    smem_opt_in(tc::gemm_kernel<BN, NPASS>, (size_t)G::SMEM, granted);
    CUtensorMap ma = make_map(A.hi, M, K, A.ld, tc::BM);
    CUtensorMap mb = make_map(B.hi, N, K, B.ld, BN);
    CUtensorMap ma2 = NPASS == 3 ? make_map(A.lo, M, K, A.ld, tc::BM) : ma;
    CUtensorMap mb2 = NPASS == 3 ? make_map(B.lo, N, K, B.ld, BN) : mb;
    dim3 grid((N + BN - 1) / BN, (M + tc::BM - 1) / tc::BM);
    if (grid.y > 65535) fail(KH_EINVAL, "tc gemm: M too large");
    tc::gemm_kernel<BN, NPASS><<<grid, tc::THREADS, G::SMEM, st>>>(ma, mb, ma2, mb2, C, M, N, K, ldc, alpha, beta,
                                                                   colscale, err);
    KH_LAUNCHED();
}

template <int NPASS>
static void dispatch_bn(const TcOperand& A, const TcOperand& B, float* C, int M, int N, int K, long long ldc,
                        float alpha, float beta, const float* colscale, int* err, cudaStream_t st) {
    const long long mt = (M + tc::BM - 1) / tc::BM;
    // widest tile that still gives ~one wave of CTAs over the 152 SMs
    if (N <= 16) launch_tc<16, NPASS>(A, B, C, M, N, K, ldc, alpha, beta, colscale, err, st);
    else if (N <= 32) launch_tc<32, NPASS>(A, B, C, M, N, K, ldc, alpha, beta, colscale, err, st);
    else if (N <= 64 || mt * ((N + 127) / 128) < 120) launch_tc<64, NPASS>(A, B, C, M, N, K, ldc, alpha, beta, colscale, err, st);
    else launch_tc<128, NPASS>(A, B, C, M, N, K, ldc, alpha, beta, colscale, err, st);
}

void tc_gemm(const TcOperand& A, const TcOperand& B, float* C, int M, int N, int K, long long ldc, float alpha,
             float beta, const float* colscale, int npass, int* err, cudaStream_t st) {
    if (M <= 0 || N <= 0 || K <= 0) return;
    if (npass == 3) dispatch_bn<3>(A, B, C, M, N, K, ldc, alpha, beta, colscale, err, st);
    else dispatch_bn<1>(A, B, C, M, N, K, ldc, alpha, beta, colscale, err, st);
}

void tc_split(const float* x, float* hi, float* lo, long long n, cudaStream_t st) {
    tc::split_kernel<<<grid_for(n), 256, 0, st>>>(x, hi, lo, n);
    KH_LAUNCHED();
}

}  // namespace kh
