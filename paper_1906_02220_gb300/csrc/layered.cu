// Layered (ket layer, then bra layer) site contraction of the enlarged
// corners and edge absorptions, Fig. 4 and Sec. III of arXiv:1906.02220, as
// one persistent tcgen05 kernel for sm_103a.  The shapes, the operand images
// and the index conventions are in layered.cuh.
//
// One CTA per SM loops over tiles of 128 rows (b, ib) (bt = 128 / D^2 blocks
// b per tile).  Per tile and chunk c of pc physical indices:
//   warp 0 (lanes 0, 1)  bulk-copies the chunk's ket (B1) and bra (B2) operand
//                        images into shared-memory rings (or once, when all
//                        chunks fit: resident images);
//   warp 1               allocates tensor memory; one lane issues the ket GEMMs
//                          acc1[c % 2]  = Y_tile * B1_c    (A, B in shared memory)
//   warps 2, 3           one lane each issues half of the bra GEMMs' MMAs
//                          out         += Z_c   * B2_c    (A = Z in tensor memory)
//                        (each group committed to an mbarrier);
//   warps 4-7 (workers)  load the Y tile (hi/lo split, or BF16) into shared
//                        memory (the next tile's values fetched into registers
//                        while this tile's chunks run), read acc1 row (b, ib)
//                        per thread, scatter it into a shared-memory buffer in
//                        (b, ok) row order, read back row (b, ok), split it into
//                        TF32 hi/lo (or round it to BF16 pairs) and store it to
//                        tensor memory as the bra GEMM's A operand; at the end
//                        of a tile they read the output accumulators and store
//                        out rows (b, ok).
// With 3 passes every product is A_hi B_hi + A_hi B_lo + A_lo B_hi (FP32-level
// accuracy from TF32 inputs); BF16 runs one kind::f16 pass (K = 16 per MMA).
// The MMAs of each GEMM are spread round-robin over independent accumulators
// (summed when read) and, for the bra GEMM, over two issuing threads: these
// narrow MMAs are bound by their issue, not by the tensor pipe.  Every wait is bounded: on time-out the kernel
// raises a flag, the roles drain, tensor memory is freed and the kernel
// returns with bits set in *err (8 producer, 16 MMA issuer, 32 workers).
#include <atomic>

#include <cuda_bf16.h>

#include "engine.cuh"
#include "layered.cuh"
#include "tc_ptx.cuh"

namespace kh {

namespace lay {

using namespace tc;

constexpr int NSET = 1;                        // worker sets (4 warps each), chunks split by index mod NSET
// issuing threads (one per warp) of the ket and the bra GEMMs; the bra GEMM
// has four times the MMAs of the ket GEMM at D = 4.  Eight warps in all keep
// the per-thread register limit at 255 (a ninth warp on one SM sub-partition
// would cut it to 168 and spill the workers).
constexpr int NI1 = 1, NI2 = 2;
constexpr int WORKER0 = 1 + NI1 + NI2;          // first worker warp
constexpr int THREADS = 32 * WORKER0 + 128 * NSET;   // producer, issuers, workers
constexpr int MAXST = 16;

__device__ __forceinline__ float tf32_hi(float v) { return __uint_as_float(__float_as_uint(v) & 0xFFFFE000u); }

// instruction descriptor: FP32 accumulator, A and B TF32 (kind::tf32) or BF16
// (kind::f16), K-major, N and M = 128
constexpr uint32_t idesc(int n, bool bf16) {
    const uint32_t fmt = bf16 ? 1u : 2u;
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// packs two FP32 values as BF16 (round to nearest even), a in the low half
__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    const uint32_t lo = __bfloat16_as_ushort(__float2bfloat16_rn(a));
    const uint32_t hi = __bfloat16_as_ushort(__float2bfloat16_rn(b));
    return lo | (hi << 16);
}

struct Bars {
    uint64_t b1_full[MAXST], b1_empty[MAXST], b2_full[MAXST], b2_empty[MAXST];
    uint64_t acc1_full[2], acc1_empty[2], a2_full[2], a2_empty[2];
    uint64_t zs_w[NSET], zs_r[NSET];
    uint64_t a1_full, a1_empty, out_full, out_empty, drain[NI1 + NI2];
};

// Bounded wait made uniform over the warp: false on time-out or abort.
__device__ __forceinline__ bool wait_warp(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
    const bool ok = mbar_wait(bar, parity, abort_flag);
    return __all_sync(0xffffffffu, ok);
}

// Wait that ignores the abort flag (used while draining).
__device__ __forceinline__ bool wait_drain(uint64_t* bar, uint32_t parity) {
    for (uint32_t it = 0; it < (1u << 22); ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

template <int D, int NPASS, bool BF>
__global__ void __launch_bounds__(THREADS, 1)
layered_kernel(const float* __restrict__ Y, long long nb, int nc, const uint8_t* __restrict__ img1,
               const uint8_t* __restrict__ img2, float* __restrict__ out, int ntiles, int nst1, int nst2,
               int* err) {
    static_assert(!BF || NPASS == 1, "BF16 runs one pass");
    constexpr Plan P = make_plan(D, NPASS, BF);
    constexpr int D2 = P.d2;
    constexpr int NPL = NPASS == 3 ? 2 : 1;
    constexpr int KS = P.kstep;
    constexpr uint32_t ID1 = idesc(P.n1p, BF), ID2 = idesc(P.n2p, BF);
    constexpr int A1_SZ = NPL * P.a1_bytes, B1_SZ = NPL * P.b1_bytes, B2_SZ = NPL * P.b2_bytes;

    extern __shared__ uint8_t smem_raw[];
    __shared__ Bars bars;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool res1 = nst1 == nc, res2 = nst2 == nc;      // images loaded once
    uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA1 = base;
    uint8_t* sB1 = sA1 + A1_SZ;
    uint8_t* sB2 = sB1 + (size_t)nst1 * B1_SZ;
    float* sZ = (float*)(sB2 + (size_t)nst2 * B2_SZ);

    if (threadIdx.x == 0) {
        for (int s = 0; s < MAXST; ++s) {
            mbar_init(&bars.b1_full[s], 1);
            mbar_init(&bars.b1_empty[s], NI1);
            mbar_init(&bars.b2_full[s], 1);
            mbar_init(&bars.b2_empty[s], NI2);
        }
        for (int j = 0; j < 2; ++j) {
            mbar_init(&bars.acc1_full[j], NI1);
            mbar_init(&bars.acc1_empty[j], 128);
            mbar_init(&bars.a2_full[j], 128);
            mbar_init(&bars.a2_empty[j], NI2);
        }
        mbar_init(&bars.a1_full, 128 * NSET);
        mbar_init(&bars.a1_empty, NI1);
        mbar_init(&bars.out_full, NI2);
        mbar_init(&bars.out_empty, 128);
        for (int s = 0; s < NSET; ++s) {
            mbar_init(&bars.zs_w[s], 128);
            mbar_init(&bars.zs_r[s], 128);
        }
        for (int q = 0; q < NI1 + NI2; ++q) mbar_init(&bars.drain[q], 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"((uint32_t)P.tmem)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = s_tmem;
    volatile int* abort_flag = &s_abort;

    if (warp == 0) {
        // ---------------------------------------------------------- producer
        if (lane < 2) {
            const bool ket = lane == 0;
            const int nst = ket ? nst1 : nst2;
            const bool res = ket ? res1 : res2;
            const int sz = ket ? B1_SZ : B2_SZ;
            uint8_t* ring = ket ? sB1 : sB2;
            const uint8_t* img = ket ? img1 : img2;
            uint64_t* full = ket ? bars.b1_full : bars.b2_full;
            uint64_t* empty = ket ? bars.b1_empty : bars.b2_empty;
            int armed[MAXST];
            for (int s = 0; s < MAXST; ++s) armed[s] = 0;
            if (res) {
                if (blockIdx.x < ntiles)
                    for (int c = 0; c < nc; ++c) {
                        mbar_expect_tx(&full[c], (uint32_t)sz);
                        bulk_load(ring + (size_t)c * sz, img + (size_t)c * sz, (uint32_t)sz, &full[c]);
                        armed[c] = 1;
                    }
            } else {
                long long g = 0;
                for (int tile = blockIdx.x; tile < ntiles && !*abort_flag; tile += gridDim.x) {
                    for (int c = 0; c < nc; ++c, ++g) {
                        const int s = (int)(g % nst);
                        const uint32_t u = (uint32_t)(g / nst);
                        if (!mbar_wait(&empty[s], (u & 1) ^ 1, abort_flag)) {
                            s_abort = 1;
                            atomicOr(err, 8);
                            break;
                        }
                        mbar_expect_tx(&full[s], (uint32_t)sz);
                        bulk_load(ring + (size_t)s * sz, img + (size_t)c * sz, (uint32_t)sz, &full[s]);
                        armed[s] = (int)u + 1;
                    }
                }
            }
            // copies still in flight land before the CTA exits
            for (int s = 0; s < MAXST; ++s)
                if (armed[s] && !wait_drain(&full[s], (uint32_t)(armed[s] - 1) & 1)) atomicOr(err, 8);
        }
    } else if (warp < WORKER0) {
        // ---------------------------------------------------------- MMA issuers
        // NI1 threads (warps 1 ..) issue the ket GEMMs, NI2 threads (the next
        // warps) the bra GEMMs, one thread per warp: these narrow MMAs are
        // bounded by their issue, not by the tensor pipe, so several issuers
        // keep more of them in flight.  Issuer q of a GEMM issues the MMAs of
        // the accumulators a with a % NI == q.
        if (lane == 0) {
            bool ok = true;
            long long g0 = 0;
            int it = 0;
            const bool ket = warp <= NI1;
            const int qi = ket ? warp - 1 : warp - 1 - NI1;   // issuer index within its GEMM
            if (ket) {
                for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++it, g0 += nc) {
                    if (!mbar_wait(&bars.a1_full, it & 1, abort_flag)) { ok = false; break; }
                    fence_after();
                    for (int c = 0; c < nc; ++c) {                      // ket layer of chunk c
                        const long long g = g0 + c;
                        const int s1 = res1 ? c : (int)(g % nst1);
                        const uint32_t ph1 = res1 ? 0u : (uint32_t)((g / nst1) & 1);
                        const int j = (int)(g & 1);
                        if (!mbar_wait(&bars.b1_full[s1], ph1, abort_flag) ||
                            !mbar_wait(&bars.acc1_empty[j], (uint32_t)((g >> 1) & 1) ^ 1, abort_flag)) {
                            ok = false;
                            break;
                        }
                        fence_after();
                        // MMAs round-robin over the buffer's nacc1 accumulators
                        const uint32_t d0 = tmem + P.c_acc1 + j * P.nacc1 * P.acc1_cols;
                        const uint32_t a0 = smem_u32(sA1), b0 = smem_u32(sB1 + (size_t)s1 * B1_SZ);
#pragma unroll
                        for (int pass = 0; pass < NPASS; ++pass) {
                            const uint32_t ab = a0 + (pass == 2 ? P.a1_bytes : 0);
                            const uint32_t bb = b0 + (pass == 1 ? P.b1_bytes : 0);
#pragma unroll
                            for (int ks = 0; ks < P.k1p / KS; ++ks) {
                                const int i = pass * (P.k1p / KS) + ks;
                                if ((i % P.nacc1) % NI1 != qi) continue;
                                // 32 bytes of K per MMA, four per 128-byte block
                                const uint64_t da = smem_desc(ab + (ks >> 2) * (128 * 128) + (ks & 3) * 32);
                                const uint64_t db = smem_desc(bb + (ks >> 2) * (P.n1p * 128) + (ks & 3) * 32);
                                const uint32_t dd = d0 + (i % P.nacc1) * P.acc1_cols;
                                if constexpr (BF) umma_f16(dd, da, db, ID1, i >= P.nacc1 ? 1u : 0u);
                                else umma_tf32(dd, da, db, ID1, i >= P.nacc1 ? 1u : 0u);
                            }
                        }
                        umma_commit(&bars.acc1_full[j]);
                        if (!res1) umma_commit(&bars.b1_empty[s1]);
                        if (c == nc - 1) umma_commit(&bars.a1_empty);
                    }
                }
            } else {
                for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++it, g0 += nc) {
                    for (int cc = 0; cc < nc; ++cc) {                   // bra layer of chunk cc
                        const long long g = g0 + cc;
                        const int s2 = res2 ? cc : (int)(g % nst2);
                        const uint32_t ph2 = res2 ? 0u : (uint32_t)((g / nst2) & 1);
                        const int ja = (int)(g % P.na2);
                        const uint32_t pa = (uint32_t)((g / P.na2) & 1);
                        if (!mbar_wait(&bars.b2_full[s2], ph2, abort_flag) ||
                            !mbar_wait(&bars.a2_full[ja], pa, abort_flag) ||
                            (cc == 0 && !mbar_wait(&bars.out_empty, (uint32_t)(it & 1) ^ 1, abort_flag))) {
                            ok = false;
                            break;
                        }
                        fence_after();
                        // MMAs round-robin over the nacc2 output accumulators
                        const uint32_t d0 = tmem + P.c_out;
                        const uint32_t a2 = tmem + P.c_a2 + ja * NPL * P.a2_cols;
                        const uint32_t b0 = smem_u32(sB2 + (size_t)s2 * B2_SZ);
#pragma unroll
                        for (int pass = 0; pass < NPASS; ++pass) {
                            const uint32_t aa = a2 + (pass == 2 ? P.a2_cols : 0);
                            const uint32_t bb = b0 + (pass == 1 ? P.b2_bytes : 0);
#pragma unroll
                            for (int ks = 0; ks < P.k2p / KS; ++ks) {
                                const int i = pass * (P.k2p / KS) + ks;
                                if ((i % P.nacc2) % NI2 != qi) continue;
                                const uint64_t db = smem_desc(bb + (ks >> 2) * (P.n2p * 128) + (ks & 3) * 32);
                                const uint32_t dd = d0 + (i % P.nacc2) * P.out_cols;
                                const uint32_t acc = (cc > 0 || i >= P.nacc2) ? 1u : 0u;
                                // 8 tensor-memory columns of Z per MMA (8 TF32 or 16 BF16 values)
                                if constexpr (BF) umma_f16_tmem_a(dd, aa + ks * 8, db, ID2, acc);
                                else umma_tf32_tmem_a(dd, aa + ks * 8, db, ID2, acc);
                            }
                        }
                        umma_commit(&bars.a2_empty[ja]);
                        if (!res2) umma_commit(&bars.b2_empty[s2]);
                        if (cc == nc - 1) umma_commit(&bars.out_full);
                    }
                }
            }
            if (!ok) {
                s_abort = 1;
                atomicOr(err, 16);
            }
            // every MMA this thread issued completes before tensor memory is freed
            uint64_t* dr = &bars.drain[warp - 1];
            umma_commit(dr);
            if (!wait_drain(dr, 0)) atomicOr(err, 16);
        }
    } else {
        // ---------------------------------------------------------- workers
        const int wt = threadIdx.x - 32 * WORKER0;       // 0 .. 128 NSET - 1
        const int set = wt >> 7;                         // chunks g with g % NSET == set
        const int q = warp & 3;                          // tensor-memory lane quadrant
        const int t = 32 * q + lane;                     // tile row of this thread
        const uint32_t lane_base = (uint32_t)(32 * q) << 16;
        const long long total_rows = nb * D2;
        float* zbuf = sZ + set * 128 * P.zs;
        bool ok = true;

        // zero the Y tile images once: padding rows and columns stay zero
        for (int i = wt; i < A1_SZ / 16; i += 128 * NSET) ((float4*)sA1)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        asm volatile("bar.sync 1, %0;" ::"r"(128 * NSET) : "memory");   // zeros land before the first tile's values

        // the tile's R D^2 values of Y (contiguous), all loads in flight at once:
        // fetched into registers, then written (hi/lo split) into the tile image
        constexpr int YPER = (P.rows * D2 + 128 * NSET - 1) / (128 * NSET);
        auto fetch_y = [&](int tile, float (&yv)[YPER]) {
            const long long e0 = (long long)tile * P.rows * D2, etot = total_rows * D2;
#pragma unroll
            for (int j = 0; j < YPER; ++j) {
                const int i = wt + 128 * NSET * j;
                const long long e = e0 + i;
                yv[j] = (i < P.rows * D2 && e < etot) ? __ldg(Y + e) : 0.f;
            }
        };
        auto store_y = [&](const float (&yv)[YPER]) {
#pragma unroll
            for (int j = 0; j < YPER; ++j) {
                const int i = wt + 128 * NSET * j;
                if (i < P.rows * D2) {
                    const int o = swz_offset(i / D2, i % D2, 128, P.esz);
                    if constexpr (BF) {
                        *(__nv_bfloat16*)(sA1 + o) = __float2bfloat16_rn(yv[j]);
                    } else if (NPASS == 3) {
                        const float h = tf32_hi(yv[j]);
                        *(float*)(sA1 + o) = h;
                        *(float*)(sA1 + P.a1_bytes + o) = yv[j] - h;
                    } else {
                        *(float*)(sA1 + o) = yv[j];
                    }
                }
            }
            fence_proxy_async();
            mbar_arrive(&bars.a1_full);
        };
        auto load_y = [&](int tile) {
            float yv[YPER];
            fetch_y(tile, yv);
            store_y(yv);
        };
        // the next tile's values are fetched while this tile's chunks run (where
        // the registers allow it), so their latency leaves the critical path
        constexpr bool kPrefetch = YPER <= 32;
        float ynext[kPrefetch ? YPER : 1];

        if ((int)blockIdx.x < ntiles) load_y(blockIdx.x);
        long long g0 = 0;
        int it = 0;
        uint32_t zcount = 0;                             // chunks this set has transposed
        for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++it, g0 += nc) {
            for (int c = 0; c < nc && ok; ++c) {
                const long long g = g0 + c;
                if ((int)(g % NSET) != set) continue;
                const int j = (int)(g & 1);
                // ---- ket accumulator row (b, ib) -> transpose buffer rows (b, ok)
                if (!wait_warp(&bars.acc1_full[j], (uint32_t)((g >> 1) & 1), abort_flag)) { ok = false; break; }
                fence_after();
                // the buffer's nacc1 accumulators, summed
                uint32_t vr[P.nacc1][P.n1p / 16][16];
#pragma unroll
                for (int a = 0; a < P.nacc1; ++a)
#pragma unroll
                    for (int c0 = 0; c0 < P.n1p; c0 += 16)
                        tmem_ld16_async(tmem + lane_base +
                                            (uint32_t)(P.c_acc1 + (j * P.nacc1 + a) * P.acc1_cols + c0),
                                        vr[a][c0 / 16]);
                tmem_ld_wait();
#pragma unroll
                for (int a = 0; a < P.nacc1; ++a)
#pragma unroll
                    for (int c0 = 0; c0 < P.n1p; c0 += 16) tmem_regs_ready(vr[a][c0 / 16]);
                auto v = [&](int n) {
                    float x = __uint_as_float(vr[0][n >> 4][n & 15]);
#pragma unroll
                    for (int a = 1; a < P.nacc1; ++a) x += __uint_as_float(vr[a][n >> 4][n & 15]);
                    return x;
                };
                fence_before();
                mbar_arrive(&bars.acc1_empty[j]);
                if constexpr (kPrefetch) {
                    if (c == 0 && tile + (int)gridDim.x < ntiles) fetch_y(tile + gridDim.x, ynext);
                }
                if (t < P.rows) {
                    const int b = t / D2, ib = t % D2;
#pragma unroll
                    for (int ok_ = 0; ok_ < D2; ++ok_) {
                        float* dst = zbuf + (b * D2 + ok_) * P.zs + ib * P.pc;
                        if constexpr (P.pc % 4 == 0) {
#pragma unroll
                            for (int pl = 0; pl < P.pc; pl += 4)
                                *(float4*)(dst + pl) = make_float4(v(pl * D2 + ok_), v((pl + 1) * D2 + ok_),
                                                                   v((pl + 2) * D2 + ok_), v((pl + 3) * D2 + ok_));
                        } else if constexpr (P.pc == 2) {
                            *(float2*)dst = make_float2(v(ok_), v(D2 + ok_));
                        } else {
                            *dst = v(ok_);
                        }
                    }
                }
                mbar_arrive(&bars.zs_w[set]);
                if (!wait_warp(&bars.zs_w[set], zcount & 1, abort_flag)) { ok = false; break; }
                // ---- row (b, ok) of Z -> tensor memory (bra GEMM A operand)
                const int ja = (int)(g % P.na2);
                if (!wait_warp(&bars.a2_empty[ja], (uint32_t)((g / P.na2) & 1) ^ 1, abort_flag)) {
                    ok = false;
                    break;
                }
                fence_after();
                constexpr int K2R = pad_to(P.k2, 4);          // values read per row
                constexpr int K2S = pad_to(P.k2p, BF ? 32 : 16);   // values stored per row (whole 16-column groups)
                float z[K2S];
#pragma unroll
                for (int i = 0; i < K2S; ++i) z[i] = 0.f;
                if (t < P.rows) {
                    const float* src = zbuf + t * P.zs;
#pragma unroll
                    for (int i = 0; i < K2R; i += 4) {
                        const float4 w = *(const float4*)(src + i);
                        z[i] = w.x;
                        if (i + 1 < P.k2) z[i + 1] = w.y;
                        if (i + 2 < P.k2) z[i + 2] = w.z;
                        if (i + 3 < P.k2) z[i + 3] = w.w;
                    }
                }
                const uint32_t a2 = tmem + lane_base + (uint32_t)(P.c_a2 + ja * NPL * P.a2_cols);
                if constexpr (BF) {
                    // two BF16 values per column, the lower K index in the low half
#pragma unroll
                    for (int c0 = 0; c0 < K2S / 2; c0 += 16) {
                        float w[16];
#pragma unroll
                        for (int i = 0; i < 16; ++i)
                            w[i] = __uint_as_float(pack_bf16x2(z[2 * (c0 + i)], z[2 * (c0 + i) + 1]));
                        tmem_st16(a2 + (uint32_t)c0, w);
                    }
                } else {
#pragma unroll
                    for (int c0 = 0; c0 < K2S; c0 += 16) {
                        float hi[16], lo[16];
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const float x = z[c0 + i];
                            hi[i] = NPASS == 3 ? tf32_hi(x) : x;
                            lo[i] = x - hi[i];
                        }
                        tmem_st16(a2 + (uint32_t)c0, hi);
                        if (NPASS == 3) tmem_st16(a2 + (uint32_t)(P.a2_cols + c0), lo);
                    }
                }
                tmem_st_wait();
                fence_before();
                mbar_arrive(&bars.a2_full[ja]);
                mbar_arrive(&bars.zs_r[set]);
                if (!wait_warp(&bars.zs_r[set], zcount & 1, abort_flag)) { ok = false; break; }
                ++zcount;
            }
            if (!ok) break;
            // next tile's Y once the ket GEMMs of this tile have read it
            const int next = tile + gridDim.x;
            if (next < ntiles) {
                if (!wait_warp(&bars.a1_empty, it & 1, abort_flag)) { ok = false; break; }
                if constexpr (kPrefetch) store_y(ynext);
                else load_y(next);
            }
            if (set != 0) continue;
            // ---- output rows (b, ok) (first set)
            if (!wait_warp(&bars.out_full, it & 1, abort_flag)) { ok = false; break; }
            fence_after();
            uint32_t orr[P.nacc2][P.n2p / 16][16];
#pragma unroll
            for (int a = 0; a < P.nacc2; ++a)
#pragma unroll
                for (int c0 = 0; c0 < P.n2p; c0 += 16)
                    tmem_ld16_async(tmem + lane_base + (uint32_t)(P.c_out + a * P.out_cols + c0), orr[a][c0 / 16]);
            tmem_ld_wait();
            float o[P.n2p];
#pragma unroll
            for (int c0 = 0; c0 < P.n2p; c0 += 16) {
#pragma unroll
                for (int a = 0; a < P.nacc2; ++a) tmem_regs_ready(orr[a][c0 / 16]);
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    float x = __uint_as_float(orr[0][c0 / 16][i]);
#pragma unroll
                    for (int a = 1; a < P.nacc2; ++a) x += __uint_as_float(orr[a][c0 / 16][i]);
                    o[c0 + i] = x;
                }
            }
            fence_before();
            mbar_arrive(&bars.out_empty);
            const long long row = (long long)tile * P.rows + t;
            if (t < P.rows && row < total_rows) {
                float* dst = out + row * D2;
                if constexpr (D2 % 4 == 0) {
#pragma unroll
                    for (int i = 0; i < D2; i += 4) *(float4*)(dst + i) = make_float4(o[i], o[i + 1], o[i + 2], o[i + 3]);
                } else {
#pragma unroll
                    for (int i = 0; i < D2; ++i) dst[i] = o[i];
                }
            }
        }
        if (!ok) {
            s_abort = 1;
            if (lane == 0) atomicOr(err, 32);
        }
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)P.tmem)
                     : "memory");
    }
}

}  // namespace lay

// ------------------------------------------------------------------ host side

namespace {

int sm_count() {
    static std::atomic<int> cache[kMaxDevices] = {};
    int dev = 0;
    KH_CUDA(cudaGetDevice(&dev));
    const int i = dev < kMaxDevices ? dev : 0;
    int v = cache[i].load();
    if (v == 0) {
        KH_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev));
        cache[i].store(v);
    }
    return v;
}

int smem_optin_max() {
    static std::atomic<int> cache[kMaxDevices] = {};
    int dev = 0;
    KH_CUDA(cudaGetDevice(&dev));
    const int i = dev < kMaxDevices ? dev : 0;
    int v = cache[i].load();
    if (v == 0) {
        KH_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        cache[i].store(v);
    }
    return v;
}

template <int D, int NPASS, bool BF>
void launch_layered(const float* Y, long long nb, int p, const float* img1, const float* img2, float* out, int* err,
                    cudaStream_t st) {
    constexpr lay::Plan P = lay::make_plan(D, NPASS, BF);
    static_assert(P.pc > 0, "no tensor-memory plan");
    constexpr int NPL = NPASS == 3 ? 2 : 1;
    const int nc = lay::n_chunks(P, p);
    const long long ntiles_ll = (nb + P.bt - 1) / P.bt;
    if (ntiles_ll > 0x7fffffffLL) fail(KH_EINVAL, "layered site contraction: too many tiles");
    const int ntiles = (int)ntiles_ll;
    if (ntiles == 0) return;
    const size_t fixed = 1024 + (size_t)NPL * P.a1_bytes + (size_t)lay::NSET * 128 * P.zs * 4;
    const size_t s1 = (size_t)NPL * P.b1_bytes, s2 = (size_t)NPL * P.b2_bytes;
    const size_t cap = (size_t)smem_optin_max() - 2048;   // the static barriers share the per-block limit
    int nst1 = 0, nst2 = 0;
    if (nc <= lay::MAXST && fixed + nc * (s1 + s2) <= cap) {
        nst1 = nst2 = nc;                                  // resident images
    } else {
        const int tries[4][2] = {{2, 2}, {2, 1}, {1, 2}, {1, 1}};
        for (auto& tr : tries) {
            const int a = tr[0] < nc ? tr[0] : nc, b = tr[1] < nc ? tr[1] : nc;
            if (fixed + a * s1 + b * s2 <= cap) {
                nst1 = a;
                nst2 = b;
                break;
            }
        }
    }
    if (nst1 == 0) fail(KH_EINVAL, "layered site contraction: shared memory too small");
    size_t smem = fixed + nst1 * s1 + nst2 * s2;
    // more than half the tensor memory: keep a second CTA off the SM (it
    // would only wait in tcgen05.alloc)
    if (P.tmem > 256 && smem <= cap / 2) smem = cap / 2 + 1024;
    static std::atomic<size_t> granted[kMaxDevices] = {};
    smem_opt_in(lay::layered_kernel<D, NPASS, BF>, smem, granted);
    const int grid = ntiles < sm_count() ? ntiles : sm_count();
    lay::layered_kernel<D, NPASS, BF><<<grid, lay::THREADS, smem, st>>>(
        Y, nb, nc, (const uint8_t*)img1, (const uint8_t*)img2, out, ntiles, nst1, nst2, err);
    KH_LAUNCHED();
}

template <int NPASS, bool BF>
void dispatch_d(const float* Y, long long nb, int D, int p, const float* img1, const float* img2, float* out,
                int* err, cudaStream_t st) {
    switch (D) {
        case 1: launch_layered<1, NPASS, BF>(Y, nb, p, img1, img2, out, err, st); break;
        case 2: launch_layered<2, NPASS, BF>(Y, nb, p, img1, img2, out, err, st); break;
        case 3: launch_layered<3, NPASS, BF>(Y, nb, p, img1, img2, out, err, st); break;
        case 4: launch_layered<4, NPASS, BF>(Y, nb, p, img1, img2, out, err, st); break;
        case 5: launch_layered<5, NPASS, BF>(Y, nb, p, img1, img2, out, err, st); break;
        case 6: launch_layered<6, NPASS, BF>(Y, nb, p, img1, img2, out, err, st); break;
        case 7: launch_layered<7, NPASS, BF>(Y, nb, p, img1, img2, out, err, st); break;
        case 8: launch_layered<8, NPASS, BF>(Y, nb, p, img1, img2, out, err, st); break;
        default: fail(KH_EINVAL, "layered site contraction: D out of range");
    }
}

}  // namespace

long long layered_img1_floats(int D, int p, int npass, bool bf16) {
    const lay::Plan P = lay::make_plan(D, npass, bf16);
    if (P.pc == 0) return 0;
    return (long long)lay::n_chunks(P, p) * (npass == 3 ? 2 : 1) * P.b1_bytes / 4;
}

long long layered_img2_floats(int D, int p, int npass, bool bf16) {
    const lay::Plan P = lay::make_plan(D, npass, bf16);
    if (P.pc == 0) return 0;
    return (long long)lay::n_chunks(P, p) * (npass == 3 ? 2 : 1) * P.b2_bytes / 4;
}

void site_layered_tc(const float* Y, long long nb, int D, int p, const float* img1, const float* img2, float* out,
                     int npass, bool bf16, int* err, cudaStream_t st) {
    if (nb <= 0) return;
    if (((uintptr_t)img1 & 15) || ((uintptr_t)img2 & 15) || ((uintptr_t)out & 15) || ((uintptr_t)Y & 3))
        fail(KH_EINVAL, "layered site contraction: misaligned operand");
    if (bf16) {
        if (npass != 1) fail(KH_EINVAL, "layered site contraction: BF16 runs one pass");
        dispatch_d<1, true>(Y, nb, D, p, img1, img2, out, err, st);
    } else if (npass == 3) {
        dispatch_d<3, false>(Y, nb, D, p, img1, img2, out, err, st);
    } else {
        dispatch_d<1, false>(Y, nb, D, p, img1, img2, out, err, st);
    }
}

}  // namespace kh
