// Layered two-layer site contraction on the tensor cores: the shapes and the
// operand images shared by the kernel (layered.cu) and by the image builder
// (bond.cu).
//
// For nb blocks b (the chi^2 environment index pairs of an enlarged corner or
// an edge) the contraction is
//   out[b][ok][ob] = sum_p sum_{ik,ib} TL[ik][p][ok] Y[b][ib][ik] TL[ib][p][ob]
// with ik, ib, ok, ob pairs of virtual legs (D^2 values each) and p the
// physical index.  It runs as two GEMMs per tile of rows (b, ib):
//   ket layer  Z[(b,ib)][(p,ok)]  = sum_ik Y[(b,ib)][ik] TL[ik][(p,ok)]
//   bra layer  out[(b,ok)][ob]   += sum_(ib,p) Z[(b,ok)][(ib,p)] TL[(ib,p)][ob]
// over chunks of pc physical indices.  Z never leaves the SM: the ket GEMM
// accumulates it in tensor memory, the worker warps move it through shared
// memory into the (b,ok)-row layout, and the bra GEMM reads it back from
// tensor memory as its A operand.  The D^2 x D^2 double-layer index is never
// formed.
#pragma once

namespace kh {
namespace lay {

__host__ __device__ constexpr int pad_to(int x, int m) { return (x + m - 1) / m * m; }

// Tile shapes for bond dimension D (D^2 = d2), 1 or 3 MMA passes, and the
// operand type: TF32 (4-byte elements, K = 8 per MMA) or BF16 (2-byte
// elements, K = 16 per MMA, one pass).  Both move 32 bytes of K per MMA, so the
// shared-memory K blocks (128 bytes: 32 TF32 or 64 BF16 values) and the
// descriptor steps are the same; a tensor-memory column holds one TF32 or two
// BF16 values of the Z operand.
struct Plan {
    int esz = 4, kstep = 8;                  // element bytes; K per MMA
    int d2 = 0, bt = 0, rows = 0;            // D^2; blocks b per tile; rows (b, ib) used of 128
    int pc = 0, na2 = 0;                     // physical indices per chunk; Z buffers in tensor memory
    int nacc1 = 0, nacc2 = 0;                // independent accumulators of the ket and the bra GEMM
    int n1 = 0, n1p = 0, k1p = 0, kb1 = 0;   // ket GEMM: N = pc D^2 (padded to 16), K = D^2 (padded to kstep)
    int n2p = 0, k2 = 0, k2p = 0, kb2 = 0;   // bra GEMM: N = D^2 (padded to 16), K = pc D^2 (padded to kstep)
    int zs = 0;                              // row stride (floats) of the shared-memory transpose buffer
    int acc1_cols = 0, out_cols = 0;         // columns of one ket / bra accumulator (32-aligned)
    int c_acc1 = 0, c_a2 = 0, a2_cols = 0, c_out = 0, tmem = 0;   // tensor-memory columns
    int a1_bytes = 0, b1_bytes = 0, b2_bytes = 0;                 // one (hi or lo) operand image
};

// The tensor core runs consecutive MMAs into one accumulator as a dependent
// chain; these GEMMs are thin (N = D^2 for the bra layer), so the chain's
// latency, not the MMA throughput, sets the time.  Each GEMM therefore
// spreads its MMAs round-robin over nacc independent accumulators (summed
// when read).  The plan picks pc (a power of two <= 16), the accumulator
// counts and the Z double buffering that fit the 512 tensor-memory columns
// (every region 32-column aligned: two ket buffers of nacc1 accumulators, na2
// Z buffers (hi and lo with 3 passes), nacc2 bra accumulators), minimising a
// latency model: per chunk one worker hand-off plus the two dependent MMA
// chains (0.1 of a hand-off per chained MMA).  Shared-memory operands use the
// 128-byte-swizzle K-major layout in K blocks of 128 bytes.
__host__ __device__ constexpr Plan make_plan(int D, int npass, bool bf16 = false) {
    Plan P{};
    P.esz = bf16 ? 2 : 4;
    P.kstep = bf16 ? 16 : 8;
    const int per_block = 128 / P.esz;                  // K values per 128-byte block
    P.d2 = D * D;
    P.bt = P.d2 > 0 ? 128 / P.d2 : 0;
    P.rows = P.bt * P.d2;
    P.k1p = pad_to(P.d2, P.kstep);
    P.kb1 = (P.k1p + per_block - 1) / per_block;
    P.n2p = pad_to(P.d2, 16);
    if (P.bt < 1 || (bf16 && npass != 1)) return P;
    const int npl = npass == 3 ? 2 : 1;
    double best = 1e30;
    for (int pc = 16; pc >= 1; pc /= 2) {
        const int n1p = pad_to(pc * P.d2, 16);
        if (n1p > 256) continue;
        const int k2p = pad_to(pc * P.d2, P.kstep);
        const int zcols = k2p * P.esz / 4;                // tensor-memory columns of one Z operand
        const int nc = (16 + pc - 1) / pc;                // chunks at p = 16
        const int mm1 = (P.k1p / P.kstep) * npass, mm2 = (k2p / P.kstep) * npass;
        for (int nacc2 = 4; nacc2 >= 1; nacc2 /= 2)
            for (int nacc1 = 2; nacc1 >= 1; --nacc1)
                for (int na2 = 2; na2 >= 1; --na2) {
                    if (nacc1 > mm1 || nacc2 > mm2) continue;
                    const int cols = 2 * nacc1 * pad_to(n1p, 32) + na2 * npl * pad_to(zcols, 32) +
                                     nacc2 * pad_to(P.n2p, 32);
                    if (cols > 512) continue;
                    const double cost = nc * (1.0 + 0.1 * ((mm1 + nacc1 - 1) / nacc1) +
                                              0.1 * ((mm2 + nacc2 - 1) / nacc2)) - 0.01 * na2;
                    if (cost >= best) continue;
                    best = cost;
                    P.pc = pc;
                    P.na2 = na2;
                    P.nacc1 = nacc1;
                    P.nacc2 = nacc2;
                    P.n1 = pc * P.d2;
                    P.n1p = n1p;
                    P.k2 = pc * P.d2;
                    P.k2p = k2p;
                    P.kb2 = (k2p + per_block - 1) / per_block;
                    P.zs = pad_to(P.k2, 4);
                    if ((P.zs / 4) % 2 == 0) P.zs += 4;          // odd 16-byte stride: conflict-free row reads
                    P.acc1_cols = pad_to(n1p, 32);
                    P.out_cols = pad_to(P.n2p, 32);
                    P.c_acc1 = 0;
                    P.c_a2 = 2 * nacc1 * P.acc1_cols;
                    P.a2_cols = pad_to(zcols, 32);
                    P.c_out = P.c_a2 + na2 * npl * P.a2_cols;
                    P.tmem = 32;
                    while (P.tmem < P.c_out + nacc2 * P.out_cols) P.tmem *= 2;
                    P.a1_bytes = 128 * P.kb1 * 128;
                    P.b1_bytes = n1p * P.kb1 * 128;
                    P.b2_bytes = P.n2p * P.kb2 * 128;
                }
    }
    return P;
}

// Byte offset of element (row r, k) of esz bytes in a K-major operand of
// `rows` rows with 128-byte swizzle: K blocks of 128 bytes, each block rows x
// 128 bytes, the 16-byte chunks of row r permuted by r mod 8.
__host__ __device__ inline int swz_offset(int r, int k, int rows, int esz = 4) {
    const int byte = k * esz, kb = byte >> 7, kc = byte & 127;
    return kb * rows * 128 + r * 128 + ((((kc >> 4) ^ (r & 7)) << 4) | (kc & 15));
}

// Inverse of swz_offset for an esz-aligned offset o: (row, k).
__host__ __device__ inline void swz_position(int o, int rows, int& r, int& k, int esz = 4) {
    const int kb = o / (rows * 128), rem = o % (rows * 128);
    r = rem / 128;
    const int ch = (rem % 128) >> 4;
    k = (kb * 128 + (((ch ^ (r & 7)) << 4) | (rem & 15))) / esz;
}

// Chunks of pc physical indices covering p.
__host__ __device__ inline int n_chunks(const Plan& P, int p) { return (p + P.pc - 1) / P.pc; }

}  // namespace lay

// Image sizes (floats) of one (kind, frame) operand set for p physical
// indices: ket images of all chunks, then bra images (hi, lo per chunk with
// 3 passes).  Zero when D has no tensor-core plan.
long long layered_img1_floats(int D, int p, int npass, bool bf16 = false);
long long layered_img2_floats(int D, int p, int npass, bool bf16 = false);

// Operand images of all (kind, frame) pairs from the FP64 site tensor
// Tm[p][D^4] (legs l, u, r, d of frame 0): img1 holds 8 x per1 floats, img2
// 8 x per2 (per1, per2 at least layered_img1_floats / layered_img2_floats for
// p), layout [kind][frame][chunk][hi, lo].  With Tbra given, the bra images
// come from Tbra (same shape) and the ket images from Tm: the mixed double
// layer of an operator applied to the ket layer only.
void build_layered_images(const double* Tm, int p, int D, int npass, bool bf16, float* img1, float* img2,
                          long long per1, long long per2, cudaStream_t st, const double* Tbra = nullptr);

// out[b][ok][ob] (row-major, nb x D^2 x D^2) from Y[b][ib][ik] (row-major,
// nb x D^2 x D^2) and the operand images of one (kind, frame).  Tensor-core
// passes npass = 1 (TF32, or BF16 with bf16 set) or 3 (3xTF32).  Time-outs
// set bits of *err.
void site_layered_tc(const float* Y, long long nb, int D, int p, const float* img1, const float* img2, float* out,
                     int npass, bool bf16, int* err, cudaStream_t st);

}  // namespace kh
