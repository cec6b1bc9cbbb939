// Gate application and environment-weighted bond update, Fig. 3(b) and Sec. III
// of arXiv:1906.02220, plus the observables of Sec. V (energy per site,
// sublattice magnetisations).
//
// Composite for mapping gamma (Fig. 4(b)): with (alpha, alpha') the other two
// bond directions in cyclic order, T'[p'; l,u,r,d] =
//   sum_{sA,sB} g[(sA',sB'),(sA,sB)] sum_k A[sA,aA; u=alpha', r=alpha, k=gamma]
//                                         B[sB,aB; d=alpha', l=alpha, k=gamma].
// Bond update: minimise d = <T''-T'|N|T''-T'> over A''[sA,aA,u,r,k],
// B''[sB,aB,d,l,k] (k < D) with the CTMRG metric N; start from the truncated
// SVD of T' as a (4D^2)x(4D^2) matrix; alternate the two quadratic
// subproblems (R + reg tr(R)/m I) X = S (FP64 Cholesky); balanced gauge from
// the Gram matrices of A'' and B''.
#include <cuda_bf16.h>

#include "engine.cuh"
#include "layered.cuh"

namespace kh {

struct Mat4 { double v[16]; };
struct Mat4x3 { double v[48]; };

// ------------------------------------------------------------------ composite

__device__ __forceinline__ void bond_strides(int gamma, int D, int& s_u, int& s_r, int& s_k) {
    // site tensor A[s][a][x][y][z]: bond strides x: D^2, y: D, z: 1
    int str[3] = {D * D, D, 1};
    int al = (gamma + 1) % 3, alp = (gamma + 2) % 3;
    s_u = str[alp];
    s_r = str[al];
    s_k = str[gamma];
}

__global__ void composite_kernel(const double* __restrict__ A, const double* __restrict__ B, int D, int gamma,
                                 Mat4 g, int has_gate, double* __restrict__ T) {
    const int D4 = D * D * D * D, D3 = D * D * D;
    int tot = 16 * D4;
    int su, sr, sk;
    bond_strides(gamma, D, su, sr, sk);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += gridDim.x * blockDim.x) {
        int p = i / D4, leg = i % D4;
        int l = leg / (D * D * D), u = (leg / (D * D)) % D, r = (leg / D) % D, d = leg % D;
        int sAo = (p >> 3) & 1, aA = (p >> 2) & 1, sBo = (p >> 1) & 1, aB = p & 1;
        double acc = 0.0;
        for (int sA = 0; sA < 2; ++sA)
            for (int sB = 0; sB < 2; ++sB) {
                double gv = has_gate ? g.v[(sAo * 2 + sBo) * 4 + sA * 2 + sB] : ((sA == sAo && sB == sBo) ? 1.0 : 0.0);
                if (gv == 0.0) continue;
                const double* a = A + (sA * 2 + aA) * D3 + u * su + r * sr;
                const double* b = B + (sB * 2 + aB) * D3 + d * su + l * sr;
                double s = 0.0;
                for (int k = 0; k < D; ++k) s += a[k * sk] * b[k * sk];
                acc += gv * s;
            }
        T[i] = acc;
    }
}

// Rotated operand layouts for frames f = 0..3 (counter-clockwise quarter
// turns: new (l,u,r,d) = old (u,r,d,l)):
//   Tcor_f[l][u][p][r][d], Tedg_f[l][d][p][u][r]  (frame-f legs).
template <typename T>
__global__ void derived_kernel(const double* __restrict__ Tm, int p, int D, int pmax, T* Tcor, T* Tedg) {
    const int D4 = D * D * D * D;
    int tot = 4 * p * D4;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += gridDim.x * blockDim.x) {
        int f = i / (p * D4), rem = i % (p * D4);
        int pp = rem / D4, leg = rem % D4;
        int L = leg / (D * D * D), Uu = (leg / (D * D)) % D, Rr = (leg / D) % D, Dd = leg % D;
        // frame-f legs (L,U,R,D) -> original legs: undo f rotations
        int l = L, u = Uu, r = Rr, d = Dd;
        for (int t = 0; t < f; ++t) {
            int ol = d, ou = l, orr = u, od = r;   // old legs of one rotation
            l = ol; u = ou; r = orr; d = od;
        }
        double v = Tm[pp * D4 + ((l * D + u) * D + r) * D + d];
        // Tcor_f[L][U][p][R][D]
        long long ic = (long long)f * pmax * D4 + (((long long)(L * D + Uu) * p + pp) * D + Rr) * D + Dd;
        // Tedg_f[L][D][p][U][R]
        long long ie = (long long)f * pmax * D4 + (((long long)(L * D + Dd) * p + pp) * D + Uu) * D + Rr;
        Tcor[ic] = (T)v;
        Tedg[ie] = (T)v;
    }
}

// Original-frame offset (l,u,r,d) of the frame-f legs (L,U,R,D) of T.
__device__ __forceinline__ int frame_offset(int f, int L, int U, int R, int Dd, int D) {
    int l = L, u = U, r = R, d = Dd;
    for (int t = 0; t < f; ++t) {
        int ol = d, ou = l, orr = u, od = r;
        l = ol; u = ou; r = orr; d = od;
    }
    return ((l * D + u) * D + r) * D + d;
}

// Double-layer operands of the site contraction, in the K-major layout of a
// GEMM's second operand: for kind 0 (corner, TL = [L,U][p][R,D]) and kind 1
// (edge, TL = [L,D][p][U,R]) of frame f,
//   Wt_f[(ok,ob)][(ib,ik)] = sum_p TL_f[ik][p][ok] TL_f[ib][p][ob]
// summed in FP64.  With lo != null the value is stored as its TF32 head
// (13 low mantissa bits cleared) in W and the FP32 remainder in lo.
template <typename T>
__global__ void wt_kernel(const double* __restrict__ Tm, int p, int D, T* Wc, T* We, T* Wc_lo, T* We_lo) {
    const int d2 = D * D, d4 = d2 * d2;
    const long long per = (long long)d4 * d4;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 8 * per;
         i += (long long)gridDim.x * blockDim.x) {
        const int kind = (int)(i / (4 * per));
        const long long rem = i % (4 * per);
        const int f = (int)(rem / per);
        const long long idx = rem % per;
        const int nn = (int)(idx / d4), kk = (int)(idx % d4);
        const int ok = nn / d2, ob = nn % d2, ib = kk / d2, ik = kk % d2;
        int ok_, ob_;
        if (kind == 0) {     // in = (L,U), out = (R,D)
            ok_ = frame_offset(f, ik / D, ik % D, ok / D, ok % D, D);
            ob_ = frame_offset(f, ib / D, ib % D, ob / D, ob % D, D);
        } else {             // in = (L,D), out = (U,R)
            ok_ = frame_offset(f, ik / D, ok / D, ok % D, ik % D, D);
            ob_ = frame_offset(f, ib / D, ob / D, ob % D, ib % D, D);
        }
        const long long D4 = d4;
        double sacc = 0.0;
        for (int pp = 0; pp < p; ++pp) sacc += Tm[pp * D4 + ok_] * Tm[pp * D4 + ob_];
        T* W = (kind == 0 ? Wc : We) + rem;
        T* Wl = kind == 0 ? Wc_lo : We_lo;
        if (Wl) {
            float v = (float)sacc;
            float h = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
            *W = (T)h;
            Wl[rem] = (T)(v - h);
        } else {
            *W = (T)sacc;
        }
    }
}

// Operand images of the layered tensor-core site contraction (layered.cuh)
// for kind 0 (corner, TL = [L,U][p][R,D]) and kind 1 (edge, TL = [L,D][p][U,R])
// of frame f.  Per chunk c of pc physical indices, the ket image
//   B1_c[(pl, ok)][ik] = TL_f[ik][c pc + pl][ok]
// and the bra image
//   B2_c[ob][(ib, pl)] = TL_f[ib][c pc + pl][ob],
// each stored byte for byte as its 128-byte-swizzled K-major shared-memory
// tile (the TF32 head, then the FP32 remainder, with 3 passes), zero outside
// the operand.  Layout [kind][frame][chunk][hi, lo], per1 / per2 floats per
// (kind, frame).
__global__ void layered_img_kernel(const double* __restrict__ Tm, const double* __restrict__ Tb, int p, int D,
                                   lay::Plan P, int npass, float* __restrict__ img1, float* __restrict__ img2,
                                   long long per1, long long per2) {
    // per1, per2 in floats; elements of P.esz bytes (TF32 values or BF16)
    const int npl = npass == 3 ? 2 : 1;
    const int epf = 4 / P.esz;                                 // elements per float slot
    const long long e1 = per1 * epf, e2 = per2 * epf;          // elements per (kind, frame)
    const long long tot1 = 8 * e1, tot = tot1 + 8 * e2;
    const long long D4 = (long long)D * D * D * D;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
         i += (long long)gridDim.x * blockDim.x) {
        const bool ket = i < tot1;
        const long long e = ket ? i : i - tot1;
        const long long per = ket ? e1 : e2;
        const int kf = (int)(e / per), kind = kf >> 2, f = kf & 3;
        const long long rem = e % per;
        const int sub = (ket ? P.b1_bytes : P.b2_bytes) / P.esz;  // elements of one hi or lo image
        const int idx = (int)(rem / sub), c = idx / npl, hl = idx % npl;
        int r, k;
        lay::swz_position((int)(rem % sub) * P.esz, ket ? P.n1p : P.n2p, r, k, P.esz);
        int in = -1, out = -1, pp = p;
        if (ket && r < P.n1 && k < P.d2) {                 // row (pl, ok), column ik
            in = k;
            out = r % P.d2;
            pp = c * P.pc + r / P.d2;
        } else if (!ket && r < P.d2 && k < P.k2) {         // row ob, column (ib, pl)
            in = k / P.pc;
            out = r;
            pp = c * P.pc + k % P.pc;
        }
        double v = 0.0;
        if (in >= 0 && pp < p) {
            const int off = kind == 0 ? frame_offset(f, in / D, in % D, out / D, out % D, D)
                                      : frame_offset(f, in / D, out / D, out % D, in % D, D);
            v = (ket ? Tm : Tb)[pp * D4 + off];
        }
        if (P.esz == 2) {
            __nv_bfloat16* dst = (__nv_bfloat16*)(ket ? img1 : img2);
            dst[e] = __double2bfloat16(v);
        } else {
            float x = (float)v;
            if (npass == 3) {
                const float h = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
                x = hl == 0 ? h : x - h;
            }
            (ket ? img1 : img2)[e] = x;
        }
    }
}

void build_layered_images(const double* Tm, int p, int D, int npass, bool bf16, float* img1, float* img2,
                          long long per1, long long per2, cudaStream_t st, const double* Tbra) {
    const long long tot = 8 * (per1 + per2) * (bf16 ? 2 : 1);
    layered_img_kernel<<<grid_for(tot), 256, 0, st>>>(Tm, Tbra ? Tbra : Tm, p, D, lay::make_plan(D, npass, bf16),
                                                      npass, img1, img2, per1, per2);
    KH_LAUNCHED();
}

template <typename T>
void derive_operands(const double* Tm, int p, int D, int pmax, T* Tcor, T* Tedg, cudaStream_t st) {
    derived_kernel<T><<<grid_for(4LL * p * D * D * D * D), 256, 0, st>>>(Tm, p, D, pmax, Tcor, Tedg);
    KH_LAUNCHED();
}
template void derive_operands<float>(const double*, int, int, int, float*, float*, cudaStream_t);
template void derive_operands<double>(const double*, int, int, int, double*, double*, cudaStream_t);

template <typename T>
void Engine<T>::build_derived(Slot<T>& sl) {
    int tot = 4 * sl.p * dm.D4;
    derived_kernel<T><<<grid_for(tot), 256, 0, st>>>(sl.Ts, sl.p, dm.D, dm.pmax, sl.Tcor, sl.Tedg);
    KH_LAUNCHED();
    // the double-layer form costs D^8 per block against 2 p D^6 layer by layer
    sl.dl = dm.dl_alloc && dm.d2 <= 2 * sl.p;
    if (dm.lay && !sl.dl)
        build_layered_images(sl.Ts, sl.p, dm.D, dm.npass, dm.bf16, (float*)sl.L1, (float*)sl.L2, dm.lay1, dm.lay2,
                             st);
    if (sl.dl) {
        const bool split = sizeof(T) == 4 && tc_npass == 3 && dm.D4 % 4 == 0;
        const long long tot8 = 8LL * dm.D4 * dm.D4;
        wt_kernel<T><<<grid_for(tot8), 256, 0, st>>>(sl.Ts, sl.p, dm.D, sl.Wcor, sl.Wedg,
                                                     split ? sl.Wcor_lo : nullptr, split ? sl.Wedg_lo : nullptr);
        KH_LAUNCHED();
    }
}

template <typename T>
void Engine<T>::set_tensor(int slot, const double* Tin, int p) {
    if (p < 1 || p > dm.pmax) fail(KH_EINVAL, "p out of range");
    Slot<T>& sl = slots[slot];
    KH_CUDA(cudaMemcpyAsync(sl.Ts, Tin, sizeof(double) * p * dm.D4, cudaMemcpyDeviceToDevice, st));
    sl.p = p;
    build_derived(sl);
}

template <typename T>
void Engine<T>::build_composite(int slot, int gamma, const double* gate) {
    if (gamma < 0 || gamma > 2) fail(KH_EINVAL, "gamma must be 0, 1 or 2");
    if (dm.pmax < 16) fail(KH_EINVAL, "composites need p_max = 16");
    Slot<T>& sl = slots[slot];
    Mat4 g;
    for (int i = 0; i < 16; ++i) g.v[i] = gate ? gate[i] : 0.0;
    composite_kernel<<<grid_for(16 * dm.D4), 256, 0, st>>>(A, B, dm.D, gamma, g, gate != nullptr, sl.Ts);
    KH_LAUNCHED();
    sl.p = 16;
    build_derived(sl);
}

template <typename T>
void Engine<T>::set_state(const double* Ain, const double* Bin) {
    const size_t b = sizeof(double) * 4 * dm.D * dm.D * dm.D;
    KH_CUDA(cudaMemcpyAsync(A, Ain, b, cudaMemcpyDeviceToDevice, st));
    KH_CUDA(cudaMemcpyAsync(B, Bin, b, cudaMemcpyDeviceToDevice, st));
}

template <typename T>
void Engine<T>::get_state(double* Aout, double* Bout) {
    const size_t b = sizeof(double) * 4 * dm.D * dm.D * dm.D;
    KH_CUDA(cudaMemcpyAsync(Aout, A, b, cudaMemcpyDeviceToDevice, st));
    KH_CUDA(cudaMemcpyAsync(Bout, B, b, cudaMemcpyDeviceToDevice, st));
    KH_CUDA(cudaStreamSynchronize(st));
}

// ------------------------------------------------------------------ ALS kernels

// Leg positions in the composite row index (l,u,r,d): A owns (u,r), B owns (d,l).
// side 0 (solve A): own (o1,o2) = (u,r), other (t1,t2) = (d,l) = layout of B''.
// side 1 (solve B): own (o1,o2) = (d,l), other (t1,t2) = (u,r) = layout of A''.
__device__ __forceinline__ int row_index(int side, int o1, int o2, int t1, int t2, int D) {
    int l, u, r, d;
    if (side == 0) { u = o1; r = o2; d = t1; l = t2; }
    else { d = o1; l = o2; u = t1; r = t2; }
    return ((l * D + u) * D + r) * D + d;
}

// X[(o1,o2)][j][(ph,k)] = sum_{t1,t2} N[row(o,t)][j] Oth[ph][t1][t2][k]
__global__ void als_x_kernel(const double* __restrict__ N, const double* __restrict__ Oth, int D, int side,
                             double* __restrict__ X, const int* skip) {
    if (skip && *skip) return;
    const int D4 = D * D * D * D, d2 = D * D;
    long long tot = (long long)d2 * D4 * 4 * D;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
         i += (long long)gridDim.x * blockDim.x) {
        int k = (int)(i % D);
        int ph = (int)((i / D) % 4);
        int j = (int)((i / (4 * D)) % D4);
        int o = (int)(i / ((long long)4 * D * D4));
        int o1 = o / D, o2 = o % D;
        double s = 0.0;
        for (int t1 = 0; t1 < D; ++t1)
            for (int t2 = 0; t2 < D; ++t2)
                s += N[(long long)row_index(side, o1, o2, t1, t2, D) * D4 + j] * Oth[((ph * D + t1) * D + t2) * D + k];
        X[i] = s;
    }
}

// R[(o1,o2,k)][(o1',o2',k')] = sum_{t1',t2',ph} X[(o1,o2)][row(o',t')][(ph,k)] Oth[ph][t1'][t2'][k']
// (one thread per entry)
__global__ void als_r_kernel(const double* __restrict__ X, const double* __restrict__ Oth, int D, int side,
                             double* __restrict__ R, const int* skip) {
    if (skip && *skip) return;
    const int D4 = D * D * D * D, m = D * D * D;
    const long long totR = (long long)m * m;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < totR;
         i += (long long)gridDim.x * blockDim.x) {
        int a = (int)(i / m), b = (int)(i % m);
        int o1 = a / (D * D), o2 = (a / D) % D, k = a % D;
        int q1 = b / (D * D), q2 = (b / D) % D, kp = b % D;
        const double* x = X + (long long)(o1 * D + o2) * D4 * 4 * D;
        double s = 0.0;
        for (int t1 = 0; t1 < D; ++t1)
            for (int t2 = 0; t2 < D; ++t2) {
                int j = row_index(side, q1, q2, t1, t2, D);
                for (int ph = 0; ph < 4; ++ph)
                    s += x[((long long)j * 4 + ph) * D + k] * Oth[((ph * D + t1) * D + t2) * D + kp];
            }
        R[i] = s;
    }
}

// S[(o1,o2,k)][q] = sum_{j,ph} X[(o1,o2)][j][(ph,k)] Tp[pidx(q,ph)][j]
// (one warp per entry, lanes over j: D^4 4 terms each)
__global__ void als_s_kernel(const double* __restrict__ X, const double* __restrict__ Tp, int D, int side,
                             double* __restrict__ S, const int* skip) {
    if (skip && *skip) return;
    const int D4 = D * D * D * D, m = D * D * D;
    const int lane = threadIdx.x & 31;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long e = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; e < 4LL * m; e += nwarps) {
        int a = (int)(e / 4), q = (int)(e % 4);
        int o1 = a / (D * D), o2 = (a / D) % D, k = a % D;
        const double* x = X + (long long)(o1 * D + o2) * D4 * 4 * D;
        double s = 0.0;
        for (int j = lane; j < D4; j += 32)
            for (int ph = 0; ph < 4; ++ph) {
                int pidx = (side == 0) ? (q * 4 + ph) : (ph * 4 + q);
                s += x[((long long)j * 4 + ph) * D + k] * Tp[(long long)pidx * D4 + j];
            }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) S[a * 4 + q] = s;
    }
}

// One-CTA solve of (R + delta I) X = S (m x m, 4 right-hand sides) by a
// right-looking FP64 Cholesky, in shared memory when smem != 0 (dynamic size
// (m^2 + 4m) doubles), else in the global work copy Wg.  Thread 0 forms each
// pivot (FP64 division and square root are slow, so they are done once);
// the columns are scaled after the factorisation.  X is written to the own
// tensor in layout [ph][o1][o2][k] = Own[ph][a].  flag[0] |= 1 on a
// non-positive pivot.  skip: if *skip, do nothing.
__global__ void chol_solve_kernel(const double* __restrict__ R, const double* __restrict__ S, int m, double reg,
                                  double* __restrict__ Wg, double* __restrict__ Own, int* flag, const int* skip,
                                  int smem) {
    if (skip && *skip) return;
    extern __shared__ double sh_w[];
    __shared__ double s_delta, s_rd;
    __shared__ double s_sq[512], s_rsq[512];
    double* W = smem ? sh_w : Wg;
    // shared memory: odd row stride, so that walking a column hits distinct banks
    const long long ld = smem ? m + 1 : m;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    if (warp == 0) {
        double tr = 0.0;
        for (int i = lane; i < m; i += 32) tr += R[(long long)i * m + i];
        for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
        if (lane == 0) s_delta = reg * tr / m;
    }
    __syncthreads();
    for (long long e = tid; e < (long long)m * m; e += nt) {
        int i = (int)(e / m), j = (int)(e % m);
        W[i * ld + j] = R[e] + ((i == j) ? s_delta : 0.0);
    }
    double* y = W + (long long)m * ld;  // m x 4
    for (int e = tid; e < 4 * m; e += nt) y[e] = S[e];
    __syncthreads();
    for (int j = 0; j < m; ++j) {
        if (tid == 0) {
            double dj = W[(long long)j * ld + j];
            if (!(dj > 0.0)) { flag[0] |= 1; dj = 1e-300; W[(long long)j * ld + j] = dj; }
            s_rd = rcp_nr(dj);
        }
        __syncthreads();
        const double rd = s_rd;
        for (int i = j + 1 + warp; i < m; i += nw) {             // rows by warps, columns by lanes
            const double lij = W[(long long)i * ld + j] * rd;
            for (int c = j + 1 + lane; c <= i; c += 32) W[(long long)i * ld + c] -= lij * W[(long long)c * ld + j];
        }
        __syncthreads();
    }
    for (int j = tid; j < m; j += nt) {
        const double d = W[(long long)j * ld + j];
        s_rsq[j] = rsqrt_nr(d);
        s_sq[j] = d * s_rsq[j];
    }
    __syncthreads();
    for (long long e = tid; e < (long long)m * m; e += nt) {     // L_ij = a_ij / sqrt(d_j)
        int i = (int)(e / m), j = (int)(e % m);
        if (i > j) W[i * ld + j] *= s_rsq[j];
        else if (i == j) W[i * ld + j] = s_sq[j];
    }
    __syncthreads();
    // forward: L y = S
    for (int j = 0; j < m; ++j) {
        if (tid < 4) y[j * 4 + tid] *= s_rsq[j];
        __syncthreads();
        for (int e = tid; e < (m - j - 1) * 4; e += nt) {
            int i = j + 1 + e / 4, q = e % 4;
            y[i * 4 + q] -= W[(long long)i * ld + j] * y[j * 4 + q];
        }
        __syncthreads();
    }
    // backward: L^T x = y
    for (int j = m - 1; j >= 0; --j) {
        if (tid < 4) y[j * 4 + tid] *= s_rsq[j];
        __syncthreads();
        for (int e = tid; e < j * 4; e += nt) {
            int i = e / 4, q = e % 4;
            y[i * 4 + q] -= W[(long long)j * ld + i] * y[j * 4 + q];
        }
        __syncthreads();
    }
    for (int e = tid; e < 4 * m; e += nt) {
        int a = e / 4, q = e % 4;
        Own[q * m + a] = y[e];
    }
}

// cost d = sum_ph b^T R b - 2 b.S + c, with b = Own (layout [ph][a]); c = cost[0].
// Blocks add partial sums into cost[4]; the last block to finish forms
// d, writes cost[1], compares with the previous value -> done[0], counts the
// iteration in cost[3] and resets the accumulator (counter in done[1]).
// skip: if *skip, do nothing.
__global__ void als_cost_kernel(const double* __restrict__ R, const double* __restrict__ S,
                                const double* __restrict__ Own, int m, double* cost, int* done, double tol,
                                int first, const int* skip) {
    if (skip && *skip) return;
    __shared__ double red[32];
    __shared__ int s_last;
    const int tid = threadIdx.x, nt = blockDim.x;
    const long long gid = blockIdx.x * (long long)nt + tid, gst = (long long)gridDim.x * nt;
    double s = 0.0;
    for (long long e = gid; e < (long long)m * m; e += gst) {
        int a = (int)(e / m), b = (int)(e % m);
        double r = R[e];
        for (int q = 0; q < 4; ++q) s += Own[q * m + a] * r * Own[q * m + b];
    }
    for (long long e = gid; e < 4 * m; e += gst) {
        int a = (int)(e / 4), q = (int)(e % 4);
        s -= 2.0 * Own[q * m + a] * S[e];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((tid & 31) == 0) red[tid >> 5] = s;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < nt / 32; ++w) t += red[w];
        atomicAdd(&cost[4], t);
        __threadfence();
        s_last = (atomicAdd(&done[1], 1) == (int)gridDim.x - 1);
    }
    __syncthreads();
    if (s_last && tid == 0) {
        __threadfence();
        const double t = atomicAdd(&cost[4], 0.0);
        const double c = cost[0];
        const double dnew = t + c;
        if (!first) {
            const double dold = cost[1];
            if (c == 0.0 || fabs(dold - dnew) / c < tol) done[0] = 1;
        }
        cost[1] = dnew;
        cost[3] += 1.0;     // evaluations counted
        cost[4] = 0.0;
        done[1] = 0;
    }
}

// c = <T'|N|T'> = sum_p T'_p N T'_p
__global__ void tnt_kernel(const double* __restrict__ Tp, const double* __restrict__ N, int D4, double* out) {
    double s = 0.0;
    long long tot = 16LL * D4 * D4;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
         i += (long long)gridDim.x * blockDim.x) {
        int p = (int)(i / ((long long)D4 * D4));
        int a = (int)((i / D4) % D4), b = (int)(i % D4);
        s += Tp[(long long)p * D4 + a] * N[(long long)a * D4 + b] * Tp[(long long)p * D4 + b];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

// truncated-SVD start from the singular triplets of Tm (descending sv):
// A''[(sA,aA,u,r)][k] = U[:,k] s_k^{1/2}; colscale for B'' = Tm^T U s^{-1/2}
template <typename TJ>
__global__ void svd_init_kernel(const TJ* Ut, const TJ* sv, int mT, int D, double* A2m, double* colsc, double* Wd) {
    double s0 = (double)sv[0];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < mT * D; i += gridDim.x * blockDim.x) {
        int r = i / D, k = i % D;
        double sk = (k < mT) ? (double)sv[k] : 0.0;
        bool ok = (s0 > 0.0) && (sk > 1e-14 * s0);
        double w = (double)Ut[(long long)r * mT + k];
        A2m[i] = ok ? w * sqrt_nr(sk) : 0.0;
        Wd[i] = w;
        if (r == 0) colsc[k] = ok ? rsqrt_nr(sk) : 0.0;
    }
}

// Start of the wide bonds (4 D^2 > 160, D = 7, 8): the leading left singular
// pairs of Tm from a subspace iteration (engine's bond_start_subspace); U
// (mT x kq, FP64) and the Ritz eigenvalues e (descending) of Tm Tm^T are
// stored as the FP32 triplets svd_init_kernel reads: Ut[r][j] = U[r][j]
// (row stride mT), sv[j] = sqrt(max(e_j, 0)), zero past kq.
__global__ void start_store_kernel(const double* __restrict__ U, const double* __restrict__ ev, int mT, int kq,
                                   float* __restrict__ Ut, float* __restrict__ sv) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < mT * kq; i += gridDim.x * blockDim.x) {
        const int r = i / kq, j = i % kq;
        Ut[(long long)r * mT + j] = (float)U[i];
        if (r == 0) sv[j] = (float)sqrt(fmax(ev[j], 0.0));
    }
    for (int j = kq + blockIdx.x * blockDim.x + threadIdx.x; j < mT; j += gridDim.x * blockDim.x) sv[j] = 0.0f;
}

__global__ void uniform_fill_kernel(double* __restrict__ V, long long n, uint64_t seed, uint64_t stream) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        V[i] = rnd_uniform(seed, stream, (uint64_t)i);
}

// ------------------------------------------------------------------ gauge

__device__ void jacobi_serial(double* A, double* V, int n) {
    for (int i = 0; i < n * n; ++i) V[i] = (i / n == i % n) ? 1.0 : 0.0;
    for (int sw = 0; sw < 60; ++sw) {
        double off = 0.0, dg = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                if (i == j) dg += A[i * n + j] * A[i * n + j];
                else off += A[i * n + j] * A[i * n + j];
            }
        if (off <= 1e-30 * dg || off == 0.0) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = A[p * n + q];
                if (apq == 0.0) continue;
                double tau = (A[q * n + q] - A[p * n + p]) * rcp_nr(2.0 * apq);
                double t = rcp_nr(fabs(tau) + sqrt_nr(1.0 + tau * tau));
                if (tau < 0.0) t = -t;
                double c = rsqrt_nr(1.0 + t * t), s = t * c;
                for (int k = 0; k < n; ++k) {
                    double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - s * akq;
                    A[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - s * aqk;
                    A[q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    double vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = c * vkp - s * vkq;
                    V[k * n + q] = s * vkp + c * vkq;
                }
            }
    }
}

// Balanced gauge: G_A = A^T A, G_B = B^T B (D x D); X = G_A^-1/2 U mu^1/4,
// Y = G_A^1/2 U mu^-1/4 with U mu U^T = G_A^1/2 G_B G_A^1/2 (mu descending);
// A <- A X, B <- B Y; column signs so the largest |A| entry is positive;
// unit Frobenius norms; then written back to the site layouts.
__global__ void gauge_kernel(const double* __restrict__ A2, const double* __restrict__ B2, int D, int gamma,
                             double* __restrict__ Asite, double* __restrict__ Bsite) {
    __shared__ double GA[64], GB[64], WA[64], H[64], Uh[64], SA[64], SAi[64], Xg[64], Yg[64], mu[8], lam[8];
    __shared__ int perm[8];
    __shared__ double sgn[8], nrm[2];
    extern __shared__ double sh[];           // An[mR*D], Bn[mR*D]
    const int tid = threadIdx.x, nt = blockDim.x;
    const int mR = 4 * D * D;                // rows (ph, o1, o2)
    // own layouts: A2[ph][u][r][k] -> row (ph,u,r); B2[ph][d][l][k] -> row (ph,d,l)
    for (int e = tid; e < D * D; e += nt) {
        int i = e / D, j = e % D;
        double sa = 0.0, sb = 0.0;
        for (int r = 0; r < mR; ++r) {
            sa += A2[r * D + i] * A2[r * D + j];
            sb += B2[r * D + i] * B2[r * D + j];
        }
        GA[e] = sa;
        GB[e] = sb;
    }
    __syncthreads();
    if (tid == 0) {
        double tmp[64];
        for (int i = 0; i < D * D; ++i) tmp[i] = GA[i];
        jacobi_serial(tmp, WA, D);
        double lmax = 0.0;
        for (int i = 0; i < D; ++i) { lam[i] = tmp[i * D + i]; lmax = fmax(lmax, lam[i]); }
        for (int i = 0; i < D; ++i)
            for (int j = 0; j < D; ++j) {
                double a = 0.0, b = 0.0;
                for (int k = 0; k < D; ++k) {
                    bool ok = lam[k] > 1e-28 * lmax && lam[k] > 0.0;
                    double isq = ok ? rsqrt_nr(lam[k]) : 0.0;
                    double sq = ok ? lam[k] * isq : 0.0;
                    a += WA[i * D + k] * sq * WA[j * D + k];
                    b += WA[i * D + k] * isq * WA[j * D + k];
                }
                SA[i * D + j] = a;
                SAi[i * D + j] = b;
            }
        // H = SA GB SA
        for (int i = 0; i < D; ++i)
            for (int j = 0; j < D; ++j) {
                double s = 0.0;
                for (int a = 0; a < D; ++a)
                    for (int b = 0; b < D; ++b) s += SA[i * D + a] * GB[a * D + b] * SA[b * D + j];
                H[i * D + j] = s;
            }
        for (int i = 0; i < D * D; ++i) tmp[i] = H[i];
        jacobi_serial(tmp, Uh, D);
        // sort descending
        for (int i = 0; i < D; ++i) perm[i] = i;
        for (int i = 0; i < D; ++i)
            for (int j = i + 1; j < D; ++j)
                if (tmp[perm[j] * D + perm[j]] > tmp[perm[i] * D + perm[i]]) { int t = perm[i]; perm[i] = perm[j]; perm[j] = t; }
        double m0 = tmp[perm[0] * D + perm[0]];
        for (int c = 0; c < D; ++c) {
            int src = perm[c];
            mu[c] = tmp[src * D + src];
            bool ok = m0 > 0.0 && mu[c] > 1e-28 * m0;
            const double r2 = ok ? sqrt_nr(mu[c]) : 0.0;                 // mu^(1/2)
            double q4 = ok ? sqrt_nr(r2) : 0.0, iq4 = ok ? rsqrt_nr(r2) : 0.0;
            for (int i = 0; i < D; ++i) {
                double x = 0.0, y = 0.0;
                for (int a = 0; a < D; ++a) {
                    x += SAi[i * D + a] * Uh[a * D + src];
                    y += SA[i * D + a] * Uh[a * D + src];
                }
                Xg[i * D + c] = x * q4;
                Yg[i * D + c] = y * iq4;
            }
        }
    }
    __syncthreads();
    double* An = sh;
    double* Bn = sh + mR * D;
    for (int e = tid; e < mR * D; e += nt) {
        int r = e / D, c = e % D;
        double a = 0.0, b = 0.0;
        for (int k = 0; k < D; ++k) {
            a += A2[r * D + k] * Xg[k * D + c];
            b += B2[r * D + k] * Yg[k * D + c];
        }
        An[e] = a;
        Bn[e] = b;
    }
    __syncthreads();
    if (tid < D) {
        int c = tid;
        double best = 0.0, v = 0.0;
        for (int r = 0; r < mR; ++r) {
            double x = An[r * D + c];
            if (fabs(x) > best) { best = fabs(x); v = x; }
        }
        sgn[c] = (v < 0.0) ? -1.0 : 1.0;
    }
    if (tid == 0) {
        double sa = 0.0, sb = 0.0;
        for (int e = 0; e < mR * D; ++e) { sa += An[e] * An[e]; sb += Bn[e] * Bn[e]; }
        nrm[0] = sa > 0.0 ? rsqrt_nr(sa) : 1.0;
        nrm[1] = sb > 0.0 ? rsqrt_nr(sb) : 1.0;
    }
    __syncthreads();
    // write back: A''[ph][u][r][k] -> Asite[ph][x][y][z] with u = alpha', r = alpha, k = gamma
    int str[3] = {D * D, D, 1};
    int al = (gamma + 1) % 3, alp = (gamma + 2) % 3;
    const int D3 = D * D * D;
    for (int e = tid; e < mR * D; e += nt) {
        int r = e / D, c = e % D;
        int ph = r / (D * D), o1 = (r / D) % D, o2 = r % D;
        int off = ph * D3 + o1 * str[alp] + o2 * str[al] + c * str[gamma];
        Asite[off] = An[e] * sgn[c] * nrm[0];
        Bsite[off] = Bn[e] * sgn[c] * nrm[1];
    }
}

// Gradient of the bond cost d = <T''-T'|N|T''-T'> with respect to one factor
// (Own, layout [ph][a], a = (o1, o2, k)) with the other fixed, from the
// normal-equation matrices of that side (d = sum_ph Own_ph^T R Own_ph
// - 2 sum Own[ph][a] S[a][ph] + <T'|N|T'>):
//   G[ph][a] = sum_a' (R[a][a'] + R[a'][a]) Own[ph][a'] - 2 S[a][ph];
// the quadratic and linear parts of d are added into *e.
__global__ void cost_grad_kernel(const double* __restrict__ R, const double* __restrict__ S,
                                 const double* __restrict__ Own, int m, double* __restrict__ G, double* e) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 4 * m; i += gridDim.x * blockDim.x) {
        const int ph = i / m, a = i % m;
        const double* own = Own + (long long)ph * m;
        double sym = 0.0, row = 0.0;
        for (int b = 0; b < m; ++b) {
            const double r1 = R[(long long)a * m + b], r2 = R[(long long)b * m + a];
            sym += (r1 + r2) * own[b];
            row += r1 * own[b];
        }
        const double sa = S[(long long)a * 4 + ph];
        G[i] = sym - 2.0 * sa;
        atomicAdd(e, own[a] * (row - 2.0 * sa));
    }
}

template <typename T>
void Engine<T>::normal_equations(const double* oth, int side, const int* skip) {
    const int D = dm.D, D4 = dm.D4, m = D * D * D;
    const int threads = 256;
    const long long nX = 4LL * dm.d2 * D4 * D, nR = (long long)m * m;
    const int sgrid = (int)((4LL * m * 32 + threads - 1) / threads);
    als_x_kernel<<<grid_for(nX), threads, 0, st>>>(N, oth, D, side, XA, skip);
    KH_LAUNCHED();
    als_r_kernel<<<grid_for(nR), threads, 0, st>>>(XA, oth, D, side, R, skip);
    KH_LAUNCHED();
    als_s_kernel<<<sgrid, threads, 0, st>>>(XA, slots[als_slot].Ts, D, side, S, skip);
    KH_LAUNCHED();
}

template <typename T>
void Engine<T>::cost_gradient(int gamma, const double* gate, const double* A2in, const double* B2in, int mx, int mn,
                              double tol, double* gA, double* gB, double* cost_out) {
    if (gamma < 0 || gamma > 2) fail(KH_EINVAL, "gamma must be 0, 1 or 2");
    if (dm.nslots < 3) fail(KH_EINVAL, "eeFU needs n_slots >= 3");
    if (mx < 0) fail(KH_EINVAL, "ctm_max_sweeps < 0");
    Slot<T>& sl = slots[gamma];
    if (mx == 0 && !sl.env_valid) fail(KH_EINVAL, "no environment to reuse (ctm_max_sweeps = 0)");
    build_composite(gamma, gamma, gate);
    if (mx > 0) {
        double delta = 0.0;
        sweep(gamma, mx, mn, tol, &delta);
    } else {
        refresh_operands(sl);
    }
    compute_metric(sl, N);
    const int D = dm.D, m = D * D * D;
    const long long own = 4LL * m;
    KH_CUDA(cudaMemcpyAsync(A2, A2in, sizeof(double) * own, cudaMemcpyDeviceToDevice, st));
    KH_CUDA(cudaMemcpyAsync(B2, B2in, sizeof(double) * own, cudaMemcpyDeviceToDevice, st));
    KH_CUDA(cudaMemsetAsync(cost, 0, 8 * sizeof(double), st));
    tnt_kernel<<<grid_for(16LL * dm.D4 * dm.D4), 256, 0, st>>>(sl.Ts, N, dm.D4, cost);
    KH_LAUNCHED();
    als_slot = gamma;
    normal_equations(B2, 0, nullptr);                      // A side (B'' fixed)
    cost_grad_kernel<<<grid_for(own), 256, 0, st>>>(R, S, A2, m, gA, cost + 5);
    KH_LAUNCHED();
    normal_equations(A2, 1, nullptr);                      // B side (A'' fixed)
    cost_grad_kernel<<<grid_for(own), 256, 0, st>>>(R, S, B2, m, gB, cost + 6);
    KH_LAUNCHED();
    double h[8];
    KH_CUDA(cudaMemcpyAsync(h, cost, sizeof(h), cudaMemcpyDeviceToHost, st));
    KH_CUDA(cudaStreamSynchronize(st));
    if (!(h[5] == h[5]) || !(h[6] == h[6])) fail(KH_ENUMERIC, "NaN in the bond cost");
    cost_out[0] = h[5] + h[0];          // d from the A side
    cost_out[1] = h[0];                 // <T'|N|T'>
    cost_out[2] = h[6] + h[0];          // d from the B side (equal up to rounding)
}

// ------------------------------------------------------------------ ALS driver

// Leading left singular vectors of Tm (mT x mT, FP64) for the start of a bond
// too wide for the one-CTA Jacobi (4 D^2 > 160): subspace iteration on
// Tm Tm^T with a block of kq = D + 8 columns from a seeded uniform draw,
// V <- orth(Tm (Tm^T V)) (ordered CholQR2) twelve times, then the
// Rayleigh-Ritz step H = Z^T Z with Z = Tm^T V, H = W diag(e) W^T (Jacobi),
// U = V W.  The start only seeds the ALS, which converges in FP64.  Scratch:
// Gt (four mT x kq blocks), Wt (kq x kq blocks).
template <typename T>
void Engine<T>::bond_start_subspace(int mT, int D) {
    const int kq = std::min(mT, D + 8);
    const long long blk = (long long)mT * kq;
    double *V = Gt, *Z = Gt + blk, *Y = Gt + 2 * blk, *tmp = Gt + 3 * blk;
    double *Xk = Wt, *dG = Wt + kq * kq, *H = Wt + 2 * kq * kq, *W = Wt + 3 * kq * kq, *ev = Wt + 4 * kq * kq;
    uniform_fill_kernel<<<grid_for(blk), 256, 0, st>>>(V, blk, cfg.seed, 0xb0adULL);
    KH_LAUNCHED();
    for (int it = 0; it < 12; ++it) {
        gemm_rm<double>(mT, kq, mT, Tm, true, V, false, Z, st);     // Z = Tm^T V
        gemm_rm<double>(mT, kq, mT, Tm, false, Z, false, Y, st);    // Y = Tm Z
        cholqr2<double>(Y, mT, kq, 1e-12, tmp, Xk, dG, V, st);
    }
    gemm_rm<double>(mT, kq, mT, Tm, true, V, false, Z, st);
    gemm_rm<double>(kq, kq, mT, Z, true, Z, false, H, st);          // H = Z^T Z
    jacobi_eig<double>(H, kq, kq, 0, W, kq, 0, ev, 0, 1, 60, 1e-14, nullptr, nullptr, st);
    gemm_rm<double>(mT, kq, kq, V, false, W, false, Y, st);         // U = V W
    start_store_kernel<<<grid_for(blk), 256, 0, st>>>(Y, ev, mT, kq, Wtf, Ltf);
    KH_LAUNCHED();
}

template <typename T>
int Engine<T>::als_run(int gamma, double* rel_cost) {
    const int D = dm.D, D4 = dm.D4, m = D * D * D, mT = 4 * dm.d2;
    Slot<T>& sl = slots[gamma];
    const double* Tp = sl.Ts;
    // <T'|N|T'>
    KH_CUDA(cudaMemsetAsync(cost, 0, 8 * sizeof(double), st));
    KH_CUDA(cudaMemsetAsync(flags, 0, 8 * sizeof(int), st));
    tnt_kernel<<<grid_for(16LL * D4 * D4), 256, 0, st>>>(Tp, N, D4, cost);
    KH_LAUNCHED();
    // truncated SVD start: Tm[(sA,aA,u,r)][(sB,aB,d,l)] from T'[sA,aA,sB,aB,l,u,r,d]
    permute<double, double>(Tp, Tm, {2, 2, 2, 2, D, D, D, D}, {0, 1, 5, 6, 2, 3, 7, 4}, st);
    double* colsc = dwork;
    double* Wd = dwork + 64;
    // The start only seeds the ALS, which then converges to tolerance in
    // FP64, so the singular vectors come from the FP32 one-sided Jacobi of
    // Tm^T (Tm^T Q = L S, so Tm = Q S L^T and U = Q); only the D leading
    // triplets are used, so only the D + 4 largest columns must converge
    // (the near-null tail of Tm would otherwise keep the sweeps going).
    if (mT <= jacobi_kmax<float>()) {
        permute<double, float>(Tm, Gtf, {mT, mT}, {1, 0}, st);
        svd_jacobi<float>(Gtf, mT, Ltf, (float*)Gt, Wtf, 60, 2e-6, 0.0, st, nullptr, D + 4);
    } else {
        bond_start_subspace(mT, D);
    }
    svd_init_kernel<float><<<grid_for(mT * D), 256, 0, st>>>(Wtf, Ltf, mT, D, A2, colsc, Wd);
    KH_LAUNCHED();
    // B''[(sB,aB,d,l)][k] = sum_i Tm[i][.] Wd[i][k] colsc[k]
    gemm_rm<double>(mT, D, mT, Tm, true, Wd, false, B2, st, 1.0, 0.0, colsc);
    // initial cost with (A'', B'') from the start: B-side normal equations from A''
    const int threads = 256;
    const long long nR = (long long)m * m;
    const int cgrid = (int)std::min<long long>(32, (nR + threads - 1) / threads);
    const size_t chol_sm = sizeof(double) * ((size_t)m * (m + 1) + 4 * m);
    const int chol_smem = chol_sm <= 200 * 1024 ? 1 : 0;
    if (chol_smem) {
        static std::atomic<size_t> granted[kMaxDevices] = {};
        smem_opt_in(chol_solve_kernel, chol_sm, granted);
    }
    const int* done = flags + 1;
    als_slot = gamma;
    auto normal_eqs = [&](const double* oth, int side) { normal_equations(oth, side, done); };
    normal_eqs(A2, 1);
    als_cost_kernel<<<cgrid, threads, 0, st>>>(R, S, B2, m, cost, flags + 1, cfg.als_tol, 1, nullptr);
    KH_LAUNCHED();
    // Sweeps run on the device until the relative cost change is below the
    // tolerance (flags[1] set by the cost kernel, after which every kernel of
    // the loop returns at once); the host looks at the flags every few sweeps.
    constexpr int kCheckEvery = 4;
    for (int it = 1; it <= cfg.als_max_iter; ++it) {
        normal_eqs(B2, 0);                                   // A step (fixed B'')
        chol_solve_kernel<<<1, 512, chol_smem ? chol_sm : 0, st>>>(R, S, m, cfg.als_reg, Xmat, A2, flags, done,
                                                                   chol_smem);
        KH_LAUNCHED();
        normal_eqs(A2, 1);                                   // B step (fixed A'')
        chol_solve_kernel<<<1, 512, chol_smem ? chol_sm : 0, st>>>(R, S, m, cfg.als_reg, Xmat, B2, flags, done,
                                                                   chol_smem);
        KH_LAUNCHED();
        als_cost_kernel<<<cgrid, threads, 0, st>>>(R, S, B2, m, cost, flags + 1, cfg.als_tol, 0, done);
        KH_LAUNCHED();
        if (it % kCheckEvery == 0 || it == cfg.als_max_iter) {
            int hf[2];
            KH_CUDA(cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, st));
            KH_CUDA(cudaStreamSynchronize(st));
            if (hf[0]) fail(KH_ENUMERIC, "ALS: Cholesky breakdown (metric not positive)");
            if (hf[1]) break;
        }
    }
    double hc[4];
    int hf0 = 0;
    KH_CUDA(cudaMemcpyAsync(hc, cost, sizeof(hc), cudaMemcpyDeviceToHost, st));
    KH_CUDA(cudaMemcpyAsync(&hf0, flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    KH_CUDA(cudaStreamSynchronize(st));
    if (hf0) fail(KH_ENUMERIC, "ALS: Cholesky breakdown (metric not positive)");
    *rel_cost = hc[0] != 0.0 ? hc[1] / hc[0] : 0.0;
    return (int)hc[3] - 1;                                   // sweeps (the first evaluation is the start)
}

template <typename T>
void Engine<T>::gauge_and_store(int gamma) {
    const int D = dm.D, mR = 4 * D * D;
    size_t sm = sizeof(double) * 2 * mR * D;
    gauge_kernel<<<1, 256, sm, st>>>(A2, B2, D, gamma, A, B);
    KH_LAUNCHED();
}

template <typename T>
void Engine<T>::apply_gate(int gamma, const double* gate, int mx, int mn, double tol, double* info) {
    if (gamma < 0 || gamma > 2) fail(KH_EINVAL, "gamma must be 0, 1 or 2");
    if (dm.nslots < 3) fail(KH_EINVAL, "eeFU needs n_slots >= 3");
    build_composite(gamma, gamma, gate);
    double delta = 0.0;
    int sw = sweep(gamma, mx, mn, tol, &delta);
    compute_metric(slots[gamma], N);
    double rel = 0.0;
    prof_begin(6);
    int it = als_run(gamma, &rel);
    gauge_and_store(gamma);
    prof_end(6, 0.0);
    if (info) {
        double tr[4];
        KH_CUDA(cudaMemcpyAsync(tr, slots[gamma].trunc, sizeof(tr), cudaMemcpyDeviceToHost, st));
        KH_CUDA(cudaStreamSynchronize(st));
        info[0] = rel;
        info[1] = sw;
        info[2] = it;
        info[3] = fmax(fmax(tr[0], tr[1]), fmax(tr[2], tr[3]));
    }
}

// ------------------------------------------------------------------ observables

// X[p][q] = (T N T^T)[p][q] for the three mappings -> E_site etc.
__global__ void obs_kernel(const double* __restrict__ Xs, Mat4x3 H, double hA, double hB, double* out) {
    if (threadIdx.x != 0) return;
    double Hg[3];
    for (int g = 0; g < 3; ++g) {
        const double* X = Xs + g * 256;
        double tr = 0.0, s = 0.0;
        for (int a = 0; a < 16; ++a) tr += X[a * 16 + a];
        // sum H4[(sA' sB'),(sA sB)] X[(sA',aA,sB',aB)][(sA,aA,sB,aB)]
        for (int sAo = 0; sAo < 2; ++sAo)
            for (int sBo = 0; sBo < 2; ++sBo)
                for (int sA = 0; sA < 2; ++sA)
                    for (int sB = 0; sB < 2; ++sB) {
                        double h = H.v[g * 16 + (sAo * 2 + sBo) * 4 + sA * 2 + sB];
                        if (h == 0.0) continue;
                        for (int aA = 0; aA < 2; ++aA)
                            for (int aB = 0; aB < 2; ++aB) {
                                int pa = ((sAo * 2 + aA) * 2 + sBo) * 2 + aB;
                                int pb = ((sA * 2 + aA) * 2 + sB) * 2 + aB;
                                s += h * X[pa * 16 + pb];
                            }
                    }
        Hg[g] = s / tr;
    }
    // site moments from the z mapping: S^x = sigma^x/2, S^z = sigma^z/2 (S^y gives 0 on real X)
    const double* X = Xs + 2 * 256;
    double tr = 0.0;
    for (int a = 0; a < 16; ++a) tr += X[a * 16 + a];
    double sxA = 0, szA = 0, sxB = 0, szB = 0;
    for (int a = 0; a < 16; ++a) {
        int sA = (a >> 3) & 1, sB = (a >> 1) & 1;
        szA += (sA ? -0.5 : 0.5) * X[a * 16 + a];
        szB += (sB ? -0.5 : 0.5) * X[a * 16 + a];
        sxA += 0.5 * X[(a ^ 8) * 16 + a];
        sxB += 0.5 * X[(a ^ 2) * 16 + a];
    }
    sxA /= tr; szA /= tr; sxB /= tr; szB /= tr;
    out[0] = 0.5 * (Hg[0] + Hg[1] + Hg[2]) - 0.5 * (hA * szA + hB * szB);
    out[1] = Hg[0]; out[2] = Hg[1]; out[3] = Hg[2];
    out[4] = sxA; out[5] = 0.0; out[6] = szA;
    out[7] = sxB; out[8] = 0.0; out[9] = szB;
}

template <typename T>
void Engine<T>::observables(const double* Hh, double hA, double hB, int mx, int mn, double tol, double* out) {
    if (dm.nslots < 6) fail(KH_EINVAL, "observables need n_slots >= 6");
    // The three mappings are independent CTMRG problems: slot 3 + g runs on
    // lane g (its own scratch and stream), forked from and joined back to the
    // context's stream.
    struct Rebind {
        Engine* e;
        ~Rebind() { e->bind(0); }
    } rebind{this};
    const int nl = nlanes >= 3 ? 3 : 1;
    auto lane_of = [&](int g) { return nl == 3 ? g : 0; };
    bind(0);
    if (nl == 3) {
        KH_CUDA(cudaEventRecord(lane_ev[0], lanes[0].st));
        for (int i = 1; i < 3; ++i) KH_CUDA(cudaStreamWaitEvent(lanes[i].st, lane_ev[0], 0));
    }
    for (int g = 0; g < 3; ++g) {
        bind(lane_of(g));
        const int s = 3 + g;
        if (!slots[s].env_valid || slots[s].p == 0) {
            if (slots[g].p != 0) copy_env(s, g);
            else init_env(s, nullptr);
        }
        build_composite(s, g, nullptr);
    }
    int sweeps = 0;
    if (nl == 3) {
        const int ids[3] = {3, 4, 5};
        sweeps = sweep_lanes(ids, 3, mx, mn, tol);
    } else {
        for (int g = 0; g < 3; ++g) sweeps += sweep(3 + g, mx, mn, tol, nullptr);
    }
    for (int g = 0; g < 3; ++g) {
        bind(lane_of(g));
        const int s = 3 + g;
        compute_metric(slots[s], N);
        gemm_rm<double>(16, dm.D4, dm.D4, slots[s].Ts, false, N, false, dwork, st);
        gemm_rm<double>(16, 16, dm.D4, dwork, false, slots[s].Ts, true, Xs + g * 256, st);
    }
    if (nl == 3) {
        for (int i = 1; i < 3; ++i) {
            KH_CUDA(cudaEventRecord(lane_ev[i], lanes[i].st));
            KH_CUDA(cudaStreamWaitEvent(lanes[0].st, lane_ev[i], 0));
        }
    }
    bind(0);
    Mat4x3 H;
    for (int i = 0; i < 48; ++i) H.v[i] = Hh[i];
    double* dout = dscr + DscrOff::kObsOut;
    obs_kernel<<<1, 32, 0, st>>>(Xs, H, hA, hB, dout);
    KH_LAUNCHED();
    double tr[12];
    KH_CUDA(cudaMemcpyAsync(out, dout, sizeof(double) * 10, cudaMemcpyDeviceToHost, st));
    for (int g = 0; g < 3; ++g)
        KH_CUDA(cudaMemcpyAsync(tr + 4 * g, slots[3 + g].trunc, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
    KH_CUDA(cudaStreamSynchronize(st));
    double mt = 0.0;
    for (int i = 0; i < 12; ++i) mt = fmax(mt, tr[i]);
    out[10] = mt;
    out[11] = sweeps;
}

template struct Engine<double>;
template struct Engine<float>;

}  // namespace kh
