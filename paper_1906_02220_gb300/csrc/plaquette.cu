// Products of operators on a 2 x 2 plaquette of the square lattice and the
// plaquette flux W of the hexagonal lattice (Sec. V: the average of Kitaev's
// plaquette operator, whose ordering marks the lower crossover of the pure
// Kitaev model).
//
// The cluster of four sites in the CTM environment is the ring of the four
// enlarged corners of one plaquette, Z = Tr(Q_0 Q_1 Q_2 Q_3): Q_f is the
// enlarged corner of frame f (0 upper-left, 1 upper-right, 2 lower-right,
// 3 lower-left: the frame-f corner C_f E_f E_{f+3} and the site turned f
// quarters), contracted exactly as in a CTM move (edge GEMMs, then the
// two-layer site contraction) and stored as [(w, dk, db)][(z, rk, rb)] -- the
// row index is the cut to the previous corner of the ring, the column index
// the cut to the next one, so consecutive corners chain as matrices.  An
// operator O_f at position f enters through the ket layer of corner f's site
// contraction (ket operand O_f T, bra operand T), and
//   <O_0 O_1 O_2 O_3> = Z[O] / Z[1].
// Both clusters run through the same kernels (the plain one with O = 1), so
// the ratio sees the same rounding in numerator and denominator.
#include "engine.cuh"
#include "layered.cuh"

namespace kh {

namespace {

// out += sum_i a[i] b[i], FP64 accumulation, one atomic per warp
template <typename T>
__global__ void dot64_kernel(const T* __restrict__ a, const T* __restrict__ b, long long n, double* out) {
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        s += (double)a[i] * (double)b[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

}  // namespace

// Pauli matrices in the basis s = 0 (S^z = +1/2), 1; sigma^y = i Yt.
static const double kPauliX[4] = {0.0, 1.0, 1.0, 0.0};
static const double kPauliYt[4] = {0.0, -1.0, 1.0, 0.0};
static const double kPauliZ[4] = {1.0, 0.0, 0.0, -1.0};
static const double kId2[4] = {1.0, 0.0, 0.0, 1.0};

// 16 x 16 operator OA (x) 1_aA (x) OB (x) 1_aB on p = (sA, aA, sB, aB)
static void composite_op(const double* OA, const double* OB, double* out) {
    for (int r = 0; r < 16; ++r)
        for (int c = 0; c < 16; ++c) {
            const int sa = r >> 3, aa = (r >> 2) & 1, sb = (r >> 1) & 1, ab = r & 1;
            const int ta = c >> 3, ba = (c >> 2) & 1, tb = (c >> 1) & 1, bb = c & 1;
            out[r * 16 + c] = (aa == ba && ab == bb) ? OA[sa * 2 + ta] * OB[sb * 2 + tb] : 0.0;
        }
}

// Geometry of the gamma mapping: composite (i, j) holds A(i,j), B(i,j)
// joined by gamma; its leg r = A.alpha meets leg l = B.alpha of composite
// (i+1, j), its leg u = A.alpha' meets leg d = B.alpha' of (i, j+1) above,
// with (alpha, alpha') = (gamma+1, gamma+2) mod 3.  The hexagon
//   A(0,0) -alpha- B(1,0) -gamma- A(1,0) -alpha'- B(1,1) -alpha- A(0,1)
//          -gamma- B(0,1) -alpha'- A(0,0)
// spans the plaquette (0,1) upper-left, (1,1) upper-right, (1,0) lower-right,
// (0,0) lower-left; at each site W_p takes the Pauli component of the bond
// leaving the hexagon there.
void flux_operators(int gamma, double* ops) {
    const double* pauli[3] = {kPauliX, kPauliYt, kPauliZ};
    const int al = (gamma + 1) % 3, alp = (gamma + 2) % 3;
    composite_op(pauli[alp], pauli[al], ops);              // (0,1): A alpha', B alpha
    composite_op(kId2, pauli[gamma], ops + 256);           // (1,1): B gamma
    composite_op(pauli[al], pauli[alp], ops + 512);        // (1,0): A alpha, B alpha'
    composite_op(pauli[gamma], kId2, ops + 768);           // (0,0): A gamma
}

// Enlarged corner of frame f with ket operand Tk (FP64 [p][D^4], frame-0
// legs) and the slot's own tensor as the bra operand, into out as
// [(w, dk, db)][(z, rk, rb)].  Scratch: X1[0], Y1, Yp, Qt (Zk on the CUDA
// cores), the plaquette's operand buffers.
template <typename T>
void Engine<T>::plaquette_corner(Slot<T>& sl, int f, const double* Tk, T* out) {
    const int chi = dm.chi, d2 = dm.d2, D = dm.D, p = sl.p;
    const long long chi2 = (long long)chi * chi, E1 = (long long)chi * d2 * chi;
    const T* C1 = Cop + f * chi2;
    const T* E1p = Eop + f * E1;
    const T* E4 = Eop + ((f + 3) & 3) * E1;
    gemm_rm<T>(chi, d2 * chi, chi, C1, false, E1p, false, X1[0], st);            // [x4][(uk,ub,z)]
    gemm_rm<T>(chi * d2, d2 * chi, chi, E4, false, X1[0], false, Y1, st);        // [(w,lk,lb)][(uk,ub,z)]
    permute<T, T>(Y1, Yp, {chi, D, D, D, D, chi}, {0, 5, 2, 4, 1, 3}, st);      // [w][z][lb][ub][lk][uk]
    if (dm.lay) {
        build_layered_images(Tk, p, D, dm.npass, dm.bf16, (float*)pq_img1, (float*)pq_img2, dm.lay1, dm.lay2, st,
                             sl.Ts);
        site_layer(Yp, chi2, nullptr, pq_img1 + f * dm.lay1, pq_img2 + f * dm.lay2, p, Qt, nullptr, nullptr);
    } else {
        derive_operands<T>(Tk, p, D, dm.pmax, pq_cor, pq_edg, st);
        const long long fo = (long long)f * dm.pmax * dm.D4;
        site_layer(Yp, chi2, pq_cor + fo, nullptr, nullptr, p, Qt, nullptr, nullptr, false, sl.Tcor + fo);
    }
    permute<T, T>(Qt, out, {chi, chi, D, D, D, D}, {0, 3, 5, 1, 2, 4}, st);     // [(w,dk,db)][(z,rk,rb)]
}

template <typename T>
void Engine<T>::plaquette(int slot, const double* ops, double* out) {
    Slot<T>& sl = slots[slot];
    if (sl.p <= 0 || !sl.env_valid) fail(KH_EINVAL, "slot has no tensor or environment");
    const int p = sl.p, n = dm.n;             // p <= p_max <= 16: four p x p operators fit the staging area
    const long long nn = (long long)n * n;
    refresh_operands(sl);
    double* dops = dscr + DscrOff::kStage;             // 4 p^2 <= 1024 doubles
    double* z = dscr + DscrOff::kExpvalOut;            // Z[1], Z[O]
    KH_CUDA(cudaMemcpyAsync(dops, ops, sizeof(double) * 4 * p * p, cudaMemcpyHostToDevice, st));
    KH_CUDA(cudaMemsetAsync(z, 0, 2 * sizeof(double), st));
    for (int pass = 0; pass < 2; ++pass) {             // 0: the plain cluster, 1: with the operators
        for (int half = 0; half < 2; ++half) {
            for (int q = 0; q < 2; ++q) {
                const int f = 2 * half + q;
                const double* Tk = sl.Ts;
                if (pass == 1) {                       // O_f T: [p'][D^4] = O_f[p'][p] T[p][D^4]
                    gemm_rm<double>(p, dm.D4, p, dops + (long long)f * p * p, false, sl.Ts, false, pq_T, st);
                    Tk = pq_T;
                }
                plaquette_corner(sl, f, Tk, Q[q]);
            }
            if (half == 0)                             // Q_0 Q_1
                gemm_rm<T>(n, n, n, Q[0], false, Q[1], false, Mt, st);
            else                                       // (Q_2 Q_3)^T = Q_3^T Q_2^T
                gemm_rm<T>(n, n, n, Q[1], true, Q[0], true, mup, st);
        }
        // Tr(Q_0 Q_1 Q_2 Q_3) = sum_ij (Q_0 Q_1)[i][j] ((Q_2 Q_3)^T)[i][j]
        dot64_kernel<T><<<sumsq_grid(nn), 256, 0, st>>>(Mt, mup, nn, z + pass);
        KH_LAUNCHED();
    }
    double h[2];
    int terr = 0;
    KH_CUDA(cudaMemcpyAsync(h, z, sizeof(h), cudaMemcpyDeviceToHost, st));
    if (tc_npass) KH_CUDA(cudaMemcpyAsync(&terr, tc_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    KH_CUDA(cudaStreamSynchronize(st));
    if (terr) fail(KH_ETIMEOUT, "tensor-core kernel wait timed out (flag " + std::to_string(terr) + ")");
    if (!(h[0] == h[0]) || !(h[1] == h[1]) || h[0] == 0.0 || std::isinf(h[0]) || std::isinf(h[1]))
        fail(KH_ENUMERIC, "plaquette cluster zero or not finite");
    out[0] = h[1] / h[0];
    out[1] = h[0];
}

template struct Engine<double>;
template struct Engine<float>;

}  // namespace kh
