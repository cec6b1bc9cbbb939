// CTMRG on the rhombic (square) lattice of composites, Fig. 4(c) and Sec. III
// of arXiv:1906.02220.  Ket and bra layers are contracted separately (the
// D^2 double-layer index is never formed): every enlarged corner and every
// edge absorption applies the site tensor twice, once per layer.
//
// One move (the left move in a frame rotated by s quarter turns):
//   Q_f   = C1 E1 E4 (T, T)         upper-left enlarged corner of frame f,
//           rows c = (E4 leg, d_ket, d_bra), cols (E1 leg, r_ket, r_bra);
//   the lower-left corner of frame s is Q_{s+3}^T, so the half-system
//   product is M = Q_s^T Q_{s+3}^T and we form Mt = M^T = Q_{s+3} Q_s;
//   top-chi SVD M = U S V^T by subspace iteration with Rayleigh-Ritz steps
//   (Jacobi on the k x k Gram matrices), warm-started from the previous
//   subspace of the same direction;
//   P = Q_{s+3}^T V S^-1/2, P~^T = Q_s U S^-1/2;
//   C1 <- P^T (C1 E1), C4 <- (C4 E3) P~^T, E4 <- P^T (E4 T T) P~^T,
//   each divided by its Frobenius norm (FP64).
#define KH_JACOBI_KERNEL
#include "engine.cuh"
#include "layered.cuh"

namespace kh {

// ------------------------------------------------------------------ config

void validate(const kh_config& c) {
    if (c.D < 1 || c.D > 8) fail(KH_EINVAL, "D must be in [1, 8]");
    if (c.chi < 1 || c.chi > 256) fail(KH_EINVAL, "chi must be in [1, 256]");
    if (c.prec < KH_FP64 || c.prec > KH_BF16) fail(KH_EINVAL, "unknown precision");
    if (c.n_slots < 1 || c.n_slots > 16) fail(KH_EINVAL, "n_slots must be in [1, 16]");
    if (c.p_max < 1 || c.p_max > 16) fail(KH_EINVAL, "p_max must be in [1, 16]");
    if (c.svd_oversample < 0 || c.svd_iters_cold < 1 || c.svd_iters_warm < 1)
        fail(KH_EINVAL, "bad subspace iteration settings");
    if (c.jacobi_max_sweeps < 1) fail(KH_EINVAL, "jacobi_max_sweeps < 1");
    if (!(c.svd_cut >= 0.0) || !(c.als_reg >= 0.0) || c.als_max_iter < 0) fail(KH_EINVAL, "bad tolerances");
    if (c.proj_fp64 != 0 && c.proj_fp64 != 1) fail(KH_EINVAL, "proj_fp64 must be 0 or 1");
    if (c.site_form < 0 || c.site_form > 2) fail(KH_EINVAL, "site_form must be 0, 1 or 2");
}

Dims make_dims(const kh_config& c, bool fp64) {
    Dims d;
    d.D = c.D;
    d.d2 = c.D * c.D;
    d.D4 = d.d2 * d.d2;
    d.chi = c.chi;
    d.n = c.chi * d.d2;
    d.pmax = c.p_max;
    d.nslots = c.n_slots;
    d.npass = fp64 ? 0 : ((c.prec == KH_TF32 || c.prec == KH_BF16) ? 1 : (c.prec == KH_TF32X3 ? 3 : 0));
    d.bf16 = !fp64 && c.prec == KH_BF16;
    // site contraction form: layered on the tensor cores unless the double-layer
    // operand is asked for; on the CUDA cores the double-layer operand where it
    // halves the flops, unless the layered form is asked for
    d.dl_alloc = d.d2 <= 2 * c.p_max && (c.site_form == 2 || (c.site_form == 0 && d.npass == 0));
    d.lay = d.npass != 0;
    d.lay1 = d.lay ? layered_img1_floats(c.D, c.p_max, d.npass, d.bf16) : 0;
    d.lay2 = d.lay ? layered_img2_floats(c.D, c.p_max, d.npass, d.bf16) : 0;
    if (d.lay && (d.lay1 == 0 || d.lay2 == 0)) fail(KH_EINVAL, "no tensor-core plan for this D");
    int kmax = fp64 ? 112 : 160;      // the one-CTA Jacobi limits (FP64, FP32)
    if (d.n <= kmax) {
        d.kk = d.n;
        d.full = true;
    } else {
        d.kk = c.chi + c.svd_oversample;
        if (d.kk > d.n) d.kk = d.n;
        d.full = false;
        if (d.kk > kmax) fail(KH_EINVAL, "chi + svd_oversample exceeds the Jacobi limit");
    }
    return d;
}

template <typename T>
void Engine<T>::layout(Carver& cv) {
    const Dims& d = dm;
    const long long chi2 = (long long)d.chi * d.chi, E1 = (long long)d.chi * d.d2 * d.chi;
    const long long n = d.n, n2 = n * n, D3 = (long long)d.D * d.D * d.D, kk = d.kk;
    A = cv.take<double>(4 * D3);
    B = cv.take<double>(4 * D3);
    slots.assign(d.nslots, Slot<T>());
    for (auto& s : slots) {
        s.Ts = cv.take<double>((long long)d.pmax * d.D4);
        s.C = cv.take<double>(4 * chi2);
        s.E = cv.take<double>(4 * E1);
        s.Tcor = cv.take<T>(4LL * d.pmax * d.D4);
        s.Tedg = cv.take<T>(4LL * d.pmax * d.D4);
        if (d.dl_alloc) {
            const long long w = 4LL * d.D4 * d.D4;
            s.Wcor = cv.take<T>(w);
            s.Wedg = cv.take<T>(w);
            if (sizeof(T) == 4) {
                s.Wcor_lo = cv.take<T>(w);
                s.Wedg_lo = cv.take<T>(w);
            }
        }
        if (d.lay) {
            s.L1 = cv.take<T>(8 * d.lay1);
            s.L2 = cv.take<T>(8 * d.lay2);
        }
        s.Vw = cv.take<T>(4 * n * kk);
        s.spec = cv.take<double>(4LL * d.chi);
        s.prev = cv.take<double>(4LL * d.chi);
        s.trunc = cv.take<double>(4);
        s.delta = cv.take<double>(1);
        s.live = cv.take<int>(4LL * d.kk);
    }
    carve_lane(cv);
    save_lane(0);
    const long long mT = 4LL * d.d2;                 // rows of T' as [(sA,aA,u,r)]
    const long long m = D3;                          // size of R
    A2 = cv.take<double>(4 * D3);
    B2 = cv.take<double>(4 * D3);
    XA = cv.take<double>(4LL * d.D4 * d.d2 * d.D);  // [(o1,o2)][D^4][(ph,k)]
    R = cv.take<double>(m * m);
    S = cv.take<double>(m * 4);
    Xs = cv.take<double>(3LL * 16 * 16 + 64);
    Tm = cv.take<double>(mT * mT);
    Gt = cv.take<double>(mT * mT);
    Wt = cv.take<double>(mT * mT);
    Lt = cv.take<double>(mT);
    Gtf = cv.take<float>(mT * mT);
    Wtf = cv.take<float>(mT * mT);
    Ltf = cv.take<float>(mT);
    Xmat = cv.take<double>(m * m + 4 * m);
    cost = cv.take<double>(64);
    flags = cv.take<int>(64);
    tc_err = cv.take<int>(64);
    pq_T = cv.take<double>((long long)d.pmax * d.D4);
    if (d.lay) {
        pq_img1 = cv.take<T>(8 * d.lay1);
        pq_img2 = cv.take<T>(8 * d.lay2);
    } else {
        pq_cor = cv.take<T>(4LL * d.pmax * d.D4);
        pq_edg = cv.take<T>(4LL * d.pmax * d.D4);
    }
    nlanes = d.nslots >= 6 ? 3 : 1;
    for (int i = 1; i < nlanes; ++i) {
        carve_lane(cv);
        save_lane(i);
    }
    bind(0);
}

// Scratch of one lane (the buffers a CTM move, the metric and the
// observables' contractions write).
template <typename T>
void Engine<T>::carve_lane(Carver& cv) {
    const Dims& d = dm;
    const long long chi2 = (long long)d.chi * d.chi, E1 = (long long)d.chi * d.d2 * d.chi;
    const long long n = d.n, n2 = n * n, kk = d.kk;
    Cop = cv.take<T>(4 * chi2);
    Eop = cv.take<T>(4 * E1);
    X1[0] = cv.take<T>(E1);
    X1[1] = cv.take<T>(E1);
    Y1 = cv.take<T>(n2);
    Yp = cv.take<T>(n2);
    // the layered CUDA-core form's chi^2 D^4 p intermediate (the tensor-core
    // form keeps it on chip)
    Zk = d.lay ? nullptr : cv.take<T>((long long)d.pmax * n2);
    Qt = cv.take<T>(n2);
    Q[0] = cv.take<T>(n2);
    Q[1] = cv.take<T>(n2);
    Mt = cv.take<T>(n2);
    V0 = cv.take<T>(n * kk);
    Z1 = cv.take<T>(n * kk);
    U = cv.take<T>(n * kk);
    Z2 = cv.take<T>(n * kk);
    Vo = cv.take<T>(n * kk);
    Uf = cv.take<T>(n * kk);
    Xk = cv.take<T>(kk * kk);
    Hk = cv.take<T>(kk * kk);
    Lk = cv.take<T>(kk * kk);
    Qk = cv.take<T>(kk * kk);
    Sk = cv.take<T>(kk);
    isq = cv.take<T>(kk > d.chi ? kk : d.chi);
    P = cv.take<T>(n * d.chi);
    PtT = cv.take<T>(n * d.chi);
    C4E3 = cv.take<T>(n * d.chi);
    C1n = cv.take<T>(chi2);
    C4n = cv.take<T>(chi2);
    E4n = cv.take<T>(E1);
    dscr = cv.take<double>(DscrOff::kFixed + kk * kk);
    mt1 = cv.take<T>(E1);
    mt2 = cv.take<T>(E1);
    mup = cv.take<T>(n2);
    mdn = cv.take<T>(n2);
    mupp = cv.take<T>(n2);
    mdnp = cv.take<T>(n2);
    mN4 = cv.take<T>((long long)d.D4 * d.D4);
    N = cv.take<double>((long long)d.D4 * d.D4);
    dwork = cv.take<double>(4 * E1 + 16LL * d.D4 + 64);
    if (proj64()) {
        Hd = cv.take<double>(kk * kk);
        Ld = cv.take<double>(kk * kk);
        Qd = cv.take<double>(kk * kk);
        Lr = cv.take<double>(kk * kk);
        Qr = cv.take<double>(kk * kk);
        Sd = cv.take<double>(kk);
        Rw = cv.take<double>(svd_refine_scratch((int)kk));
    }
    sk_elems = 16LL * n * (kk > d.chi ? kk : d.chi);
    skbuf = cv.take<T>(sk_elems);
}

template <typename T>
void Engine<T>::save_lane(int i) {
    Lane<T>& L = lanes[i];
#define KH_SAVE(f) L.f = f;
    KH_LANE_PTRS(KH_SAVE)
    KH_LANE_DPTRS(KH_SAVE)
#undef KH_SAVE
    L.X1[0] = X1[0]; L.X1[1] = X1[1];
    L.Q[0] = Q[0]; L.Q[1] = Q[1];
}

template <typename T>
void Engine<T>::bind(int i) {
    const Lane<T>& L = lanes[i];
#define KH_BIND(f) f = L.f;
    KH_LANE_PTRS(KH_BIND)
    KH_LANE_DPTRS(KH_BIND)
#undef KH_BIND
    X1[0] = L.X1[0]; X1[1] = L.X1[1];
    Q[0] = L.Q[0]; Q[1] = L.Q[1];
    st = L.st;
}

template <typename T>
Engine<T>::~Engine() {
    if (own_streams) {
        for (int i = 1; i < 3; ++i)
            if (lanes[i].st) cudaStreamDestroy(lanes[i].st);
    }
    for (auto& e : lane_ev)
        if (e) cudaEventDestroy(e);
}

template <typename T>
size_t Engine<T>::bytes_needed(const kh_config& c) {
    Engine<T> e;
    e.cfg = c;
    e.dm = make_dims(c, sizeof(T) == 8);
    Carver cv(nullptr, 0);
    e.layout(cv);
    return cv.off + 256;
}

// beta = 0 purification: spin maximally entangled with its ancilla, virtual index 0
__global__ void init_state_kernel(double* A, double* B, int D) {
    if (threadIdx.x == 0) {
        long long D3 = (long long)D * D * D;
        A[0] = 1.0; A[3 * D3] = 1.0;
        B[0] = 1.0; B[3 * D3] = 1.0;
    }
}

template <typename T>
Engine<T>::Engine(const kh_config& c, void* ws, size_t bytes, cudaStream_t s) {
    memcpy(&cfg, &c, sizeof(kh_config));   // byte copy: a checkpoint holds the caller's exact configuration
    st = s;
    lanes[0].st = s;
    dm = make_dims(c, sizeof(T) == 8);
    tc_npass = (c.prec == KH_TF32 || c.prec == KH_BF16) ? 1 : (c.prec == KH_TF32X3 ? 3 : 0);
    Carver cv(ws, bytes);
    layout(cv);
    for (int i = 1; i < nlanes; ++i) {
        KH_CUDA(cudaStreamCreateWithFlags(&lanes[i].st, cudaStreamNonBlocking));
        own_streams = true;
    }
    for (int i = 0; i < nlanes; ++i) KH_CUDA(cudaEventCreateWithFlags(&lane_ev[i], cudaEventDisableTiming));
    bind(0);
    KH_CUDA(cudaMemsetAsync(ws, 0, cv.off, st));
    init_state_kernel<<<1, 32, 0, st>>>(A, B, dm.D);
    KH_LAUNCHED();
    for (int i = 0; i < dm.nslots; ++i) init_env(i, nullptr);
}

// ------------------------------------------------------------------ kernels

template <typename T>
__global__ void identity_kernel(T* V, int n, int k) {
    long long tot = (long long)n * k;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
         i += (long long)gridDim.x * blockDim.x) {
        int r = (int)(i / k), c = (int)(i % k);
        V[i] = (r == c) ? T(1) : T(0);
    }
}

template <typename T>
__global__ void rand_kernel(T* V, long long tot, uint64_t seed, uint64_t stream) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
         i += (long long)gridDim.x * blockDim.x)
        V[i] = (T)rnd_uniform(seed, stream, (uint64_t)i);
}

// Gram G = Z^T Z (Z: n x k row-major, k <= 16 KT): one CTA per chunk of rows,
// staged in shared memory; thread (ti, tj) of a 16 x 16 grid holds the
// KT x KT register tile G[ti + 16 a][tj + 16 b] and accumulates it over the
// chunk (in T), then adds it to the FP64 result.
template <typename T, int KT>
__global__ void __launch_bounds__(256) gram_kernel(const T* __restrict__ Z, const T* __restrict__ Z2, int n, int k,
                                                   double* __restrict__ G, int rows_per) {
    extern __shared__ unsigned char smem_raw[];
    T* Ys = reinterpret_cast<T*>(smem_raw);   // rows_per x k (Z), then rows_per x k (Z2) when given
    T* Ys2 = Z2 ? Ys + rows_per * k : Ys;
    const int r0 = blockIdx.x * rows_per, nr = min(rows_per, n - r0);
    for (int e = threadIdx.x; e < nr * k; e += blockDim.x) Ys[e] = Z[(long long)r0 * k + e];
    if (Z2)
        for (int e = threadIdx.x; e < nr * k; e += blockDim.x) Ys2[e] = Z2[(long long)r0 * k + e];
    __syncthreads();
    const int ti = threadIdx.x >> 4, tj = threadIdx.x & 15;
    T acc[KT][KT];
#pragma unroll
    for (int a = 0; a < KT; ++a)
#pragma unroll
        for (int b = 0; b < KT; ++b) acc[a][b] = T(0);
    for (int r = 0; r < nr; ++r) {
        const T* y = Ys + r * k;
        const T* y2 = Ys2 + r * k;
        T yi[KT], yj[KT];
#pragma unroll
        for (int a = 0; a < KT; ++a) {
            const int i = ti + 16 * a, j = tj + 16 * a;
            yi[a] = i < k ? y[i] : T(0);
            yj[a] = j < k ? y2[j] : T(0);
        }
#pragma unroll
        for (int a = 0; a < KT; ++a)
#pragma unroll
            for (int b = 0; b < KT; ++b) acc[a][b] = fma(yi[a], yj[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < KT; ++a)
#pragma unroll
        for (int b = 0; b < KT; ++b) {
            const int i = ti + 16 * a, j = tj + 16 * b;
            if (i < k && j < k) atomicAdd(&G[i * k + j], (double)acc[a][b]);
        }
}

// G = Z^T Z2 (Z2 = Z when null), k x k, accumulated in T over chunks of 16
// rows and in FP64 across chunks.
template <typename T>
void gram(const T* Z, int n, int k, double* dG, cudaStream_t st, const T* Z2 = nullptr) {
    if (k > 160) fail(KH_EINVAL, "gram: k > 160");
    KH_CUDA(cudaMemsetAsync(dG, 0, sizeof(double) * k * k, st));
    const int nmat = Z2 ? 2 : 1;
    int rows_per = (int)((48 * 1024) / (sizeof(T) * k * nmat));   // stay within the default shared-memory limit
    if (rows_per > 16) rows_per = 16;
    const int grid = (n + rows_per - 1) / rows_per;
    const size_t sm = sizeof(T) * rows_per * k * nmat;
    switch ((k + 15) / 16) {
#define KH_GRAM(KT) case KT: gram_kernel<T, KT><<<grid, 256, sm, st>>>(Z, Z2, n, k, dG, rows_per); break;
        KH_GRAM(1) KH_GRAM(2) KH_GRAM(3) KH_GRAM(4) KH_GRAM(5)
        KH_GRAM(6) KH_GRAM(7) KH_GRAM(8) KH_GRAM(9) KH_GRAM(10)
#undef KH_GRAM
    }
    KH_LAUNCHED();
}

template <typename T>
void gram2(const T* A, const T* B, int n, int k, double* dG, cudaStream_t st) {
    gram<T>(A, n, k, dG, st, B);
}
template void gram2<float>(const float*, const float*, int, int, double*, cudaStream_t);
template void gram2<double>(const double*, const double*, int, int, double*, cudaStream_t);

// max that keeps a NaN once it has seen one (fmax drops NaN operands): a
// non-finite environment must reach the host's spectrum check
__device__ __forceinline__ double nan_max(double a, double b) { return (b > a || b != b) ? b : a; }

// spectrum (first chi values, zero-padded), S^-1/2 with cut-off, discarded
// weight.  One block; every element handled by its own thread (a serial loop
// here would pay a global-memory round trip per value).  A NaN singular value
// is passed on to the spectrum and the discarded weight (not clamped to 0).
template <typename TS, typename T>
__global__ void finalize_spectrum_kernel(const TS* sv, int k, int chi, double cut, const double* normM2,
                                         double* spec, T* isq, double* trunc) {
    __shared__ double red[32];
    const int nkeep = min(chi, k);
    const double s0 = fmax((double)sv[0], 0.0);
    double kept = 0.0;
    for (int j = threadIdx.x; j < chi; j += blockDim.x) {
        const double raw = (j < nkeep) ? (double)sv[j] : 0.0;
        const double s = raw != raw ? raw : fmax(raw, 0.0);
        kept += s * s;
        bool keep = (s0 > 0.0) && (s > cut * s0);
        spec[j] = s != s ? s : (keep ? s : 0.0);
        isq[j] = keep ? (T)rsqrt(s) : T(0);
    }
    for (int o = 16; o > 0; o >>= 1) kept += __shfl_xor_sync(0xffffffffu, kept, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = kept;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        double tot = *normM2;
        double tr = (tot > 0.0) ? (tot - t) / tot : (tot != tot ? tot : 0.0);
        *trunc = tr != tr ? tr : (tr > 0.0 ? tr : 0.0);
    }
}

template <typename T>
__global__ void store_normalized_kernel(const T* x, long long n, const double* sumsq, double* master, T* op) {
    double s = *sumsq;
    double inv = s > 0.0 ? 1.0 / sqrt(s) : 1.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        double v = (double)x[i] * inv;
        master[i] = v;
        op[i] = (T)v;
    }
}

__global__ void delta_kernel(const double* spec, double* prev, int chi, int prev_valid, double* delta) {
    // one block: direction-wise normalised spectra, max |change| against the
    // previous sweep; warp q < 4 normalises direction q
    __shared__ double inv[4];
    __shared__ double red[32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (w < 4) {
        double s = 0.0;
        for (int j = lane; j < chi; j += 32) { double v = spec[w * chi + j]; s += v * v; }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) inv[w] = s > 0.0 ? rsqrt(s) : 1.0;
    }
    __syncthreads();
    // the previous spectra count only when they belong to the same run: after
    // a reset (prev_valid == 0) they may hold anything, a NaN of a failed run
    // included, and only the current spectra can make the change NaN
    double d = 0.0;
    for (int e = t; e < 4 * chi; e += blockDim.x) {
        double v = spec[e] * inv[e / chi];
        d = nan_max(d, prev_valid ? fabs(v - prev[e]) : (v != v ? v : 0.0));
        prev[e] = v;
    }
    for (int o = 16; o > 0; o >>= 1) d = nan_max(d, __shfl_xor_sync(0xffffffffu, d, o));
    if (lane == 0) red[w] = d;
    __syncthreads();
    if (t == 0) {
        double m = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = nan_max(m, red[i]);
        *delta = m != m ? m : (prev_valid ? m : INFINITY);   // NaN is reported even on a first sweep
    }
}

__global__ void init_env_kernel(double* C, double* E, int chi, int d2, const double* edge, int has_edge, int D) {
    long long chi2 = (long long)chi * chi, E1 = (long long)chi * d2 * chi;
    long long tot = 4 * chi2 + 4 * E1;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
         i += (long long)gridDim.x * blockDim.x) {
        if (i < 4 * chi2) {
            long long j = i % chi2;
            C[i] = (j == 0) ? 1.0 : 0.0;
        } else {
            long long q = i - 4 * chi2;
            long long j = q % E1;
            long long x = j / ((long long)d2 * chi), rem = j % ((long long)d2 * chi);
            long long m = rem / chi, y = rem % chi;
            double v = 0.0;
            if (x == 0 && y == 0) {
                if (has_edge) v = edge[m];
                else v = ((m / D) == (m % D)) ? 1.0 : 0.0;
            }
            E[q] = v;
        }
    }
}

// symmetrise N (n x n) in place: N = (N + N^T)/2
__global__ void symmetrize_kernel(double* Nm, int n) {
    long long tot = (long long)n * n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
         i += (long long)gridDim.x * blockDim.x) {
        int r = (int)(i / n), c = (int)(i % n);
        if (r < c) {
            double a = Nm[(long long)r * n + c], b = Nm[(long long)c * n + r];
            double m = 0.5 * (a + b);
            Nm[(long long)r * n + c] = m;
            Nm[(long long)c * n + r] = m;
        }
    }
}

// out = sum_i a[i] * b[perm(i)] in FP64 via strided index maps (small sizes)
__global__ void dot_kernel(const double* a, const double* b, long long n, double* out) {
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        s += a[i] * b[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

// Z10-type ring closure: sum_{h,m,f} t3[(h*d2+m)*chi+f] * u[(f*d2+m)*chi+h]
__global__ void ring_close_kernel(const double* t3, const double* u, int chi, int d2, double* out) {
    long long tot = (long long)chi * d2 * chi;
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
         i += (long long)gridDim.x * blockDim.x) {
        int h = (int)(i / ((long long)d2 * chi));
        int m = (int)((i / chi) % d2);
        int f = (int)(i % chi);
        s += t3[i] * u[((long long)f * d2 + m) * chi + h];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

// Z01-type: sum_{a,m,e} t3[(a*d2+m)*chi+e] * u[e*(d2*chi) + m*chi + a]
__global__ void ring_close2_kernel(const double* t3, const double* u, int chi, int d2, double* out) {
    long long tot = (long long)chi * d2 * chi;
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
         i += (long long)gridDim.x * blockDim.x) {
        int a = (int)(i / ((long long)d2 * chi));
        int m = (int)((i / chi) % d2);
        int e = (int)(i % chi);
        s += t3[i] * u[(long long)e * d2 * chi + (long long)m * chi + a];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

// vals[i] = sum_ab O_i[a][b] X[a][b] / tr X
__global__ void expval_kernel(const double* ops, int n_ops, int p, const double* X, double* vals) {
    int i = threadIdx.x;
    if (i >= n_ops) return;
    double tr = 0.0, s = 0.0;
    for (int a = 0; a < p; ++a) tr += X[a * p + a];
    for (int a = 0; a < p * p; ++a) s += ops[(long long)i * p * p + a] * X[a];
    vals[i] = s / tr;
}

// ------------------------------------------------------------------ env management

template <typename T>
void Engine<T>::init_env(int slot, const double* edge) {
    Slot<T>& sl = slots[slot];
    const int d2 = dm.d2;
    double* dedge = dscr + DscrOff::kStage;
    if (edge) KH_CUDA(cudaMemcpyAsync(dedge, edge, sizeof(double) * d2, cudaMemcpyHostToDevice, st));
    long long tot = 4LL * dm.chi * dm.chi + 4LL * dm.chi * d2 * dm.chi;
    init_env_kernel<<<grid_for(tot), 256, 0, st>>>(sl.C, sl.E, dm.chi, d2, dedge, edge != nullptr, dm.D);
    KH_LAUNCHED();
    sl.env_valid = true;
    sl.prev_valid = false;
    for (int q = 0; q < 4; ++q) sl.warm[q] = false;
    if (edge) KH_CUDA(cudaStreamSynchronize(st));   // dscr is reused
}

template <typename T>
void Engine<T>::copy_env(int dst, int src) {
    Slot<T>& a = slots[dst];
    Slot<T>& b = slots[src];
    const long long chi2 = (long long)dm.chi * dm.chi, E1 = (long long)dm.chi * dm.d2 * dm.chi;
    KH_CUDA(cudaMemcpyAsync(a.C, b.C, sizeof(double) * 4 * chi2, cudaMemcpyDeviceToDevice, st));
    KH_CUDA(cudaMemcpyAsync(a.E, b.E, sizeof(double) * 4 * E1, cudaMemcpyDeviceToDevice, st));
    KH_CUDA(cudaMemcpyAsync(a.Vw, b.Vw, sizeof(T) * 4LL * dm.n * dm.kk, cudaMemcpyDeviceToDevice, st));
    // the live-column masks belong to the warm subspaces: without them the
    // first warm move would refill columns by the destination's old mask
    KH_CUDA(cudaMemcpyAsync(a.live, b.live, sizeof(int) * 4LL * dm.kk, cudaMemcpyDeviceToDevice, st));
    a.env_valid = b.env_valid;
    a.prev_valid = false;
    for (int q = 0; q < 4; ++q) a.warm[q] = b.warm[q];
}

template <typename T>
void Engine<T>::refresh_operands(Slot<T>& sl) {
    cast<double, T>(sl.C, Cop, 4LL * dm.chi * dm.chi, st);
    cast<double, T>(sl.E, Eop, 4LL * dm.chi * dm.d2 * dm.chi, st);
}

// ------------------------------------------------------------------ contractions

// Two-layer site contraction: for each of nb blocks,
//   out[b][(o1k,o2k)][(o1b,o2b)] = sum_p sum TL[(i1k,i2k)][p][(o1k,o2k)]
//                                  Y[b][(i1b,i2b)][(i1k,i2k)] TL[(i1b,i2b)][p][(o1b,o2b)]
// with TL = T permuted to [in1][in2][p][out1][out2].
//  Wt given (D^2 <= 2p): one GEMM with the double-layer tensor,
//    out[b][(ok,ob)] = sum_{(ib,ik)} Y[b][(ib,ik)] Wt[(ok,ob)][(ib,ik)]   (2 nb D^8 flops),
//    on the tensor cores when the precision asks for them;
//  otherwise layer by layer: the ket layer as one GEMM (K = D^2), then the
//    bra layer batched over b (K = p D^2)                                  (4 nb p D^6 flops);
//    with TLb given, the bra layer reads TLb instead of TL (an operator on
//    the ket layer only).
// The double-layer site contraction runs as a 3xTF32 tensor-core GEMM: its
// Y operand is then written directly as the (hi, lo) pair into (mup, mdn).
template <typename T>
bool Engine<T>::site_presplit(const Slot<T>& sl) const {
    return sl.dl && tc_npass == 3 && sizeof(T) == 4 && dm.D4 % 4 == 0;
}

// Y permuted into the site contraction's block layout: into Yp, or as the
// split pair (mup, mdn) when site_presplit.
template <typename T>
void Engine<T>::site_operand(const Slot<T>& sl, const T* Y, T* Yp, const std::vector<long long>& shape,
                             const std::vector<int>& order) {
    if (site_presplit(sl)) permute_split((const float*)Y, (float*)mup, (float*)mdn, shape, order, st);
    else permute<T, T>(Y, Yp, shape, order, st);
}

template <typename T>
void Engine<T>::site_layer(const T* Ybuf, long long nb, const T* TL, const T* L1, const T* L2, int p, T* out,
                           const T* Wt, const T* Wt_lo, bool presplit, const T* TLb) {
    const int d2 = dm.d2, d4 = dm.D4;
    prof_begin(1);
    if (!Wt && L1) {                                   // layered, on the tensor cores
        site_layered_tc((const float*)Ybuf, nb, dm.D, p, (const float*)L1, (const float*)L2, (float*)out,
                        tc_npass, dm.bf16, tc_err, st);
        prof_end(1, 4.0 * (double)nb * p * d2 * (double)d2 * d2);
        return;
    }
    if (Wt) {
        if (tc_npass && sizeof(T) == 4 && d4 % 4 == 0) {       // TMA rows must be 16-byte multiples
            TcOperand a{(const float*)Ybuf, nullptr, d4}, b{(const float*)Wt, nullptr, d4};
            if (tc_npass == 3) {
                float *yh = (float*)mup, *yl = (float*)mdn;     // nb D^4 = n^2 elements
                if (!presplit) tc_split((const float*)Ybuf, yh, yl, nb * d4, st);
                a = TcOperand{yh, yl, d4};
                b = TcOperand{(const float*)Wt, (const float*)Wt_lo, d4};
            }
            tc_gemm(a, b, (float*)out, (int)nb, d4, d4, d4, 1.f, 0.f, nullptr, tc_npass, tc_err, st);
        } else {
            gemm_rm<T>((int)nb, d4, d4, Ybuf, false, Wt, true, out, st);
        }
        prof_end(1, 2.0 * (double)nb * d4 * (double)d4);
        return;
    }
    gemm_rm<T>((int)(nb * d2), p * d2, d2, Ybuf, false, TL, false, Zk, st);
    for (long long b0 = 0; b0 < nb; b0 += 65535) {
        GemmArgs<T> g;
        g.M = d2; g.N = d2; g.K = d2 * p;
        g.batch = (int)((nb - b0) < 65535 ? (nb - b0) : 65535);
        g.A = Zk + b0 * (long long)d2 * p * d2; g.sAm = 1; g.sAk = d2; g.sAb = (long long)d2 * p * d2;
        g.B = TLb ? TLb : TL; g.sBk = d2; g.sBn = 1; g.sBb = 0;
        g.C = out + b0 * (long long)d2 * d2; g.sCm = d2; g.sCn = 1; g.sCb = (long long)d2 * d2;
        g.alpha = T(1); g.beta = T(0); g.colscale = nullptr;
        gemm<T>(g, st);
    }
    prof_end(1, 4.0 * (double)nb * p * d2 * (double)d2 * d2);
}

template <typename T>
void Engine<T>::corner(Slot<T>& sl, int f, int which) {
    const int chi = dm.chi, d2 = dm.d2, D = dm.D;
    const long long chi2 = (long long)chi * chi, E1 = (long long)chi * d2 * chi;
    const T* C1 = Cop + f * chi2;
    const T* E1p = Eop + f * E1;
    const T* E4 = Eop + ((f + 3) & 3) * E1;
    T* X = X1[which];
    gemm_rm<T>(chi, d2 * chi, chi, C1, false, E1p, false, X, st);            // [x4][(uk,ub,z)]
    gemm_rm<T>(chi * d2, d2 * chi, chi, E4, false, X, false, Y1, st);        // [(w,lk,lb)][(uk,ub,z)]
    site_operand(sl, Y1, Yp, {chi, D, D, D, D, chi}, {0, 5, 2, 4, 1, 3});     // [w][z][lb][ub][lk][uk]
    const long long w4 = (long long)f * dm.D4 * dm.D4;
    site_layer(Yp, chi2, sl.Tcor + (long long)f * dm.pmax * dm.D4, lay_img(sl, 1, 0, f), lay_img(sl, 2, 0, f), sl.p,
               Qt, sl.dl ? sl.Wcor + w4 : nullptr,
               sl.dl && sl.Wcor_lo ? sl.Wcor_lo + w4 : nullptr, site_presplit(sl));   // [w][z][rk][dk][rb][db]
    // Q_0 stored transposed, [(z,rk,rb)][(w,dk,db)], as the K-major operand of
    // Mt = Q_{s+3} Q_s on tensor cores; with 3xTF32 the (hi, lo) pairs of both
    // operands are written by the same pass (Q_1: q1_hi, q1_lo; Q_0: mupp, mdnp)
    const std::vector<int> order = (which == 0 && tc_npass) ? std::vector<int>{1, 2, 4, 0, 3, 5}
                                                            : std::vector<int>{0, 3, 5, 1, 2, 4};
    if (mt_presplit())
        permute_split((const float*)Qt, (float*)(which == 1 ? q1_hi : mupp), (float*)(which == 1 ? q1_lo : mdnp),
                      {chi, chi, D, D, D, D}, order, st, (float*)Q[which]);
    else
        permute<T, T>(Qt, Q[which], {chi, chi, D, D, D, D}, order, st);
}

// Orthonormal basis of the columns of Y (n x k) by two passes of the ordered
// Cholesky-QR (cholqr_factor): Uo = Y X_1 X_2, dropped directions become zero
// columns.  The second pass, in the first pass's column order, restores the
// orthogonality that the first loses to the conditioning of Y (by a single
// Newton-Schulz step when that loss is already small).  Scratch: tmp (n x k), Xk (k x k), dG (k x k FP64).
template <typename T>
void cholqr2(const T* Y, int n, int k, double cut, T* tmp, T* Xk, double* dG, T* Uo, cudaStream_t st) {
    const double tau = sizeof(T) == 8 ? 1e-12 : 1e-5;
    // FP64: pivots below k 2^-53 / tau, whose acceptance could lift the
    // rounding noise of a later, exactly dependent column above tau, are
    // deferred.  FP32 defers none: there an accepted noise direction is only a
    // surplus basis vector that the Rayleigh-Ritz step discards, and the same
    // bound (k 2^-24 / 1e-5, about 0.5) would reorder most columns of an early,
    // poorly converged iteration.
    const double defer = sizeof(T) == 8 ? k * 0x1p-53 / tau : 0.0;
    gram<T>(Y, n, k, dG, st);
    cholqr_factor<T>(dG, k, cut, tau, Xk, st, true, 0.0, defer);
    gemm_rm<T>(n, k, k, Y, false, Xk, false, tmp, st);
    gram<T>(tmp, n, k, dG, st);
    // the second pass sees nearly orthonormal columns: a Newton-Schulz step
    // (3I - G)/2 suffices when G is within 1e-4 (FP32) / 1e-8 (FP64) of I
    cholqr_factor<T>(dG, k, 1e-3, tau, Xk, st, false, sizeof(T) == 8 ? 1e-8 : 1e-4);
    gemm_rm<T>(n, k, k, tmp, false, Xk, false, Uo, st);
}
template void cholqr2<float>(const float*, int, int, double, float*, float*, double*, float*, cudaStream_t);
template void cholqr2<double>(const double*, int, int, double, double*, double*, double*, double*, cudaStream_t);

// Algorithmic flops of one CholQR2 of an n x k block: two symmetric Gram
// matrices (n k (k+1) each), one Cholesky factor and triangular inverse
// (k^3/3 each; the second pass is a Newton-Schulz step, O(k^2)), Q1 = Y X1
// with triangular X1 (n k^2) and Q = Q1 X2 with dense X2 (2 n k^2).
static double cholqr2_flops(int n, int k) {
    const double N = n, K = k;
    return 5.0 * N * K * K + 2.0 * N * K + 2.0 * K * K * K / 3.0;
}

template <typename T>
void Engine<T>::orth(const T* Y, int n, int k, T* Uo) {
    prof_begin(8);
    cholqr2<T>(Y, n, k, cfg.svd_cut, Qt, Xk, dscr + DscrOff::kGram, Uo, st);
    prof_end(8, cholqr2_flops(n, k));
}

// Half-system product Mt = Q_{s+3} Q_s (= M^T), the largest single GEMM of a
// move: on tensor cores (TF32 or 3xTF32) when the precision asks for it.
template <typename T>
bool Engine<T>::mt_presplit() const {
    return tc_npass == 3 && sizeof(T) == 4 && dm.n % 4 == 0;
}

template <typename T>
void Engine<T>::half_system_product(int n) {
    prof_begin(0);
    if (tc_npass && sizeof(T) == 4 && n % 4 == 0) {     // TMA rows must be 16-byte multiples
        const float* Qb = (const float*)Q[1];
        const float* QaT = (const float*)Q[0];
        TcOperand a{Qb, nullptr, n}, b{QaT, nullptr, n};
        if (tc_npass == 3) {       // operands split when Q_0, Q_1 were written (mt_presplit)
            float *ah = (float*)q1_hi, *al = (float*)q1_lo, *bh = (float*)mupp, *bl = (float*)mdnp;
            a = TcOperand{ah, al, n};
            b = TcOperand{bh, bl, n};
        }
        tc_gemm(a, b, (float*)Mt, n, n, n, n, 1.f, 0.f, nullptr, tc_npass, tc_err, st);
    } else {      // Q_0 is stored transposed whenever the tensor cores are enabled
        gemm_rm<T>(n, n, n, Q[1], false, Q[0], tc_npass != 0, Mt, st);
    }
    prof_end(0, 2.0 * n * (double)n * n);
}

// Mask kernel for the warm subspace basis: live columns to Vl, dead columns
// (live[c] == 0) to R as fresh random vectors.
template <typename T>
__global__ void warm_split_kernel(const T* Vw, const int* live, int n, int k, T* Vl, T* Rr, uint64_t seed,
                                  uint64_t stream) {
    long long tot = (long long)n * k;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
         i += (long long)gridDim.x * blockDim.x) {
        int c = (int)(i % k);
        bool lv = live[c] != 0;
        Vl[i] = lv ? Vw[i] : T(0);
        Rr[i] = lv ? T(0) : (T)rnd_uniform(seed, stream, (uint64_t)i);
    }
}

// A warm-basis column is kept unless it is (near) zero, i.e. its direction
// was dropped by the orthonormalisation: kept tail directions keep
// converging by power iteration instead of restarting from random vectors.
// Column squared norms: block b sums rows b*parts + part (+ gridDim parts, ...),
// thread (part, c) reading consecutive columns of a row (coalesced); the
// per-block sums go to acc by atomics and the last block to finish forms
// live[] and clears acc and the block counter for the next call.
template <typename T>
__global__ void live_mask_kernel(const T* __restrict__ V, int n, int k, int* live, float* acc, int* counter) {
    extern __shared__ float s_part[];                 // parts x k
    __shared__ int s_last;
    const int parts = blockDim.x / k;
    const int c = threadIdx.x % k, part = threadIdx.x / k;
    if (part < parts) {
        float a = 0.f;
        for (int r = blockIdx.x * parts + part; r < n; r += gridDim.x * parts) {
            float v = (float)V[(long long)r * k + c];
            a = fmaf(v, v, a);
        }
        s_part[part * k + c] = a;
    }
    __syncthreads();
    for (int cc = threadIdx.x; cc < k; cc += blockDim.x) {
        float a = 0.f;
        for (int q = 0; q < parts; ++q) a += s_part[q * k + cc];
        atomicAdd(&acc[cc], a);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(counter, 1) == (int)gridDim.x - 1);
    __syncthreads();
    if (s_last) {
        __threadfence();
        for (int cc = threadIdx.x; cc < k; cc += blockDim.x) {
            const float a = atomicAdd(&acc[cc], 0.f);
            live[cc] = (a > 0.25f) ? 1 : 0;
            acc[cc] = 0.f;
        }
        if (threadIdx.x == 0) *counter = 0;
    }
}

// b <- a * alpha + b
template <typename T>
__global__ void axpby_kernel(const T* a, T* b, long long n, T alpha) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] += alpha * a[i];
}

template <typename T>
__global__ void add_kernel(const T* a, T* b, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] += a[i];
}

// The small SVD of the projector (X Q = L S, X k x k): in T by the one-sided
// Jacobi kernel, or, with proj_fp64 in a single-precision engine, by the FP64
// kernel on an FP64 copy of X (S stays in Sd for the spectrum and S^-1/2; L
// and Q are rounded to T for the basis products).
template <typename T>
void Engine<T>::rr_svd(const T* X, int k, T* L, T* Qm, double jtol, int nrel, const double* Xd) {
    svd_jacobi<T>(X, k, Sk, L, Qm, cfg.jacobi_max_sweeps, jtol, 0.0, st, flags + 48, nrel);
    if (proj64()) {
        // FP64 matrix: the FP64-accumulated one when given, else X widened
        if (!Xd) {
            cast<T, double>(X, Hd, (long long)k * k, st);
            Xd = Hd;
        }
        cast<T, double>(L, Ld, (long long)k * k, st);
        cast<T, double>(Qm, Qd, (long long)k * k, st);
        svd_refine_fp64(Xd, k, Ld, Qd, Sd, Lr, Qr, Rw, 1e-5, st);
        cast<double, T>(Lr, L, (long long)k * k, st);
        cast<double, T>(Qr, Qm, (long long)k * k, st);
    }
}

// Top-chi SVD of M = Mt^T, written into (Sk, V = Z1, U = Uf).
//  full mode (n within the Jacobi limit): one-sided Jacobi SVD of Y = M V_w
//    (V_w the previous right vectors, identity when cold): Y Q = L S, so
//    M = L S (V_w Q)^T exactly; singular values to ~eps s_1 absolute.  V is
//    kept orthonormal by one Newton-Schulz step V <- V (3 - V^T V)/2.
//  subspace mode: Y = M V, U = orth(Y), Z = M^T U, V' = orth(Z), then the
//    one-sided Jacobi SVD of G = Z^T V' (G Q = L S) gives M ~ (U L) S (V' Q)^T.  The warm
//    basis keeps its live columns and replaces dead ones by random vectors
//    projected off the live span, so new tail directions are picked up.
template <typename T>
void Engine<T>::projector(Slot<T>& sl, int dir, int slot_id) {
    const int n = dm.n, k = dm.kk, chi = dm.chi;
    const double cut = cfg.svd_cut;
    // a few times the rounding floor sqrt(k) eps of the solver's arithmetic
    const double jtol = sizeof(T) == 8 ? 1e-14 : 2e-6;
    const T* Qa = Q[0];
    const T* Qb = Q[1];
    half_system_product(n);
    double* normM2 = dscr + DscrOff::kNormM2;
    KH_CUDA(cudaMemsetAsync(normM2, 0, sizeof(double), st));
    sumsq_kernel<T><<<sumsq_grid((long long)n * n), 256, 0, st>>>(Mt, (long long)n * n, normM2);
    KH_LAUNCHED();
    uint64_t stream = (uint64_t)slot_id * 4 + dir;
    T* Vw = sl.Vw + (long long)dir * n * k;
    int* live = sl.live + dir * k;
    if (dm.full) {
        if (!sl.warm[dir]) {
            identity_kernel<T><<<grid_for((long long)n * k), 256, 0, st>>>(Vw, n, k);
            KH_LAUNCHED();
        }
        gemm_rm<T>(n, n, n, Mt, true, Vw, false, Y1, st);                      // Y = M V_w
        prof_begin(7);
        rr_svd(Y1, n, Uf, Lk, jtol, chi + 8);                                  // Y Q = L S
        prof_end(7, 0.0);
        gemm_rm<T>(n, n, n, Vw, false, Lk, false, Z1, st);                     // V = V_w Q
        gemm_rm<T>(n, n, n, Z1, true, Z1, false, Y1, st);                      // V^T V
        gemm_rm<T>(n, n, n, Z1, false, Y1, false, Z2, st, T(-0.5), T(0));      // Newton-Schulz:
        // V <- 1.5 V - V (V^T V)/2
        axpby_kernel<T><<<grid_for((long long)n * n), 256, 0, st>>>(Z1, Z2, (long long)n * n, T(1.5));
        KH_LAUNCHED();
        KH_CUDA(cudaMemcpyAsync(Vw, Z2, sizeof(T) * (size_t)n * n, cudaMemcpyDeviceToDevice, st));
        KH_CUDA(cudaMemcpyAsync(Z1, Z2, sizeof(T) * (size_t)n * n, cudaMemcpyDeviceToDevice, st));
        sl.warm[dir] = true;
    } else {
        const T* Vin;
        int q;
        if (!sl.warm[dir]) {
            rand_kernel<T><<<grid_for((long long)n * k), 256, 0, st>>>(V0, (long long)n * k, cfg.seed,
                                                                      stream * 1000003ULL + (rng_counter++));
            KH_LAUNCHED();
            orth(V0, n, k, U);
            Vin = U;
            q = cfg.svd_iters_cold;
        } else {
            warm_split_kernel<T><<<grid_for((long long)n * k), 256, 0, st>>>(
                Vw, live, n, k, Vo, Z2, cfg.seed, stream * 1000003ULL + (rng_counter++));
            KH_LAUNCHED();
            for (int r = 0; r < 2; ++r) {                                       // R <- R - Vl (Vl^T R), twice
                gemm_rm<T>(k, k, n, Vo, true, Z2, false, Xk, st, T(1), T(0), nullptr, skbuf, sk_elems);
                gemm_rm<T>(n, k, k, Vo, false, Xk, false, Z2, st, T(-1), T(1));
            }
            add_kernel<T><<<grid_for((long long)n * k), 256, 0, st>>>(Vo, Z2, (long long)n * k);
            KH_LAUNCHED();
            // no orthonormalisation needed: only span(M V) matters, and with
            // the complement projected off the live span, M V keeps the
            // trusted (large) columns first for the ordered CholQR below
            Vin = Z2;
            q = cfg.svd_iters_warm;
        }
        for (int it = 0; it < q; ++it) {
            prof_begin(9);
            gemm_rm<T>(n, k, n, Mt, true, Vin, false, Z1, st, T(1), T(0), nullptr, skbuf, sk_elems);                 // Y = M V
            prof_end(9, 2.0 * n * (double)n * k);
            orth(Z1, n, k, U);                                                 // U = orth(Y)
            prof_begin(9);
            gemm_rm<T>(n, k, n, Mt, false, U, false, Z2, st, T(1), T(0), nullptr, skbuf, sk_elems);                  // Z = M^T U
            prof_end(9, 2.0 * n * (double)n * k);
            orth(Z2, n, k, Vo);                                                // V' = orth(Z)
            Vin = Vo;
        }
        // G = H^T = Z^T V' with H = V'^T Z the Rayleigh-Ritz matrix (M ~ U G V'^T).
        // V' = orth(Z) by the ordered CholQR makes H a column-permuted
        // triangular factor with graded rows, so G's columns (H's rows) are
        // nearly orthogonal already: the one-sided Jacobi of G is the
        // QR-preconditioned Jacobi SVD and needs fewer sweeps than that of H.
        if (proj64()) {        // FP64-accumulated G for the FP64 refinement, its rounding for the Jacobi
            gram2<T>(Z2, Vo, n, k, Hd, st);
            cast<double, T>(Hd, Hk, (long long)k * k, st);
        } else {
            gemm_rm<T>(k, k, n, Z2, true, Vo, false, Hk, st, T(1), T(0), nullptr, skbuf, sk_elems);
        }
        prof_begin(7);
        rr_svd(Hk, k, Lk, Qk, jtol, chi + 8, proj64() ? Hd : nullptr);         // G Q = L S
        prof_end(7, 0.0);
        gemm_rm<T>(n, k, k, Vo, false, Qk, false, Z1, st);                     // right vectors of M: V' Q
        gemm_rm<T>(n, k, k, U, false, Lk, false, Uf, st);                      // left vectors of M: U L
        KH_CUDA(cudaMemcpyAsync(Vw, Z1, sizeof(T) * (size_t)n * k, cudaMemcpyDeviceToDevice, st));
        {
            const int thr = 256 / k > 0 ? 256 / k * k : k;
            live_mask_kernel<T><<<16, thr, sizeof(float) * thr, st>>>(
                Z1, n, k, live, (float*)(dscr + DscrOff::kLiveAcc), (int*)(dscr + DscrOff::kLiveCount));
        }
        KH_LAUNCHED();
        sl.warm[dir] = true;
    }
    if (proj64())
        finalize_spectrum_kernel<double, T><<<1, 128, 0, st>>>(Sd, k, chi, cut, normM2, sl.spec + (long long)dir * chi,
                                                               isq, sl.trunc + dir);
    else
        finalize_spectrum_kernel<T, T><<<1, 128, 0, st>>>(Sk, k, chi, cut, normM2, sl.spec + (long long)dir * chi,
                                                          isq, sl.trunc + dir);
    KH_LAUNCHED();
    const int nkeep = chi < k ? chi : k;
    if (nkeep < chi) {
        KH_CUDA(cudaMemsetAsync(P, 0, sizeof(T) * (size_t)n * chi, st));
        KH_CUDA(cudaMemsetAsync(PtT, 0, sizeof(T) * (size_t)n * chi, st));
    }
    // P and P~^T are independent: P on the side lane (its own split-K scratch)
    const bool side = side_lane();
    if (side) fork_side();
    {   // P = Qb^T V S^-1/2
        GemmArgs<T> g;
        g.M = n; g.N = nkeep; g.K = n; g.batch = 1;
        g.A = Qb; g.sAm = 1; g.sAk = n; g.sAb = 0;
        g.B = Z1; g.sBk = k; g.sBn = 1; g.sBb = 0;
        g.C = P; g.sCm = chi; g.sCn = 1; g.sCb = 0;
        g.alpha = T(1); g.beta = T(0); g.colscale = isq;
        g.sk = side ? lanes[1].skbuf : skbuf; g.sk_elems = sk_elems;
        gemm<T>(g, side ? lanes[1].st : st);
    }
    {   // P~^T = Qa U S^-1/2  (Qa stored transposed when tensor cores are used)
        GemmArgs<T> g;
        g.M = n; g.N = nkeep; g.K = n; g.batch = 1;
        g.A = Qa; g.sAm = tc_npass ? 1 : n; g.sAk = tc_npass ? n : 1; g.sAb = 0;
        g.B = Uf; g.sBk = k; g.sBn = 1; g.sBb = 0;
        g.C = PtT; g.sCm = chi; g.sCn = 1; g.sCb = 0;
        g.alpha = T(1); g.beta = T(0); g.colscale = isq;
        g.sk = skbuf; g.sk_elems = sk_elems;
        gemm<T>(g, st);
    }
    if (side) join_side();
}

// Absorption: the corner updates C1n = P^T X1a, C4n = (C4 E3) P~^T (on the
// side lane when free, with that lane's split-K and norm scratch) and the
// edge update E4n = [E4^T P, site, permute] P~^T (on the move's lane), each
// normalised and stored to the FP64 masters and the operand copies.
template <typename T>
void Engine<T>::absorb(Slot<T>& sl, int s) {
    const int chi = dm.chi, d2 = dm.d2, D = dm.D, n = dm.n;
    const long long chi2 = (long long)chi * chi, E1 = (long long)chi * d2 * chi;
    const bool side = side_lane();
    if (side) fork_side();
    {
        cudaStream_t cs = side ? lanes[1].st : st;
        T* csk = side ? lanes[1].skbuf : skbuf;
        double* cns = (side ? lanes[1].dscr : dscr) + DscrOff::kNorms;
        {   // C1n = P^T X1a
            GemmArgs<T> g;
            g.M = chi; g.N = chi; g.K = n; g.batch = 1;
            g.A = P; g.sAm = 1; g.sAk = chi; g.sAb = 0;
            g.B = X1[0]; g.sBk = chi; g.sBn = 1; g.sBb = 0;
            g.C = C1n; g.sCm = chi; g.sCn = 1; g.sCb = 0;
            g.alpha = T(1); g.beta = T(0); g.colscale = nullptr;
            g.sk = csk; g.sk_elems = sk_elems;
            gemm<T>(g, cs);
        }
        const T* C4 = Cop + ((s + 3) & 3) * chi2;
        const T* E3 = Eop + ((s + 2) & 3) * E1;
        {   // C4E3[v][y4][(dk,db)] = sum_x3 C4[x3][y4] E3[v][(dk,db)][x3]
            GemmArgs<T> g;
            g.M = chi; g.N = d2; g.K = chi; g.batch = chi;
            g.A = C4; g.sAm = 1; g.sAk = chi; g.sAb = 0;
            g.B = E3; g.sBk = 1; g.sBn = chi; g.sBb = (long long)d2 * chi;
            g.C = C4E3; g.sCm = d2; g.sCn = 1; g.sCb = n;
            g.alpha = T(1); g.beta = T(0); g.colscale = nullptr;
            gemm<T>(g, cs);
        }
        gemm_rm<T>(chi, chi, n, C4E3, false, PtT, false, C4n, cs, T(1), T(0), nullptr, csk, sk_elems);   // C4n = C4E3 P~^T
        KH_CUDA(cudaMemsetAsync(cns, 0, 2 * sizeof(double), cs));
        sumsq_kernel<T><<<sumsq_grid(chi2), 256, 0, cs>>>(C1n, chi2, cns);
        KH_LAUNCHED();
        sumsq_kernel<T><<<sumsq_grid(chi2), 256, 0, cs>>>(C4n, chi2, cns + 1);
        KH_LAUNCHED();
        store_normalized_kernel<T><<<grid_for(chi2), 256, 0, cs>>>(C1n, chi2, cns, sl.C + s * chi2, Cop + s * chi2);
        KH_LAUNCHED();
        store_normalized_kernel<T><<<grid_for(chi2), 256, 0, cs>>>(C4n, chi2, cns + 1, sl.C + ((s + 3) & 3) * chi2,
                                                                   Cop + ((s + 3) & 3) * chi2);
        KH_LAUNCHED();
    }
    const T* E4 = Eop + ((s + 3) & 3) * E1;
    gemm_rm<T>(d2 * chi, d2 * chi, chi, E4, true, P, false, Y1, st);             // [(lk,lb,x4)][(dk,db,a)]
    site_operand(sl, Y1, Yp, {D, D, chi, D, D, chi}, {2, 5, 1, 4, 0, 3});         // [x4][a][lb][db][lk][dk]
    const long long w4 = (long long)s * dm.D4 * dm.D4;
    site_layer(Yp, chi2, sl.Tedg + (long long)s * dm.pmax * dm.D4, lay_img(sl, 1, 1, s), lay_img(sl, 2, 1, s), sl.p,
               Qt, sl.dl ? sl.Wedg + w4 : nullptr,
               sl.dl && sl.Wedg_lo ? sl.Wedg_lo + w4 : nullptr, site_presplit(sl));   // [x4][a][uk][rk][ub][rb]
    permute<T, T>(Qt, Y1, {chi, chi, D, D, D, D}, {1, 3, 5, 0, 2, 4}, st);       // [a][rk][rb][x4][uk][ub]
    gemm_rm<T>(chi * d2, chi, n, Y1, false, PtT, false, E4n, st, T(1), T(0), nullptr, skbuf, sk_elems);   // [a][rk][rb][a_up]
    double* ns = dscr + DscrOff::kNorms;
    KH_CUDA(cudaMemsetAsync(ns + 2, 0, sizeof(double), st));
    sumsq_kernel<T><<<sumsq_grid(E1), 256, 0, st>>>(E4n, E1, ns + 2);
    KH_LAUNCHED();
    store_normalized_kernel<T><<<grid_for(E1), 256, 0, st>>>(E4n, E1, ns + 2, sl.E + ((s + 3) & 3) * E1,
                                                            Eop + ((s + 3) & 3) * E1);
    KH_LAUNCHED();
    if (side) join_side();
}

// Algorithmic flops of a move's steps, counted as the layered (ket, then
// bra) contraction whatever form runs: one enlarged corner is X = C E
// (2 chi^3 D^2), Y = E X (2 chi^3 D^4) and the two site layers (4 p chi^2 D^6);
// the absorption is C' = P^T (C E), C4 E3 and (C4 E3) P~^T (6 chi^3 D^2 in all),
// E^T P (2 chi^3 D^4), the two site layers and the product with P~^T
// (2 chi^3 D^4).
static double corner_flops(int chi, int D, int p) {
    const double c = chi, d2 = (double)D * D, d4 = d2 * d2, d6 = d4 * d2;
    return 2.0 * c * c * c * d2 + 2.0 * c * c * c * d4 + 4.0 * p * c * c * d6;
}
static double absorb_flops(int chi, int D, int p) {
    const double c = chi, d2 = (double)D * D, d4 = d2 * d2, d6 = d4 * d2;
    return 6.0 * c * c * c * d2 + 4.0 * c * c * c * d4 + 4.0 * p * c * c * d6;
}

template <typename T>
void Engine<T>::move(Slot<T>& sl, int s, int slot_id) {
    prof_begin(2);
    if (nlanes >= 2 && !in_lanes) {
        // The two enlarged corners are independent: corner s+3 runs on lane 1
        // (its own stream and scratch) reading lane 0's environment operands
        // and writing Q_{s+3} (and its split, into lane 1's mupp/mdnp) where
        // the half-system product reads them; lane 0 waits before the projector.
        KH_CUDA(cudaEventRecord(lane_ev[0], st));
        KH_CUDA(cudaStreamWaitEvent(lanes[1].st, lane_ev[0], 0));
        corner(sl, s, 0);
        struct Rebind {
            Engine* e;
            ~Rebind() { e->bind(0); }
        } rebind{this};
        bind(1);
        Cop = lanes[0].Cop;
        Eop = lanes[0].Eop;
        X1[1] = lanes[0].X1[1];
        Q[1] = lanes[0].Q[1];
        q1_hi = lanes[1].mupp;
        q1_lo = lanes[1].mdnp;
        corner(sl, (s + 3) & 3, 1);
        KH_CUDA(cudaEventRecord(lane_ev[1], st));
        bind(0);
        KH_CUDA(cudaStreamWaitEvent(st, lane_ev[1], 0));
    } else {
        q1_hi = mup;
        q1_lo = mdn;
        corner(sl, s, 0);
        corner(sl, (s + 3) & 3, 1);
    }
    prof_end(2, 2.0 * corner_flops(dm.chi, dm.D, sl.p));
    prof_begin(3);
    projector(sl, s, slot_id);
    prof_end(3, 0.0);
    prof_begin(4);
    absorb(sl, s);
    prof_end(4, absorb_flops(dm.chi, dm.D, sl.p));
}

template <typename T>
int Engine<T>::sweep(int slot, int max_sweeps, int min_sweeps, double tol, double* delta_out) {
    Slot<T>& sl = slots[slot];
    if (sl.p <= 0) fail(KH_EINVAL, "slot has no site tensor");
    if (!sl.env_valid) init_env(slot, nullptr);
    refresh_operands(sl);
    double delta = INFINITY;
    int done = 0;
    for (int it = 1; it <= max_sweeps; ++it) {
        for (int s = 0; s < 4; ++s) move(sl, s, slot);
        delta_kernel<<<1, 256, 0, st>>>(sl.spec, sl.prev, dm.chi, sl.prev_valid ? 1 : 0, sl.delta);
        KH_LAUNCHED();
        sl.prev_valid = true;
        done = it;
        if (tol >= 0.0) {
            KH_CUDA(cudaMemcpyAsync(&delta, sl.delta, sizeof(double), cudaMemcpyDeviceToHost, st));
            int terr = 0;
            if (tc_npass) KH_CUDA(cudaMemcpyAsync(&terr, tc_err, sizeof(int), cudaMemcpyDeviceToHost, st));
            KH_CUDA(cudaStreamSynchronize(st));
            if (terr) fail(KH_ETIMEOUT, "tensor-core kernel wait timed out (flag " + std::to_string(terr) + ")");
            if (!(delta == delta)) fail(KH_ENUMERIC, "NaN in CTM spectra");
            if (it >= min_sweeps && delta < tol) break;
        }
    }
    sl.sweeps_done += done;
    if (delta_out) *delta_out = delta;
    return done;
}

// Sweeps of up to three slots at once, slot_ids[i] on lane i: the moves are
// issued round-robin over the lanes (each lane's stream orders its own
// work, the lanes run concurrently on the GPU); with tol >= 0 the host reads
// every active slot's spectrum change after each sweep.  Returns the total
// number of sweeps.
template <typename T>
int Engine<T>::sweep_lanes(const int* slot_ids, int count, int mx, int mn, double tol) {
    struct Rebind {
        Engine* e;
        ~Rebind() {
            e->bind(0);
            e->in_lanes = false;
        }
    } rebind{this};
    if (count < 1 || count > nlanes) fail(KH_EINVAL, "sweep_lanes: bad lane count");
    in_lanes = count > 1;
    bool active[3] = {false, false, false};
    int done[3] = {0, 0, 0};
    double delta[3] = {INFINITY, INFINITY, INFINITY};
    for (int i = 0; i < count; ++i) {
        bind(i);
        Slot<T>& sl = slots[slot_ids[i]];
        if (sl.p <= 0) fail(KH_EINVAL, "slot has no site tensor");
        if (!sl.env_valid) init_env(slot_ids[i], nullptr);
        refresh_operands(sl);
        active[i] = true;
    }
    for (int it = 1; it <= mx; ++it) {
        for (int s = 0; s < 4; ++s)
            for (int i = 0; i < count; ++i)
                if (active[i]) {
                    bind(i);
                    move(slots[slot_ids[i]], s, slot_ids[i]);
                }
        for (int i = 0; i < count; ++i)
            if (active[i]) {
                bind(i);
                Slot<T>& sl = slots[slot_ids[i]];
                delta_kernel<<<1, 256, 0, st>>>(sl.spec, sl.prev, dm.chi, sl.prev_valid ? 1 : 0, sl.delta);
                KH_LAUNCHED();
                sl.prev_valid = true;
                done[i] = it;
                if (tol >= 0.0) KH_CUDA(cudaMemcpyAsync(&delta[i], sl.delta, sizeof(double), cudaMemcpyDeviceToHost, st));
            }
        if (tol >= 0.0) {
            int terr = 0;
            for (int i = 0; i < count; ++i)
                if (active[i]) {
                    bind(i);
                    KH_CUDA(cudaStreamSynchronize(st));
                }
            if (tc_npass) {
                bind(0);
                KH_CUDA(cudaMemcpyAsync(&terr, tc_err, sizeof(int), cudaMemcpyDeviceToHost, st));
                KH_CUDA(cudaStreamSynchronize(st));
                if (terr) fail(KH_ETIMEOUT, "tensor-core kernel wait timed out (flag " + std::to_string(terr) + ")");
            }
            bool any = false;
            for (int i = 0; i < count; ++i)
                if (active[i]) {
                    if (!(delta[i] == delta[i])) fail(KH_ENUMERIC, "NaN in CTM spectra");
                    if (it >= mn && delta[i] < tol) active[i] = false;
                    any = any || active[i];
                }
            if (!any) break;
        }
    }
    int total = 0;
    for (int i = 0; i < count; ++i) {
        slots[slot_ids[i]].sweeps_done += done[i];
        total += done[i];
    }
    return total;
}

template <typename T>
void Engine<T>::projectors_out(int slot, int dir, double* spec, double* trunc) {
    Slot<T>& sl = slots[slot];
    if (spec)
        KH_CUDA(cudaMemcpyAsync(spec, sl.spec + (long long)dir * dm.chi, sizeof(double) * dm.chi,
                                cudaMemcpyDeviceToDevice, st));
    if (trunc) {
        KH_CUDA(cudaMemcpyAsync(trunc, sl.trunc + dir, sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    KH_CUDA(cudaStreamSynchronize(st));
}

template <typename T>
void Engine<T>::get_env(int slot, double* C, double* E) {
    Slot<T>& sl = slots[slot];
    const long long chi2 = (long long)dm.chi * dm.chi, E1 = (long long)dm.chi * dm.d2 * dm.chi;
    if (C) KH_CUDA(cudaMemcpyAsync(C, sl.C, sizeof(double) * 4 * chi2, cudaMemcpyDeviceToDevice, st));
    if (E) KH_CUDA(cudaMemcpyAsync(E, sl.E, sizeof(double) * 4 * E1, cudaMemcpyDeviceToDevice, st));
    KH_CUDA(cudaStreamSynchronize(st));
}

// ------------------------------------------------------------------ metric, kappa, expval

template <typename T>
void Engine<T>::compute_metric(Slot<T>& sl, double* N_out) {
    prof_begin(5);
    const int chi = dm.chi, d2 = dm.d2, D = dm.D;
    const long long chi2 = (long long)chi * chi, E1 = (long long)chi * d2 * chi;
    refresh_operands(sl);
    const T *C1 = Cop, *C2 = Cop + chi2, *C3 = Cop + 2 * chi2, *C4 = Cop + 3 * chi2;
    const T *E1p = Eop, *E2 = Eop + E1, *E3 = Eop + 2 * E1, *E4 = Eop + 3 * E1;
    gemm_rm<T>(chi, d2 * chi, chi, C1, false, E1p, false, mt1, st);          // [h][(u,b)]
    gemm_rm<T>(chi * d2, chi, chi, mt1, false, C2, false, mt2, st);           // [(h,u)][c]
    gemm_rm<T>(chi * d2, d2 * chi, chi, mt2, false, E2, false, mup, st);      // [(h,u)][(r,e)]
    gemm_rm<T>(chi, d2 * chi, chi, C3, false, E3, false, mt1, st);           // [e][(d,g)]
    gemm_rm<T>(chi * d2, chi, chi, mt1, false, C4, false, mt2, st);           // [(e,d)][i]
    gemm_rm<T>(chi * d2, d2 * chi, chi, mt2, false, E4, false, mdn, st);      // [(e,d)][(l,h)]
    permute<T, T>(mup, mupp, {chi, D, D, D, D, chi}, {1, 2, 3, 4, 0, 5}, st);  // [uk][ub][rk][rb][h][e]
    permute<T, T>(mdn, mdnp, {chi, D, D, D, D, chi}, {5, 0, 1, 2, 3, 4}, st);  // [h][e][dk][db][lk][lb]
    gemm_rm<T>(d2 * d2, d2 * d2, chi * chi, mupp, false, mdnp, false, mN4, st, T(1), T(0), nullptr, skbuf,
               sk_elems);                                                      // K = chi^2: split over CTAs
    permute<T, double>(mN4, N_out, {D, D, D, D, D, D, D, D}, {6, 0, 2, 4, 7, 1, 3, 5}, st);
    symmetrize_kernel<<<grid_for((long long)dm.D4 * dm.D4), 256, 0, st>>>(N_out, dm.D4);
    KH_LAUNCHED();
    prof_end(5, 0.0);
}

template <typename T>
void Engine<T>::metric(int slot, double* N_out) {
    compute_metric(slots[slot], N);
    KH_CUDA(cudaMemcpyAsync(N_out, N, sizeof(double) * dm.D4 * dm.D4, cudaMemcpyDeviceToDevice, st));
    KH_CUDA(cudaStreamSynchronize(st));
}

template <typename T>
double Engine<T>::kappa(int slot) {
    Slot<T>& sl = slots[slot];
    const int chi = dm.chi, d2 = dm.d2, p = sl.p, D4 = dm.D4;
    const long long chi2 = (long long)chi * chi, E1 = (long long)chi * d2 * chi;
    compute_metric(sl, N);
    double* z = dscr + DscrOff::kKappa;    // Z11, Z00, Z10, Z01
    KH_CUDA(cudaMemsetAsync(z, 0, 4 * sizeof(double), st));
    double* w1 = dwork;
    double* w2 = dwork + E1;
    double* w3 = dwork + 2 * E1;
    double* w4 = dwork + 3 * E1;
    // Z11 = sum_p T_p N T_p
    gemm_rm<double>(p, D4, D4, sl.Ts, false, N, false, w1, st);
    dot_kernel<<<grid_for((long long)p * D4), 256, 0, st>>>(w1, sl.Ts, (long long)p * D4, z);
    KH_LAUNCHED();
    const double *C1 = sl.C, *C2 = sl.C + chi2, *C3 = sl.C + 2 * chi2, *C4 = sl.C + 3 * chi2;
    const double *E1p = sl.E, *E2 = sl.E + E1, *E3 = sl.E + 2 * E1, *E4 = sl.E + 3 * E1;
    // Z00 = Tr(C1 C2 C3 C4)
    gemm_rm<double>(chi, chi, chi, C1, false, C2, false, w1, st);
    gemm_rm<double>(chi, chi, chi, w1, false, C3, false, w2, st);
    // Tr(w2 C4) = sum_ij w2[i][j] (C4^T)[i][j]
    permute<double, double>(C4, w4, {chi, chi}, {1, 0}, st);
    dot_kernel<<<grid_for(chi2), 256, 0, st>>>(w2, w4, chi2, z + 1);
    KH_LAUNCHED();
    // Z10 = C1 E1 C2 C3 E3 C4 with E1.m = E3.m
    gemm_rm<double>(chi, d2 * chi, chi, C1, false, E1p, false, w1, st);      // [h][(m,b)]
    gemm_rm<double>(chi * d2, chi, chi, w1, false, C2, false, w2, st);       // [(h,m)][c]
    gemm_rm<double>(chi * d2, chi, chi, w2, false, C3, false, w3, st);       // [(h,m)][f]
    gemm_rm<double>(chi * d2, chi, chi, E3, false, C4, false, w4, st);       // [(f,m)][h]
    ring_close_kernel<<<grid_for(E1), 256, 0, st>>>(w3, w4, chi, d2, z + 2);
    KH_LAUNCHED();
    // Z01 = C1 C2 E2 C3 C4 E4 with E2.m = E4.m
    gemm_rm<double>(chi, chi, chi, C1, false, C2, false, w1, st);             // [a][c]
    gemm_rm<double>(chi, d2 * chi, chi, w1, false, E2, false, w2, st);        // [a][(m,d)]
    gemm_rm<double>(chi * d2, chi, chi, w2, false, C3, false, w3, st);       // [(a,m)][e]
    gemm_rm<double>(chi, d2 * chi, chi, C4, false, E4, false, w4, st);        // [e][(m,a)]
    ring_close2_kernel<<<grid_for(E1), 256, 0, st>>>(w3, w4, chi, d2, z + 3);
    KH_LAUNCHED();
    double h[4];
    KH_CUDA(cudaMemcpyAsync(h, z, sizeof(h), cudaMemcpyDeviceToHost, st));
    KH_CUDA(cudaStreamSynchronize(st));
    return h[0] * h[1] / (h[2] * h[3]);
}

template <typename T>
void Engine<T>::expval(int slot, const double* ops, int n_ops, double* vals) {
    Slot<T>& sl = slots[slot];
    const int p = sl.p, D4 = dm.D4;
    if (n_ops < 1 || n_ops > 16) fail(KH_EINVAL, "n_ops must be in [1, 16]");
    compute_metric(sl, N);
    double* X = Xs;
    double* TN = dwork;
    gemm_rm<double>(p, D4, D4, sl.Ts, false, N, false, TN, st);
    gemm_rm<double>(p, p, D4, TN, false, sl.Ts, true, X, st);
    double* dops = dscr + DscrOff::kStage;
    double* dvals = dscr + DscrOff::kExpvalOut;
    KH_CUDA(cudaMemcpyAsync(dops, ops, sizeof(double) * n_ops * p * p, cudaMemcpyHostToDevice, st));
    expval_kernel<<<1, 32, 0, st>>>(dops, n_ops, p, X, dvals);
    KH_LAUNCHED();
    KH_CUDA(cudaMemcpyAsync(vals, dvals, sizeof(double) * n_ops, cudaMemcpyDeviceToHost, st));
    KH_CUDA(cudaStreamSynchronize(st));
}

template <typename T>
void jacobi_eig(const T* G, int k, int ldg, long long sG, T* W, int ldw, long long sW, T* evals, long long sE,
                int batch, int max_sweeps, double tol, int* sweeps, const int* skip, cudaStream_t st) {
    if (k > jacobi_kmax<T>()) fail(KH_EINVAL, "jacobi: k beyond limit");
    size_t sm = jacobi_smem<T>(k);
    static std::atomic<size_t> granted[kMaxDevices] = {};   // per T
    smem_opt_in(jacobi_eig_kernel<T>, sm, granted);
    jacobi_eig_kernel<T><<<batch, kJacobiThreads, sm, st>>>(G, k, ldg, sG, W, ldw, sW, evals, sE, max_sweeps, tol,
                                                           sweeps, skip);
    KH_LAUNCHED();
}
template <typename T, int LP, int R>
static void svd_jacobi_launch(const T* X, int k, T* sv, T* L, T* Qm, int max_sweeps, double tol, double cut,
                              cudaStream_t st, int* sweep_count, int nrel) {
    const int kp = (k + 1) & ~1;
    size_t sm = (size_t)2 * kp * svdj_ld<T>(LP * R) * sizeof(T);
    static std::atomic<size_t> granted[kMaxDevices] = {};   // per instantiation
    smem_opt_in(svd_jacobi_kernel<T, LP, R>, sm, granted);
    const int threads = ((kp / 2) * LP + 31) / 32 * 32;
    svd_jacobi_kernel<T, LP, R><<<1, threads, sm, st>>>(X, k, sv, L, Qm, max_sweeps, tol, cut, sweep_count, nrel);
    KH_LAUNCHED();
}

// Rows per lane chosen at compile time: 8 lanes per column pair, R (even)
// rows per lane with 8 R >= kp (at most 640 threads).
template <typename T>
void svd_jacobi(const T* X, int k, T* sv, T* L, T* Qm, int max_sweeps, double tol, double cut, cudaStream_t st,
                int* sweep_count, int nrel) {
    if (k > jacobi_kmax<T>() || k < 1) fail(KH_EINVAL, "svd_jacobi: k beyond limit");
    const int kp = (k + 1) & ~1;
#define KH_SVDJ(LP, R) svd_jacobi_launch<T, LP, R>(X, k, sv, L, Qm, max_sweeps, tol, cut, st, sweep_count, nrel)
    if (kp <= 16) KH_SVDJ(8, 2);
    else if (kp <= 32) KH_SVDJ(8, 4);
    else if (kp <= 48) KH_SVDJ(8, 6);
    else if (kp <= 64) KH_SVDJ(8, 8);
    else if (kp <= 80) KH_SVDJ(8, 10);
    else if (kp <= 96) KH_SVDJ(8, 12);
    else if (kp <= 112) KH_SVDJ(8, 14);
    else if constexpr (sizeof(T) == 4) {     // FP64 stops at k = 112
        if (kp <= 128) KH_SVDJ(8, 16);
        else if (kp <= 144) KH_SVDJ(8, 18);
        else KH_SVDJ(8, 20);
    }
#undef KH_SVDJ
}
template <typename T>
void cholqr_factor(const double* dG, int k, double cut_abs, double tau, T* X, cudaStream_t st, bool sorted,
                   double ns_tol, double defer) {
    if (k > jacobi_kmax<T>()) fail(KH_EINVAL, "cholqr: k beyond limit");
    const size_t sm = (size_t)2 * k * (k | 1) * sizeof(T);
    static std::atomic<size_t> granted[kMaxDevices] = {};
    smem_opt_in(cholqr_kernel<T>, sm, granted);
    cholqr_kernel<T><<<1, 1024, sm, st>>>(dG, k, cut_abs, tau, X, sorted ? 1 : 0, ns_tol, defer);
    KH_LAUNCHED();
}
template void cholqr_factor<float>(const double*, int, double, double, float*, cudaStream_t, bool, double, double);
template void cholqr_factor<double>(const double*, int, double, double, double*, cudaStream_t, bool, double, double);

template void svd_jacobi<float>(const float*, int, float*, float*, float*, int, double, double, cudaStream_t, int*,
                                int);
template void svd_jacobi<double>(const double*, int, double*, double*, double*, int, double, double, cudaStream_t,
                                 int*, int);

template void jacobi_eig<float>(const float*, int, int, long long, float*, int, long long, float*, long long, int, int,
                                double, int*, const int*, cudaStream_t);
template void jacobi_eig<double>(const double*, int, int, long long, double*, int, long long, double*, long long, int,
                                 int, double, int*, const int*, cudaStream_t);

template struct Engine<double>;
template struct Engine<float>;

}  // namespace kh
