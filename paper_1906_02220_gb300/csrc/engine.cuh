// eeFU engine: context layout and the declarations shared by the CTMRG
// (ctm.cu), bond-update (bond.cu) and C-ABI (abi.cu) translation units.
#pragma once
#include "common.cuh"
#include "jacobi.cuh"

namespace kh {

// ------------------------------------------------------------------ per-slot state

template <typename T>
struct Slot {
    double* Ts = nullptr;     // master site tensor [p][D^4]
    int p = 0;                // physical dimension of the loaded tensor (0 = none)
    double* C = nullptr;      // 4 x chi x chi
    double* E = nullptr;      // 4 x chi x D^2 x chi
    T* Tcor = nullptr;        // 4 frames x [l][u][p][r][d]  (corner layer operand)
    T* Tedg = nullptr;        // 4 frames x [l][d][p][u][r]  (edge layer operand)
    // double-layer operands (when D^2 <= 2p): 4 frames x [(ok,ob)][(ib,ik)],
    // with their 3xTF32 low parts when the tensor cores run three passes
    T* Wcor = nullptr;
    T* Wedg = nullptr;
    T* Wcor_lo = nullptr;
    T* Wedg_lo = nullptr;
    bool dl = false;          // the loaded tensor uses the double-layer operands
    // operand images of the layered tensor-core site contraction (layered.cuh):
    // [kind (corner, edge)][frame][chunk][hi, lo], ket images in L1, bra in L2
    T* L1 = nullptr;
    T* L2 = nullptr;
    T* Vw = nullptr;          // 4 dirs x n x kk  (warm projector subspaces)
    double* spec = nullptr;   // 4 x chi  last kept spectra (descending)
    double* prev = nullptr;   // 4 x chi  normalised spectra of the previous sweep
    double* trunc = nullptr;  // 4        discarded weight per move
    double* delta = nullptr;  // 1        last sweep's spectrum change
    int* live = nullptr;      // 4 x kk   live columns of the warm subspaces
    bool env_valid = false;   // environment initialised
    bool prev_valid = false;  // prev holds a sweep
    bool warm[4] = {false, false, false, false};
    int sweeps_done = 0;
};

struct Dims {
    int D, d2, D4, chi, n, kk, pmax, nslots;
    bool full;                 // kk == n: exact Rayleigh-Ritz on the whole space
    bool dl_alloc;             // double-layer operands allocated (D^2 <= 2 p_max and the site form allows)
    bool lay;                  // layered tensor-core site contraction (tensor-core precisions)
    int npass;                 // tensor-core passes: 0 (CUDA cores), 1 (TF32 or BF16), 3 (3xTF32)
    bool bf16;                 // layered site contraction with BF16 operands (kind::f16)
    long long lay1, lay2;      // floats per (kind, frame) of the ket and bra operand images
};

// ------------------------------------------------------------------ engine

// Kernel categories: an NVTX range each (always; a no-op unless a tracing
// tool is attached) and CUDA-event timing (bench instrumentation, when on):
// 0 = half-system product Mt = Q_{s+3} Q_s, 1 = two-layer site contractions,
// 2 = enlarged corners (all), 3 = projector SVD (excluding Mt),
// 4 = absorption, 5 = environment metric, 6 = ALS + gauge,
// 7 = one-sided Jacobi SVD, 8 = CholQR orthonormalisation, 9 = subspace GEMMs.
constexpr const char* kProfNames[10] = {"half_system_product", "site_layer", "corners", "projector_svd",
                                        "absorb", "metric", "als_gauge", "svd_jacobi", "cholqr_orth",
                                        "subspace_gemm"};
struct ProfCat {
    std::vector<cudaEvent_t> a, b;
    int used = 0;
    double flops = 0.0;
};

struct EngineBase {
    virtual ~EngineBase() {
        for (auto& c : prof)
            for (size_t i = 0; i < c.a.size(); ++i) { cudaEventDestroy(c.a[i]); cudaEventDestroy(c.b[i]); }
    }
    bool prof_on = false;
    static constexpr int kProfCats = 10;
    ProfCat prof[kProfCats];
    void prof_begin(int cat) {
        nvtxRangePushA(kProfNames[cat]);
        if (!prof_on) return;
        ProfCat& c = prof[cat];
        if (c.used == (int)c.a.size()) {
            cudaEvent_t x, y;
            KH_CUDA(cudaEventCreate(&x));
            KH_CUDA(cudaEventCreate(&y));
            c.a.push_back(x);
            c.b.push_back(y);
        }
        KH_CUDA(cudaEventRecord(c.a[c.used], st));
    }
    void prof_end(int cat, double flops) {
        nvtxRangePop();
        if (!prof_on) return;
        ProfCat& c = prof[cat];
        KH_CUDA(cudaEventRecord(c.b[c.used], st));
        c.used++;
        c.flops += flops;
    }
    kh_config cfg;
    Dims dm;
    double beta = 0.0;        // inverse temperature reached by eefu_evolve from the initial state
    cudaStream_t st = 0;
    std::string err;
    virtual void set_state(const double* A, const double* B) = 0;
    virtual void get_state(double* A, double* B) = 0;
    virtual void reset_counters() = 0;
    virtual double read_counter() = 0;
    virtual void set_tensor(int slot, const double* Tin, int p) = 0;
    virtual void build_composite(int slot, int gamma, const double* gate) = 0;
    virtual void init_env(int slot, const double* edge) = 0;
    virtual void copy_env(int dst, int src) = 0;
    virtual int sweep(int slot, int max_sweeps, int min_sweeps, double tol, double* delta) = 0;
    virtual void projectors_out(int slot, int dir, double* spec, double* trunc) = 0;
    virtual void get_env(int slot, double* C, double* E) = 0;
    virtual void metric(int slot, double* N_out) = 0;
    virtual double kappa(int slot) = 0;
    virtual void expval(int slot, const double* ops, int n_ops, double* vals) = 0;
    virtual void correlation_length(int slot, int dir, int max_iter, double tol, double* out) = 0;
    virtual void plaquette(int slot, const double* ops, double* out) = 0;
    virtual int slot_p(int slot) const = 0;    // physical dimension of slot's tensor (0 = none)
    virtual void apply_gate(int gamma, const double* gate, int mx, int mn, double tol, double* info) = 0;
    virtual void cost_gradient(int gamma, const double* gate, const double* A2, const double* B2, int mx, int mn,
                               double tol, double* gA, double* gB, double* cost) = 0;
    virtual void observables(const double* H, double hA, double hB, int mx, int mn, double tol,
                             double* out) = 0;
    // persistent state to / from an open checkpoint file (checkpoint.cu)
    virtual void save_checkpoint(std::FILE* f) = 0;
    virtual void load_checkpoint(std::FILE* f) = 0;
};

// Per-lane scratch of the CTM moves and the metric.  Lane 0 serves every
// call on the context's stream; lanes 1 and 2 (own streams) let the
// observables run the CTMs of the three bond mappings concurrently (each
// move is latency-bound and leaves most SMs idle).
#define KH_LANE_PTRS(X) X(Cop) X(Eop) X(Y1) X(Yp) X(Zk) X(Qt) X(Mt) X(V0) X(Z1) X(U) X(Z2) X(Vo) X(Uf) \
    X(Xk) X(Hk) X(Lk) X(Qk) X(Sk) X(isq) X(P) X(PtT) X(C4E3) X(C1n) \
    X(C4n) X(E4n) X(mt1) X(mt2) X(mup) X(mdn) X(mupp) X(mdnp) X(mN4) X(skbuf)
// Fixed regions of the small FP64 scratch dscr that every lane owns (offsets
// in doubles); the Gram matrix of the orthonormalisation (kk^2) comes last.
struct DscrOff {
    static constexpr int kStage = 0;         // host->device staging: edge vector (D^2) or <= 16 operators (p^2 each)
    static constexpr int kExpvalOut = 4096;  // <= 16 expectation values
    static constexpr int kObsOut = 4200;     // 10 observables
    static constexpr int kLiveAcc = 7000;    // column norms of the live mask, k <= 160 floats
    static constexpr int kLiveCount = 7100;  // its last-block counter (int)
    static constexpr int kNormM2 = 8000;     // ||Mt||^2 of the half-system product
    static constexpr int kNorms = 8010;      // sums of squares of C1n, C4n, E4n
    static constexpr int kKappa = 8020;      // Z11, Z00, Z10, Z01 of the free energy
    static constexpr int kGram = 8192;       // FP64 Gram matrix, kk^2
    static constexpr int kFixed = kGram;     // doubles before the Gram matrix
};
static_assert(DscrOff::kStage + 16 * 16 * 16 <= DscrOff::kExpvalOut && DscrOff::kExpvalOut + 16 <= DscrOff::kObsOut &&
                  DscrOff::kObsOut + 10 <= DscrOff::kLiveAcc && DscrOff::kLiveAcc + 160 / 2 <= DscrOff::kLiveCount &&
                  DscrOff::kLiveCount + 1 <= DscrOff::kNormM2 && DscrOff::kNormM2 + 1 <= DscrOff::kNorms &&
                  DscrOff::kNorms + 3 <= DscrOff::kKappa && DscrOff::kKappa + 4 <= DscrOff::kGram,
              "dscr regions overlap");

// FP64 scratch of the projector's Rayleigh-Ritz SVD in the single-precision
// engines with proj_fp64: the matrix Hd, the single-precision factors Ld, Qd,
// the refined factors Lr, Qr (kk x kk each), singular values Sd (kk) and the
// refinement's work Rw (svd_refine_scratch(kk)).
#define KH_LANE_DPTRS(X) X(dscr) X(N) X(dwork) X(Hd) X(Ld) X(Qd) X(Sd) X(Lr) X(Qr) X(Rw)
template <typename T>
struct Lane {
#define KH_DECL(f) T* f = nullptr;
    KH_LANE_PTRS(KH_DECL)
#undef KH_DECL
#define KH_DECL(f) double* f = nullptr;
    KH_LANE_DPTRS(KH_DECL)
#undef KH_DECL
    T* X1[2] = {nullptr, nullptr};
    T* Q[2] = {nullptr, nullptr};
    cudaStream_t st = 0;
};

template <typename T>
struct Engine : EngineBase {
    // persistent
    double* A = nullptr;       // 4 D^3 site tensors
    double* B = nullptr;
    std::vector<Slot<T>> slots;
    // operand copies of the environment of the slot being swept
    T *Cop = nullptr, *Eop = nullptr;
    // CTM scratch
    T *X1[2] = {nullptr, nullptr}, *Y1 = nullptr, *Yp = nullptr, *Zk = nullptr, *Qt = nullptr;
    T *Q[2] = {nullptr, nullptr}, *Mt = nullptr;
    T *V0 = nullptr, *Z1 = nullptr, *U = nullptr, *Z2 = nullptr, *Vo = nullptr, *Uf = nullptr;
    T *Xk = nullptr, *Hk = nullptr, *Lk = nullptr, *Qk = nullptr, *Sk = nullptr;
    T *isq = nullptr, *P = nullptr, *PtT = nullptr, *C4E3 = nullptr;
    T *C1n = nullptr, *C4n = nullptr, *E4n = nullptr;
    double* dscr = nullptr;    // small FP64 scratch (norms etc.), regions in DscrOff
    // metric / bond scratch (FP64 unless noted)
    T *mt1 = nullptr, *mt2 = nullptr, *mup = nullptr, *mdn = nullptr, *mupp = nullptr, *mdnp = nullptr, *mN4 = nullptr;
    double *N = nullptr, *Tp = nullptr, *A2 = nullptr, *B2 = nullptr, *XA = nullptr, *R = nullptr,
           *S = nullptr, *Xs = nullptr, *Tm = nullptr, *Gt = nullptr, *Wt = nullptr, *Lt = nullptr,
           *Xmat = nullptr, *cost = nullptr, *dwork = nullptr;
    double *Hd = nullptr, *Ld = nullptr, *Qd = nullptr, *Sd = nullptr, *Lr = nullptr, *Qr = nullptr, *Rw = nullptr;
    // projector factorisations in FP64 while the contractions run in T = float
    bool proj64() const { return sizeof(T) == 4 && cfg.proj_fp64 != 0; }
    float *Gtf = nullptr, *Wtf = nullptr, *Ltf = nullptr;
    int* flags = nullptr;
    int* tc_err = nullptr;     // tensor-core kernels' time-out flag
    T* skbuf = nullptr;        // split-K partial sums of skinny GEMMs
    long long sk_elems = 0;
    int tc_npass = 0;          // 0: CUDA-core GEMMs; 1: TF32; 3: 3xTF32
    unsigned long long rng_counter = 0;
    Lane<T> lanes[3];
    int nlanes = 1;            // 3 when the context has the six slots of the observables
    bool own_streams = false;
    cudaEvent_t lane_ev[3] = {nullptr, nullptr, nullptr};
    bool in_lanes = false;     // lanes 1, 2 busy with other slots (sweep_lanes)
    T *q1_hi = nullptr, *q1_lo = nullptr;   // where the 3xTF32 split of Q_{s+3} was written
    // Side lane for independent pieces of a move (lane 1), when not busy:
    // fork makes lane 1 wait for lane 0's work so far, join the reverse.
    bool side_lane() const { return nlanes >= 2 && !in_lanes; }
    void fork_side() {
        KH_CUDA(cudaEventRecord(lane_ev[0], lanes[0].st));
        KH_CUDA(cudaStreamWaitEvent(lanes[1].st, lane_ev[0], 0));
    }
    void join_side() {
        KH_CUDA(cudaEventRecord(lane_ev[1], lanes[1].st));
        KH_CUDA(cudaStreamWaitEvent(lanes[0].st, lane_ev[1], 0));
    }
    void bind(int i);          // lane i's scratch and stream become the members used by the moves
    void save_lane(int i);
    void carve_lane(Carver& cv);
    int sweep_lanes(const int* slot_ids, int count, int mx, int mn, double tol);
    ~Engine() override;
    void half_system_product(int n);
    bool mt_presplit() const;

    Engine() {}
    Engine(const kh_config& c, void* ws, size_t bytes, cudaStream_t s);
    static size_t bytes_needed(const kh_config& c);
    void layout(Carver& cv);

    // CTM internals
    void refresh_operands(Slot<T>& sl);
    void corner(Slot<T>& sl, int frame, int which);
    void site_layer(const T* Ybuf, long long nb, const T* TL, const T* L1, const T* L2, int p, T* out,
                    const T* Wt, const T* Wt_lo,
                    bool presplit = false, const T* TLb = nullptr);
    bool site_presplit(const Slot<T>& sl) const;
    // operand image (1 = ket, 2 = bra) of the layered tensor-core contraction
    // for (kind: 0 corner, 1 edge; frame f), or null when the slot uses
    // another form
    const T* lay_img(const Slot<T>& sl, int img, int kind, int f) const {
        if (sl.dl || !sl.L1) return nullptr;
        return img == 1 ? sl.L1 + (kind * 4 + f) * dm.lay1 : sl.L2 + (kind * 4 + f) * dm.lay2;
    }
    void site_operand(const Slot<T>& sl, const T* Y, T* Yp, const std::vector<long long>& shape,
                      const std::vector<int>& order);
    void projector(Slot<T>& sl, int dir, int slot_id);
    void orth(const T* Y, int n, int k, T* Uo);
    void rr_svd(const T* X, int k, T* L, T* Qm, double jtol, int nrel, const double* Xd = nullptr);
    void absorb(Slot<T>& sl, int s);
    void move(Slot<T>& sl, int s, int slot_id);
    void compute_metric(Slot<T>& sl, double* N_out);
    void build_derived(Slot<T>& sl);

    // bond internals
    int als_run(int gamma, double* rel_cost);
    void bond_start_subspace(int mT, int D);
    void gauge_and_store(int gamma);

    // API
    void set_state(const double* A, const double* B) override;
    void get_state(double* A, double* B) override;
    void reset_counters() override { KH_CUDA(cudaMemsetAsync(flags + 48, 0, sizeof(int), st)); }
    double read_counter() override {
        int h = 0;
        KH_CUDA(cudaMemcpyAsync(&h, flags + 48, sizeof(int), cudaMemcpyDeviceToHost, st));
        KH_CUDA(cudaStreamSynchronize(st));
        return h;
    }
    void set_tensor(int slot, const double* Tin, int p) override;
    void build_composite(int slot, int gamma, const double* gate) override;
    void init_env(int slot, const double* edge) override;
    void copy_env(int dst, int src) override;
    int sweep(int slot, int max_sweeps, int min_sweeps, double tol, double* delta) override;
    void projectors_out(int slot, int dir, double* spec, double* trunc) override;
    void get_env(int slot, double* C, double* E) override;
    void metric(int slot, double* N_out) override;
    double kappa(int slot) override;
    void expval(int slot, const double* ops, int n_ops, double* vals) override;
    void correlation_length(int slot, int dir, int max_iter, double tol, double* out) override;   // xi.cu
    void plaquette(int slot, const double* ops, double* out) override;                            // plaquette.cu
    int slot_p(int slot) const override { return slots[slot].p; }
    void plaquette_corner(Slot<T>& sl, int f, const double* Tk, T* out);
    // scratch of the plaquette: the operator-dressed site tensor (FP64) and
    // its site-contraction operands (layered images, or frame layouts)
    double* pq_T = nullptr;
    T *pq_img1 = nullptr, *pq_img2 = nullptr, *pq_cor = nullptr, *pq_edg = nullptr;
    void apply_gate(int gamma, const double* gate, int mx, int mn, double tol, double* info) override;
    void cost_gradient(int gamma, const double* gate, const double* A2in, const double* B2in, int mx, int mn,
                       double tol, double* gA, double* gB, double* cost_out) override;
    void normal_equations(const double* oth, int side, const int* skip);   // R, S of one ALS side
    int als_slot = 0;          // slot whose composite T' the normal equations read
    void observables(const double* H, double hA, double hB, int mx, int mn, double tol,
                     double* out) override;
    void save_checkpoint(std::FILE* f) override;
    void load_checkpoint(std::FILE* f) override;
};

// Tensor-core GEMM (tcgen05.cu): C = alpha colscale (A B^T) + beta C with A
// (M x K) and B (N x K) row-major FP32 read as TF32; npass = 3 uses the
// hi/lo split operands (lo may be null for npass = 1).
struct TcOperand {
    const float* hi;
    const float* lo;
    long long ld;
};
void tc_gemm(const TcOperand& A, const TcOperand& B, float* C, int M, int N, int K, long long ldc, float alpha,
             float beta, const float* colscale, int npass, int* err, cudaStream_t st);
void tc_split(const float* x, float* hi, float* lo, long long n, cudaStream_t st);

// Orthonormal basis of the columns of Y (n x k, k <= the Jacobi limit) by the
// ordered CholQR2 (ctm.cu); see Engine::orth.
template <typename T>
void cholqr2(const T* Y, int n, int k, double cut, T* tmp, T* Xk, double* dG, T* Uo, cudaStream_t st);
// G = A^T B (n x k each, T) accumulated in FP64 across row chunks (ctm.cu)
template <typename T>
void gram2(const T* A, const T* B, int n, int k, double* dG, cudaStream_t st);

// Three FP64 Newton steps on a single-precision SVD G Q ~ L diag(s) of a k x k
// FP64 matrix G (refine.cu): refined factors to Lo, Qo, singular values to s.
size_t svd_refine_scratch(int k);
void svd_refine_fp64(const double* G, int k, const double* L, const double* Q, double* s, double* Lo, double* Qo,
                     double* work, double rel_gap, cudaStream_t st);

// Frame layouts of a site tensor Tm[p][D^4] for the two-layer site
// contraction (bond.cu): Tcor, Tedg 4 frames x pmax D^4 each.
template <typename T>
void derive_operands(const double* Tm, int p, int D, int pmax, T* Tcor, T* Tedg, cudaStream_t st);

// The four 16 x 16 composite-site operators of the plaquette flux W_p in the
// gamma mapping (plaquette.cu), real form: sigma^y enters as i Ytilde with
// Ytilde = [[0, -1], [1, 0]], and W_p = -(product of these) since W_p holds
// sigma^y on exactly two sites.
void flux_operators(int gamma, double* ops);

Dims make_dims(const kh_config& c, bool fp64);
void validate(const kh_config& c);

// ------------------------------------------------------------------ small kernels

// counter-based uniform(-1,1): splitmix64 of (seed, stream, index)
__device__ __forceinline__ double rnd_uniform(uint64_t seed, uint64_t stream, uint64_t i) {
    uint64_t z = seed + 0x9E3779B97F4A7C15ULL * (stream * 0x100000001B3ULL + i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z = z ^ (z >> 31);
    return ((double)(z >> 11) * (1.0 / 9007199254740992.0)) * 2.0 - 1.0;
}

}  // namespace kh
