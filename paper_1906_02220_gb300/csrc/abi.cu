// extern "C" boundary of the eeFU library (declarations and contracts in
// include/eefu.h).  Every entry point converts internal errors into a
// kh_status and a one-line message; nothing throws across the boundary.
#include <cmath>
#include <thread>
#include <vector>

#include "engine.cuh"

namespace kh {
std::atomic<unsigned long long> g_launches{0};
}

struct kh_ctx {
    kh::EngineBase* eng = nullptr;
    std::string err;
    int device = 0;           // device current at creation
};

namespace {

constexpr int kTrajCols = 13;   // beta, the 10 observables, truncation, C

// NVTX range over one ABI call, named after it (tracing; a no-op unless a
// tool is attached)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};
#define KH_RANGE() NvtxRange kh_nvtx_range_(__func__)

template <typename F>
kh_status guard(kh_ctx* ctx, F&& f) {
    if (!ctx || !ctx->eng) return KH_EINVAL;
    try {
        f();
        ctx->err.clear();
        return KH_OK;
    } catch (const kh::Error& e) {
        ctx->err = e.msg;
        return e.st;
    } catch (const std::exception& e) {
        ctx->err = e.what();
        return KH_EINVAL;
    }
}

bool slot_ok(kh_ctx* ctx, int slot) { return slot >= 0 && slot < ctx->eng->dm.nslots; }

// Cyclic Jacobi for a symmetric 4x4 (host, FP64): A -> diag, V eigenvectors.
void jacobi4(double A[16], double V[16]) {
    for (int i = 0; i < 16; ++i) V[i] = (i / 4 == i % 4) ? 1.0 : 0.0;
    for (int sw = 0; sw < 50; ++sw) {
        double off = 0.0;
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j)
                if (i != j) off += A[i * 4 + j] * A[i * 4 + j];
        if (off < 1e-60) break;
        for (int p = 0; p < 3; ++p)
            for (int q = p + 1; q < 4; ++q) {
                double apq = A[p * 4 + q];
                if (apq == 0.0) continue;
                double tau = (A[q * 4 + q] - A[p * 4 + p]) / (2.0 * apq);
                double t = (tau >= 0.0) ? 1.0 / (tau + std::sqrt(1.0 + tau * tau))
                                        : -1.0 / (-tau + std::sqrt(1.0 + tau * tau));
                double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
                for (int k = 0; k < 4; ++k) {
                    double akp = A[k * 4 + p], akq = A[k * 4 + q];
                    A[k * 4 + p] = c * akp - s * akq;
                    A[k * 4 + q] = s * akp + c * akq;
                }
                for (int k = 0; k < 4; ++k) {
                    double apk = A[p * 4 + k], aqk = A[q * 4 + k];
                    A[p * 4 + k] = c * apk - s * aqk;
                    A[q * 4 + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 4; ++k) {
                    double vkp = V[k * 4 + p], vkq = V[k * 4 + q];
                    V[k * 4 + p] = c * vkp - s * vkq;
                    V[k * 4 + q] = s * vkp + c * vkq;
                }
            }
    }
}

void bond_h(int gamma, double J, double Kg, double hA, double hB, double H[16]) {
    // sigma^a (x) sigma^a on (sA,sB), row 2*sA'+sB', col 2*sA+sB
    static const double XX[16] = {0, 0, 0, 1, 0, 0, 1, 0, 0, 1, 0, 0, 1, 0, 0, 0};
    static const double YY[16] = {0, 0, 0, -1, 0, 0, 1, 0, 0, 1, 0, 0, -1, 0, 0, 0};
    static const double ZZ[16] = {1, 0, 0, 0, 0, -1, 0, 0, 0, 0, -1, 0, 0, 0, 0, 1};
    const double* G[3] = {XX, YY, ZZ};
    for (int i = 0; i < 16; ++i) H[i] = 0.25 * J * (XX[i] + YY[i] + ZZ[i]) + 0.25 * Kg * G[gamma][i];
    // -hA S^z_A - hB S^z_B: S^z (x) 1 = diag(1,1,-1,-1)/2, 1 (x) S^z = diag(1,-1,1,-1)/2
    const double zA[4] = {0.5, 0.5, -0.5, -0.5}, zB[4] = {0.5, -0.5, 0.5, -0.5};
    for (int i = 0; i < 4; ++i) H[i * 4 + i] -= hA * zA[i] + hB * zB[i];
}

void gate_from_h(const double* Hin, double tau, double g[16]) {
    double A[16], V[16];
    for (int i = 0; i < 16; ++i) A[i] = 0.5 * (Hin[i] + Hin[(i % 4) * 4 + i / 4]);
    jacobi4(A, V);
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            double s = 0.0;
            for (int k = 0; k < 4; ++k) s += V[i * 4 + k] * std::exp(-tau * A[k * 4 + k]) * V[j * 4 + k];
            g[i * 4 + j] = s;
        }
}

}  // namespace

extern "C" {

void kh_config_defaults(kh_config* c) {
    if (!c) return;
    memset(c, 0, sizeof(*c));
    c->D = 2;
    c->chi = 16;
    c->prec = KH_FP64;
    c->n_slots = 6;
    c->p_max = 16;
    c->svd_oversample = 16;
    c->svd_iters_cold = 4;
    c->svd_iters_warm = 1;
    c->jacobi_max_sweeps = 40;    // per Rayleigh-Ritz SVD; converged environments need 2-3
    c->svd_cut = 1e-12;
    c->als_tol = 1e-12;
    c->als_max_iter = 50;
    c->als_reg = 1e-12;
    c->seed = 0x5eed;
}

size_t kh_workspace_bytes(const kh_config* c) {
    if (!c) return 0;
    try {
        kh::validate(*c);
        if (c->prec == KH_FP64) return kh::Engine<double>::bytes_needed(*c);
        return kh::Engine<float>::bytes_needed(*c);
    } catch (...) {
        return 0;
    }
}

kh_status kh_create(kh_ctx** out, const kh_config* c, void* ws, size_t bytes, void* stream) {
    KH_RANGE();
    if (!out || !c) return KH_EINVAL;
    *out = nullptr;
    kh_ctx* ctx = new kh_ctx();
    try {
        kh::validate(*c);
        if ((uintptr_t)ws % 256 != 0) kh::fail(KH_EINVAL, "workspace must be 256-byte aligned");
        size_t need = kh_workspace_bytes(c);
        if (bytes < need) kh::fail(KH_ENOMEM, "workspace smaller than kh_workspace_bytes()");
        cudaStream_t st = (cudaStream_t)stream;
        KH_CUDA(cudaGetDevice(&ctx->device));
        if (c->prec == KH_FP64) ctx->eng = new kh::Engine<double>(*c, ws, bytes, st);
        else ctx->eng = new kh::Engine<float>(*c, ws, bytes, st);
        KH_CUDA(cudaStreamSynchronize(st));
    } catch (const kh::Error& e) {
        delete ctx->eng;
        delete ctx;
        return e.st;
    }
    *out = ctx;
    return KH_OK;
}

void kh_destroy(kh_ctx* ctx) {
    if (!ctx) return;
    delete ctx->eng;
    delete ctx;
}

const char* kh_last_error(const kh_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

const char* kh_version(void) { return "eefu-gb300 0.1 (sm_103a)"; }

// ------------------------------------------------------------------ checkpoint / resume

namespace {

const char kCheckpointMagic[8] = {'K', 'H', 'C', 'K', 'P', 'T', '0', '1'};

struct FileCloser {
    std::FILE* f;
    ~FileCloser() {
        if (f) std::fclose(f);
    }
};

// Opens a checkpoint and reads its header (magic, configuration); the file
// is left positioned at the engine payload.
kh_status read_checkpoint_header(const char* path, std::FILE** out, kh_config* cfg) {
    *out = nullptr;
    if (!path || !cfg) return KH_EINVAL;
    std::FILE* f = std::fopen(path, "rb");
    if (!f) return KH_EINVAL;
    char magic[8];
    if (std::fread(magic, 1, 8, f) != 8 || memcmp(magic, kCheckpointMagic, 8) != 0 ||
        std::fread(cfg, 1, sizeof(kh_config), f) != sizeof(kh_config)) {
        std::fclose(f);
        return KH_EINVAL;
    }
    *out = f;
    return KH_OK;
}

}  // namespace

kh_status kh_save(kh_ctx* ctx, const char* path) {
    KH_RANGE();
    return guard(ctx, [&] {
        if (!path) kh::fail(KH_EINVAL, "null path");
        FileCloser fc{std::fopen(path, "wb")};
        if (!fc.f) kh::fail(KH_EINVAL, std::string("cannot open ") + path + " for writing");
        if (std::fwrite(kCheckpointMagic, 1, 8, fc.f) != 8 ||
            std::fwrite(&ctx->eng->cfg, 1, sizeof(kh_config), fc.f) != sizeof(kh_config))
            kh::fail(KH_EINVAL, "checkpoint: write failed");
        ctx->eng->save_checkpoint(fc.f);
        if (std::fflush(fc.f) != 0) kh::fail(KH_EINVAL, "checkpoint: write failed");
    });
}

kh_status kh_load_config(const char* path, kh_config* cfg) {
    KH_RANGE();
    std::FILE* f = nullptr;
    kh_status st = read_checkpoint_header(path, &f, cfg);
    if (f) std::fclose(f);
    return st;
}

kh_status kh_load(kh_ctx** out, const char* path, void* ws, size_t bytes, void* stream) {
    KH_RANGE();
    if (!out) return KH_EINVAL;
    *out = nullptr;
    kh_config cfg;
    std::FILE* f = nullptr;
    kh_status st = read_checkpoint_header(path, &f, &cfg);
    if (st != KH_OK) return st;
    FileCloser fc{f};
    st = kh_create(out, &cfg, ws, bytes, stream);
    if (st != KH_OK) return st;
    return guard(*out, [&] { (*out)->eng->load_checkpoint(fc.f); });
}

kh_status kh_set_state(kh_ctx* ctx, const double* A, const double* B) {
    KH_RANGE();
    return guard(ctx, [&] {
        if (!A || !B) kh::fail(KH_EINVAL, "null tensor");
        ctx->eng->set_state(A, B);
    });
}

kh_status kh_get_state(kh_ctx* ctx, double* A, double* B) {
    KH_RANGE();
    return guard(ctx, [&] {
        if (!A || !B) kh::fail(KH_EINVAL, "null tensor");
        ctx->eng->get_state(A, B);
    });
}

kh_status ctm_set_tensor(kh_ctx* ctx, int slot, const double* T, int p) {
    KH_RANGE();
    return guard(ctx, [&] {
        if (!slot_ok(ctx, slot) || !T) kh::fail(KH_EINVAL, "bad slot or tensor");
        ctx->eng->set_tensor(slot, T, p);
    });
}

kh_status ctm_build_composite(kh_ctx* ctx, int slot, int gamma, const double* gate) {
    KH_RANGE();
    return guard(ctx, [&] {
        if (!slot_ok(ctx, slot)) kh::fail(KH_EINVAL, "bad slot");
        ctx->eng->build_composite(slot, gamma, gate);
    });
}

kh_status ctm_init(kh_ctx* ctx, int slot, const double* edge) {
    KH_RANGE();
    return guard(ctx, [&] {
        if (!slot_ok(ctx, slot)) kh::fail(KH_EINVAL, "bad slot");
        ctx->eng->init_env(slot, edge);
    });
}

kh_status ctm_copy_env(kh_ctx* ctx, int dst, int src) {
    KH_RANGE();
    return guard(ctx, [&] {
        if (!slot_ok(ctx, dst) || !slot_ok(ctx, src)) kh::fail(KH_EINVAL, "bad slot");
        ctx->eng->copy_env(dst, src);
    });
}

kh_status ctm_sweep(kh_ctx* ctx, int slot, int max_sweeps, int min_sweeps, double tol, int* done,
                    double* delta) {
    KH_RANGE();
    kh_status s = KH_OK;
    int n = 0;
    double dl = 0.0;
    s = guard(ctx, [&] {
        if (!slot_ok(ctx, slot) || max_sweeps < 1) kh::fail(KH_EINVAL, "bad slot or sweep count");
        n = ctx->eng->sweep(slot, max_sweeps, min_sweeps, tol, &dl);
    });
    if (s != KH_OK) return s;
    if (done) *done = n;
    if (delta) *delta = dl;
    if (tol >= 0.0 && !(dl < tol)) {
        ctx->err = "CTM did not reach the tolerance within max_sweeps";
        return KH_ENOCONV;
    }
    return KH_OK;
}

kh_status ctm_projectors(kh_ctx* ctx, int slot, int dir, double* spec, double* trunc) {
    KH_RANGE();
    return guard(ctx, [&] {
        if (!slot_ok(ctx, slot) || dir < 0 || dir > 3) kh::fail(KH_EINVAL, "bad slot or dir");
        ctx->eng->projectors_out(slot, dir, spec, trunc);
    });
}

kh_status ctm_get_env(kh_ctx* ctx, int slot, double* C, double* E) {
    KH_RANGE();
    return guard(ctx, [&] {
        if (!slot_ok(ctx, slot)) kh::fail(KH_EINVAL, "bad slot");
        ctx->eng->get_env(slot, C, E);
    });
}

kh_status ctm_metric(kh_ctx* ctx, int slot, double* N) {
    KH_RANGE();
    return guard(ctx, [&] {
        if (!slot_ok(ctx, slot) || !N) kh::fail(KH_EINVAL, "bad slot");
        ctx->eng->metric(slot, N);
    });
}

kh_status ctm_kappa(kh_ctx* ctx, int slot, double* kappa) {
    KH_RANGE();
    return guard(ctx, [&] {
        if (!slot_ok(ctx, slot) || !kappa) kh::fail(KH_EINVAL, "bad slot");
        *kappa = ctx->eng->kappa(slot);
    });
}

kh_status ctm_correlation_length(kh_ctx* ctx, int slot, int direction, int max_iter, double tol,
                                 double* host_out) {
    KH_RANGE();
    return guard(ctx, [&] {
        if (!slot_ok(ctx, slot) || !host_out || max_iter < 1 || !(tol >= 0.0)) kh::fail(KH_EINVAL, "bad arguments");
        ctx->eng->correlation_length(slot, direction, max_iter, tol, host_out);
    });
}

kh_status ctm_plaquette(kh_ctx* ctx, int slot, const double* host_ops, double* host_out) {
    KH_RANGE();
    return guard(ctx, [&] {
        if (!slot_ok(ctx, slot) || !host_ops || !host_out) kh::fail(KH_EINVAL, "bad arguments");
        ctx->eng->plaquette(slot, host_ops, host_out);
    });
}

kh_status ctm_flux(kh_ctx* ctx, int slot, int gamma, double* host_out) {
    KH_RANGE();
    return guard(ctx, [&] {
        if (!slot_ok(ctx, slot) || !host_out || gamma < 0 || gamma > 2) kh::fail(KH_EINVAL, "bad arguments");
        if (ctx->eng->slot_p(slot) != 16) kh::fail(KH_EINVAL, "slot does not hold a composite (p = 16)");
        std::vector<double> ops(4 * 256);
        kh::flux_operators(gamma, ops.data());
        double r[2];
        ctx->eng->plaquette(slot, ops.data(), r);
        host_out[0] = -r[0];         // sigma^y sigma^y = -Ytilde Ytilde
        host_out[1] = r[1];
    });
}

kh_status ctm_expval(kh_ctx* ctx, int slot, const double* ops, int n_ops, double* vals) {
    KH_RANGE();
    return guard(ctx, [&] {
        if (!slot_ok(ctx, slot) || !ops || !vals) kh::fail(KH_EINVAL, "bad arguments");
        ctx->eng->expval(slot, ops, n_ops, vals);
    });
}

kh_status eefu_apply_gate(kh_ctx* ctx, int gamma, const double* gate, int mx, int mn, double tol,
                          double* info) {
    KH_RANGE();
    return guard(ctx, [&] {
        if (!gate || mx < 1) kh::fail(KH_EINVAL, "bad gate or sweep count");
        ctx->eng->apply_gate(gamma, gate, mx, mn, tol, info);
    });
}

kh_status eefu_cost_gradient(kh_ctx* ctx, int gamma, const double* gate, const double* A2, const double* B2, int mx,
                             int mn, double tol, double* gA, double* gB, double* cost) {
    KH_RANGE();
    return guard(ctx, [&] {
        if (!gate || !A2 || !B2 || !gA || !gB || !cost || mx < 0) kh::fail(KH_EINVAL, "bad arguments");
        ctx->eng->cost_gradient(gamma, gate, A2, B2, mx, mn, tol, gA, gB, cost);
    });
}

kh_status observables(kh_ctx* ctx, const double* H, double hA, double hB, int mx, int mn, double tol,
                      double* out) {
    KH_RANGE();
    return guard(ctx, [&] {
        if (!H || !out || mx < 1) kh::fail(KH_EINVAL, "bad arguments");
        ctx->eng->observables(H, hA, hB, mx, mn, tol, out);
    });
}

kh_status kh_bond_hamiltonian(int gamma, double J, double Kg, double hA, double hB, double* H) {
    KH_RANGE();
    if (gamma < 0 || gamma > 2 || !H) return KH_EINVAL;
    bond_h(gamma, J, Kg, hA, hB, H);
    return KH_OK;
}

kh_status kh_gate(const double* H, double tau, double* g) {
    KH_RANGE();
    if (!H || !g) return KH_EINVAL;
    gate_from_h(H, tau, g);
    return KH_OK;
}

kh_status kh_flux_operators(int gamma, double* ops) {
    KH_RANGE();
    if (!ops || gamma < 0 || gamma > 2) return KH_EINVAL;
    kh::flux_operators(gamma, ops);
    return KH_OK;
}

kh_status eefu_trotter_step(kh_ctx* ctx, double J, const double* Kxyz, double hA, double hB, double dbeta,
                            int mx, int mn, double tol, double* info) {
    KH_RANGE();
    return guard(ctx, [&] {
        if (!Kxyz || mx < 1) kh::fail(KH_EINVAL, "bad arguments");
        static const int order[5] = {0, 1, 2, 1, 0};
        const double taus[5] = {dbeta / 4, dbeta / 4, dbeta / 2, dbeta / 4, dbeta / 4};
        double worst = 0.0, sweeps = 0.0, iters = 0.0, tr = 0.0;
        for (int l = 0; l < 5; ++l) {
            int g = order[l];
            double H[16], G[16], inf[4];
            bond_h(g, J, Kxyz[g], g == 2 ? hA : 0.0, g == 2 ? hB : 0.0, H);
            gate_from_h(H, taus[l], G);
            ctx->eng->apply_gate(g, G, mx, mn, tol, info ? inf : nullptr);
            if (info) {
                worst = std::fmax(worst, inf[0]);
                sweeps += inf[1];
                iters += inf[2];
                tr = std::fmax(tr, inf[3]);
            }
        }
        if (info) { info[0] = worst; info[1] = sweeps; info[2] = iters; info[3] = tr; }
    });
}

namespace {

// The trajectory of eefu_evolve for one context (throws kh::Error).
void evolve_one(kh_ctx* ctx, double J, const double* Kxyz, double hA, double hB, double dbeta, int n_steps,
                int measure_every, int mx, int mn, double tol, int obs_mx, int obs_mn, double obs_tol,
                double* traj, double* wflux = nullptr) {
    if (!Kxyz || !traj || mx < 1 || obs_mx < 1 || n_steps < 1 || measure_every < 1 || !(dbeta > 0.0))
        kh::fail(KH_EINVAL, "bad arguments");
    std::vector<double> wops;
    if (wflux) {                       // the flux from the z mapping's observables slot
        if (ctx->eng->dm.nslots < 6) kh::fail(KH_EINVAL, "the flux needs the six slots of the observables");
        wops.resize(4 * 256);
        kh::flux_operators(2, wops.data());
    }
    static const int order[5] = {0, 1, 2, 1, 0};
    const double taus[5] = {dbeta / 4, dbeta / 4, dbeta / 2, dbeta / 4, dbeta / 4};
    double H3[48], G[5][16];
    for (int g = 0; g < 3; ++g) bond_h(g, J, Kxyz[g], 0.0, 0.0, H3 + 16 * g);
    for (int l = 0; l < 5; ++l) {
        double H[16];
        const int g = order[l];
        bond_h(g, J, Kxyz[g], g == 2 ? hA : 0.0, g == 2 ? hB : 0.0, H);
        gate_from_h(H, taus[l], G[l]);
    }
    const int nm = n_steps / measure_every;
    const double beta0 = ctx->eng->beta;
    for (int n = 1; n <= n_steps; ++n) {
        for (int l = 0; l < 5; ++l) ctx->eng->apply_gate(order[l], G[l], mx, mn, tol, nullptr);
        ctx->eng->beta += dbeta;
        if (n % measure_every == 0) {
            double* row = traj + (long long)(n / measure_every - 1) * kTrajCols;
            double out[12];
            ctx->eng->observables(H3, hA, hB, obs_mx, obs_mn, obs_tol, out);
            row[0] = beta0 + n * dbeta;
            for (int i = 0; i < 10; ++i) row[1 + i] = out[i];
            row[11] = out[10];
            if (wflux) {
                double r[2];
                ctx->eng->plaquette(5, wops.data(), r);
                wflux[n / measure_every - 1] = -r[0];       // sigma^y sigma^y = -Ytilde Ytilde
            }
        }
    }
    // C = dE/dT = -beta^2 dE/dbeta by central differences on the uniform
    // measurement grid; NaN at the two ends
    for (int i = 0; i < nm; ++i) {
        double* row = traj + (long long)i * kTrajCols;
        if (i == 0 || i == nm - 1) {
            row[12] = NAN;
            continue;
        }
        const double* lo = row - kTrajCols;
        const double* hi = row + kTrajCols;
        row[12] = -row[0] * row[0] * (hi[1] - lo[1]) / (hi[0] - lo[0]);
    }
}

}  // namespace

kh_status eefu_evolve(kh_ctx* ctx, double J, const double* Kxyz, double hA, double hB, double dbeta, int n_steps,
                      int measure_every, int mx, int mn, double tol, int obs_mx, int obs_mn, double obs_tol,
                      double* traj) {
    KH_RANGE();
    return guard(ctx, [&] {
        evolve_one(ctx, J, Kxyz, hA, hB, dbeta, n_steps, measure_every, mx, mn, tol, obs_mx, obs_mn, obs_tol, traj);
    });
}

kh_status eefu_evolve_flux(kh_ctx* ctx, double J, const double* Kxyz, double hA, double hB, double dbeta,
                           int n_steps, int measure_every, int mx, int mn, double tol, int obs_mx, int obs_mn,
                           double obs_tol, double* traj, double* host_flux) {
    KH_RANGE();
    return guard(ctx, [&] {
        if (!host_flux) kh::fail(KH_EINVAL, "bad arguments");
        evolve_one(ctx, J, Kxyz, hA, hB, dbeta, n_steps, measure_every, mx, mn, tol, obs_mx, obs_mn, obs_tol, traj,
                   host_flux);
    });
}

kh_status eefu_evolve_batch(kh_ctx* const* ctxs, int n, const double* J, const double* Kxyz, const double* hA,
                            const double* hB, double dbeta, int n_steps, int measure_every, int mx, int mn,
                            double tol, int obs_mx, int obs_mn, double obs_tol, double* traj, kh_status* status) {
    KH_RANGE();
    if (!ctxs || n < 1 || !J || !Kxyz || !traj || measure_every < 1 || n_steps < 1) return KH_EINVAL;
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i] || !ctxs[i]->eng) return KH_EINVAL;
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return KH_EINVAL;          // one thread per context
    }
    const long long rows = (long long)(n_steps / measure_every) * kTrajCols;
    std::vector<kh_status> st(n, KH_OK);
    std::vector<std::thread> pool;
    pool.reserve(n);
    for (int i = 0; i < n; ++i)
        pool.emplace_back([&, i] {
            kh_ctx* c = ctxs[i];
            st[i] = guard(c, [&] {
                KH_CUDA(cudaSetDevice(c->device));
                evolve_one(c, J[i], Kxyz + 3 * i, hA ? hA[i] : 0.0, hB ? hB[i] : 0.0, dbeta, n_steps,
                           measure_every, mx, mn, tol, obs_mx, obs_mn, obs_tol, traj + i * rows);
            });
        });
    for (auto& t : pool) t.join();
    kh_status first = KH_OK;
    for (int i = 0; i < n; ++i) {
        if (status) status[i] = st[i];
        if (first == KH_OK && st[i] != KH_OK) first = st[i];
    }
    return first;
}

unsigned long long kh_launch_count(void) { return kh::g_launches.load(std::memory_order_relaxed); }

kh_status kh_profile(kh_ctx* ctx, int enable, double* out) {
    KH_RANGE();
    return guard(ctx, [&] {
        kh::EngineBase* e = ctx->eng;
        if (enable) {
            for (auto& c : e->prof) { c.used = 0; c.flops = 0.0; }
            e->prof_on = true;
            e->reset_counters();
            return;
        }
        KH_CUDA(cudaStreamSynchronize(e->st));
        e->prof_on = false;
        for (int k = 0; k < kh::EngineBase::kProfCats; ++k) {
            double ms = 0.0;
            for (int i = 0; i < e->prof[k].used; ++i) {
                float t = 0.f;
                KH_CUDA(cudaEventElapsedTime(&t, e->prof[k].a[i], e->prof[k].b[i]));
                ms += t;
            }
            if (out) {
                out[3 * k + 0] = e->prof[k].used;
                out[3 * k + 1] = ms;
                out[3 * k + 2] = e->prof[k].flops;
            }
        }
        if (out) out[3 * 7 + 2] = e->read_counter();   // one-sided Jacobi: total sweeps
    });
}

}  // extern "C"
