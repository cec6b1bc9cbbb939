// Checkpoint and resume of a context: the persistent state only.  Scratch is
// not saved, and the operands derived from a slot's site tensor (rotated
// frames, double-layer operands, their 3xTF32 low parts) are rebuilt from
// the saved FP64 master on load, exactly as loading the tensor would.
//
// Payload after the header written by kh_save (magic, kh_config):
//   int32 {sizeof(T), D, chi, n, kk, n_slots}, uint64 rng counter,
//   A, B (4 D^3 doubles each),
//   per slot: int32 {p, env_valid, prev_valid, warm[0..3], sweeps_done},
//     Ts (p_max D^4 doubles), C (4 chi^2), E (4 chi D^2 chi), Vw (4 n kk, in
//     the compute type), spec (4 chi), prev (4 chi), trunc (4), delta (1),
//     live (4 kk int32).
// Native byte order and widths: a checkpoint is read back on the same kind
// of machine that wrote it.
#include "engine.cuh"

namespace kh {

namespace {

void put(std::FILE* f, const void* p, size_t n) {
    if (n && std::fwrite(p, 1, n, f) != n) fail(KH_EINVAL, "checkpoint: write failed");
}

void get(std::FILE* f, void* p, size_t n) {
    if (n && std::fread(p, 1, n, f) != n) fail(KH_EINVAL, "checkpoint: file truncated");
}

// device array <-> file through one reused host buffer
void put_dev(std::FILE* f, const void* dev, size_t n, cudaStream_t st, std::vector<unsigned char>& buf) {
    buf.resize(n);
    KH_CUDA(cudaMemcpyAsync(buf.data(), dev, n, cudaMemcpyDeviceToHost, st));
    KH_CUDA(cudaStreamSynchronize(st));
    put(f, buf.data(), n);
}

void get_dev(std::FILE* f, void* dev, size_t n, cudaStream_t st, std::vector<unsigned char>& buf) {
    buf.resize(n);
    get(f, buf.data(), n);
    KH_CUDA(cudaMemcpyAsync(dev, buf.data(), n, cudaMemcpyHostToDevice, st));
    KH_CUDA(cudaStreamSynchronize(st));     // the buffer is reused by the next array
}

}  // namespace

template <typename T>
void Engine<T>::save_checkpoint(std::FILE* f) {
    bind(0);                                // every call has joined its lanes into lane 0
    const Dims& d = dm;
    const size_t chi2 = (size_t)d.chi * d.chi, E1 = (size_t)d.chi * d.d2 * d.chi, D3 = (size_t)d.D * d.D * d.D;
    const int32_t hdr[6] = {(int32_t)sizeof(T), d.D, d.chi, d.n, d.kk, d.nslots};
    put(f, hdr, sizeof(hdr));
    put(f, &rng_counter, sizeof(rng_counter));
    std::vector<unsigned char> buf;
    put_dev(f, A, sizeof(double) * 4 * D3, st, buf);
    put_dev(f, B, sizeof(double) * 4 * D3, st, buf);
    for (const Slot<T>& s : slots) {
        const int32_t meta[8] = {s.p, s.env_valid, s.prev_valid, s.warm[0], s.warm[1], s.warm[2], s.warm[3],
                                 s.sweeps_done};
        put(f, meta, sizeof(meta));
        put_dev(f, s.Ts, sizeof(double) * (size_t)d.pmax * d.D4, st, buf);
        put_dev(f, s.C, sizeof(double) * 4 * chi2, st, buf);
        put_dev(f, s.E, sizeof(double) * 4 * E1, st, buf);
        put_dev(f, s.Vw, sizeof(T) * 4 * (size_t)d.n * d.kk, st, buf);
        put_dev(f, s.spec, sizeof(double) * 4 * d.chi, st, buf);
        put_dev(f, s.prev, sizeof(double) * 4 * d.chi, st, buf);
        put_dev(f, s.trunc, sizeof(double) * 4, st, buf);
        put_dev(f, s.delta, sizeof(double), st, buf);
        put_dev(f, s.live, sizeof(int) * 4 * (size_t)d.kk, st, buf);
    }
}

template <typename T>
void Engine<T>::load_checkpoint(std::FILE* f) {
    bind(0);
    const Dims& d = dm;
    const size_t chi2 = (size_t)d.chi * d.chi, E1 = (size_t)d.chi * d.d2 * d.chi, D3 = (size_t)d.D * d.D * d.D;
    int32_t hdr[6];
    get(f, hdr, sizeof(hdr));
    if (hdr[0] != (int32_t)sizeof(T) || hdr[1] != d.D || hdr[2] != d.chi || hdr[3] != d.n || hdr[4] != d.kk ||
        hdr[5] != d.nslots)
        fail(KH_EINVAL, "checkpoint: layout does not match its own configuration");
    unsigned long long rc = 0;
    get(f, &rc, sizeof(rc));
    std::vector<unsigned char> buf;
    get_dev(f, A, sizeof(double) * 4 * D3, st, buf);
    get_dev(f, B, sizeof(double) * 4 * D3, st, buf);
    for (Slot<T>& s : slots) {
        int32_t meta[8];
        get(f, meta, sizeof(meta));
        if (meta[0] < 0 || meta[0] > d.pmax) fail(KH_EINVAL, "checkpoint: physical dimension out of range");
        get_dev(f, s.Ts, sizeof(double) * (size_t)d.pmax * d.D4, st, buf);
        get_dev(f, s.C, sizeof(double) * 4 * chi2, st, buf);
        get_dev(f, s.E, sizeof(double) * 4 * E1, st, buf);
        get_dev(f, s.Vw, sizeof(T) * 4 * (size_t)d.n * d.kk, st, buf);
        get_dev(f, s.spec, sizeof(double) * 4 * d.chi, st, buf);
        get_dev(f, s.prev, sizeof(double) * 4 * d.chi, st, buf);
        get_dev(f, s.trunc, sizeof(double) * 4, st, buf);
        get_dev(f, s.delta, sizeof(double), st, buf);
        get_dev(f, s.live, sizeof(int) * 4 * (size_t)d.kk, st, buf);
        s.p = meta[0];
        s.env_valid = meta[1] != 0;
        s.prev_valid = meta[2] != 0;
        for (int q = 0; q < 4; ++q) s.warm[q] = meta[3 + q] != 0;
        s.sweeps_done = meta[7];
        if (s.p > 0) build_derived(s);
    }
    rng_counter = rc;
    KH_CUDA(cudaStreamSynchronize(st));
}

template void Engine<double>::save_checkpoint(std::FILE*);
template void Engine<float>::save_checkpoint(std::FILE*);
template void Engine<double>::load_checkpoint(std::FILE*);
template void Engine<float>::load_checkpoint(std::FILE*);

}  // namespace kh
