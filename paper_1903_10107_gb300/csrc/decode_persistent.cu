// Host side of the persistent mixed-rate decoder: argument checks, group
// width, grid sizing, message scratch, dispatch to the kernel of the code's
// unroll width, and the C ABI.  The kernel is in decode_persistent.cuh.
#include <string>
#include <vector>

#include "decode_persistent.cuh"

namespace {

using ldpc_dec::PersistArgs;
using ldpc_dec::smem_bytes;

int dispatch(const ldpc_code* c, const PersistArgs& A, int W, int ctas_per_sm, int threads, int* grid, bool dry,
             cudaStream_t st) {
    switch (ldpc_dec::pick_maxh(c->max_deg)) {
#define LDPC_PERSIST_CASE(M) \
    case M:                  \
        return ldpc_dec::persist_launch<M>(c, A, W, ctas_per_sm, threads, grid, dry, st);
        LDPC_MAXH_LIST(LDPC_PERSIST_CASE)
#undef LDPC_PERSIST_CASE
        default:
            return ldpc::fail(LDPC_EUNSUPPORTED, "persistent decode: row degree above 64");
    }
}

}  // namespace

extern "C" {

int ldpc_code_reserve_persistent(ldpc_code* code, int list_len, int words, int ctas_per_sm, int threads) {
    if (!code || list_len < 0) return ldpc::fail(LDPC_EINVAL, "ldpc_code_reserve_persistent: bad argument");
    if (list_len == 0) return LDPC_OK;
    const int W = words > 0 ? words : 1;
    if (W != 1 && W != 2 && W != 4) return ldpc::fail(LDPC_EINVAL, "ldpc_code_reserve_persistent: bad words");
    PersistArgs A{};
    A.list_len = list_len;
    int grid = 0;
    int rc = dispatch(code, A, W, ctas_per_sm, threads, &grid, true, nullptr);
    if (rc) return rc;
    return ldpc::ensure_arena(code, (size_t)grid * 4 * W * (size_t)code->edges);
}

}  // extern "C"

namespace {

int reconcile_common(const ldpc_code* c, const uint8_t* bob_bits, const int8_t* llr_mag, const int32_t* rank,
                     const int32_t* n_short, const int32_t* n_punct, const uint8_t* known,
                     const uint8_t* target_syndrome, int batch, const int32_t* frame_list, int list_len, int max_iter,
                     int stall_window, const int32_t* reveal, int max_rounds, int words, int ctas_per_sm,
                     int threads, uint8_t* out_bits, int32_t* out_iters, uint8_t* out_ok, int32_t* out_rounds,
                     void* stream, int epoch_iters = 0, int resume = 0, void* epoch_state = nullptr,
                     size_t epoch_state_bytes = 0, int32_t* out_claimed = nullptr) {
    using ldpc::fail;
    if (!c) return fail(LDPC_EINVAL, "persistent decode: NULL code");
    if (list_len < 0 || batch < 0 || max_iter < 1 || stall_window < 0)
        return fail(LDPC_EINVAL, "persistent decode: bad batch, list length, max_iter or stall window");
    if (stall_window > 0 && c->m > 0xFFFF)
        return fail(LDPC_EUNSUPPORTED, "persistent decode: the stall window counts checks in 16 bits (m <= 65535)");
    if (!frame_list && list_len > batch) return fail(LDPC_EINVAL, "persistent decode: list_len > batch");
    if (list_len == 0 && epoch_iters <= 0) return LDPC_OK;  // an epoch also runs the lanes already in flight
    if (!bob_bits || !llr_mag || !target_syndrome || !out_bits || !out_iters || !out_ok)
        return fail(LDPC_EINVAL, "persistent decode: NULL buffer");
    if ((n_short || n_punct) && !rank) return fail(LDPC_EINVAL, "persistent decode: counts need a rank table");
    if (n_short && !known) return fail(LDPC_EINVAL, "persistent decode: shortening needs known values");
    const int smem_limit = ldpc::max_dyn_smem(c->device);
    int W = words;
    if (W == 0) {
        int sms = 0;
        LDPC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
        W = 1;
        for (int cand = 4; cand >= 2; cand >>= 1)  // wider groups only while every SM still gets two
            if ((int64_t)smem_bytes(c, cand) <= smem_limit && (int64_t)list_len >= (int64_t)cand * 4 * 2 * sms) {
                W = cand;
                break;
            }
    }
    if ((W != 1 && W != 2 && W != 4) || (int64_t)smem_bytes(c, W) > smem_limit)
        return fail(LDPC_EINVAL, "persistent decode: unsupported words per row");
    if (epoch_iters > 0 && words <= 0) return fail(LDPC_EINVAL, "epoch decode: give words explicitly");
    PersistArgs A{};
    A.tab = c->d_tab;
    A.Mb = c->Mb;
    A.nblk = c->nblk;
    A.Z = c->Z;
    A.n = c->n;
    A.m = c->m;
    A.bob = bob_bits;
    A.mag = llr_mag;
    A.rank = rank;
    A.n_short = n_short;
    A.n_punct = n_punct;
    A.known = known;
    A.syn = target_syndrome;
    A.list = frame_list;
    A.batch = batch;
    A.list_len = list_len;
    A.max_iter = max_iter;
    A.stall = stall_window;
    A.out_bits = out_bits;
    A.out_iters = out_iters;
    A.out_ok = out_ok;
    A.reveal = reveal;
    A.max_rounds = reveal ? max_rounds : 0;
    A.out_rounds = out_rounds;
    A.queue = c->d_queue;
    A.epoch_iters = epoch_iters > 0 ? epoch_iters : 0;
    A.resume = resume ? 1 : 0;
    int grid = 0;
    int rc = dispatch(c, A, W, ctas_per_sm, threads, &grid, true, (cudaStream_t)stream);
    if (rc) return rc;
    if (A.epoch_iters) {
        const ldpc_dec::EpochLayout L = ldpc_dec::epoch_layout(c->n, c->m, W, grid);
        if (!epoch_state || epoch_state_bytes < L.total)
            return fail(LDPC_EINVAL, "epoch decode: the lane-state buffer needs " + std::to_string(L.total) +
                                         " bytes for this launch shape (ldpc_epoch_state_bytes)");
        if (reinterpret_cast<uintptr_t>(epoch_state) % 256)
            return fail(LDPC_EINVAL, "epoch decode: the lane-state buffer must be 256-byte aligned");
        uint8_t* base = static_cast<uint8_t*>(epoch_state);
        A.lane_save = reinterpret_cast<int32_t*>(base + L.lanes);
        A.word_save = reinterpret_cast<uint32_t*>(base + L.words);
        A.e_save = reinterpret_cast<uint32_t*>(base + L.soft);
        A.syn_save = base + L.syn;
    }
    const size_t need = (size_t)grid * 4 * W * (size_t)c->edges;
    rc = ldpc::ensure_arena(const_cast<ldpc_code*>(c), need);
    if (rc) return rc;
    A.msg = reinterpret_cast<uint32_t*>(c->arena);
    rc = dispatch(c, A, W, ctas_per_sm, threads, &grid, false, (cudaStream_t)stream);
    if (rc || !out_claimed) return rc;
    LDPC_CUDA_TRY(cudaMemcpyAsync(out_claimed, c->d_queue, sizeof(int32_t), cudaMemcpyDeviceToDevice,
                                  (cudaStream_t)stream));
    return LDPC_OK;
}

}  // namespace

extern "C" {

int ldpc_epoch_state_bytes(const ldpc_code* code, int words, int ctas_per_sm, int threads, size_t* bytes,
                           int* grid) {
    using ldpc::fail;
    if (!code || !bytes || (words != 1 && words != 2 && words != 4))
        return fail(LDPC_EINVAL, "ldpc_epoch_state_bytes: bad argument (words must be 1, 2 or 4)");
    PersistArgs A{};
    A.list_len = 1;
    A.epoch_iters = 1;
    int g = 0;
    int rc = dispatch(code, A, words, ctas_per_sm, threads, &g, true, nullptr);
    if (rc) return rc;
    *bytes = ldpc_dec::epoch_layout(code->n, code->m, words, g).total;
    if (grid) *grid = g;
    return LDPC_OK;
}

int ldpc_reconcile_epoch(const ldpc_code* code, const uint8_t* bob_bits, const int8_t* llr_mag, const int32_t* rank,
                         const int32_t* n_short, const int32_t* n_punct, const uint8_t* known,
                         const uint8_t* target_syndrome, int batch, const int32_t* frame_list, int list_len,
                         int max_iter, int stall_window, int epoch_iters, int resume, void* lane_state,
                         size_t lane_state_bytes, int words, int ctas_per_sm, int threads, uint8_t* out_bits,
                         int32_t* out_iters, uint8_t* out_ok, int32_t* out_claimed, void* stream) {
    using ldpc::fail;
    if (epoch_iters < 1) return fail(LDPC_EINVAL, "epoch decode: epoch_iters must be >= 1");
    if (!out_claimed) return fail(LDPC_EINVAL, "epoch decode: NULL out_claimed");
    return reconcile_common(code, bob_bits, llr_mag, rank, n_short, n_punct, known, target_syndrome, batch,
                            frame_list, list_len, max_iter, stall_window, nullptr, 0, words, ctas_per_sm, threads,
                            out_bits, out_iters, out_ok, nullptr, stream, epoch_iters, resume, lane_state,
                            lane_state_bytes, out_claimed);
}

int ldpc_reconcile_persistent(const ldpc_code* code, const uint8_t* bob_bits, const int8_t* llr_mag,
                              const int32_t* rank, const int32_t* n_short, const int32_t* n_punct,
                              const uint8_t* known, const uint8_t* target_syndrome, int batch,
                              const int32_t* frame_list, int list_len, int max_iter, int stall_window,
                              int words, int ctas_per_sm, int threads, uint8_t* out_bits, int32_t* out_iters,
                              uint8_t* out_ok, void* stream) {
    return reconcile_common(code, bob_bits, llr_mag, rank, n_short, n_punct, known, target_syndrome, batch,
                            frame_list, list_len, max_iter, stall_window, nullptr, 0, words, ctas_per_sm, threads,
                            out_bits, out_iters, out_ok, nullptr, stream);
}

int ldpc_reconcile_interactive(const ldpc_code* code, const uint8_t* bob_bits, const int8_t* llr_mag,
                               const int32_t* rank, const int32_t* n_short, const int32_t* n_punct,
                               const uint8_t* known, const uint8_t* target_syndrome, int batch,
                               const int32_t* frame_list, int list_len, int max_iter, int stall_window,
                               const int32_t* reveal, int max_rounds, int words, int ctas_per_sm, int threads,
                               uint8_t* out_bits, int32_t* out_iters, uint8_t* out_ok, int32_t* out_rounds,
                               void* stream) {
    using ldpc::fail;
    if (!reveal || !out_rounds || max_rounds < 0)
        return fail(LDPC_EINVAL, "interactive decode: needs the reveal table, out_rounds and max_rounds >= 0");
    if (!rank || !n_short || !n_punct || !known)
        return fail(LDPC_EINVAL, "interactive decode: needs the rank table, both counts and the known values");
    return reconcile_common(code, bob_bits, llr_mag, rank, n_short, n_punct, known, target_syndrome, batch,
                            frame_list, list_len, max_iter, stall_window, reveal, max_rounds, words, ctas_per_sm,
                            threads, out_bits, out_iters, out_ok, out_rounds, stream);
}

int ldpc_reconcile_interactive_host(const ldpc_code* code, const uint8_t* bob_bits, const int8_t* llr_mag,
                                    const int32_t* rank, const int32_t* n_short, const int32_t* n_punct,
                                    const uint8_t* known, const uint8_t* target_syndrome, int batch,
                                    const int32_t* frame_list, int list_len, int max_iter, int stall_window,
                                    const int32_t* reveal, int max_rounds, int words, int ctas_per_sm, int threads,
                                    uint8_t* out_bits, int32_t* out_iters, uint8_t* out_ok, int32_t* out_rounds,
                                    int64_t* h2d_bytes, int64_t* d2h_bytes, void* stream) {
    using ldpc::fail;
    if (!code) return fail(LDPC_EINVAL, "interactive decode (host buffers): NULL code");
    if (batch < 0 || list_len < 0 || max_rounds < 0)
        return fail(LDPC_EINVAL, "interactive decode (host buffers): bad batch, list length or max_rounds");
    if (!bob_bits || !llr_mag || !rank || !n_short || !n_punct || !known || !target_syndrome || !reveal ||
        !out_bits || !out_iters || !out_ok || !out_rounds)
        return fail(LDPC_EINVAL, "interactive decode (host buffers): NULL buffer");
    if (!frame_list && list_len > batch)
        return fail(LDPC_EINVAL, "interactive decode (host buffers): list_len > batch");
    ldpc_code* c = const_cast<ldpc_code*>(code);
    const size_t B = (size_t)batch, nb = ((size_t)c->n + 7) / 8, mb = ((size_t)c->m + 7) / 8;
    const size_t R1 = (size_t)max_rounds + 1, L = frame_list ? (size_t)list_len : 0;
    // the device copies, each part 256-byte aligned
    size_t off = 0;
    auto part = [&off](size_t bytes) {
        const size_t o = off;
        off = (off + bytes + 255) & ~(size_t)255;
        return o;
    };
    const size_t o_bob = part(B * nb), o_known = part(B * nb), o_syn = part(B * mb), o_mag = part(B);
    const size_t o_ns = part(4 * B), o_np = part(4 * B), o_rev = part(4 * B * R1), o_rank = part(4 * (size_t)c->n);
    const size_t o_list = part(4 * L), o_bits = part(B * nb), o_it = part(4 * B), o_ok = part(B), o_rd = part(4 * B);
    int rc = ldpc::ensure_io(c, off > 0 ? off : 256);
    if (rc) return rc;
    uint8_t* d = static_cast<uint8_t*>(c->io);
    cudaStream_t st = (cudaStream_t)stream;
    int64_t in = 0, out = 0;
    auto h2d = [&](size_t o, const void* src, size_t bytes) -> int {
        if (!bytes) return LDPC_OK;
        LDPC_CUDA_TRY(cudaMemcpyAsync(d + o, src, bytes, cudaMemcpyHostToDevice, st));
        in += (int64_t)bytes;
        return LDPC_OK;
    };
    if ((rc = h2d(o_bob, bob_bits, B * nb)) || (rc = h2d(o_known, known, B * nb)) ||
        (rc = h2d(o_syn, target_syndrome, B * mb)) || (rc = h2d(o_mag, llr_mag, B)) ||
        (rc = h2d(o_ns, n_short, 4 * B)) || (rc = h2d(o_np, n_punct, 4 * B)) ||
        (rc = h2d(o_rev, reveal, 4 * B * R1)) || (rc = h2d(o_rank, rank, 4 * (size_t)c->n)) ||
        (rc = h2d(o_list, frame_list, 4 * L)))
        return rc;
    // Frames the list leaves out keep their outputs: when it does not cover every frame, the device
    // outputs start as copies of the caller's.
    bool covers = !frame_list && list_len >= batch;
    if (frame_list) {
        std::vector<char> seen(B, 0);
        size_t distinct = 0;
        for (size_t i = 0; i < L; ++i) {
            const int32_t f = frame_list[i];
            if (f >= 0 && f < batch && !seen[(size_t)f]) {
                seen[(size_t)f] = 1;
                ++distinct;
            }
        }
        covers = distinct == B;
    }
    if (!covers && ((rc = h2d(o_bits, out_bits, B * nb)) || (rc = h2d(o_it, out_iters, 4 * B)) ||
                    (rc = h2d(o_ok, out_ok, B)) || (rc = h2d(o_rd, out_rounds, 4 * B))))
        return rc;
    auto at = [d](size_t o) { return d + o; };
    rc = reconcile_common(c, at(o_bob), reinterpret_cast<const int8_t*>(at(o_mag)),
                          reinterpret_cast<const int32_t*>(at(o_rank)), reinterpret_cast<const int32_t*>(at(o_ns)),
                          reinterpret_cast<const int32_t*>(at(o_np)), at(o_known), at(o_syn), batch,
                          frame_list ? reinterpret_cast<const int32_t*>(at(o_list)) : nullptr, list_len, max_iter,
                          stall_window, reinterpret_cast<const int32_t*>(at(o_rev)), max_rounds, words, ctas_per_sm,
                          threads, at(o_bits), reinterpret_cast<int32_t*>(at(o_it)), at(o_ok),
                          reinterpret_cast<int32_t*>(at(o_rd)), stream);
    if (rc) return rc;
    auto d2h = [&](void* dst, size_t o, size_t bytes) -> int {
        if (!bytes) return LDPC_OK;
        LDPC_CUDA_TRY(cudaMemcpyAsync(dst, d + o, bytes, cudaMemcpyDeviceToHost, st));
        out += (int64_t)bytes;
        return LDPC_OK;
    };
    if ((rc = d2h(out_bits, o_bits, B * nb)) || (rc = d2h(out_iters, o_it, 4 * B)) || (rc = d2h(out_ok, o_ok, B)) ||
        (rc = d2h(out_rounds, o_rd, 4 * B)))
        return rc;
    LDPC_CUDA_TRY(cudaStreamSynchronize(st));
    if (h2d_bytes) *h2d_bytes = in;
    if (d2h_bytes) *d2h_bytes = out;
    return LDPC_OK;
}

}  // extern "C"
