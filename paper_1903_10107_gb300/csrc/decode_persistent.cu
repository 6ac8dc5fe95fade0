// Host side of the persistent mixed-rate decoder: argument checks, group
// width, grid sizing, message scratch, dispatch to the kernel of the code's
// unroll width, and the C ABI.  The kernel is in decode_persistent.cuh.
#include <string>

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

}  // extern "C"
