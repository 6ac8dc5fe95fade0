// Host side of the batch decoder: argument checks, group width, message
// scratch, dispatch to the kernel of the code's unroll width, and the C ABI.
// The kernel and its launch are in decode_int8.cuh.
#include <mutex>
#include <string>

#include "decode_int8.cuh"

namespace {

using ldpc_dec::DecodeArgs;
using ldpc_dec::smem_bytes;

int launch(const ldpc_code* c, const DecodeArgs& A, int groups, int W, bool tables, cudaStream_t st) {
    switch (ldpc_dec::pick_maxh(c->max_deg)) {
#define LDPC_DECODE_CASE(M) \
    case M:                 \
        return ldpc_dec::decode_launch<M>(c, A, groups, W, tables, st);
        LDPC_MAXH_LIST(LDPC_DECODE_CASE)
#undef LDPC_DECODE_CASE
        default:
            return ldpc::fail(LDPC_EUNSUPPORTED, "decode: row degree above 64");
    }
}

// One word (4 frames) per CTA: a group holds its SM until the slowest of its
// frames stops, so the smallest group wins whenever iteration counts are
// uneven -- n = 4096, 16384 frames at QBER 2 % (max 50): 5.45 ms at one word
// against 6.88 at two and 9.32 at four (the several-words-per-thread kernel),
// 8.26 and 12.07 with one word per thread at two and four -- and loses at
// most 4 % when every frame runs to the cap (QBER 3.5 %, 20 iterations: 4.70
// against 4.53 and 4.48).  ldpc_decode_batch_words takes 2 or 4 explicitly.
int pick_words(const ldpc_code*, int, int, int) { return 1; }

int decode_common(const ldpc_code* c, const int8_t* llr, const uint8_t* syn, int batch, int max_iter,
                  const uint8_t* sq, const int8_t* oq, uint8_t* bits, int32_t* iters, uint8_t* ok,
                  void* stream, int force_words) {
    using ldpc::fail;
    if (!c) return fail(LDPC_EINVAL, "decode: NULL code");
    if (batch < 0) return fail(LDPC_EINVAL, "decode: negative batch");
    if (max_iter < 1) return fail(LDPC_EINVAL, "decode: max_iter must be >= 1");
    if (batch == 0) return LDPC_OK;
    if (!llr || !syn || !bits || !iters || !ok) return fail(LDPC_EINVAL, "decode: NULL buffer");
    const int smem_limit = ldpc::max_dyn_smem(c->device);
    if ((int64_t)smem_bytes(c, 1) > smem_limit)
        return fail(LDPC_EUNSUPPORTED, "decode: soft values of four frames exceed shared memory");
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    int W = force_words > 0 ? force_words : pick_words(c, batch, smem_limit, sms);
    if ((W != 1 && W != 2 && W != 4) || (int64_t)smem_bytes(c, W) > smem_limit)
        return fail(LDPC_EINVAL, "decode: unsupported words per row");
    const int64_t groups = (batch + 4 * W - 1) / (4 * W);
    if (groups > 0x7FFFFFFF) return fail(LDPC_EINVAL, "decode: batch too large");
    const size_t need = (size_t)groups * 4 * W * (size_t)c->edges;
    int rc = ldpc::ensure_arena(const_cast<ldpc_code*>(c), need);
    if (rc) return rc;
    DecodeArgs A{c->d_tab, c->Mb, c->nblk, c->Z, c->n, c->m, llr, syn, batch, max_iter, sq, oq, bits, iters, ok,
                 reinterpret_cast<uint32_t*>(c->arena)};
    return launch(c, A, (int)groups, W, sq || oq, (cudaStream_t)stream);
}

}  // namespace

namespace {

// ---------------------------------------------------------------------------
// Decoding without any device allocation.
//
// Some callers cannot let the library call cudaMalloc: a reconciliation
// daemon that sized all of its device memory at start-up and must not grow it
// while keys stream in, a process whose GPU memory belongs to another
// allocator's fixed pool, or a latency-critical loop that cannot take the
// device-wide synchronisation an allocation or free may cause.  For them the
// decoder's message scratch comes from a fixed array compiled into this
// library instead of the handle's arena.  The array occupies kStaticMsgBytes
// on every GPU that loads the library, until the process exits.
// ---------------------------------------------------------------------------
constexpr size_t kStaticMsgBytes = (size_t)32 << 20;  // 32 MiB of message scratch
__device__ __align__(256) uint32_t g_static_msg[kStaticMsgBytes / sizeof(uint32_t)];

// Cached device addresses of g_static_msg, one per CUDA context.  A context
// is identified by the driver's context id, which is never reused within a
// process: after cudaDeviceReset the primary context is created anew (and
// the library's module loaded again, possibly at another address), and a
// caller's own non-primary context on the same device is another context,
// so neither can pick up a stale address.
struct StaticAddr {
    unsigned long long ctx_id;
    uint32_t* addr;
};
constexpr int kAddrSlots = 64;
std::mutex g_static_mu;
StaticAddr g_static_addr[kAddrSlots] = {};
int g_static_next = 0;

// Driver entry points, resolved through the runtime (the library does not
// link the driver library itself).
typedef int (*ctx_get_current_fn)(void** ctx);
typedef int (*ctx_get_id_fn)(void* ctx, unsigned long long* id);

// Id of the calling thread's current context, or 0 if there is none yet
// (the runtime creates and binds it lazily) or the driver lacks the query.
unsigned long long current_context_id() {
    static ctx_get_current_fn get_cur = nullptr;
    static ctx_get_id_fn get_id = nullptr;
    static bool resolved = false;
    if (!resolved) {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult st;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &st) == cudaSuccess &&
            st == cudaDriverEntryPointSuccess)
            get_cur = reinterpret_cast<ctx_get_current_fn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &st) == cudaSuccess &&
            st == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<ctx_get_id_fn>(f);
        resolved = true;
    }
    void* ctx = nullptr;
    unsigned long long id = 0;
    if (!get_cur || !get_id || get_cur(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
    return id;
}

// Device address of g_static_msg in the current context.  Host code only
// knows the array's host-side stand-in; the address is looked up with
// cudaGetSymbolAddress once per context (the first call in a context also
// loads the library's module there) and cached by context id.
int static_msg_address(uint32_t** out) {
    std::lock_guard<std::mutex> lock(g_static_mu);
    unsigned long long id = current_context_id();
    if (id) {
        for (const StaticAddr& e : g_static_addr)
            if (e.ctx_id == id) {
                *out = e.addr;
                return LDPC_OK;
            }
    }
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_msg);
    if (e != cudaSuccess) return ldpc::cuda_fail(e, "noalloc decode: cudaGetSymbolAddress");
    if (!id) id = current_context_id();  // the lookup has made the context current
    if (id) {
        g_static_addr[g_static_next] = StaticAddr{id, static_cast<uint32_t*>(p)};
        g_static_next = (g_static_next + 1) % kAddrSlots;
    }
    *out = static_cast<uint32_t*>(p);
    return LDPC_OK;
}

}  // namespace

extern "C" {

int ldpc_decode_batch(const ldpc_code* code, const int8_t* llr_in, const uint8_t* target_syndrome, int batch,
                      int max_iter, uint8_t* out_bits, int32_t* out_iters, uint8_t* out_ok, void* stream) {
    return decode_common(code, llr_in, target_syndrome, batch, max_iter, nullptr, nullptr, out_bits, out_iters,
                         out_ok, stream, 0);
}

int ldpc_decode_batch_ex(const ldpc_code* code, const int8_t* llr_in, const uint8_t* target_syndrome,
                         int batch, int max_iter, const uint8_t* scale_q4, const int8_t* offset_q,
                         uint8_t* out_bits, int32_t* out_iters, uint8_t* out_ok, void* stream) {
    return decode_common(code, llr_in, target_syndrome, batch, max_iter, scale_q4, offset_q, out_bits, out_iters,
                         out_ok, stream, 0);
}

// Decode with an explicit number of 32-bit words (4 frames each) per check
// row and CTA: 1, 2 or 4.  Used by the autotuner; 0 picks automatically.
int ldpc_decode_batch_words(const ldpc_code* code, const int8_t* llr_in, const uint8_t* target_syndrome,
                            int batch, int max_iter, int words, uint8_t* out_bits, int32_t* out_iters,
                            uint8_t* out_ok, void* stream) {
    return decode_common(code, llr_in, target_syndrome, batch, max_iter, nullptr, nullptr, out_bits, out_iters,
                         out_ok, stream, words);
}

int ldpc_code_reserve(ldpc_code* code, int batch) {
    if (!code || batch < 0) return ldpc::fail(LDPC_EINVAL, "ldpc_code_reserve: bad argument");
    const size_t need = (size_t)((batch + 15) / 16) * 16 * (size_t)code->edges;
    return ldpc::ensure_arena(code, need);
}

// Same decode as ldpc_decode_batch, with the message scratch taken from the
// library's fixed device array instead of the handle's arena; see the header.
int ldpc_decode_batch_noalloc(const ldpc_code* code, const int8_t* llr_in, const uint8_t* target_syndrome,
                              int batch, int max_iter, uint8_t* out_bits, int32_t* out_iters, uint8_t* out_ok,
                              void* stream) {
    using ldpc::fail;
    const ldpc_code* c = code;
    if (!c) return fail(LDPC_EINVAL, "noalloc decode: NULL code");
    if (batch < 0) return fail(LDPC_EINVAL, "noalloc decode: negative batch");
    if (max_iter < 1) return fail(LDPC_EINVAL, "noalloc decode: max_iter must be >= 1");
    if (batch == 0) return LDPC_OK;
    if (!llr_in || !target_syndrome || !out_bits || !out_iters || !out_ok)
        return fail(LDPC_EINVAL, "noalloc decode: NULL buffer");
    int cur = -1;
    LDPC_CUDA_TRY(cudaGetDevice(&cur));
    if (cur != c->device) return fail(LDPC_EINVAL, "noalloc decode: make the code's device current first");
    const int smem_limit = ldpc::max_dyn_smem(c->device);
    if ((int64_t)smem_bytes(c, 1) > smem_limit)
        return fail(LDPC_EUNSUPPORTED, "noalloc decode: soft values of four frames exceed shared memory");
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    const int W = pick_words(c, batch, smem_limit, sms);
    const int64_t groups = (batch + 4 * W - 1) / (4 * W);
    const size_t need = (size_t)groups * 4 * W * (size_t)c->edges;
    if (need > kStaticMsgBytes)
        return fail(LDPC_EINVAL, "noalloc decode: " + std::to_string(batch) + " frames need " + std::to_string(need) +
                                     " bytes of message scratch; the fixed scratch holds " +
                                     std::to_string(kStaticMsgBytes) + " bytes (decode fewer frames per call)");
    uint32_t* msg = nullptr;
    int rc = static_msg_address(&msg);
    if (rc) return rc;
    DecodeArgs A{c->d_tab, c->Mb, c->nblk, c->Z, c->n, c->m, llr_in, target_syndrome, batch, max_iter, nullptr,
                 nullptr, out_bits, out_iters, out_ok, msg};
    return launch(c, A, (int)groups, W, false, (cudaStream_t)stream);
}

}  // extern "C"
