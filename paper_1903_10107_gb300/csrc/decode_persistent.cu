// Host side of the persistent mixed-rate decoder: argument checks, group
// width, grid sizing, message scratch, dispatch to the kernel of the code's
// unroll width, and the C ABI.  The kernel is in decode_persistent.cuh.
#include "decode_persistent.cuh"

namespace {

using ldpc_dec::PersistArgs;
using ldpc_dec::smem_bytes;

int dispatch(const ldpc_code* c, const PersistArgs& A, int W, int ctas_per_sm, int* grid, bool dry,
             cudaStream_t st) {
    switch (ldpc_dec::pick_maxh(c->max_deg)) {
#define LDPC_PERSIST_CASE(M) \
    case M:                  \
        return ldpc_dec::persist_launch<M>(c, A, W, ctas_per_sm, grid, dry, st);
        LDPC_MAXH_LIST(LDPC_PERSIST_CASE)
#undef LDPC_PERSIST_CASE
        default:
            return ldpc::fail(LDPC_EUNSUPPORTED, "persistent decode: row degree above 64");
    }
}

}  // namespace

extern "C" {

int ldpc_code_reserve_persistent(ldpc_code* code, int list_len, int words, int ctas_per_sm) {
    if (!code || list_len < 0) return ldpc::fail(LDPC_EINVAL, "ldpc_code_reserve_persistent: bad argument");
    if (list_len == 0) return LDPC_OK;
    const int W = words > 0 ? words : 1;
    if (W != 1 && W != 2 && W != 4) return ldpc::fail(LDPC_EINVAL, "ldpc_code_reserve_persistent: bad words");
    PersistArgs A{};
    A.list_len = list_len;
    int grid = 0;
    int rc = dispatch(code, A, W, ctas_per_sm, &grid, true, nullptr);
    if (rc) return rc;
    return ldpc::ensure_arena(code, (size_t)grid * 4 * W * (size_t)code->edges);
}

int ldpc_reconcile_persistent(const ldpc_code* code, const uint8_t* bob_bits, const double* qber,
                              const int32_t* rank, const int32_t* n_short, const int32_t* n_punct,
                              const uint8_t* known, const uint8_t* target_syndrome, int batch,
                              const int32_t* frame_list, int list_len, int max_iter, double llr_scale, int words,
                              int ctas_per_sm, uint8_t* out_bits, int32_t* out_iters, uint8_t* out_ok,
                              void* stream) {
    using ldpc::fail;
    const ldpc_code* c = code;
    if (!c) return fail(LDPC_EINVAL, "persistent decode: NULL code");
    if (list_len < 0 || batch < 0 || max_iter < 1)
        return fail(LDPC_EINVAL, "persistent decode: bad batch, list length or max_iter");
    if (!frame_list && list_len > batch) return fail(LDPC_EINVAL, "persistent decode: list_len > batch");
    if (list_len == 0) return LDPC_OK;
    if (!bob_bits || !qber || !target_syndrome || !out_bits || !out_iters || !out_ok)
        return fail(LDPC_EINVAL, "persistent decode: NULL buffer");
    if ((n_short || n_punct) && !rank) return fail(LDPC_EINVAL, "persistent decode: counts need a rank table");
    if (n_short && !known) return fail(LDPC_EINVAL, "persistent decode: shortening needs known values");
    if (!(llr_scale > 0.0)) return fail(LDPC_EINVAL, "persistent decode: bad LLR scale");
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
    PersistArgs A{c->d_tab, c->Mb, c->nblk, c->Z, c->n, c->m, bob_bits, qber, rank, n_short, n_punct, known,
                  target_syndrome, frame_list, batch, list_len, max_iter, llr_scale, out_bits, out_iters, out_ok,
                  nullptr, c->d_queue};
    int grid = 0;
    int rc = dispatch(c, A, W, ctas_per_sm, &grid, true, (cudaStream_t)stream);
    if (rc) return rc;
    const size_t need = (size_t)grid * 4 * W * (size_t)c->edges;
    rc = ldpc::ensure_arena(const_cast<ldpc_code*>(c), need);
    if (rc) return rc;
    A.msg = reinterpret_cast<uint32_t*>(c->arena);
    return dispatch(c, A, W, ctas_per_sm, &grid, false, (cudaStream_t)stream);
}

}  // extern "C"
