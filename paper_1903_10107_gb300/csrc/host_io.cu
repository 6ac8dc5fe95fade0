// Host-buffer entry points of the C ABI: the library's own copies between the
// caller's host memory and a device staging area owned by the code handle,
// around one call of the device-pointer entry point.  No kernel lives here.
#include <vector>

#include "common.cuh"

extern "C" {

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
    // Once a copy is queued, every return waits for the stream first: the
    // caller may release its host buffers as soon as the call returns, so no
    // copy may still be reading or writing them, on success or on error.
    auto drain = [st](int r) {
        cudaStreamSynchronize(st);
        return r;
    };
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
        return drain(rc);
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
        return drain(rc);
    auto at = [d](size_t o) { return d + o; };
    rc = ldpc_reconcile_interactive(
        c, at(o_bob), reinterpret_cast<const int8_t*>(at(o_mag)), reinterpret_cast<const int32_t*>(at(o_rank)),
        reinterpret_cast<const int32_t*>(at(o_ns)), reinterpret_cast<const int32_t*>(at(o_np)), at(o_known),
        at(o_syn), batch, frame_list ? reinterpret_cast<const int32_t*>(at(o_list)) : nullptr, list_len, max_iter,
        stall_window, reinterpret_cast<const int32_t*>(at(o_rev)), max_rounds, words, ctas_per_sm, threads,
        at(o_bits), reinterpret_cast<int32_t*>(at(o_it)), at(o_ok), reinterpret_cast<int32_t*>(at(o_rd)), stream);
    if (rc) return drain(rc);
    auto d2h = [&](void* dst, size_t o, size_t bytes) -> int {
        if (!bytes) return LDPC_OK;
        LDPC_CUDA_TRY(cudaMemcpyAsync(dst, d + o, bytes, cudaMemcpyDeviceToHost, st));
        out += (int64_t)bytes;
        return LDPC_OK;
    };
    if ((rc = d2h(out_bits, o_bits, B * nb)) || (rc = d2h(out_iters, o_it, 4 * B)) || (rc = d2h(out_ok, o_ok, B)) ||
        (rc = d2h(out_rounds, o_rd, 4 * B)))
        return drain(rc);
    LDPC_CUDA_TRY(cudaStreamSynchronize(st));
    if (h2d_bytes) *h2d_bytes = in;
    if (d2h_bytes) *d2h_bytes = out;
    return LDPC_OK;
}

}  // extern "C"
