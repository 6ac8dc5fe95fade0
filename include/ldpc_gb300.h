/*
 * ldpc_gb300.h -- C ABI of the GB300 (sm_103a) quantised LDPC reconciliation
 * decoder.
 *
 * The decoder is the paper's (Mao, Li, Han, Guo, "High Throughput and Low Cost
 * LDPC Reconciliation for Quantum Key Distribution"): layered belief
 * propagation (section 2) on quasi-cyclic codes (section 4.1) with 8-bit
 * messages (section 3.1), the improved RCBP check-node table of Algorithm 1
 * (section 3.2), the saturation-oriented variable-node rule of Algorithm 2
 * (section 3.3) and a parity-check stopping test after every iteration
 * (section 2), run syndrome-based: Bob decodes his key against Alice's
 * syndrome.
 *
 * General rules for every entry point:
 *   - Pointers marked "device" are CUDA device pointers; "host" pointers are
 *     ordinary host memory.  The caller owns every input and output buffer.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Device
 *     work is enqueued on it and the call returns without synchronising,
 *     except where a function says otherwise.
 *   - Return value: LDPC_OK (0) or a negative LDPC_E* code.  Nothing is
 *     thrown across the ABI.  ldpc_last_error() gives a message for the most
 *     recent failure on the calling thread.
 *   - Bit vectors are packed LSB-first: bit j of a frame is bit (j & 7) of
 *     byte (j >> 3); a frame of n bits takes ceil(n/8) bytes.
 *   - Circulant convention: base entry s >= 0 at block (i, k) connects check
 *     row r of block row i to variable node k*Z + ((r + s) mod Z).
 *   - A code handle owns its device tables and a message scratch arena that
 *     grows on demand (cudaMalloc) and is freed by ldpc_code_destroy.  Two
 *     decodes that use one handle must not run concurrently on different
 *     streams; use one handle per concurrent stream.
 */
#ifndef LDPC_GB300_H
#define LDPC_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LDPC_OK 0
#define LDPC_EINVAL (-1)      /* bad argument: dimensions, shift >= Z, NULL pointer, size */
#define LDPC_ENOMEM (-2)      /* device allocation failed */
#define LDPC_ECUDA (-3)       /* a CUDA call or kernel launch failed (see ldpc_last_error) */
#define LDPC_EUNSUPPORTED (-4) /* shape outside what the kernels are built for */
#define LDPC_EKERNEL (-5)     /* a kernel reported an internal bound violation */

typedef struct ldpc_code ldpc_code;

/* Create a code from a quasi-cyclic base matrix (section 4.1: every nonzero
 * base entry becomes a Z x Z cyclically shifted identity, every zero entry
 * an all-zero block).
 *   base : host, int32[Mb][Nb] row-major; -1 = zero block, else shift in [0, Z).
 *   Mb, Nb, Z : base dimensions and lifting size; n = Nb*Z, m = Mb*Z.
 *   out  : receives the new handle.
 * One block row is one layer of the layered schedule (section 2).  Row degrees
 * up to 64 are supported.  Errors: LDPC_EINVAL (dims <= 0, shift out of range,
 * NULL), LDPC_EUNSUPPORTED (a row degree above 64 or n*4 bytes of state per
 * frame group beyond shared memory), LDPC_ENOMEM, LDPC_ECUDA. */
int ldpc_code_create(const int32_t* base, int Mb, int Nb, int Z, ldpc_code** out);

/* Free the handle, its tables and its scratch arena (synchronises the device). */
void ldpc_code_destroy(ldpc_code* code);

/* n, m, edges per frame (number of ones in H) and the largest row degree.
 * Any output pointer may be NULL. */
int ldpc_code_info(const ldpc_code* code, int* n, int* m, int64_t* edges, int* max_row_deg);

/* Grow the scratch arena for decodes of up to `batch` frames now, so that
 * later calls allocate nothing (needed before capturing a decode in a CUDA
 * graph).  Synchronous. */
int ldpc_code_reserve(ldpc_code* code, int batch);

/* Per-frame channel LLR magnitude of section 3.1 for a binary symmetric
 * channel, computed on the host: mag[f] = round-half-away(ln((1-q_f)/q_f) *
 * scale), clamped to 127.  Host code with the host C library's log, so that
 * every caller on one machine (and the reference CPU decoder) gets the same
 * integer even where the product lands next to a half-integer; the kernels
 * take these magnitudes instead of evaluating the logarithm on the device.
 *   qber    : host, double[batch] per-frame QBER in (0, 0.5).
 *   scale   : LSB per nat (> 0).
 *   mag_out : host, int8[batch].
 * Errors: LDPC_EINVAL (NULL, scale <= 0, a QBER outside (0, 0.5)). */
int ldpc_llr_magnitudes(const double* qber, int batch, double scale, int8_t* mag_out);

/* Channel LLRs of section 3.1, quantised to int8: a key position gets
 * +llr_mag[f] for a received 0 and -llr_mag[f] for a 1; punctured positions
 * 0; shortened positions +127 (known bit 0) or -127 (known bit 1).  Rate
 * adaptation of section 4.1: with `rank` given, position j of frame f is
 * shortened when rank[j] < n_short[f], punctured when n_short[f] <= rank[j] <
 * n_short[f] + n_punct[f], a key bit otherwise.
 *   bob_bits : device, uint8[batch][ceil(n/8)] Bob's key.
 *   llr_mag  : device, int8[batch] per-frame magnitudes (ldpc_llr_magnitudes).
 *   rank     : device, int32[n] puncturing order, or NULL (all key bits).
 *   n_short, n_punct : device, int32[batch], or NULL (zero).
 *   known    : device, uint8[batch][ceil(n/8)] values of shortened positions
 *              (only those positions are read), or NULL when n_short is NULL.
 *   llr_out  : device, int8[batch][n].  batch <= 65535. */
int ldpc_llr_from_bsc(const ldpc_code* code, const uint8_t* bob_bits, const int8_t* llr_mag, const int32_t* rank,
                      const int32_t* n_short, const int32_t* n_punct, const uint8_t* known, int batch,
                      int8_t* llr_out, void* stream);

/* Syndrome s = H x (mod 2) of a batch of packed bit vectors: the message
 * Alice sends in the syndrome-based protocol (section 4.1).
 *   bits    : device, uint8[batch][ceil(n/8)].
 *   syn_out : device, uint8[batch][ceil(m/8)]. */
int ldpc_syndrome(const ldpc_code* code, const uint8_t* bits, int batch, uint8_t* syn_out, void* stream);

/* Layered decoding of a batch against target syndromes (sections 2 and 3):
 * each iteration runs every block row in order; per check row, L_ji =
 * sat8(E_j - L_ij) (Eq. 8), sign = syndrome sign x product of the other
 * signs (Eq. 1), magnitude = repeated box-plus of the other magnitudes with
 * the tau table of Algorithm 1 (Eq. 7, folded forward-backward in ascending
 * variable order), E_j = sat8(L_ji + L_ij) unless |E_j| = 127 (Algorithm 2);
 * after every iteration the parity checks are tested with the latest E_j and
 * a frame stops at its first match (section 2).
 *   llr_in          : device, int8[batch][n] channel LLRs (e.g. from
 *                     ldpc_llr_from_bsc; 0 = punctured, +-127 = shortened).
 *   target_syndrome : device, uint8[batch][ceil(m/8)].
 *   batch >= 0, max_iter >= 1.
 *   out_bits  : device, uint8[batch][ceil(n/8)] hard decisions (E_j < 0 -> 1)
 *               at the first matching iteration, or after max_iter.
 *   out_iters : device, int32[batch] iterations run (1..max_iter).
 *   out_ok    : device, uint8[batch] 1 if the syndrome matched.
 * Results are bit-exact to the reference CPU decoder and independent of the
 * batch composition. */
int ldpc_decode_batch(const ldpc_code* code, const int8_t* llr_in, const uint8_t* target_syndrome, int batch,
                      int max_iter, uint8_t* out_bits, int32_t* out_iters, uint8_t* out_ok, void* stream);

/* ldpc_decode_batch with per-iteration, per-layer check-node tables: the
 * magnitude m from the box-plus fold becomes
 *   m' = clamp(((m * scale_q4[t][i] + 8) >> 4) - offset_q[t][i], 0, 127)
 * for iteration t (0-based) and layer i.  scale 16 / offset 0 is the plain
 * decoder; tables are the integer form of the scaled/offset check-node
 * corrections the paper lists as alternatives in section 2 (OMS/NMS).
 *   scale_q4 : device, uint8[max_iter][Mb], or NULL (all 16).
 *   offset_q : device, int8[max_iter][Mb], or NULL (all 0). */
int ldpc_decode_batch_ex(const ldpc_code* code, const int8_t* llr_in, const uint8_t* target_syndrome,
                         int batch, int max_iter, const uint8_t* scale_q4, const int8_t* offset_q,
                         uint8_t* out_bits, int32_t* out_iters, uint8_t* out_ok, void* stream);

/* ldpc_decode_batch with an explicit frame-group width: `words` 32-bit words
 * of four int8 lanes per check row and CTA (1, 2 or 4, i.e. 4, 8 or 16
 * frames per CTA); 0 picks automatically.  Results do not depend on it.
 * Errors: LDPC_EINVAL for another value or one whose state does not fit in
 * shared memory. */
int ldpc_decode_batch_words(const ldpc_code* code, const int8_t* llr_in, const uint8_t* target_syndrome,
                            int batch, int max_iter, int words, uint8_t* out_bits, int32_t* out_iters,
                            uint8_t* out_ok, void* stream);

/* Persistent mixed-rate reconciliation: ldpc_llr_from_bsc fused into the
 * layered decoder of ldpc_decode_batch, in one launch of resident CTAs that
 * pull frames from a device work counter (frames of different rates, QBERs
 * and iteration counts share the mother code; section 4.1).  Every byte lane
 * of a CTA decodes one frame at a time and, when the frame stops, takes the
 * next one, so uneven iteration counts do not hold the others back.  A CTA
 * whose oldest frame has run far longer than the mean leaves its free lanes
 * idle while the rest of the queue fits the other lanes before that frame
 * ends (it then runs without refills); results do not depend on the schedule.
 *   bob_bits, llr_mag, rank, n_short, n_punct, known : as in
 *       ldpc_llr_from_bsc, indexed by frame id.
 *   target_syndrome : device, uint8[batch][ceil(m/8)], indexed by frame id.
 *   batch : number of frames in the per-frame arrays.
 *   frame_list : device, int32[list_len] frame ids to decode (e.g. the frames
 *       still failing after an interactive reveal), or NULL for 0..list_len-1
 *       (then list_len <= batch).  Ids outside [0, batch) are skipped.
 *   max_iter : iteration cap.
 *   stall_window : K >= 0.  With K > 0 a frame also stops, as a failure,
 *       after iteration t when its number of unsatisfied parity checks has
 *       set no new minimum since iteration t - K (the minimum and the
 *       iteration that first reached it are tracked per frame from iteration
 *       1).  K = 0 is the plain decoder: it stops only at a syndrome match or
 *       max_iter.  Not in the paper: a stopping criterion for frames that
 *       have stopped converging (they would run to max_iter), in the spirit
 *       of the paper's remark that early termination adds throughput; the
 *       reference CPU decoder implements the same rule.  Needs m <= 65535.
 *   words : 32-bit lane words per CTA (1, 2, 4; 0 = automatic).
 *   ctas_per_sm : resident CTAs per SM (0 = as many as fit).
 *   threads : threads per CTA (0 = one thread pair per check row of a
 *       layer, at most 1024 (512 for rows of more than 32 edges)); otherwise
 *       a multiple of 32*words no larger than that, each thread pair then
 *       taking several rows of a layer.  Results do not depend on it.
 *   out_bits, out_iters, out_ok : device, indexed by frame id; entries of
 *       frames not in the list are left untouched.
 * Per-frame results equal ldpc_decode_batch on the LLRs of
 * ldpc_llr_from_bsc.  Capturable in a CUDA graph once the scratch arena is
 * large enough (ldpc_code_reserve_persistent). */
int ldpc_reconcile_persistent(const ldpc_code* code, const uint8_t* bob_bits, const int8_t* llr_mag,
                              const int32_t* rank, const int32_t* n_short, const int32_t* n_punct,
                              const uint8_t* known, const uint8_t* target_syndrome, int batch,
                              const int32_t* frame_list, int list_len, int max_iter, int stall_window,
                              int words, int ctas_per_sm, int threads, uint8_t* out_bits, int32_t* out_iters,
                              uint8_t* out_ok, void* stream);

/* The interactive rate-adaptive protocol of sections 4.1 and 4.2 in one
 * persistent launch: ldpc_reconcile_persistent, where a frame whose decode
 * fails (no syndrome match by max_iter, or the stall rule) and has rounds
 * left is rebuilt in its lane at the next round's state -- more of its
 * puncturing order revealed by Alice, punctured positions first, every
 * revealed position then shortened with her value -- and decoded again from
 * its channel LLRs.  Rounds of different frames overlap; no round waits for
 * the slowest frame of the one before.  Per-frame results equal decoding
 * each round separately (ldpc_reconcile_persistent with the round's
 * counts), round after round, until a match or the last round.
 *   n_short, n_punct : device, int32[batch] the counts of round 0 (the rate
 *       plan for the starting efficiency).  In round r frame f has
 *       n_short[f] + R and max(n_punct[f] - R, 0) of them, R = reveal[f][r].
 *   reveal : device, int32[batch][max_rounds + 1] cumulative revealed counts,
 *       reveal[f][0] = 0, non-decreasing, R <= n - n_short[f]; the paper
 *       does not fix how many bits a round reveals, the caller chooses.
 *   max_rounds : rounds after the first (>= 0).
 *   out_iters : iterations summed over the frame's rounds.
 *   out_rounds : device, int32[batch] index of the frame's last round.
 *   rank, known are required; the other arguments as in
 *   ldpc_reconcile_persistent. */
int ldpc_reconcile_interactive(const ldpc_code* code, const uint8_t* bob_bits, const int8_t* llr_mag,
                               const int32_t* rank, const int32_t* n_short, const int32_t* n_punct,
                               const uint8_t* known, const uint8_t* target_syndrome, int batch,
                               const int32_t* frame_list, int list_len, int max_iter, int stall_window,
                               const int32_t* reveal, int max_rounds, int words, int ctas_per_sm, int threads,
                               uint8_t* out_bits, int32_t* out_iters, uint8_t* out_ok, int32_t* out_rounds,
                               void* stream);

/* ldpc_reconcile_interactive from host buffers, for callers whose frames
 * and results live in host memory (the end-to-end form of the protocol of
 * sections 4.1 and 4.2): every input is copied into device buffers that the
 * code handle owns, the one persistent launch runs, and the outputs are
 * copied back; the call returns once they are in host memory (it
 * synchronises `stream`).
 *   Every pointer argument is host memory with the layout and meaning of the
 *   same argument of ldpc_reconcile_interactive, rank included (int32[n],
 *   copied on every call).  Page-locked memory (cudaHostAlloc, or torch's
 *   pin_memory) makes the copies asynchronous DMA; pageable memory works,
 *   the driver then stages it.
 *   Outputs of frames that frame_list does not contain keep the values the
 *   caller's buffers held (they are copied in first when the list does not
 *   cover every frame).
 *   h2d_bytes, d2h_bytes : host, int64[1] each, or NULL: the bytes this call
 *   copied to and from the device.
 * The device copies are cached on the handle and grow on demand (cudaMalloc
 * when a call needs more than an earlier one), so the call is not for CUDA
 * graph capture, and two calls on one handle must not run concurrently
 * (from two host threads) -- they share the copies.  Errors as for
 * ldpc_reconcile_interactive; LDPC_ENOMEM if the copies cannot be
 * allocated.  On an error after the first copy was queued the call still
 * waits for `stream` before it returns, so the caller's host buffers are
 * free to reuse whatever the outcome. */
int ldpc_reconcile_interactive_host(const ldpc_code* code, const uint8_t* bob_bits, const int8_t* llr_mag,
                                    const int32_t* rank, const int32_t* n_short, const int32_t* n_punct,
                                    const uint8_t* known, const uint8_t* target_syndrome, int batch,
                                    const int32_t* frame_list, int list_len, int max_iter, int stall_window,
                                    const int32_t* reveal, int max_rounds, int words, int ctas_per_sm, int threads,
                                    uint8_t* out_bits, int32_t* out_iters, uint8_t* out_ok, int32_t* out_rounds,
                                    int64_t* h2d_bytes, int64_t* d2h_bytes, void* stream);

/* Bytes of the lane-state buffer that ldpc_reconcile_epoch needs for a launch
 * shape (words 1, 2 or 4 explicitly; ctas_per_sm and threads as in
 * ldpc_reconcile_persistent), and the grid that shape runs (`grid` may be
 * NULL).  Host only. */
int ldpc_epoch_state_bytes(const ldpc_code* code, int words, int ctas_per_sm, int threads, size_t* bytes,
                           int* grid);

/* One epoch of a continuously batched persistent decode, for serving: the
 * persistent decoder of ldpc_reconcile_persistent where every CTA runs at
 * most `epoch_iters` decoder iterations and then saves its lanes -- each
 * frame's iteration count and stall-rule state, its soft values and
 * syndrome bits -- into `lane_state` and returns.  Its messages stay in the
 * code handle's arena, in the region of the same CTA.  The next call with
 * `resume` = 1 restores the lanes and continues their frames where they
 * stopped; lanes that are free (their frame finished) take frames from this
 * call's frame_list.  Frames thus join and leave between epochs while the
 * others' decoding state stays on the device; nothing on the device waits
 * for the host.  A frame's results equal those of one
 * ldpc_reconcile_persistent call, however its decode is split.
 *   Per-frame arrays (bob_bits ... target_syndrome, outputs) are indexed by
 *       frame id in [0, batch) as in ldpc_reconcile_persistent.  A frame's
 *       inputs are read once, when a lane takes it; its outputs are written
 *       when it finishes (out_iters >= 1 then, so a caller that zeroes
 *       out_iters at admission can see which frames are done).
 *   frame_list, list_len : the frames this epoch may start (list_len >= 0);
 *       frames a lane took are counted in *out_claimed.
 *   epoch_iters >= 1 : iterations per CTA in this call.
 *   resume : 0 for the first epoch of a lane-state buffer (every lane
 *       free), 1 afterwards.  Every epoch of one buffer must use the same
 *       code handle, words, ctas_per_sm and threads, and no other decode may
 *       use that handle in between (it owns the messages).
 *   lane_state : device, 256-byte aligned, lane_state_bytes >=
 *       ldpc_epoch_state_bytes(code, words, ctas_per_sm, threads).
 *   words : 1, 2 or 4 (no automatic choice: it fixes the lane layout).
 *   out_claimed : device, int32[1]: how many entries of frame_list were
 *       handed to a lane (claims past the list's end are counted too, so
 *       the frames taken are the first min(*out_claimed, list_len)); the
 *       rest are for a later epoch.
 * The stall window applies as in ldpc_reconcile_persistent; the claim-hold
 * rule does not (each epoch's list is short). */
int ldpc_reconcile_epoch(const ldpc_code* code, const uint8_t* bob_bits, const int8_t* llr_mag, const int32_t* rank,
                         const int32_t* n_short, const int32_t* n_punct, const uint8_t* known,
                         const uint8_t* target_syndrome, int batch, const int32_t* frame_list, int list_len,
                         int max_iter, int stall_window, int epoch_iters, int resume, void* lane_state,
                         size_t lane_state_bytes, int words, int ctas_per_sm, int threads, uint8_t* out_bits,
                         int32_t* out_iters, uint8_t* out_ok, int32_t* out_claimed, void* stream);

/* Grow the scratch arena now for a persistent decode of `list_len` frames
 * with the given `words`, `ctas_per_sm` and `threads` (0 = automatic, as in
 * ldpc_reconcile_persistent), so that the decode itself allocates nothing
 * and can be captured in a CUDA graph.  Synchronous. */
int ldpc_code_reserve_persistent(ldpc_code* code, int list_len, int words, int ctas_per_sm, int threads);

/* FP32 relaxation of the layered decoder, for learning check-node
 * corrections (the normalised/offset forms section 2 lists as alternatives).
 * Same schedule, sign rule (Eq. 1 with the syndrome sign) and forward-backward
 * fold of Eq. 7 as ldpc_decode_batch, in float and without saturation; the
 * fold uses the tempered box-plus beta_k(x,y) = k*beta(x/k, y/k) of Eq. 6,
 * which is what Algorithm 1's table (the integer form of beta at its own step
 * D_t, section 3.2) computes when LLRs are quantised at a step D (k = D/D_t;
 * k = 1 is exact belief propagation).  Each magnitude becomes
 *   alpha[t][c] * relu(fold - gamma[t][c])
 * for iteration t and the layer's row-degree class c.  A degree-1 row sends
 * 50 (the empty box-plus).  Variable update: plain Eq. 9.
 *   llr   : device, float[batch][n] channel LLRs in nats (positive = bit 0).
 *   syn   : device, uint8[batch][ceil(m/8)] target syndromes.
 *   bits  : device, uint8[batch][ceil(n/8)] Alice's bits, or NULL (no loss).
 *   alpha, gamma : device, float[iters][n_classes].
 *   layer_class  : device, int32[Mb] class of each layer (0..n_classes-1).
 *   ckE   : device, float[iters+1][batch][n]: E at the start of every
 *           iteration and the final E (checkpoints for the adjoint).
 *   ckL   : device, float[iters][batch][edges]: messages at the start of
 *           iterations 1..iters-1 (slot 0 is not written: L starts at 0).
 *   loss  : device float[1] (zeroed here), or NULL: mean over frames and bits
 *           of softplus(-(1-2x) E_final), the cross entropy against Alice.
 * Requires Z <= 512 and row degree <= 32. */
int ldpc_relaxed_forward(const ldpc_code* code, const float* llr, const uint8_t* syn, const uint8_t* bits, int batch,
                         int iters, const float* alpha, const float* gamma, const int32_t* layer_class,
                         int n_classes, float kappa, float* ckE, float* ckL, float* loss, void* stream);

/* Adjoint of ldpc_relaxed_forward's loss with respect to alpha and gamma
 * (and optionally the LLRs).  Walks the iterations backwards; each iteration
 * is recomputed from its checkpoint (ckE, ckL) and its layers reversed with
 * d beta_k/dx = s((x+y)/k) - s((x-y)/k), s the logistic function.
 *   V, gL : device scratch, float[batch][edges] each.
 *   grad_alpha, grad_gamma : device, float[iters][n_classes] (zeroed here).
 *   grad_llr : device, float[batch][n], or NULL.
 * Gradients of sign and relu at 0 are taken as 0 (as autograd does). */
int ldpc_relaxed_backward(const ldpc_code* code, const uint8_t* syn, const uint8_t* bits, int batch, int iters,
                          const float* alpha, const float* gamma, const int32_t* layer_class, int n_classes,
                          float kappa, const float* ckE, const float* ckL, float* V, float* gL, float* grad_alpha,
                          float* grad_gamma, float* grad_llr, void* stream);

/* ldpc_decode_batch for callers that must not let the library allocate
 * device memory.  The paper has no counterpart: this is a property of the
 * library, not of the method.
 *
 * Who needs it: a reconciliation service that sizes all of its GPU memory at
 * start-up and may not grow it while keys stream in; a process whose device
 * memory is owned by another allocator's fixed pool; a latency-critical loop
 * that cannot accept the device-wide synchronisation that cudaMalloc/cudaFree
 * may cause.  ldpc_decode_batch keeps its message scratch in the code handle's
 * arena and grows it with cudaMalloc; this entry point instead takes the
 * scratch from one fixed 32 MiB array compiled into the library, and calls no
 * cudaMalloc, cudaFree or allocating library routine.
 *
 * Same arguments, layouts and results as ldpc_decode_batch (bit-identical
 * outputs), with these differences:
 *   - Limit: round_up(batch, frames per CTA) * edges bytes of scratch must fit
 *     in 32 MiB (frames per CTA is 4, 8 or 16, chosen as in
 *     ldpc_decode_batch); e.g. up to 2720 frames of the n=4096 code of 12288
 *     edges, or up to 272 frames of a 122880-edge code.  Larger batches are
 *     rejected with LDPC_EINVAL and a message giving the bytes needed; split
 *     them into several calls.
 *   - The array exists on every GPU that loads the library and stays there
 *     until the process exits.
 *   - Set-up: the first call in a CUDA context (per device, and again after
 *     cudaDeviceReset or in a caller-created context) looks up the array's
 *     device address there (cudaGetSymbolAddress, which also loads the
 *     library's module into that context) and caches it by the context's
 *     id; make that first call before any stream capture.  The code's device
 *     must be the current device (else LDPC_EINVAL).
 *   - All calls share the one array, which keeps the previous call's
 *     contents.  Nothing needs clearing (the decoder never reads a message it
 *     has not written in the same call), but two calls whose kernels overlap
 *     on the GPU -- on different streams, or from different threads -- race
 *     on the array and corrupt each other's results.  Serialise them. */
int ldpc_decode_batch_noalloc(const ldpc_code* code, const int8_t* llr_in, const uint8_t* target_syndrome,
                              int batch, int max_iter, uint8_t* out_bits, int32_t* out_iters, uint8_t* out_ok,
                              void* stream);

/* Device evaluation of the check-node table of Algorithm 1 exactly as the
 * decoder's byte-lane arithmetic computes it, for every (p, q) in
 * [0,128)^2: out[p*128 + q].  out: device, uint8[16384].  For tests. */
int ldpc_debug_tau_table(uint8_t* out, void* stream);

/* Number of kernel launches this library has issued in this process. */
int64_t ldpc_launch_count(void);

/* Message for an error code, and the detailed message of the calling
 * thread's most recent failure. */
const char* ldpc_strerror(int code);
const char* ldpc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LDPC_GB300_H */
