// Persistent mixed-rate reconciliation: channel-LLR quantisation (section
// 3.1, with the punctured/shortened positions of section 4.1) fused into the
// layered int8 decoder (sections 2 and 3), with per-lane refill.
//
//   * A grid of resident CTAs pulls frames from a device work counter.  Each
//     CTA has 4*W byte lanes; every lane decodes one frame at a time with its
//     own iteration count.
//   * When a lane's frame stops (first syndrome match, or its iteration cap)
//     the CTA writes that frame's bits/iterations/flag, claims the next
//     frame for the lane and builds its soft values straight from Bob's
//     packed key bits, the frame's QBER and its rate counts.  Messages of a
//     refilled lane are treated as 0 during its first iteration, so the
//     message scratch is never cleared.
//   * Frames of any rate, QBER and iteration count mix freely in one launch:
//     puncturing and shortening only change the initial soft values of the
//     shared mother code.  Per-frame results equal those of
//     ldpc_decode_batch on the same soft values.
//   * Interactive rounds (section 4.2) run inside the same launch: a frame
//     that fails a round is rebuilt in its lane from the next round's reveal
//     state (a per-frame table of revealed counts) and decoded again, so no
//     round waits for the slowest frame of the previous one.
#pragma once

#include <string>

#include "decode_int8.cuh"

namespace ldpc_dec {

struct PersistArgs {
    const int32_t* tab;
    int Mb, nblk, Z, n, m;
    const uint8_t* bob;
    const int8_t* mag;  // per-frame channel LLR magnitude (host-computed)
    const int32_t* rank;
    const int32_t* n_short;
    const int32_t* n_punct;
    const uint8_t* known;
    const uint8_t* syn;
    const int32_t* list;
    int batch, list_len, max_iter;
    int stall;  // stall window K (0 = off): a frame whose unsatisfied-check count set no new minimum
                // in its last K iterations stops as a failure
    uint8_t* out_bits;
    int32_t* out_iters;
    uint8_t* out_ok;
    // Interactive rounds (NULL reveal = one round): reveal[f][r] bits of frame f's puncturing order are
    // revealed in round r (cumulative, reveal[f][0] = 0); a frame failing round r < max_rounds restarts
    // in its lane from round r + 1's state.  out_rounds[f] = the last round decoded.
    const int32_t* reveal;
    int max_rounds;
    int32_t* out_rounds;
    // Epoch mode (serving; epoch_iters > 0): every CTA runs at most epoch_iters iterations, then saves its
    // lanes -- lane records, soft-value image, syndrome nibbles, lane masks -- and returns; its messages
    // stay in its own arena region.  With resume set a CTA first restores what it saved, then fills its
    // free lanes from this launch's frame list.  The grid is the same in every epoch.
    int epoch_iters, resume;
    int32_t* lane_save;   // [grid][4W][kLaneRec]
    uint32_t* word_save;  // [grid][2W]: active and fresh masks
    uint32_t* e_save;     // [grid][n W]
    uint8_t* syn_save;    // [grid][m W]
    uint32_t* msg;
    int* queue;  // [0] frames claimed, [1] frames finished, [2..3] their iterations (64 bit); zeroed per launch
};

// Frame id of work-list slot `slot`, or -1 past the end of the list or for an
// id outside [0, batch).
__device__ __forceinline__ int frame_of(const PersistArgs& A, int slot) {
    if (slot >= A.list_len) return -1;
    const int f = A.list ? A.list[slot] : slot;
    return (f >= 0 && f < A.batch) ? f : -1;
}

// The claim step's hold rule: only a frame past kHoldAfter iterations can
// make its CTA hold, and only once kHoldMinDone frames have finished (for the
// mean iteration count).
constexpr int kHoldAfter = 16;
constexpr int kHoldMinDone = 64;

// Integers per saved lane: frame, iterations, round, earlier rounds' iterations, fewest unsatisfied checks
// and its iteration, LLR magnitude, shortened and punctured counts.
constexpr int kLaneRec = 9;

// Bytes of the epoch-mode save area of `grid` CTAs, and the offsets of its parts.
struct EpochLayout {
    size_t lanes, words, soft, syn, total;
};
__host__ __device__ inline EpochLayout epoch_layout(int n, int m, int W, int grid) {
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    EpochLayout L;
    L.lanes = 0;
    L.words = up(L.lanes + (size_t)grid * 4 * W * kLaneRec * sizeof(int32_t));
    L.soft = up(L.words + (size_t)grid * 2 * W * sizeof(uint32_t));
    L.syn = up(L.soft + (size_t)grid * n * W * sizeof(uint32_t));
    L.total = up(L.syn + (size_t)grid * m * W);
    return L;
}

template <int MAXH, int P, int W, int MAXT>
__global__ void __launch_bounds__(MAXT) persistent_kernel(PersistArgs A) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int n = A.n, m = A.m, Z = A.Z, Mb = A.Mb, nblk = A.nblk;
    const int nb = (n + 7) / 8, mbytes = (m + 7) / 8;
    const int tab_words = (int)ldpc_dev::tables_words(Mb, nblk);
    uint32_t* E_s = reinterpret_cast<uint32_t*>(smem);
    uint8_t* E_b = smem;
    int32_t* s_tab = reinterpret_cast<int32_t*>(smem + soft_bytes(n, W));
    uint8_t* syn_s = reinterpret_cast<uint8_t*>(s_tab + tab_words);
    constexpr int NL = 4 * W;
    __shared__ int s_frame[NL], s_it[NL], s_mag[NL], s_ns[NL], s_np[NL], s_ubest[NL], s_tbest[NL];
    __shared__ int s_round[NL], s_itsum[NL];  // interactive round of the lane's frame, iterations of its earlier rounds
    __shared__ uint8_t s_done[NL], s_okf[NL];
    __shared__ uint32_t s_active[W], s_fresh[W], s_bad[W], s_load[W], s_cnt[2 * W];
    __shared__ int s_base, s_any_load, s_any_done;

    const int tid = threadIdx.x, T = blockDim.x;
    const int w = tid % W, q = tid / W;
    const int half = (P == 2) ? (q & 1) : 0;
    const int rt = q / P, RT = T / (W * P), QT = T / W;

    const ldpc_dev::Tables TB = ldpc_dev::load_tables(s_tab, A.tab, Mb, nblk, Z, W, tid, T);
    const bool epoch = A.epoch_iters > 0;
    const int b = blockIdx.x;
    if (tid < W) {
        s_bad[tid] = 0;
        s_load[tid] = 0;
        s_cnt[2 * tid] = 0;
        s_cnt[2 * tid + 1] = 0;
    }
    if (epoch && A.resume) {
        // ---- the lanes this CTA saved at the end of the previous epoch
        if (tid < NL) {
            const int32_t* rec = A.lane_save + ((size_t)b * NL + tid) * kLaneRec;
            s_frame[tid] = (rec[0] >= 0 && rec[0] < A.batch) ? rec[0] : -1;  // a record never saved reads as free
            s_it[tid] = rec[1];
            s_round[tid] = min(max(rec[2], 0), A.max_rounds);
            s_itsum[tid] = rec[3];
            s_ubest[tid] = rec[4];
            s_tbest[tid] = rec[5];
            s_mag[tid] = rec[6];
            s_ns[tid] = rec[7];
            s_np[tid] = rec[8];
            s_done[tid] = 0;
        }
        __syncthreads();
        if (tid < W) {
            uint32_t valid = 0;
            for (int l = 0; l < 4; ++l)
                if (s_frame[4 * tid + l] >= 0) valid |= 0xFFu << (8 * l);
            s_active[tid] = A.word_save[(size_t)b * 2 * W + tid] & valid;
            s_fresh[tid] = A.word_save[(size_t)b * 2 * W + W + tid];
        }
        __syncthreads();
        uint32_t was_live = 0;
#pragma unroll
        for (int ww = 0; ww < W; ++ww) was_live |= s_active[ww];
        if (was_live) {  // the soft values and syndrome bits of the lanes in flight
            const uint32_t* es = A.e_save + (size_t)b * n * W;
            for (int i = tid; i < n * W; i += T) E_s[i] = es[i];
            const uint8_t* ss = A.syn_save + (size_t)b * m * W;
            for (int i = tid; i < m * W; i += T) syn_s[i] = ss[i];
        }
        __syncthreads();
        if (tid == 0) {  // new frames of this launch's list for the free lanes
            int k = 0;
            for (int lane = 0; lane < NL; ++lane) k += s_frame[lane] < 0 ? 1 : 0;
            const int base = k ? atomicAdd(A.queue, k) : 0;
            int i = 0, any = 0;
            for (int lane = 0; lane < NL; ++lane) {
                if (s_frame[lane] >= 0) continue;
                s_frame[lane] = frame_of(A, base + i++);
                s_round[lane] = 0;
                s_itsum[lane] = 0;
                if (s_frame[lane] >= 0) {
                    s_load[lane >> 2] |= 0xFFu << (8 * (lane & 3));
                    any = 1;
                }
            }
            s_any_load = any;
        }
    } else {
        if (tid == 0) s_base = atomicAdd(A.queue, NL);
        if (tid < W) {
            s_active[tid] = 0;
            s_fresh[tid] = 0;
        }
        __syncthreads();
        if (tid < NL) {
            const int slot = s_base + tid;
            s_frame[tid] = frame_of(A, slot);
            s_done[tid] = 0;
            s_round[tid] = 0;
            s_itsum[tid] = 0;
        }
        __syncthreads();
        if (tid < W) {
            uint32_t ld = 0;
            for (int l = 0; l < 4; ++l)
                if (s_frame[4 * tid + l] >= 0) ld |= 0xFFu << (8 * l);
            s_load[tid] = ld;
        }
        if (tid == 0) s_any_load = 1;
    }
    int cta_iters = 0;  // iterations this CTA has run in this launch

    const int* deg = TB.deg;
    const int* off = TB.off;
    RowCtx C;
    C.E_s = E_s;
    C.msg = A.msg + (size_t)blockIdx.x * nblk * Z * W;
    C.Z = Z;
    C.w = w;
    C.sq = 16;
    C.oq = 0;

    for (;;) {
        __syncthreads();
        // ---- refill: soft values and syndrome bits of newly claimed frames
        if (s_any_load) {
            if (tid < NL) {
                const int ww = tid >> 2, l = tid & 3;
                if ((s_load[ww] >> (8 * l)) & 1u) {
                    const int f = s_frame[tid];
                    const int mg = A.mag[f];
                    s_mag[tid] = mg > 127 ? 127 : (mg < -127 ? -127 : mg);
                    int ns = A.n_short ? A.n_short[f] : 0, np = A.n_punct ? A.n_punct[f] : 0;
                    if (A.reveal) {  // revealed positions: punctured ones first, all of them now shortened
                        const int rv = A.reveal[(int64_t)f * (A.max_rounds + 1) + s_round[tid]];
                        ns += rv;
                        np = max(np - rv, 0);
                    }
                    s_ns[tid] = ns;
                    s_np[tid] = np;
                    s_it[tid] = 0;
                    s_ubest[tid] = 0x7FFFFFFF;
                    s_tbest[tid] = 0;
                }
            }
            __syncthreads();
            // soft values: one byte of Bob's key (8 variables) per thread and step,
            // every load of the step issued before the stores that use them
            for (int b = tid; b < nb; b += T) {
                const int j0 = b << 3;
                int rk[8];
#pragma unroll
                for (int qq = 0; qq < 8; ++qq) rk[qq] = (A.rank && j0 + qq < n) ? A.rank[j0 + qq] : 0x7FFFFFFF;
                for (int lane = 0; lane < NL; ++lane) {
                    const int ww = lane >> 2, l = lane & 3;
                    if (!((s_load[ww] >> (8 * l)) & 1u)) continue;
                    const int64_t f = s_frame[lane];
                    const int ns = s_ns[lane], np = s_np[lane], mag = s_mag[lane];
                    const uint32_t yb = A.bob[f * nb + b];
                    const uint32_t kb = (ns > 0) ? A.known[f * nb + b] : 0u;  // shortening implies known values
#pragma unroll
                    for (int qq = 0; qq < 8; ++qq) {
                        const int j = j0 + qq;
                        if (j >= n) break;
                        int x = ((yb >> qq) & 1u) ? -mag : mag;
                        if (rk[qq] < ns) x = ((kb >> qq) & 1u) ? -127 : 127;
                        else if (rk[qq] < ns + np) x = 0;
                        E_b[((size_t)j * W + ww) * 4 + l] = (uint8_t)((int8_t)x) ^ 0x80u;
                    }
                }
            }
            // syndrome bits: one byte of each claimed frame's syndrome (8 checks) per thread and step
            for (int sb = tid; sb < mbytes; sb += T) {
                const int c0 = sb << 3;
                for (int ww = 0; ww < W; ++ww) {
                    const uint32_t ld = s_load[ww];
                    if (!ld) continue;
                    uint32_t sy[4];
#pragma unroll
                    for (int l = 0; l < 4; ++l)
                        sy[l] = ((ld >> (8 * l)) & 1u) ? A.syn[(int64_t)s_frame[4 * ww + l] * mbytes + sb] : 0u;
#pragma unroll
                    for (int qq = 0; qq < 8; ++qq) {
                        const int c = c0 + qq;
                        if (c >= m) break;
                        uint32_t nib = syn_s[c * W + ww] & 0xFu;  // lanes not being loaded keep their bits
#pragma unroll
                        for (int l = 0; l < 4; ++l)
                            if ((ld >> (8 * l)) & 1u) nib = (nib & ~(1u << l)) | (((sy[l] >> qq) & 1u) << l);
                        syn_s[c * W + ww] = (uint8_t)nib;
                    }
                }
            }
            __syncthreads();
            if (tid < W) {
                s_active[tid] |= s_load[tid];
                s_fresh[tid] |= s_load[tid];
                s_load[tid] = 0;
            }
            if (tid == 0) s_any_load = 0;
            __syncthreads();
        }
        uint32_t live = 0;
#pragma unroll
        for (int ww = 0; ww < W; ++ww) live |= s_active[ww];
        if (!live || (epoch && cta_iters >= A.epoch_iters)) {
            if (epoch) {  // save the lanes for the next epoch (none is pending a write-out or a load here)
                if (tid < NL) {
                    int32_t* rec = A.lane_save + ((size_t)b * NL + tid) * kLaneRec;
                    const int lv = (s_active[tid >> 2] >> (8 * (tid & 3))) & 1u;
                    rec[0] = lv ? s_frame[tid] : -1;
                    rec[1] = s_it[tid];
                    rec[2] = s_round[tid];
                    rec[3] = s_itsum[tid];
                    rec[4] = s_ubest[tid];
                    rec[5] = s_tbest[tid];
                    rec[6] = s_mag[tid];
                    rec[7] = s_ns[tid];
                    rec[8] = s_np[tid];
                }
                if (tid < W) {
                    A.word_save[(size_t)b * 2 * W + tid] = s_active[tid];
                    A.word_save[(size_t)b * 2 * W + W + tid] = s_fresh[tid];
                }
                if (live) {
                    uint32_t* es = A.e_save + (size_t)b * n * W;
                    for (int i = tid; i < n * W; i += T) es[i] = E_s[i];
                    uint8_t* ss = A.syn_save + (size_t)b * m * W;
                    for (int i = tid; i < m * W; i += T) ss[i] = syn_s[i];
                }
            }
            break;
        }
        ++cta_iters;

        // ---- one iteration of every active lane
        C.active = s_active[w];
        C.fresh = s_fresh[w];
        for (int i = 0; i < Mb; ++i) {
            C.d = deg[i];
            C.b0 = off[i];
            C.et = TB.et + C.b0;
            if (C.d > 0) {
                for (int r0 = 0; r0 < Z; r0 += RT) {
                    const int r = r0 + rt;
                    const bool valid = r < Z;
                    const uint32_t nib = valid ? syn_s[(i * Z + r) * W + w] : 0u;
                    ldpc_dev::row_update_any<W, false, MAXH>(C, valid ? r : 0, valid, half, nib);
                }
            }
            __syncthreads();
        }
        uint32_t bad = 0;
        uint32_t ulo = 0, uhi = 0;  // unsatisfied checks of lanes 0, 2 (ulo) and 1, 3 (uhi), 16 bits each
        {
            int i = q / Z, r = q - i * Z;
            const int di = QT / Z, dr = QT - di * Z;
            for (int c = q; c < m; c += QT) {
                uint32_t p;
                if constexpr (MAXH <= 8) {  // rows of at most 16 edges
                    p = ldpc_dev::row_parity_unrolled<W, 2 * MAXH>(E_s, TB.et + off[i], deg[i], r, Z, w,
                                                                   syn_s[c * W + w]);
                } else {
                    p = ldpc_dev::row_parity<W>(E_s, TB.et + off[i], deg[i], r, Z, w, syn_s[c * W + w]);
                }
                bad |= p;
                if (A.stall) {
                    ulo += (p >> 7) & 0x00010001u;
                    uhi += (p >> 15) & 0x00010001u;
                }
                r += dr;
                i += di;
                if (r >= Z) {
                    r -= Z;
                    ++i;
                }
            }
        }
#pragma unroll
        for (int o = 16; o >= W; o >>= 1) bad |= __shfl_xor_sync(0xffffffffu, bad, o);
        if ((tid & 31) < W && bad) atomicOr(&s_bad[w], bad);
        if (A.stall) {
#pragma unroll
            for (int o = 16; o >= W; o >>= 1) {
                ulo += __shfl_xor_sync(0xffffffffu, ulo, o);
                uhi += __shfl_xor_sync(0xffffffffu, uhi, o);
            }
            if ((tid & 31) < W && (ulo | uhi)) {
                atomicAdd(&s_cnt[2 * w], ulo);
                atomicAdd(&s_cnt[2 * w + 1], uhi);
            }
        }
        if (tid == 0) s_any_done = 0;
        __syncthreads();

        // ---- per-lane bookkeeping (one thread per word)
        if (tid < W) {
            const uint32_t failing = spread(s_bad[tid]);
            uint32_t act = s_active[tid];
            for (int l = 0; l < 4; ++l) {
                const uint32_t lm = 0xFFu << (8 * l);
                if (!(act & lm)) continue;
                const int lane = 4 * tid + l;
                const int it = ++s_it[lane];
                const bool ok = !(failing & lm);
                bool stalled = false;
                if (A.stall && !ok) {
                    const int u = (int)((s_cnt[2 * tid + (l & 1)] >> (16 * (l >> 1))) & 0xFFFFu);
                    if (u < s_ubest[lane]) {
                        s_ubest[lane] = u;
                        s_tbest[lane] = it;
                    } else {
                        stalled = it - s_tbest[lane] >= A.stall;
                    }
                }
                if (ok || stalled || it >= A.max_iter) {
                    act &= ~lm;
                    if (!ok && A.reveal && s_round[lane] < A.max_rounds) {
                        // the next interactive round: more bits revealed, decoded again in this lane
                        s_itsum[lane] += it;
                        ++s_round[lane];
                        s_load[tid] |= lm;
                        s_any_load = 1;
                    } else {
                        s_done[lane] = 1;
                        s_okf[lane] = ok ? 1 : 0;
                        s_any_done = 1;
                    }
                }
            }
            s_active[tid] = act;
            s_fresh[tid] = 0;
            s_bad[tid] = 0;
            s_cnt[2 * tid] = 0;
            s_cnt[2 * tid + 1] = 0;
        }
        __syncthreads();
        if (!s_any_done) continue;

        // ---- results of finished frames (E of a finished lane is frozen)
        for (int b = tid; b < nb; b += T) {  // one byte of output (8 variables) per thread and step
            for (int ww = 0; ww < W; ++ww) {
                uint32_t dmask = 0;  // finished lanes of this word
#pragma unroll
                for (int l = 0; l < 4; ++l) dmask |= (uint32_t)s_done[4 * ww + l] << l;
                if (!dmask) continue;
                uint32_t e[8];
#pragma unroll
                for (int qq = 0; qq < 8; ++qq) {
                    const int j = 8 * b + qq;
                    e[qq] = (j < n) ? E_s[j * W + ww] : 0xFFFFFFFFu;  // past n: bit 7 set, output bit 0
                }
                for (int l = 0; l < 4; ++l) {
                    if (!((dmask >> l) & 1u)) continue;
                    uint32_t byte = 0;
#pragma unroll
                    for (int qq = 0; qq < 8; ++qq) byte |= ((~e[qq] >> (8 * l + 7)) & 1u) << qq;  // E < 0 <=> bit 7 clear
                    A.out_bits[(int64_t)s_frame[4 * ww + l] * nb + b] = (uint8_t)byte;
                }
            }
        }
        if (tid < NL && s_done[tid]) {
            const int64_t f = s_frame[tid];
            A.out_iters[f] = s_itsum[tid] + s_it[tid];
            A.out_ok[f] = s_okf[tid];
            if (A.out_rounds) A.out_rounds[f] = s_round[tid];
        }
        __syncthreads();
        // ---- claim the next frames for the finished and the idle lanes.  A
        // CTA whose oldest live frame is long past the typical count (almost
        // surely one that runs to max_iter) holds instead -- claims nothing and
        // leaves its free lanes idle -- when the frames left in the queue, at
        // the mean iteration count of the finished ones and with half again as
        // margin, fit in the lanes of the whole grid before that frame ends:
        // it then spends its remaining iterations without refills, and the
        // queue drains through the other CTAs no later than it would have.
        if (tid == 0) {
            unsigned long long* done_iters = reinterpret_cast<unsigned long long*>(A.queue + 2);
            int fin = 0;
            unsigned long long fin_it = 0;
            int oldest = 0, oldest_end = A.max_iter;  // iterations of the oldest live frame, and when it ends at latest
            for (int lane = 0; lane < NL; ++lane) {
                if (s_done[lane]) {
                    ++fin;
                    fin_it += (unsigned)(s_itsum[lane] + s_it[lane]);
                }
                if (((s_active[lane >> 2] >> (8 * (lane & 3))) & 1u) && s_it[lane] > oldest) {
                    oldest = s_it[lane];
                    oldest_end = A.stall ? min(A.max_iter, s_tbest[lane] + A.stall) : A.max_iter;
                }
            }
            const int done_f = atomicAdd(A.queue + 1, fin) + fin;
            const unsigned long long done_i = atomicAdd(done_iters, fin_it) + fin_it;
            bool hold = false;
            if (!epoch && oldest >= kHoldAfter && done_f >= kHoldMinDone) {
                const long long left = (long long)A.list_len - atomicAdd(A.queue, 0);
                hold = left <= 0 || 3ull * (unsigned long long)left * done_i <
                                        2ull * (unsigned long long)done_f * gridDim.x * NL * (oldest_end - oldest);
            }
            int k = 0;
            for (int lane = 0; lane < NL; ++lane) k += (s_done[lane] || s_frame[lane] < 0) ? 1 : 0;
            const int base = hold ? 0 : atomicAdd(A.queue, k);
            int i = 0;
            for (int lane = 0; lane < NL; ++lane) {
                if (!s_done[lane] && s_frame[lane] >= 0) continue;  // still decoding
                s_done[lane] = 0;
                s_round[lane] = 0;
                s_itsum[lane] = 0;
                s_frame[lane] = hold ? -1 : frame_of(A, base + i++);
                if (s_frame[lane] >= 0) {
                    s_load[lane >> 2] |= 0xFFu << (8 * (lane & 3));
                    s_any_load = 1;
                }
            }
        }
    }
}


template <int MAXH, int W>
int launch_p(const ldpc_code* c, const PersistArgs& A, int ctas_per_sm, int threads, int* grid_out, bool dry,
             cudaStream_t st) {
    constexpr int P = 2;
    constexpr int MAXT = max_threads<MAXH>();
    int T = c->Z * W * P;
    if (T > MAXT) T = MAXT;
    T = (T + 31) / 32 * 32;
    if (threads > 0) {  // fewer threads than rows: each thread pair then takes several rows per layer
        if (threads % (32 * W) || threads > MAXT)
            return ldpc::fail(LDPC_EINVAL, "persistent decode: threads must be a multiple of 32*words and at most " +
                                               std::to_string(MAXT));
        T = threads;
    }
    const size_t smem = smem_bytes(c, W);
    auto kern = persistent_kernel<MAXH, P, W, MAXT>;
    LDPC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 0, sms = 0;
    LDPC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, T, smem));
    LDPC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    if (occ < 1) return ldpc::fail(LDPC_EUNSUPPORTED, "persistent decode: kernel does not fit on an SM");
    int per_sm = ctas_per_sm > 0 ? (ctas_per_sm < occ ? ctas_per_sm : occ) : occ;
    int64_t grid = (int64_t)sms * per_sm;
    const int64_t need = ((int64_t)A.list_len + 4 * W - 1) / (4 * W);
    if (grid > need && A.epoch_iters <= 0) grid = need;  // epoch mode keeps its grid: lanes belong to CTAs
    if (grid < 1) grid = 1;
    *grid_out = (int)grid;
    if (dry) return LDPC_OK;
    LDPC_CUDA_TRY(cudaMemsetAsync(A.queue, 0, 4 * sizeof(int), st));
    kern<<<(int)grid, T, smem, st>>>(A);
    ldpc::count_launch();
    LDPC_CUDA_TRY(cudaGetLastError());
    return LDPC_OK;
}

// Launch (or with dry, only size the grid of) the persistent decoder of
// width MAXH with W words per row.  Instantiated once per width, each in its
// own translation unit.
template <int MAXH>
int persist_launch(const ldpc_code* c, const PersistArgs& A, int W, int ctas_per_sm, int threads, int* grid, bool dry,
                   cudaStream_t st) {
    if (W == 1) return launch_p<MAXH, 1>(c, A, ctas_per_sm, threads, grid, dry, st);
    if (W == 2) return launch_p<MAXH, 2>(c, A, ctas_per_sm, threads, grid, dry, st);
    return launch_p<MAXH, 4>(c, A, ctas_per_sm, threads, grid, dry, st);
}

#define LDPC_PERSIST_EXTERN(M) \
    extern template int persist_launch<M>(const ldpc_code*, const PersistArgs&, int, int, int, int*, bool, \
                                          cudaStream_t);
LDPC_MAXH_LIST(LDPC_PERSIST_EXTERN)
#undef LDPC_PERSIST_EXTERN

}  // namespace ldpc_dec
