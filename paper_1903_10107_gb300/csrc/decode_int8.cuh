// Layered int8 decoding of a batch of frames (sections 2 and 3).
//
// Work decomposition
//   * A CTA owns a group of 4*W frames for the whole decode.  Frame 4w + l of
//     the group sits in byte lane l of word w, so one 32-bit operation
//     advances four frames.
//   * E (the soft values, n bytes per frame) stays in shared memory for the
//     whole decode: E_s[j*W + w].
//   * L (check-to-variable messages, one byte per edge and frame) lives in a
//     global scratch arena, edge-major with frames innermost:
//     msg[group][(block b)*Z + row][w].  Consecutive threads handle
//     consecutive rows, so every access of a warp is one contiguous run.
//   * One block row is one layer.  The Z rows of a layer touch distinct
//     variable nodes, so threads update them in parallel; layers are
//     separated by a CTA barrier.
//   * Two threads share a check row: they fold tau (Algorithm 1) forward and
//     backward over the row's edges in ascending variable order, in
//     registers (row_update.cuh), unrolled for the code's width (maxh.cuh).
//   * After each iteration all parity checks are tested with the latest E
//     (section 2); lanes whose syndrome matches are frozen and leave the
//     group's stopping test; the CTA stops when every lane has stopped.
#pragma once

#include "maxh.cuh"
#include "row_update.cuh"

namespace ldpc_dec {

using namespace lanes;
using ldpc_dev::RowCtx;

struct DecodeArgs {
    const int32_t* tab;
    int Mb, nblk, Z, n, m;
    const int8_t* llr;
    const uint8_t* syn;
    int batch, max_iter;
    const uint8_t* scale_q4;
    const int8_t* offset_q;
    uint8_t* out_bits;
    int32_t* out_iters;
    uint8_t* out_ok;
    uint32_t* msg;
};

// Shared memory of a CTA: soft values (4 n W bytes), the code tables from the
// next 16-byte boundary (their int2 edge entries need 8-byte alignment, and
// 4 n W is only a multiple of 4 when n is odd), then the syndrome nibbles.
__host__ __device__ inline size_t soft_bytes(int n, int W) { return ((size_t)4 * n * W + 15) & ~(size_t)15; }

// Threads: tid = ((row slot) * P + half) * W + w.  The two halves of a row sit
// W lanes apart in one warp.
template <int MAXH, int P, int W, bool TABLES, int MAXT>
__global__ void __launch_bounds__(MAXT) decode_kernel(DecodeArgs A) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int n = A.n, m = A.m, Z = A.Z, Mb = A.Mb, nblk = A.nblk;
    const int tab_words = (int)ldpc_dev::tables_words(Mb, nblk);
    uint32_t* E_s = reinterpret_cast<uint32_t*>(smem);
    int32_t* s_tab = reinterpret_cast<int32_t*>(smem + soft_bytes(n, W));
    uint8_t* syn_s = reinterpret_cast<uint8_t*>(s_tab + tab_words);
    __shared__ uint32_t s_bad[W], s_active[W];
    __shared__ int s_iters[4 * W];

    const int tid = threadIdx.x, T = blockDim.x;
    const int w = tid % W, q = tid / W;
    const int half = (P == 2) ? (q & 1) : 0;
    const int rt = q / P, RT = T / (W * P), QT = T / W;
    const int64_t f0 = (int64_t)blockIdx.x * 4 * W;
    const int mbytes = (m + 7) / 8;

    const ldpc_dev::Tables TB = ldpc_dev::load_tables(s_tab, A.tab, Mb, nblk, Z, W, tid, T);
    for (int idx = tid; idx < n * W; idx += T) {
        const int j = idx / W, ww = idx % W;
        uint32_t word = 0;
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const int64_t f = f0 + 4 * ww + l;
            if (f < A.batch) word |= (uint32_t)(uint8_t)A.llr[f * n + j] << (8 * l);
        }
        E_s[idx] = word ^ kHigh;  // offset binary
    }
    for (int idx = tid; idx < m * W; idx += T) {
        const int c = idx / W, ww = idx % W;
        uint32_t nib = 0;
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const int64_t f = f0 + 4 * ww + l;
            if (f < A.batch) nib |= ((A.syn[f * mbytes + (c >> 3)] >> (c & 7)) & 1u) << l;
        }
        syn_s[idx] = (uint8_t)nib;
    }
    if (tid < W) {
        uint32_t act = 0;
        for (int l = 0; l < 4; ++l)
            if (f0 + 4 * tid + l < A.batch) act |= 0xFFu << (8 * l);
        s_active[tid] = act;
        s_bad[tid] = 0;
    }
    if (tid < 4 * W) s_iters[tid] = 0;
    __syncthreads();

    const int* deg = TB.deg;
    const int* off = TB.off;

    RowCtx C;
    C.E_s = E_s;
    C.msg = A.msg + (size_t)blockIdx.x * nblk * Z * W;
    C.Z = Z;
    C.w = w;
    C.sq = 16;
    C.oq = 0;

    // the stopping test's rows of this thread: c = q + k QT, layer i, row r
    const int pq_i0 = q / Z, pq_r0 = q - pq_i0 * Z, pq_di = QT / Z, pq_dr = QT - pq_di * Z;
    for (int t = 1; t <= A.max_iter; ++t) {
        C.active = s_active[w];
        C.fresh = (t == 1) ? 0xFFFFFFFFu : 0u;  // messages start at 0 (stale scratch is never read)
        for (int i = 0; i < Mb; ++i) {          // one block row = one layer, in order
            C.d = deg[i];
            C.b0 = off[i];
            C.et = TB.et + C.b0;
            if (TABLES) {
                if (A.scale_q4) C.sq = A.scale_q4[(size_t)(t - 1) * Mb + i];
                if (A.offset_q) C.oq = A.offset_q[(size_t)(t - 1) * Mb + i];
            }
            if (C.d > 0) {
                for (int r0 = 0; r0 < Z; r0 += RT) {
                    const int r = r0 + rt;
                    const bool valid = r < Z;
                    const uint32_t nib = valid ? syn_s[(i * Z + r) * W + w] : 0u;
                    ldpc_dev::row_update_any<W, TABLES, MAXH>(C, valid ? r : 0, valid, half, nib);
                }
            }
            __syncthreads();
        }
        // stopping test: every parity check with the latest E (section 2)
        uint32_t bad = 0;
        {
            int i = pq_i0, r = pq_r0;  // layer and row of check c = q + k QT
            for (int c = q; c < m; c += QT) {
                const int d = deg[i];
                const int2* et = TB.et + off[i];
                const uint32_t nib = syn_s[c * W + w];
                bad |= ldpc_dev::row_parity<W>(E_s, et, d, r, Z, w, nib);
                r += pq_dr;
                i += pq_di;
                if (r >= Z) {
                    r -= Z;
                    ++i;
                }
            }
        }
#pragma unroll
        for (int o = 16; o >= W; o >>= 1) bad |= __shfl_xor_sync(0xffffffffu, bad, o);
        if ((tid & 31) < W && bad) atomicOr(&s_bad[w], bad);
        __syncthreads();
        if (tid < W) {
            const uint32_t failing = spread(s_bad[tid]);
            const uint32_t act = s_active[tid];
            const uint32_t newly = act & ~failing;
            for (int l = 0; l < 4; ++l)
                if ((newly >> (8 * l)) & 0xFFu) s_iters[4 * tid + l] = t;
            s_active[tid] = act & failing;
            s_bad[tid] = 0;
        }
        __syncthreads();
        uint32_t live = 0;
#pragma unroll
        for (int ww = 0; ww < W; ++ww) live |= s_active[ww];
        if (!live) break;
    }

    if (tid < 4 * W) {
        const int64_t f = f0 + tid;
        if (f < A.batch) {
            const int it = s_iters[tid];
            A.out_iters[f] = it ? it : A.max_iter;
            A.out_ok[f] = it ? 1 : 0;
        }
    }
    const int nb = (n + 7) / 8;
    for (int idx = tid; idx < 4 * W * nb; idx += T) {
        const int lane = idx / nb, b = idx - lane * nb;
        const int64_t f = f0 + lane;
        if (f >= A.batch) continue;
        const int ww = lane >> 2, sbit = 8 * (lane & 3) + 7;
        uint32_t byte = 0;
        for (int qq = 0; qq < 8; ++qq) {
            const int j = 8 * b + qq;
            if (j < n) byte |= ((~E_s[j * W + ww] >> sbit) & 1u) << qq;  // E < 0 <=> stored bit 7 clear
        }
        A.out_bits[f * nb + b] = (uint8_t)byte;
    }
}

// ---------------------------------------------------------------------------
// The same decode with all W words of a row-half in one thread.  Each edge
// slot's index arithmetic, table load, guard and loop step then serve 4W
// frames instead of 4, and a slot's message and soft-value words move as one
// 8-byte (W = 2) or 16-byte (W = 4) access.  Thread t is half (t & 1) of row
// slot t >> 1; a CTA has 2 Z threads (512 at most, so up to 128 registers).
// Used for W >= 2 where the slots' registers fit (every width up to 16 slots
// at W = 2, up to 9 at W = 4, where it spills 52 bytes and is still faster):
// 17-26 % faster than one word per thread at the same group width on the
// n = 4096 code (16384 frames: 6.88 against 8.26 ms at W = 2, 9.32 against
// 12.07 at W = 4).
// ---------------------------------------------------------------------------
template <int W>
__device__ __forceinline__ void ld_words(const uint32_t* p, uint32_t (&o)[W]) {
    if constexpr (W == 4) {
        const uint4 v = *reinterpret_cast<const uint4*>(p);
        o[0] = v.x;
        o[1] = v.y;
        o[2] = v.z;
        o[3] = v.w;
    } else if constexpr (W == 2) {
        const uint2 v = *reinterpret_cast<const uint2*>(p);
        o[0] = v.x;
        o[1] = v.y;
    } else {
        o[0] = *p;
    }
}
template <int W>
__device__ __forceinline__ void st_words(uint32_t* p, const uint32_t (&o)[W]) {
    if constexpr (W == 4) {
        *reinterpret_cast<uint4*>(p) = make_uint4(o[0], o[1], o[2], o[3]);
    } else if constexpr (W == 2) {
        *reinterpret_cast<uint2*>(p) = make_uint2(o[0], o[1]);
    } else {
        *p = o[0];
    }
}

// row_update of row_update.cuh for all W words of the row-half at once; the
// partner half is the neighbouring thread.  act: lanes whose E may change.
template <int HMAX, int W, bool TABLES>
__device__ __forceinline__ void row_update_words(uint32_t* E_s, uint32_t* msg, const int2* etab, int b0, int d, int Z,
                                                 int r, bool valid, int half, const uint32_t (&act)[W],
                                                 uint32_t fresh, const uint8_t* syn_row, uint32_t sq, int oq) {
    d = valid ? d : 0;
    const int h = (d + 1) >> 1;
    const int cnt = half ? d - h : h;
    constexpr int CH = HMAX <= 8 ? HMAX : 4;  // slots per guarded chunk, as in row_update (2-4 % here)
    const int k0 = half ? d - 1 : 0;
    const int kdir = half ? -1 : 1;
    const int2* et = etab + k0;
    uint32_t* Lp = msg + ((size_t)(b0 + k0) * Z + r) * W;
    const ptrdiff_t Lstep = (ptrdiff_t)kdir * Z * W;
    uint32_t av[HMAX][W], F[HMAX][W];
    int idx[HMAX];
    uint32_t S[W];
#pragma unroll
    for (int w = 0; w < W; ++w) S[w] = (half == 0 && valid) ? nibble_to_high(syn_row[w]) : 0u;
    const bool load_l = fresh != 0xFFFFFFFFu;
#pragma unroll
    for (int c0 = 0; c0 < HMAX; c0 += CH) {
        if (c0 < cnt) {
#pragma unroll
            for (int j = c0; j < (c0 + CH < HMAX ? c0 + CH : HMAX); ++j) {
                if (j < cnt) {
                    if (load_l) {
                        ld_words<W>(Lp + j * Lstep, av[j]);  // every message load of the row in flight first
                    } else {
        #pragma unroll
                        for (int w = 0; w < W; ++w) av[j][w] = kHigh;
                    }
                    const int2 t = et[j * kdir];
                    idx[j] = t.x + ldpc_dev::wrap(r + t.y, Z) * W;
                }
            }
        }
    }
    uint32_t tot[W];
#pragma unroll
    for (int w = 0; w < W; ++w) tot[w] = kMax;
#pragma unroll
    for (int c0 = 0; c0 < HMAX; c0 += CH) {
        if (c0 < cnt) {
#pragma unroll
            for (int j = c0; j < (c0 + CH < HMAX ? c0 + CH : HMAX); ++j) {
                if (j < cnt) {
                    uint32_t e[W];
                    ld_words<W>(&E_s[idx[j]], e);
        #pragma unroll
                    for (int w = 0; w < W; ++w) {
                        const uint32_t lb = select(fresh, kHigh, av[j][w]);  // stale lanes read as 0
                        const uint32_t sv = lt_u8(e[w], lb);
                        const uint32_t a = cap127(absdiff(e[w], lb));
                        av[j][w] = a | sv;
                        S[w] ^= sv;
                        tot[w] = (j == 0) ? a : tau(tot[w], a);
                        F[j][w] = tot[w];
                    }
                }
            }
        }
    }
    uint32_t R[W], MS[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
        R[w] = __shfl_xor_sync(0xffffffffu, tot[w], 1);
        S[w] ^= __shfl_xor_sync(0xffffffffu, S[w], 1);
        MS[w] = spread(S[w]);
    }
#pragma unroll
    for (int c0 = ((HMAX - 1) / CH) * CH; c0 >= 0; c0 -= CH) {
        if (c0 < cnt) {
#pragma unroll
            for (int j = (c0 + CH < HMAX ? c0 + CH : HMAX) - 1; j >= c0; --j) {
                if (j < cnt) {
                    uint32_t eo[W], en[W], ln[W];
                    ld_words<W>(&E_s[idx[j]], eo);
        #pragma unroll
                    for (int w = 0; w < W; ++w) {
                        const uint32_t a = av[j][w] & kMax;
                        const uint32_t Fp = F[j >= 1 ? j - 1 : 0][w];
                        uint32_t m = (j == 0) ? R[w] : tau(Fp, R[w]);
                        if (j > 0) R[w] = tau(a, R[w]);
                        if (TABLES) m = ldpc_dev::apply_table(m, sq, oq);
                        const uint32_t Msv = spread(av[j][w]);
                        const uint32_t hm = kHigh | m;
                        ln[w] = select(Msv ^ MS[w], 0x01010100u - hm, hm);
                        const uint32_t y = select(MS[w], kHigh + a - m, kHigh | cap127(a + m));
                        const uint32_t sat = spread(absdiff(eo[w], kHigh) + kOnes);  // |E| = 127
                        en[w] = select(act[w] & ~sat, select(Msv, 0x01010100u - y, y), eo[w]);
                    }
                    st_words<W>(&E_s[idx[j]], en);
                    st_words<W>(Lp + j * Lstep, ln);
                }
            }
        }
    }
}

template <int MAXH, int W, bool TABLES>
__global__ void __launch_bounds__(512) decode_words_kernel(DecodeArgs A) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int n = A.n, m = A.m, Z = A.Z, Mb = A.Mb, nblk = A.nblk;
    const int tab_words = (int)ldpc_dev::tables_words(Mb, nblk);
    uint32_t* E_s = reinterpret_cast<uint32_t*>(smem);
    int32_t* s_tab = reinterpret_cast<int32_t*>(smem + soft_bytes(n, W));
    uint8_t* syn_s = reinterpret_cast<uint8_t*>(s_tab + tab_words);
    __shared__ uint32_t s_bad[W], s_active[W];
    __shared__ int s_iters[4 * W];
    const int tid = threadIdx.x, T = blockDim.x;
    const int half = tid & 1, rt = tid >> 1, RT = T >> 1;
    const int64_t f0 = (int64_t)blockIdx.x * 4 * W;
    const int mbytes = (m + 7) / 8;
    const ldpc_dev::Tables TB = ldpc_dev::load_tables(s_tab, A.tab, Mb, nblk, Z, W, tid, T);
    for (int idx = tid; idx < n * W; idx += T) {
        const int j = idx / W, ww = idx % W;
        uint32_t word = 0;
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const int64_t f = f0 + 4 * ww + l;
            if (f < A.batch) word |= (uint32_t)(uint8_t)A.llr[f * n + j] << (8 * l);
        }
        E_s[idx] = word ^ kHigh;  // offset binary
    }
    for (int idx = tid; idx < m * W; idx += T) {
        const int c = idx / W, ww = idx % W;
        uint32_t nib = 0;
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const int64_t f = f0 + 4 * ww + l;
            if (f < A.batch) nib |= ((A.syn[f * mbytes + (c >> 3)] >> (c & 7)) & 1u) << l;
        }
        syn_s[idx] = (uint8_t)nib;
    }
    if (tid < W) {
        uint32_t act = 0;
        for (int l = 0; l < 4; ++l)
            if (f0 + 4 * tid + l < A.batch) act |= 0xFFu << (8 * l);
        s_active[tid] = act;
        s_bad[tid] = 0;
    }
    if (tid < 4 * W) s_iters[tid] = 0;
    __syncthreads();
    uint32_t* msg = A.msg + (size_t)blockIdx.x * nblk * Z * W;
    for (int t = 1; t <= A.max_iter; ++t) {
        uint32_t act[W];
#pragma unroll
        for (int w = 0; w < W; ++w) act[w] = s_active[w];
        const uint32_t fresh = (t == 1) ? 0xFFFFFFFFu : 0u;  // messages start at 0
        for (int i = 0; i < Mb; ++i) {                       // one block row = one layer, in order
            const int d = TB.deg[i], b0 = TB.off[i];
            uint32_t sq = 16;
            int oq = 0;
            if (TABLES) {
                if (A.scale_q4) sq = A.scale_q4[(size_t)(t - 1) * Mb + i];
                if (A.offset_q) oq = A.offset_q[(size_t)(t - 1) * Mb + i];
            }
            if (d > 0) {
                for (int r0 = 0; r0 < Z; r0 += RT) {
                    const int r = r0 + rt;
                    const bool valid = r < Z;
                    const int rr = valid ? r : 0;
                    row_update_words<MAXH, W, TABLES>(E_s, msg, TB.et + b0, b0, d, Z, rr, valid, half, act, fresh,
                                                      &syn_s[(i * Z + rr) * W], sq, oq);
                }
            }
            __syncthreads();
        }
        // stopping test: every parity check with the latest E (section 2)
        uint32_t bad[W];
#pragma unroll
        for (int w = 0; w < W; ++w) bad[w] = 0;
        for (int c = tid; c < m; c += T) {
            const int i = c / Z, r = c - i * Z;
#pragma unroll
            for (int w = 0; w < W; ++w)
                bad[w] |= ldpc_dev::row_parity<W>(E_s, TB.et + TB.off[i], TB.deg[i], r, Z, w, syn_s[c * W + w]);
        }
#pragma unroll
        for (int w = 0; w < W; ++w) {
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) bad[w] |= __shfl_xor_sync(0xffffffffu, bad[w], o);
            if ((tid & 31) == 0 && bad[w]) atomicOr(&s_bad[w], bad[w]);
        }
        __syncthreads();
        if (tid < W) {
            const uint32_t failing = spread(s_bad[tid]);
            const uint32_t a = s_active[tid];
            const uint32_t newly = a & ~failing;
            for (int l = 0; l < 4; ++l)
                if ((newly >> (8 * l)) & 0xFFu) s_iters[4 * tid + l] = t;
            s_active[tid] = a & failing;
            s_bad[tid] = 0;
        }
        __syncthreads();
        uint32_t live = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) live |= s_active[w];
        if (!live) break;
    }
    if (tid < 4 * W) {
        const int64_t f = f0 + tid;
        if (f < A.batch) {
            const int it = s_iters[tid];
            A.out_iters[f] = it ? it : A.max_iter;
            A.out_ok[f] = it ? 1 : 0;
        }
    }
    const int nb = (n + 7) / 8;
    for (int idx = tid; idx < 4 * W * nb; idx += T) {
        const int lane = idx / nb, b = idx - lane * nb;
        const int64_t f = f0 + lane;
        if (f >= A.batch) continue;
        const int ww = lane >> 2, sbit = 8 * (lane & 3) + 7;
        uint32_t byte = 0;
        for (int qq = 0; qq < 8; ++qq) {
            const int j = 8 * b + qq;
            if (j < n) byte |= ((~E_s[j * W + ww] >> sbit) & 1u) << qq;  // E < 0 <=> stored bit 7 clear
        }
        A.out_bits[f * nb + b] = (uint8_t)byte;
    }
}

// Whether the batch launch of width MAXH with W words per row takes the
// several-words-per-thread kernel.
template <int MAXH, int W>
constexpr bool words_per_thread() {
    return (W == 2 && MAXH <= 16) || (W == 4 && MAXH <= 9);
}

inline size_t smem_bytes(const ldpc_code* c, int W) {
    const size_t tab_words = (size_t)((2 * c->Mb + 1 + 1) & ~1) + 2 * (size_t)c->nblk;
    size_t b = soft_bytes(c->n, W) + sizeof(int32_t) * tab_words + (size_t)c->m * W;
    return (b + 15) & ~(size_t)15;
}

template <int MAXH, int W, bool TABLES>
int launch_t(const ldpc_code* c, const DecodeArgs& A, int groups, cudaStream_t st) {
    if constexpr (words_per_thread<MAXH, W>()) {
        int T = 2 * c->Z;
        if (T > 512) T = 512;
        T = (T + 31) / 32 * 32;
        const size_t smem = smem_bytes(c, W);
        auto kern = decode_words_kernel<MAXH, W, TABLES>;
        LDPC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<groups, T, smem, st>>>(A);
        ldpc::count_launch();
        LDPC_CUDA_TRY(cudaGetLastError());
        return LDPC_OK;
    } else {
        constexpr int P = 2;
        constexpr int MAXT = max_threads<MAXH>();
        int T = c->Z * W * P;
        if (T > MAXT) T = MAXT;
        T = (T + 31) / 32 * 32;
        const size_t smem = smem_bytes(c, W);
        auto kern = decode_kernel<MAXH, P, W, TABLES, MAXT>;
        LDPC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<groups, T, smem, st>>>(A);
        ldpc::count_launch();
        LDPC_CUDA_TRY(cudaGetLastError());
        return LDPC_OK;
    }
}

// Launch the batch decoder of width MAXH with W words per row, with or
// without scale/offset tables.  Instantiated once per width, each in its own
// translation unit.
template <int MAXH>
int decode_launch(const ldpc_code* c, const DecodeArgs& A, int groups, int W, bool tables, cudaStream_t st) {
    if (W == 1) return tables ? launch_t<MAXH, 1, true>(c, A, groups, st) : launch_t<MAXH, 1, false>(c, A, groups, st);
    if (W == 2) return tables ? launch_t<MAXH, 2, true>(c, A, groups, st) : launch_t<MAXH, 2, false>(c, A, groups, st);
    return tables ? launch_t<MAXH, 4, true>(c, A, groups, st) : launch_t<MAXH, 4, false>(c, A, groups, st);
}

#define LDPC_DECODE_EXTERN(M) \
    extern template int decode_launch<M>(const ldpc_code*, const DecodeArgs&, int, int, bool, cudaStream_t);
LDPC_MAXH_LIST(LDPC_DECODE_EXTERN)
#undef LDPC_DECODE_EXTERN

}  // namespace ldpc_dec
