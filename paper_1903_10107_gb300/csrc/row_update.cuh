// One check row of the layered decoder (sections 2 and 3), in byte lanes.
//
// Storage is offset binary: a soft value E (or message L) in [-127, 127] is
// kept as the byte E + 128, so |E - L| is one unsigned byte absolute
// difference and the hard decision E < 0 is "bit 7 clear".
//
// Per edge the thread forms, from the stored E_j and L_ij (Eq. 8):
//   a = min(|E_j - L_ij|, 127) = |sat8(E_j - L_ij)|, sign bit sv = [E_j < L_ij]
// and packs them as av = a | sv (bit 7).  The row's sign S is the syndrome bit
// xor every sv (Eq. 1 with the syndrome sign).  The magnitude for edge k is
// the box-plus of the other magnitudes (Eq. 7) with tau of Algorithm 1,
// folded forward-backward in ascending variable order:
//   m_k = tau(F_{k-1}, B_{k+1}),  F = left fold, B = right fold.
// The outgoing message is L_ij = (S xor sv) m and the soft value becomes
// sat8(v + L_ij) (Eq. 9) unless |E_j| = 127 (Algorithm 2):
//   S = 0 (same sign):     E = sv * min(a + m, 127)
//   S = 1 (opposite sign): E = sv * (a - m)          (already in range)
//
// Two threads share a row.  Thread 0 walks edges 0..h-1 upward, thread 1
// walks edges d-1..h downward; both fold tau over their own walk (tau is
// symmetric, so thread 1's fold is the right fold B), swap their totals and
// sign parities with one shuffle each, and walk back to produce their
// outputs.  Both threads run the same instructions.
#pragma once

#include "common.cuh"

namespace ldpc_dev {

using namespace lanes;

// m' = clamp(((m*s + 8) >> 4) - o, 0, 127) per byte, s and o the same for all
// lanes.  Even and odd bytes are widened to 16-bit lanes: m*s <= 127*255 and
// the later bias keep every lane below 2^16.
__device__ __forceinline__ uint32_t apply_table(uint32_t m, uint32_t s, int o) {
    uint32_t lo = m & 0x00FF00FFu, hi = (m >> 8) & 0x00FF00FFu;
    lo = ((lo * s + 0x00080008u) >> 4) & 0x0FFF0FFFu;
    hi = ((hi * s + 0x00080008u) >> 4) & 0x0FFF0FFFu;
    const uint32_t bias = (uint32_t)(128 - o) * 0x00010001u;  // x - o + 128 in [1, 2280]
    lo = __vmaxu2(__vminu2(lo + bias, 0x00FF00FFu), 0x00800080u) - 0x00800080u;
    hi = __vmaxu2(__vminu2(hi + bias, 0x00FF00FFu), 0x00800080u) - 0x00800080u;
    return lo | (hi << 8);
}

// (r + s) mod Z for r, s in [0, Z): the unsigned min of x and x - Z.
__device__ __forceinline__ int wrap(int x, int Z) { return (int)min((unsigned)x, (unsigned)(x - Z)); }

// Shared-memory code tables: deg[Mb], off[Mb+1], then per nonzero block
// {block column * Z * W, circulant shift}.
struct Tables {
    const int* deg;
    const int* off;
    const int2* et;
};

__device__ __forceinline__ size_t tables_words(int Mb, int nblk) {
    return (size_t)((2 * Mb + 1 + 1) & ~1) + 2 * (size_t)nblk;
}

__device__ __forceinline__ Tables load_tables(int32_t* s, const int32_t* g, int Mb, int nblk, int Z, int W,
                                              int tid, int T) {
    const int head = (2 * Mb + 1 + 1) & ~1;
    for (int i = tid; i < 2 * Mb + 1; i += T) s[i] = g[i];
    int2* et = reinterpret_cast<int2*>(s + head);
    const int32_t* col = g + 2 * Mb + 1;
    const int32_t* sh = col + nblk;
    for (int b = tid; b < nblk; b += T) et[b] = make_int2(col[b] * Z * W, sh[b]);
    return Tables{s, s + Mb, et};
}

struct RowCtx {
    uint32_t* E_s;           // shared soft values, [n][W] words
    uint32_t* msg;           // this CTA's messages, [(block)*Z + row][W] words
    const int2* et;          // edge table of the layer (ascending block column)
    int b0, d, Z, w;         // layer block offset and degree; lifting; my word
    uint32_t fresh;          // lanes whose stored L is stale (treated as 0)
    uint32_t active;         // lanes whose E may change
    uint32_t sq;             // table scale (16 = identity)
    int oq;                  // table offset
};

// `half` is 0 or 1; `valid` false makes the thread a bystander that only
// joins the shuffles.  HMAX bounds the edges walked by one thread.
template <int HMAX, int W, bool TABLES>
__device__ __forceinline__ void row_update(const RowCtx& C, int r, bool valid, int half, uint32_t syn_nib) {
    const int d = valid ? C.d : 0;
    const int h = (d + 1) >> 1;
    const int cnt = half ? d - h : h;           // edges walked by this thread
    const int Z = C.Z;
    const int k0 = half ? d - 1 : 0;             // first edge of the walk
    const int kdir = half ? -1 : 1;
    const int2* et = C.et + k0;
    uint32_t* Lp = C.msg + ((size_t)(C.b0 + k0) * Z + r) * W + C.w;
    const int Lstep = kdir * Z * W;  // 32-bit: one wide multiply-add per slot address
    uint32_t av[HMAX], F[HMAX];
    int idx[HMAX];
    uint32_t S = (half == 0 && valid) ? nibble_to_high(syn_nib) : 0u;

    const bool load_l = C.fresh != 0xFFFFFFFFu;
    // Slots are guarded in chunks of CH: a chunk wholly past the walk's count
    // is skipped by one branch, where per-slot guards alone left the idle
    // slots' instructions to be issued predicated off.  Measured on a code
    // with rows of 6-25 edges (13 slots): chunks of 4 are 5.8 % faster than
    // per-slot guards, chunks of 3 another 1.4 %, chunks of 2, 6 or 8 slower;
    // bodies of at most 8 slots are fastest as one chunk (2.5 % on rows of
    // 15-16 edges).
    constexpr int CH = HMAX <= 8 ? HMAX : 3;
#pragma unroll
    for (int c0 = 0; c0 < HMAX; c0 += CH) {
        if (c0 < cnt) {
#pragma unroll
            for (int j = c0; j < (c0 + CH < HMAX ? c0 + CH : HMAX); ++j) {
                if (j < cnt) {
                    av[j] = load_l ? Lp[j * Lstep] : kHigh;  // every message load of the row in flight first
                    const int2 t = et[j * kdir];
                    idx[j] = t.x + wrap(r + t.y, Z) * W + C.w;
                }
            }
        }
    }
    // One pass per slot: |E - L| and its sign, then the left fold.  (A
    // separate pass for each doubles the guard branches of the unrolled slots.)
    uint32_t tot = kMax;
#pragma unroll
    for (int c0 = 0; c0 < HMAX; c0 += CH) {
        if (c0 < cnt) {
#pragma unroll
            for (int j = c0; j < (c0 + CH < HMAX ? c0 + CH : HMAX); ++j) {
                if (j < cnt) {
                    const uint32_t e = C.E_s[idx[j]];
                    const uint32_t lb = select(C.fresh, kHigh, av[j]);  // stale lanes read as 0
                    const uint32_t sv = lt_u8(e, lb);    // sign of E - L
                    const uint32_t a = cap127(absdiff(e, lb));  // |sat8(E - L)|
                    av[j] = a | sv;
                    S ^= sv;
                    tot = (j == 0) ? a : tau(tot, a);
                    F[j] = tot;
                }
            }
        }
    }
    // A half that walks no edge sends tot = MSG_max: for a degree-1 row the one
    // edge then gets m = MSG_max, the box-plus over the empty set.
    uint32_t R = __shfl_xor_sync(0xffffffffu, tot, W);
    S ^= __shfl_xor_sync(0xffffffffu, S, W);
    const uint32_t MS = spread(S);

#pragma unroll
    for (int c0 = ((HMAX - 1) / CH) * CH; c0 >= 0; c0 -= CH) {
        if (c0 < cnt) {
#pragma unroll
            for (int j = (c0 + CH < HMAX ? c0 + CH : HMAX) - 1; j >= c0; --j) {
                if (j < cnt) {
                    const uint32_t a = av[j] & kMax;
                    const uint32_t Fp = F[j >= 1 ? j - 1 : 0];
                    uint32_t m = (j == 0) ? R : tau(Fp, R);
                    if (j > 0) R = tau(a, R);
                    if (TABLES) m = apply_table(m, C.sq, C.oq);
                    // Negation in offset binary: the byte 128 - x is 256 - (128 + x).  For
                    // words whose four bytes y are all >= 1, 0x01010100 - y equals the
                    // bytes 256 - y (the borrows out of bytes 0..2 are the 1s added to
                    // bytes 1..3, and the one out of byte 3 leaves the word).
                    const uint32_t Msv = spread(av[j]);
                    const uint32_t hm = kHigh | m;             // 128 + m, bytes >= 128
                    const uint32_t lnew = select(Msv ^ MS, 0x01010100u - hm, hm);
                    // y = 128 + u with E_new = sv ? -u : u, u = a - m (opposite signs,
                    // in [-127, 127]) or min(a + m, 127) (same sign); bytes >= 1
                    const uint32_t y = select(MS, kHigh + a - m, kHigh | cap127(a + m));
                    uint32_t* ep = &C.E_s[idx[j]];
                    const uint32_t eo = *ep;
                    const uint32_t sat = spread(absdiff(eo, kHigh) + kOnes);  // |E| = 127
                    *ep = select(C.active & ~sat, select(Msv, 0x01010100u - y, y), eo);
                    Lp[j * Lstep] = lnew;
                }
            }
        }
    }
}

// One body per kernel: MAXH bounds ceil(d/2) over all layers of the code (the
// smallest compiled width that holds the longest row, maxh.cuh).  A single
// body keeps register allocation tight; the guarded slots past a layer's
// degree are the price of irregular codes.
template <int W, bool TABLES, int MAXH>
__device__ __forceinline__ void row_update_any(const RowCtx& C, int r, bool valid, int half, uint32_t syn_nib) {
    row_update<MAXH, W, TABLES>(C, r, valid, half, syn_nib);
}

// Parity of check row r of a layer against its syndrome bits: bit 7 of each
// byte set where the lane's check fails.  Hard decision: E < 0, i.e. bit 7 of
// the stored byte clear, so the xor of bit 7s is flipped once per edge.
template <int W>
__device__ __forceinline__ uint32_t row_parity(const uint32_t* E_s, const int2* et, int d, int r, int Z, int w,
                                               uint32_t syn_nib) {
    uint32_t p = nibble_to_high(syn_nib) ^ ((d & 1) ? kHigh : 0u);
    int k = 0;
    for (; k + 2 <= d; k += 2) {
        const int2 t0 = et[k], t1 = et[k + 1];
        p ^= E_s[t0.x + wrap(r + t0.y, Z) * W + w] ^ E_s[t1.x + wrap(r + t1.y, Z) * W + w];
    }
    if (k < d) {
        const int2 t = et[k];
        p ^= E_s[t.x + wrap(r + t.y, Z) * W + w];
    }
    return p & kHigh;
}

// row_parity with the edge loop unrolled for at most MAXD edges: every soft-value load of the row is in
// flight before the first is used.  Worth it where the unrolled loads fit the registers without spilling
// (codes whose rows have at most 16 edges): 0.7-0.8 % on the persistent step of the n = 49152 code.
template <int W, int MAXD>
__device__ __forceinline__ uint32_t row_parity_unrolled(const uint32_t* E_s, const int2* et, int d, int r, int Z,
                                                        int w, uint32_t syn_nib) {
    uint32_t v[MAXD];
#pragma unroll
    for (int k = 0; k < MAXD; ++k) {
        if (k < d) {
            const int2 t = et[k];
            v[k] = E_s[t.x + wrap(r + t.y, Z) * W + w];
        }
    }
    uint32_t p = nibble_to_high(syn_nib) ^ ((d & 1) ? kHigh : 0u);
#pragma unroll
    for (int k = 0; k < MAXD; ++k)
        if (k < d) p ^= v[k];
    return p & kHigh;
}

}  // namespace ldpc_dev
