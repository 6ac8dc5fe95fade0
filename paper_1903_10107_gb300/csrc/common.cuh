// Shared definitions of the GB300 decoder library: the code handle, error
// plumbing and byte-lane (4 x int8 in one 32-bit word) arithmetic.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "ldpc_gb300.h"

struct ldpc_code {
    int Mb = 0, Nb = 0, Z = 0, n = 0, m = 0;
    int nblk = 0;       // nonzero circulant blocks in the base matrix
    int max_deg = 0;    // largest row (layer) degree
    int64_t edges = 0;  // ones in H = nblk * Z
    int device = 0;
    // Layer tables, block-row order, ascending block column inside a row:
    //   deg[Mb], off[Mb+1] (block offsets), col[nblk], shift[nblk]
    std::vector<int32_t> h_tab;
    int32_t* d_tab = nullptr;
    size_t tab_words = 0;
    void* arena = nullptr;  // message scratch
    size_t arena_bytes = 0;
};

namespace ldpc {

void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);
void count_launch(int64_t k = 1);
int ensure_arena(ldpc_code* c, size_t bytes);
int max_dyn_smem(int device);

inline const int32_t* tab_deg(const int32_t* t) { return t; }
inline const int32_t* tab_off(const int32_t* t, int Mb) { return t + Mb; }
inline const int32_t* tab_col(const int32_t* t, int Mb) { return t + 2 * Mb + 1; }
inline const int32_t* tab_shift(const int32_t* t, int Mb, int nblk) { return t + 2 * Mb + 1 + nblk; }

}  // namespace ldpc

#define LDPC_CUDA_TRY(expr)                                        \
    do {                                                           \
        cudaError_t _e = (expr);                                   \
        if (_e != cudaSuccess) return ldpc::cuda_fail(_e, #expr);  \
    } while (0)

// ---------------------------------------------------------------------------
// Byte lanes.  A 32-bit word carries one int8 value for each of four frames.
// Every helper below keeps each byte's arithmetic inside its byte: operands
// are restricted so that no carry or borrow crosses a byte boundary (the
// comments give the range argument).
// ---------------------------------------------------------------------------
namespace lanes {

constexpr uint32_t kHigh = 0x80808080u;  // bit 7 of every byte
constexpr uint32_t kOnes = 0x01010101u;
constexpr uint32_t kMax = 0x7F7F7F7Fu;   // +127 in every byte
constexpr uint32_t kMin = 0x81818181u;   // -127 in every byte

// prmt.b32 in its default mode: a selector nibble with bit 3 set copies the
// sign bit of the selected byte into all 8 bits.
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

// 0xFF in every byte whose bit 7 is set, 0x00 in the others.
__device__ __forceinline__ uint32_t spread(uint32_t x) { return prmt(x, 0u, 0xBA98u); }

// Bitwise select: bits of x where mask is 1, bits of y elsewhere.
__device__ __forceinline__ uint32_t select(uint32_t mask, uint32_t x, uint32_t y) {
    return (x & mask) | (y & ~mask);
}

// sat8(x - y) per byte for x, y in [-127, 127]: saturating subtraction
// (range [-128, 127]) followed by a max with -127.
__device__ __forceinline__ uint32_t sub_sat(uint32_t x, uint32_t y) {
    return __vmaxs4(__vsubss4(x, y), kMin);
}

// sat8(x + y) per byte for x, y in [-127, 127].
__device__ __forceinline__ uint32_t add_sat(uint32_t x, uint32_t y) {
    return __vmaxs4(__vaddss4(x, y), kMin);
}

// |x| per byte for x in [-127, 127].
__device__ __forceinline__ uint32_t absv(uint32_t x) {
    const uint32_t s = spread(x);
    return (x ^ s) + (s & kOnes);  // ~x + 1 = -x lies in [1, 127] for x in [-127, -1]
}

// tau(a, b) of Algorithm 1 per byte, for a, b in [0, 127] (= MSG_max, so the
// input caps are the identity).
//   l = min, g = max, d = g - l;  l > 2: l - [d<2] - [d<6];  else max(l - [d<4], 0)
// The tests are "x >= c" read from bit 7 of x + (128 - c), which stays below
// 256 for x <= 127.  For l <= 2 the correction is [d<4] only where l >= 1,
// which equals the max(., 0).
__device__ __forceinline__ uint32_t tau(uint32_t a, uint32_t b) {
    const uint32_t m = spread(a + kHigh - b);    // a + 128 - b in [1, 255]: bit 7 = (a >= b)
    const uint32_t l = select(m, b, a);
    const uint32_t g = select(m, a, b);
    const uint32_t d = g - l;                    // in [0, 127]
    const uint32_t d_ge2 = d + 0x7E7E7E7Eu;
    const uint32_t d_ge4 = d + 0x7C7C7C7Cu;
    const uint32_t d_ge6 = d + 0x7A7A7A7Au;
    const uint32_t l_ge3 = l + 0x7D7D7D7Du;
    const uint32_t l_ge1 = l + 0x7F7F7F7Fu;
    const uint32_t c2 = l_ge3 & ~d_ge2 & kHigh;                               // l>=3 and d<2
    const uint32_t c1 = ((l_ge3 & ~d_ge6) | (~l_ge3 & ~d_ge4)) & l_ge1 & kHigh; // l>=3 ? d<6 : (l>=1 and d<4)
    return l - (c2 >> 7) - (c1 >> 7);            // corrections <= l, no borrow
}

// -m in the bytes where bit 7 of s is set, m elsewhere; m in [0, 127].
__device__ __forceinline__ uint32_t apply_sign(uint32_t m, uint32_t s) {
    const uint32_t neg = (kHigh - m) ^ kHigh;    // 128 - m in [1, 128]; xor 128 gives 256 - m (0 -> 0)
    return select(spread(s), neg, m);
}

// 0xFF in the bytes with |x| = 127 (x in [-127, 127]).
__device__ __forceinline__ uint32_t saturated(uint32_t x) {
    return spread(absv(x) + kOnes);              // |x| + 1 reaches 128 only for |x| = 127
}

// Four syndrome bits (bit l = frame l) -> bit 7 of byte l.  The four partial
// products x << (7 + 7k) occupy disjoint bit ranges, so the multiply adds no
// carries.
__device__ __forceinline__ uint32_t nibble_to_high(uint32_t nib) { return (nib * 0x10204080u) & kHigh; }

// Bit 7 of each byte -> bit l of a nibble.
__device__ __forceinline__ uint32_t high_to_nibble(uint32_t x) {
    x &= kHigh;
    return ((x >> 7) | (x >> 14) | (x >> 21) | (x >> 28)) & 0xFu;
}

}  // namespace lanes
