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
    void* io = nullptr;     // device copies of the host-buffer entry points' inputs and outputs
    size_t io_bytes = 0;
    int* d_queue = nullptr; // work counter of the persistent decoder
};

namespace ldpc {

void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);
void count_launch(int64_t k = 1);
int ensure_arena(ldpc_code* c, size_t bytes);
int ensure_io(ldpc_code* c, size_t bytes);
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

// |x - y| per byte, unsigned (a native byte-lane instruction).
__device__ __forceinline__ uint32_t absdiff(uint32_t x, uint32_t y) { return __vabsdiffu4(x, y); }

// min(x, 127) per byte for x in [0, 255].
__device__ __forceinline__ uint32_t cap127(uint32_t x) { return (x | spread(x)) & kMax; }

// Bit 7 of each byte = [x < y] for unsigned bytes.  (x | 128) - (y & 127)
// stays in [1, 255] per byte, so its bit 7 is [x mod 128 >= y mod 128]; the
// top bits then decide as in a borrow chain.
__device__ __forceinline__ uint32_t lt_u8(uint32_t x, uint32_t y) {
    const uint32_t c = (x | kHigh) - (y & kMax);
    return ((~x & y) | (~(x ^ y) & ~c)) & kHigh;
}

// Integer multiply-add on the FMA pipe.  The decoder's byte-lane arithmetic
// is otherwise all integer-ALU work (adds, logic, shifts), and the ALU pipe
// issues at half the rate of the scheduler; an add written as x * 1 + c, or a
// right shift by 7 written as the high word of x * 2^25, runs on the
// multiply-add pipe instead and the two pipes then share the load.  The
// multipliers come from constant memory so that the compiler cannot fold
// them back into plain adds and shifts.
__device__ __forceinline__ uint32_t imad(uint32_t x, uint32_t y, uint32_t z) {
    uint32_t d;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(x), "r"(y), "r"(z));
    return d;
}
__device__ __forceinline__ uint32_t imad_hi(uint32_t x, uint32_t y, uint32_t z) {
    uint32_t d;
    asm("mad.hi.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(x), "r"(y), "r"(z));
    return d;
}
static __constant__ uint32_t c_mul[2] = {1u, 1u << 25};  // {x -> x, hi(x * 2^25) = x >> 7}

// tau(a, b) of Algorithm 1 per byte, for a, b in [0, 127] (= MSG_max, so the
// input caps are the identity).
//   l = min, d = |a - b|;  l > 2: l - [d<2] - [d<6];  else max(l - [d<4], 0)
// a + b - d = 2 l per byte (a + b <= 254 fits a byte); every byte of it is
// even, so the 32-bit shift by one brings a zero into each byte's bit 7 and
// yields l exactly.  The tests "x >= c" are bit 7 of x + (128 - c), which
// stays below 256 for x <= 127.  For l <= 2 the correction [d<4] is applied
// only where l >= 1, which equals max(., 0).  The result l - c1 - c2 (c1, c2
// the 0/1 corrections) is formed as l - 2 + (1 - c1) + (1 - c2): n1, n2 hold
// 1 - c1, 1 - c2 in bit 7, and the sum is exact as 32-bit arithmetic because
// the final bytes l - c1 - c2 lie in [0, 127].
__device__ __forceinline__ uint32_t tau(uint32_t a, uint32_t b) {
    const uint32_t one = c_mul[0];
    const uint32_t d = absdiff(a, b);
    const uint32_t l = (a + b - d) >> 1;
    const uint32_t d_ge2 = imad(d, one, 0x7E7E7E7Eu);
    const uint32_t d_ge4 = imad(d, one, 0x7C7C7C7Cu);
    const uint32_t d_ge6 = imad(d, one, 0x7A7A7A7Au);
    const uint32_t l_ge3 = imad(l, one, 0x7D7D7D7Du);
    const uint32_t l_ge1 = imad(l, one, 0x7F7F7F7Fu);
    const uint32_t n2 = ~(l_ge3 & ~d_ge2) & kHigh;                                  // not (l>=3 and d<2)
    const uint32_t n1 = ~(((l_ge3 & ~d_ge6) | (~l_ge3 & ~d_ge4)) & l_ge1) & kHigh;  // not (l>=3 ? d<6 : l>=1 and d<4)
    uint32_t t = imad(l, one, 0xFDFDFDFEu);                                         // l - 0x02020202 (mod 2^32)
    t = imad_hi(n1, c_mul[1], t);
    return imad_hi(n2, c_mul[1], t);
}

// Four syndrome bits (bit l = frame l) -> bit 7 of byte l.  For a 4-bit
// input the four partial products x << (7 + 7k) occupy disjoint bit ranges,
// so the multiply adds no carries; higher input bits would carry into the
// upper lanes, hence the mask.
__device__ __forceinline__ uint32_t nibble_to_high(uint32_t nib) { return ((nib & 0xFu) * 0x10204080u) & kHigh; }

// Bit 7 of each byte -> bit l of a nibble.
__device__ __forceinline__ uint32_t high_to_nibble(uint32_t x) {
    x &= kHigh;
    return ((x >> 7) | (x >> 14) | (x >> 21) | (x >> 28)) & 0xFu;
}

}  // namespace lanes
