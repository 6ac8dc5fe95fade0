// Unroll widths of the integer decoders.
//
// Two threads share a check row and each walks at most ceil(d/2) of its
// edges; the row update keeps that many slots in registers and is unrolled
// for a compile-time bound MAXH >= ceil(max_deg / 2) of the code.  Every slot
// past a layer's degree still costs guard branches and part of its index
// arithmetic, so the bound should be tight: a code gets the smallest width in
// this list that holds its longest row.  Each width is compiled in its own
// translation unit (the build generates one per entry, instantiating the
// batch and the persistent launchers), so the list can be fine-grained
// without serialising the build.
#pragma once

// X(width) for every compiled width, ascending.
#define LDPC_MAXH_LIST(X) X(4) X(6) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(16) X(24) X(32)

namespace ldpc_dec {

// Smallest compiled width holding ceil(max_deg / 2) slots, or 0 if the row
// degree exceeds the largest width's 2 * 32 = 64 edges.
inline int pick_maxh(int max_deg) {
    const int need = (max_deg + 1) / 2;
#define LDPC_MAXH_PICK(M) \
    if (need <= (M)) return (M);
    LDPC_MAXH_LIST(LDPC_MAXH_PICK)
#undef LDPC_MAXH_PICK
    return 0;
}

// Threads per CTA bound of a width: up to 16 slots the row update fits in 64
// registers, so a CTA may have 1024 threads; wider rows take 512.
template <int MAXH>
constexpr int max_threads() {
    return MAXH <= 16 ? 1024 : 512;
}

}  // namespace ldpc_dec
