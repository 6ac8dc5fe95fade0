// FP32 relaxation of the layered decoder (sections 2 and 3) and its adjoint.
//
// The relaxation keeps the layered schedule, the sign rule (Eq. 1 with the
// syndrome sign) and the forward-backward fold of Eq. 7, but in floating
// point and without saturation.  Algorithm 1's table is the integer form of
// the box-plus beta of Eq. 6 at its own quantisation step D_t; an integer
// decoder fed LLRs at a finer step D computes the tempered box-plus
//     beta_k(x, y) = k * beta(x / k, y / k),   k = D / D_t,
// so the relaxation folds beta_k (k = 1: exact belief propagation).  Each
// check-to-variable magnitude is scaled and offset per iteration t and
// row-degree class c (the normalised/offset forms listed in section 2):
//     mag = alpha[t][c] * relu(fold - gamma[t][c]).
// The variable-node update is the plain Eq. 9; the loss is the mean binary
// cross entropy of the final soft values against Alice's bits.
//
// Work decomposition: a CTA holds FR frames, two threads per (frame, check
// row).  Soft values live in shared memory; the forward writes iteration-
// boundary checkpoints of E and L to global memory.  The adjoint walks the
// iterations backwards; for each it recomputes that iteration's forward from
// its checkpoint (storing only the per-edge L_ji it needs), then reverses
// the layers.  Nothing finer than an iteration is stored across the unroll.
#include <math.h>

#include "row_update.cuh"

namespace {

constexpr float kEmpty = 50.0f;  // empty box-plus of a degree-1 row

// beta_k(x, y) = min(x, y) + k * ln((1 + e^{-(x+y)/k}) / (1 + e^{-|x-y|/k})) for
// x, y >= 0: the ratio lies in [1/2, 1], so the single logarithm of it has a
// small absolute error, and the hardware exponential, logarithm and division
// (__expf, __logf, __fdividef) replace the two log1p/exp library sequences.
// The result is symmetric in x and y bit for bit.
__device__ __forceinline__ float bplus(float x, float y, float kap, float ikap) {
    const float a = __expf(-(x + y) * ikap), b = __expf(-fabsf(x - y) * ikap);
    return fminf(x, y) + kap * __logf(__fdividef(1.0f + a, 1.0f + b));
}

__device__ __forceinline__ float sigm(float z) { return __fdividef(1.0f, 1.0f + __expf(-z)); }

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// d beta_k / dx = s((x+y)/k) - s((x-y)/k), and symmetrically for y.
__device__ __forceinline__ void bplus_grad(float x, float y, float ikap, float& dx, float& dy) {
    const float sp = sigm((x + y) * ikap);
    dx = sp - sigm((x - y) * ikap);
    dy = sp - sigm((y - x) * ikap);
}

struct RelaxArgs {
    const int32_t* tab;
    int Mb, nblk, Z, n, m;
    int64_t edges;
    const float* llr;
    const uint8_t* syn;
    const uint8_t* bits;
    int batch, iters;
    const float* alpha;
    const float* gamma;
    const int32_t* cls;
    int ncls;
    float kappa;
    float* ckE;  // [iters+1][batch][n]
    float* ckL;  // [iters][batch][edges]; slot 0 unused (L starts at 0)
    float* loss;
    float* V;    // [batch][edges] L_ji of the iteration being reversed
    float* gL;   // [batch][edges] adjoint of the stored messages
    float* g_alpha;
    float* g_gamma;
    float* g_llr;
};

__device__ __forceinline__ float syn_sign(const RelaxArgs& A, int64_t f, int c) {
    const int mbytes = (A.m + 7) / 8;
    return ((A.syn[f * mbytes + (c >> 3)] >> (c & 7)) & 1) ? -1.0f : 1.0f;
}

// Two threads share a check row, as in the integer decoder: half 0 walks the
// row's edges upward from the first, half 1 downward from the last.  Each
// folds beta over its own walk (beta is symmetric, so half 1's fold is the
// right fold B of the forward-backward scheme), the halves swap their fold
// totals and sign products with one shuffle each, and each walks back,
// extending the partner's total through its own edges, to form every
//     m_k = beta(F_{k-1}, B_{k+1})            (Eq. 7, forward-backward).
// beta is bitwise symmetric in FP32 (min, x + y and |x - y| do not depend on
// the order of the operands), so every value equals the one a single thread
// folding the whole row computes.  A half that walks no edge sends the
// empty box-plus, which is what the one edge of a degree-1 row receives.
//
// Per-thread state: own fold O[j] after slot j, and (adjoint) the partner
// chain beyond slot j, X[j] = B_{k+1} or F_{k-1} for the slot's edge k.
struct RowHalf {
    int cnt, k0, kdir;
};

__device__ __forceinline__ RowHalf row_half(int d, int half) {
    const int h = (d + 1) >> 1;
    return RowHalf{half ? d - h : h, half ? d - 1 : 0, half ? -1 : 1};
}

// Forward of one check row; Lold == nullptr means the messages are 0.
// `d` is 0 for a thread without a row (it still joins the shuffles).
template <int HMAX>
__device__ __forceinline__ void row_forward(float* E, const float* Lold, float* Lnew, float* Vout, const int2* et,
                                            int d, int half, int r, int Z, float S, float al, float ga, float kap,
                                            float ikap) {
    const RowHalf H = row_half(d, half);
    // Slots guarded in chunks (as in the integer row update): a chunk wholly
    // past the walk's count is one branch (backward 7 %, forward 2 % faster on
    // the n = 4096 code, rows of up to 18 edges).
    constexpr int CH = HMAX <= 8 ? HMAX : 4;
    float v[HMAX], O[HMAX];
    int idx[HMAX];
    float sgn = 1.0f;
#pragma unroll
    for (int c0 = 0; c0 < HMAX; c0 += CH) {
        if (c0 < H.cnt) {
#pragma unroll
            for (int j = c0; j < (c0 + CH < HMAX ? c0 + CH : HMAX); ++j) {
                if (j < H.cnt) {
                    const int k = H.k0 + j * H.kdir;
                    const int2 t = et[k];
                    idx[j] = t.x + ldpc_dev::wrap(r + t.y, Z);
                    v[j] = E[idx[j]] - (Lold ? Lold[k * Z] : 0.0f);  // Eq. 8
                    if (v[j] < 0.0f) sgn = -sgn;                              // Eq. 1
                    if (Vout) Vout[k * Z] = v[j];
                }
            }
        }
    }
    float tot = kEmpty;
#pragma unroll
    for (int c0 = 0; c0 < HMAX; c0 += CH) {
        if (c0 < H.cnt) {
#pragma unroll
            for (int j = c0; j < (c0 + CH < HMAX ? c0 + CH : HMAX); ++j) {
                if (j < H.cnt) {
                    const float a = fabsf(v[j]);
                    tot = (j == 0) ? a : bplus(tot, a, kap, ikap);
                    O[j] = tot;
                }
            }
        }
    }
    float X = __shfl_xor_sync(0xffffffffu, tot, 1);
    S *= sgn * __shfl_xor_sync(0xffffffffu, sgn, 1);
#pragma unroll
    for (int c0 = ((HMAX - 1) / CH) * CH; c0 >= 0; c0 -= CH) {
        if (c0 < H.cnt) {
#pragma unroll
            for (int j = (c0 + CH < HMAX ? c0 + CH : HMAX) - 1; j >= c0; --j) {
                if (j < H.cnt) {
                    const int k = H.k0 + j * H.kdir;
                    const float B = (j == 0) ? X : bplus(O[j >= 1 ? j - 1 : 0], X, kap, ikap);
                    if (j > 0) X = bplus(fabsf(v[j]), X, kap, ikap);
                    const float mag = al * fmaxf(B - ga, 0.0f);
                    const float Ln = (v[j] < 0.0f ? -S : S) * mag;  // own sign removed
                    E[idx[j]] = v[j] + Ln;                          // Eq. 9
                    if (Lnew) Lnew[k * Z] = Ln;
                }
            }
        }
    }
}

// Adjoint of one check row.  G holds the adjoint of E after the layer and
// receives the adjoint before it; gLrow holds the adjoint of the new messages
// and receives the adjoint of the old ones.
template <int HMAX>
__device__ __forceinline__ void row_backward(float* G, const float* Vrow, float* gLrow, const int2* et, int d,
                                             int dtrue, int half, int r, int Z, float S, float al, float ga,
                                             float kap, float ikap, float& acc_a, float& acc_g) {
    const RowHalf H = row_half(d, half);
    constexpr int CH = HMAX <= 8 ? HMAX : 4;  // slots per guarded chunk
    float a[HMAX], O[HMAX], X[HMAX], gO[HMAX], gA[HMAX];
    uint32_t neg = 0;  // bit j: v_j < 0
    float sgn = 1.0f;
#pragma unroll
    for (int c0 = 0; c0 < HMAX; c0 += CH) {
        if (c0 < H.cnt) {
#pragma unroll
            for (int j = c0; j < (c0 + CH < HMAX ? c0 + CH : HMAX); ++j) {
                if (j < H.cnt) {
                    const float v = Vrow[(size_t)(H.k0 + j * H.kdir) * Z];
                    // the message adjoint this slot reads in the ascending pass, fetched into L1 now
                    asm volatile("prefetch.global.L1 [%0];" ::"l"(gLrow + (size_t)(H.k0 + j * H.kdir) * Z));
                    a[j] = fabsf(v);
                    if (v < 0.0f) {
                        neg |= 1u << j;
                        sgn = -sgn;
                    }
                    gO[j] = gA[j] = 0.0f;
                }
            }
        }
    }
    float tot = kEmpty;
#pragma unroll
    for (int c0 = 0; c0 < HMAX; c0 += CH) {
        if (c0 < H.cnt) {
#pragma unroll
            for (int j = c0; j < (c0 + CH < HMAX ? c0 + CH : HMAX); ++j) {
                if (j < H.cnt) {
                    tot = (j == 0) ? a[j] : bplus(tot, a[j], kap, ikap);
                    O[j] = tot;
                }
            }
        }
    }
    float x = __shfl_xor_sync(0xffffffffu, tot, 1);
    S *= sgn * __shfl_xor_sync(0xffffffffu, sgn, 1);
#pragma unroll
    for (int c0 = ((HMAX - 1) / CH) * CH; c0 >= 0; c0 -= CH) {  // partner chain beyond every slot
        if (c0 < H.cnt) {
#pragma unroll
            for (int j = (c0 + CH < HMAX ? c0 + CH : HMAX) - 1; j >= c0; --j) {
                if (j < H.cnt) {
                    X[j] = x;
                    if (j > 0) x = bplus(a[j], x, kap, ikap);
                }
            }
        }
    }
    // Ascending: the magnitude m_j = beta(O_{j-1}, X_j) of every slot and its
    // adjoint, and with it the adjoint of the partner chain X_{j-1} =
    // beta(a_j, X_j), carried as one running value g (the adjoint of X_j);
    // what reaches the far end belongs to the partner's fold total.
    float g = 0.0f;
#pragma unroll
    for (int c0 = 0; c0 < HMAX; c0 += CH) {
        if (c0 < H.cnt) {
#pragma unroll
            for (int j = c0; j < (c0 + CH < HMAX ? c0 + CH : HMAX); ++j) {
                if (j < H.cnt) {
                    const int k = H.k0 + j * H.kdir;
                    const int2 t = et[k];
                    const float B = (j == 0) ? X[0] : bplus(O[j >= 1 ? j - 1 : 0], X[j], kap, ikap);
                    const float sj = ((neg >> j) & 1u) ? -S : S;
                    const float gtot = gLrow[(size_t)k * Z] + G[t.x + ldpc_dev::wrap(r + t.y, Z)];  // L_new feeds E and the next iteration
                    const float gmag = gtot * sj;
                    const bool pos = B > ga;
                    acc_a += gmag * fmaxf(B - ga, 0.0f);
                    acc_g -= pos ? gmag * al : 0.0f;
                    const float gm = (pos && dtrue > 1) ? gmag * al : 0.0f;
                    if (j == 0) {
                        g = gm;
                    } else {
                        float dx, dy, cx, cy;
                        bplus_grad(O[j >= 1 ? j - 1 : 0], X[j], ikap, dx, dy);
                        gO[j >= 1 ? j - 1 : 0] += gm * dx;
                        bplus_grad(a[j], X[j], ikap, cx, cy);
                        gA[j] += g * cx;
                        g = gm * dy + g * cy;
                    }
                }
            }
        }
    }
    // Descending: the own fold O_j = beta(O_{j-1}, a_j), starting from the
    // adjoint of the total that the partner's chain sends back; each slot's
    // adjoint is complete once its step is done, so it is written out there.
    float go = __shfl_xor_sync(0xffffffffu, g, 1);
#pragma unroll
    for (int c0 = ((HMAX - 1) / CH) * CH; c0 >= 0; c0 -= CH) {
        if (c0 < H.cnt) {
#pragma unroll
            for (int j = (c0 + CH < HMAX ? c0 + CH : HMAX) - 1; j >= c0; --j) {
                if (j < H.cnt) {
                    go += gO[j];
                    float ga_j = gA[j];
                    if (j > 0) {
                        float dx, dy;
                        bplus_grad(O[j >= 1 ? j - 1 : 0], a[j], ikap, dx, dy);
                        ga_j += go * dy;
                        go *= dx;
                    } else {
                        ga_j += go;
                    }
                    const int k = H.k0 + j * H.kdir;
                    const int2 t = et[k];
                    const int vi = t.x + ldpc_dev::wrap(r + t.y, Z);
                    const float gv = G[vi] + ga_j * (((neg >> j) & 1u) ? -1.0f : 1.0f);  // d|v|/dv = sign(v)
                    G[vi] = gv;                                                         // adjoint of E before the layer
                    gLrow[(size_t)k * Z] = -gv;                                         // adjoint of the old message (Eq. 8)
                }
            }
        }
    }
}

// CTA shape: FR frames, two threads per check row; RT rows of a frame per
// pass (RT = Z unless 2 Z FR exceeds the block, then passes over the rows).
struct Shape {
    int FR, RT, T;
};

__host__ __device__ inline Shape cta_shape(int Z) {
    int fr = 512 / (2 * Z);
    fr = fr < 1 ? 1 : (fr > 4 ? 4 : fr);
    const int rt = 2 * Z * fr <= 512 ? Z : 256;
    const int t = ((2 * rt * fr + 31) / 32) * 32;
    return Shape{fr, rt, t};
}

template <int HMAX>
__global__ void __launch_bounds__(512, 2) relaxed_forward_kernel(RelaxArgs A) {
    extern __shared__ __align__(16) float fsm[];
    const int Z = A.Z, n = A.n;
    const Shape sh = cta_shape(Z);
    const int FR = sh.FR, RT = sh.RT, T = blockDim.x;
    const int tid = threadIdx.x, half = tid & 1, q = tid >> 1;
    const int flq = q / RT, rr = q - flq * RT;
    const int fl = flq < FR ? flq : 0;
    float* E_s = fsm;
    int32_t* s_tab = reinterpret_cast<int32_t*>(fsm + (((size_t)FR * n + 3) & ~(size_t)3));  // 16-byte aligned (int2 entries)
    const ldpc_dev::Tables TB = ldpc_dev::load_tables(s_tab, A.tab, A.Mb, A.nblk, Z, 1, tid, T);
    const int64_t fbase = (int64_t)blockIdx.x * FR;
    const int64_t f = fbase + fl;
    const bool valid = flq < FR && f < A.batch;
    for (int i = tid; i < FR * n; i += T) {
        const int64_t ff = fbase + i / n;
        if (ff < A.batch) E_s[i] = A.llr[ff * n + i % n];
    }
    __syncthreads();
    float* E = E_s + (size_t)fl * n;
    const float kap = A.kappa, ikap = 1.0f / A.kappa;
    for (int t = 0; t < A.iters; ++t) {
        for (int i = tid; i < FR * n; i += T) {
            const int64_t ff = fbase + i / n;
            if (ff < A.batch) A.ckE[((int64_t)t * A.batch + ff) * n + i % n] = E_s[i];
        }
        const float* Lold = t > 0 ? A.ckL + ((int64_t)t * A.batch + f) * A.edges : nullptr;
        float* Lnew = t + 1 < A.iters ? A.ckL + ((int64_t)(t + 1) * A.batch + f) * A.edges : nullptr;
        for (int i = 0; i < A.Mb; ++i) {
            const int d = TB.deg[i], b0 = TB.off[i];
            if (d > 0) {
                const int c = A.cls[i];
                for (int r0 = 0; r0 < Z; r0 += RT) {
                    const int r = r0 + rr;
                    const bool ok = valid && r < Z;
                    const int rs = ok ? r : 0;
                    const size_t e0 = (size_t)b0 * Z + rs;
                    row_forward<HMAX>(E, Lold ? Lold + e0 : nullptr, Lnew ? Lnew + e0 : nullptr, nullptr,
                                      TB.et + b0, ok ? d : 0, half, rs, Z, ok ? syn_sign(A, f, i * Z + rs) : 1.0f,
                                      A.alpha[t * A.ncls + c], A.gamma[t * A.ncls + c], kap, ikap);
                }
            }
            __syncthreads();
        }
    }
    const int nbytes = (n + 7) / 8;
    float part = 0.0f;
    for (int i = tid; i < FR * n; i += T) {
        const int64_t ff = fbase + i / n;
        if (ff >= A.batch) continue;
        const int j = i % n;
        const float e = E_s[i];
        A.ckE[((int64_t)A.iters * A.batch + ff) * n + j] = e;
        if (A.bits && A.loss) {
            const float sgn = ((A.bits[ff * nbytes + (j >> 3)] >> (j & 7)) & 1) ? -1.0f : 1.0f;
            const float z = -sgn * e;  // BCE with logit e for bit 0: softplus(-(1-2x) e)
            part += fmaxf(z, 0.0f) + log1pf(expf(-fabsf(z)));
        }
    }
    if (A.bits && A.loss) {
        part = warp_sum(part);
        if ((tid & 31) == 0) atomicAdd(A.loss, part / ((float)A.batch * (float)n));
    }
}

template <int HMAX>
__global__ void __launch_bounds__(512, 2) relaxed_backward_kernel(RelaxArgs A) {
    extern __shared__ __align__(16) float fsm[];
    const int Z = A.Z, n = A.n;
    const Shape sh = cta_shape(Z);
    const int FR = sh.FR, RT = sh.RT, T = blockDim.x;
    const int tid = threadIdx.x, half = tid & 1, q = tid >> 1;
    const int flq = q / RT, rr = q - flq * RT;
    const int fl = flq < FR ? flq : 0;
    float* E_s = fsm;
    float* G_s = fsm + (size_t)FR * n;
    float* s_acc = G_s + (size_t)FR * n;  // [2 * ncls]
    int32_t* s_tab = reinterpret_cast<int32_t*>(s_acc + 2 * A.ncls);
    const ldpc_dev::Tables TB = ldpc_dev::load_tables(s_tab, A.tab, A.Mb, A.nblk, Z, 1, tid, T);
    const int64_t fbase = (int64_t)blockIdx.x * FR;
    const int64_t f = fbase + fl;
    const bool valid = flq < FR && f < A.batch;
    float* G = G_s + (size_t)fl * n;
    float* E = E_s + (size_t)fl * n;
    const int nbytes = (n + 7) / 8;
    const float kap = A.kappa, ikap = 1.0f / A.kappa;
    const float inv = 1.0f / ((float)A.batch * (float)n);
    for (int i = tid; i < FR * n; i += T) {
        const int64_t ff = fbase + i / n;
        if (ff >= A.batch) continue;
        const int j = i % n;
        const float e = A.ckE[((int64_t)A.iters * A.batch + ff) * n + j];
        const float sgn = ((A.bits[ff * nbytes + (j >> 3)] >> (j & 7)) & 1) ? -1.0f : 1.0f;
        G_s[i] = -sgn * sigm(-sgn * e) * inv;  // d softplus(-sgn e) / de
    }
    for (int64_t i = tid; i < (int64_t)FR * A.edges; i += T) {  // the last messages feed nothing
        const int64_t ff = fbase + i / A.edges;
        if (ff < A.batch) A.gL[ff * A.edges + i % A.edges] = 0.0f;
    }
    for (int t = A.iters - 1; t >= 0; --t) {
        for (int i = tid; i < FR * n; i += T) {
            const int64_t ff = fbase + i / n;
            if (ff < A.batch) E_s[i] = A.ckE[((int64_t)t * A.batch + ff) * n + i % n];
        }
        for (int qq = tid; qq < 2 * A.ncls; qq += T) s_acc[qq] = 0.0f;
        __syncthreads();
        const float* Lold = t > 0 ? A.ckL + ((int64_t)t * A.batch + f) * A.edges : nullptr;
        float* Vf = A.V + f * A.edges;
        for (int i = 0; i < A.Mb; ++i) {  // recompute iteration t, keeping L_ji
            const int d = TB.deg[i], b0 = TB.off[i];
            if (d > 0) {
                const int c = A.cls[i];
                for (int r0 = 0; r0 < Z; r0 += RT) {
                    const int r = r0 + rr;
                    const bool ok = valid && r < Z;
                    const int rs = ok ? r : 0;
                    const size_t e0 = (size_t)b0 * Z + rs;
                    row_forward<HMAX>(E, Lold ? Lold + e0 : nullptr, nullptr, Vf + e0, TB.et + b0, ok ? d : 0, half,
                                      rs, Z, ok ? syn_sign(A, f, i * Z + rs) : 1.0f, A.alpha[t * A.ncls + c],
                                      A.gamma[t * A.ncls + c], kap, ikap);
                }
            }
            __syncthreads();
        }
        for (int i = A.Mb - 1; i >= 0; --i) {  // reverse the layers
            const int d = TB.deg[i], b0 = TB.off[i];
            if (d > 0) {
                const int c = A.cls[i];
                float acc_a = 0.0f, acc_g = 0.0f;
                for (int r0 = 0; r0 < Z; r0 += RT) {
                    const int r = r0 + rr;
                    const bool ok = valid && r < Z;
                    const int rs = ok ? r : 0;
                    const size_t e0 = (size_t)b0 * Z + rs;
                    row_backward<HMAX>(G, Vf + e0, A.gL + f * A.edges + e0, TB.et + b0, ok ? d : 0, d, half, rs, Z,
                                       ok ? syn_sign(A, f, i * Z + rs) : 1.0f, A.alpha[t * A.ncls + c],
                                       A.gamma[t * A.ncls + c], kap, ikap, acc_a, acc_g);
                }
                // every lane of a warp works on this layer, whose class is c:
                // sum over the warp first, one shared atomic per warp
                acc_a = warp_sum(acc_a);
                acc_g = warp_sum(acc_g);
                if ((tid & 31) == 0) {
                    atomicAdd(&s_acc[c], acc_a);
                    atomicAdd(&s_acc[A.ncls + c], acc_g);
                }
            }
            __syncthreads();
        }
        for (int qq = tid; qq < A.ncls; qq += T) {
            atomicAdd(&A.g_alpha[t * A.ncls + qq], s_acc[qq]);
            atomicAdd(&A.g_gamma[t * A.ncls + qq], s_acc[A.ncls + qq]);
        }
        __syncthreads();
    }
    if (A.g_llr)
        for (int i = tid; i < FR * n; i += T) {
            const int64_t ff = fbase + i / n;
            if (ff < A.batch) A.g_llr[ff * n + i % n] = G_s[i];
        }
}

size_t tab_bytes(const ldpc_code* c) {
    return sizeof(int32_t) * ((size_t)((2 * c->Mb + 1 + 1) & ~1) + 2 * (size_t)c->nblk);
}

// Unroll width of the relaxation's kernels: the smallest of 6, 9, 12 and 16
// slots that holds half the longest row (fewer idle slots and, in the
// adjoint's five per-slot arrays, fewer registers).
template <template <int> class K>
auto pick_width(int max_deg) {
    const int h = (max_deg + 1) / 2;
    return h <= 6 ? K<6>::fn : h <= 9 ? K<9>::fn : h <= 12 ? K<12>::fn : K<16>::fn;
}
template <int H>
struct ForwardK {
    static constexpr auto fn = relaxed_forward_kernel<H>;
};
template <int H>
struct BackwardK {
    static constexpr auto fn = relaxed_backward_kernel<H>;
};

int check_common(const ldpc_code* c, int batch, int iters, int ncls, float kappa) {
    using ldpc::fail;
    if (!c) return fail(LDPC_EINVAL, "relaxed decoder: NULL code");
    if (batch < 0 || iters < 1 || ncls < 1 || !(kappa > 0.0f))
        return fail(LDPC_EINVAL, "relaxed decoder: bad batch, iterations, classes or kappa");
    if (c->Z > 512) return fail(LDPC_EUNSUPPORTED, "relaxed decoder: lifting size above 512");
    if (c->max_deg > 32) return fail(LDPC_EUNSUPPORTED, "relaxed decoder: row degree above 32");
    return LDPC_OK;
}

}  // namespace

extern "C" {

int ldpc_relaxed_forward(const ldpc_code* code, const float* llr, const uint8_t* syn, const uint8_t* bits, int batch,
                         int iters, const float* alpha, const float* gamma, const int32_t* layer_class,
                         int n_classes, float kappa, float* ckE, float* ckL, float* loss, void* stream) {
    using ldpc::fail;
    const ldpc_code* c = code;
    int rc = check_common(c, batch, iters, n_classes, kappa);
    if (rc) return rc;
    if (batch == 0) return LDPC_OK;
    if (!llr || !syn || !alpha || !gamma || !layer_class || !ckE || (!ckL && iters > 1))
        return fail(LDPC_EINVAL, "relaxed forward: NULL buffer");
    if (loss && !bits) return fail(LDPC_EINVAL, "relaxed forward: the loss needs Alice's bits");
    cudaStream_t st = (cudaStream_t)stream;
    if (loss) LDPC_CUDA_TRY(cudaMemsetAsync(loss, 0, sizeof(float), st));
    const Shape sh = cta_shape(c->Z);
    const int FR = sh.FR;
    const size_t smem = sizeof(float) * (((size_t)FR * c->n + 3) & ~(size_t)3) + tab_bytes(c);
    if ((int64_t)smem > ldpc::max_dyn_smem(c->device)) return fail(LDPC_EUNSUPPORTED, "relaxed forward: shared memory");
    RelaxArgs A{c->d_tab, c->Mb, c->nblk, c->Z, c->n, c->m, c->edges, llr, syn, bits, batch, iters, alpha, gamma,
                layer_class, n_classes, kappa, ckE, ckL, loss, nullptr, nullptr, nullptr, nullptr, nullptr};
    const int grid = (batch + FR - 1) / FR;
    auto kern = pick_width<ForwardK>(c->max_deg);
    LDPC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, sh.T, smem, st>>>(A);
    ldpc::count_launch();
    LDPC_CUDA_TRY(cudaGetLastError());
    return LDPC_OK;
}

int ldpc_relaxed_backward(const ldpc_code* code, const uint8_t* syn, const uint8_t* bits, int batch, int iters,
                          const float* alpha, const float* gamma, const int32_t* layer_class, int n_classes,
                          float kappa, const float* ckE, const float* ckL, float* V, float* gL, float* grad_alpha,
                          float* grad_gamma, float* grad_llr, void* stream) {
    using ldpc::fail;
    const ldpc_code* c = code;
    int rc = check_common(c, batch, iters, n_classes, kappa);
    if (rc) return rc;
    if (!grad_alpha || !grad_gamma) return fail(LDPC_EINVAL, "relaxed backward: NULL gradient buffer");
    cudaStream_t st = (cudaStream_t)stream;
    LDPC_CUDA_TRY(cudaMemsetAsync(grad_alpha, 0, sizeof(float) * (size_t)iters * n_classes, st));
    LDPC_CUDA_TRY(cudaMemsetAsync(grad_gamma, 0, sizeof(float) * (size_t)iters * n_classes, st));
    if (batch == 0) return LDPC_OK;
    if (!syn || !bits || !alpha || !gamma || !layer_class || !ckE || (!ckL && iters > 1) || !V || !gL)
        return fail(LDPC_EINVAL, "relaxed backward: NULL buffer");
    const Shape sh = cta_shape(c->Z);
    const int FR = sh.FR;
    const size_t smem = sizeof(float) * (2 * (size_t)FR * c->n + 2 * (size_t)n_classes) + tab_bytes(c);
    if ((int64_t)smem > ldpc::max_dyn_smem(c->device))
        return fail(LDPC_EUNSUPPORTED, "relaxed backward: shared memory");
    RelaxArgs A{c->d_tab, c->Mb, c->nblk, c->Z, c->n, c->m, c->edges, nullptr, syn, bits, batch, iters, alpha,
                gamma, layer_class, n_classes, kappa, const_cast<float*>(ckE), const_cast<float*>(ckL), nullptr,
                V, gL, grad_alpha, grad_gamma, grad_llr};
    const int grid = (batch + FR - 1) / FR;
    auto kern = pick_width<BackwardK>(c->max_deg);
    LDPC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, sh.T, smem, st>>>(A);
    ldpc::count_launch();
    LDPC_CUDA_TRY(cudaGetLastError());
    return LDPC_OK;
}

}  // extern "C"
