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
// Work decomposition: a CTA holds FR frames, one thread per (frame, check
// row).  Soft values live in shared memory; the forward writes iteration-
// boundary checkpoints of E and L to global memory.  The adjoint walks the
// iterations backwards; for each it recomputes that iteration's forward from
// its checkpoint (storing only the per-edge L_ji it needs), then reverses
// the layers.  Nothing finer than an iteration is stored across the unroll.
#include <math.h>

#include "row_update.cuh"

namespace {

constexpr float kEmpty = 50.0f;  // empty box-plus of a degree-1 row

__device__ __forceinline__ float bplus(float x, float y, float kap, float ikap) {
    return fminf(x, y) + kap * (log1pf(expf(-(x + y) * ikap)) - log1pf(expf(-fabsf(x - y) * ikap)));
}

__device__ __forceinline__ float sigm(float z) { return 1.0f / (1.0f + expf(-z)); }

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

// Forward of one check row; Lold == nullptr means the messages are 0.
template <int DMAX>
__device__ __forceinline__ void row_forward(float* E, const float* Lold, float* Lnew, float* Vout, const int2* et,
                                            int d, int r, int Z, float S, float al, float ga, float kap,
                                            float ikap) {
    float v[DMAX], a[DMAX], F[DMAX];
    int idx[DMAX];
#pragma unroll(DMAX)
    for (int k = 0; k < DMAX; ++k) {
        if (k < d) {
            const int2 t = et[k];
            idx[k] = t.x + ldpc_dev::wrap(r + t.y, Z);
            v[k] = E[idx[k]] - (Lold ? Lold[(size_t)k * Z] : 0.0f);  // Eq. 8
            a[k] = fabsf(v[k]);
            if (v[k] < 0.0f) S = -S;                                  // Eq. 1
            if (Vout) Vout[(size_t)k * Z] = v[k];
        }
    }
    F[0] = a[0];
#pragma unroll(DMAX)
    for (int k = 1; k < DMAX - 1; ++k)
        if (k <= d - 2) F[k] = bplus(F[k - 1], a[k], kap, ikap);
    float R = 0.0f;
#pragma unroll(DMAX)
    for (int kk = 0; kk < DMAX; ++kk) {
        const int k = DMAX - 1 - kk;
        if (k < d) {
            float B;
            if (d == 1) B = kEmpty;
            else if (k == d - 1) B = F[k >= 1 ? k - 1 : 0];
            else if (k == 0) B = R;
            else B = bplus(F[k >= 1 ? k - 1 : 0], R, kap, ikap);
            if (k == d - 1) R = a[k];
            else if (k > 0) R = bplus(a[k], R, kap, ikap);
            const float mag = al * fmaxf(B - ga, 0.0f);
            const float Ln = (v[k] < 0.0f ? -S : S) * mag;  // own sign removed
            E[idx[k]] = v[k] + Ln;                          // Eq. 9
            if (Lnew) Lnew[(size_t)k * Z] = Ln;
        }
    }
}

// Adjoint of one check row.  G holds the adjoint of E after the layer and
// receives the adjoint before it; gLrow holds the adjoint of the new messages
// and receives the adjoint of the old ones.
template <int DMAX>
__device__ __forceinline__ void row_backward(float* G, const float* Vrow, float* gLrow, const int2* et, int d,
                                             int r, int Z, float S, float al, float ga, float kap, float ikap,
                                             float& acc_a, float& acc_g) {
    float a[DMAX], sg[DMAX], F[DMAX], Rr[DMAX], gF[DMAX], gR[DMAX], gA[DMAX], gE[DMAX], gB[DMAX];
    int idx[DMAX];
#pragma unroll(DMAX)
    for (int k = 0; k < DMAX; ++k) {
        if (k < d) {
            const int2 t = et[k];
            idx[k] = t.x + ldpc_dev::wrap(r + t.y, Z);
            const float v = Vrow[(size_t)k * Z];
            a[k] = fabsf(v);
            sg[k] = v < 0.0f ? -1.0f : 1.0f;
            S *= sg[k];
            gF[k] = gR[k] = gA[k] = 0.0f;
        }
    }
    F[0] = a[0];
#pragma unroll(DMAX)
    for (int k = 1; k < DMAX - 1; ++k)
        if (k <= d - 2) F[k] = bplus(F[k - 1], a[k], kap, ikap);
#pragma unroll(DMAX)
    for (int kk = 0; kk < DMAX; ++kk) {
        const int k = DMAX - 1 - kk;
        if (k < d) {
            if (k == d - 1) Rr[k] = a[k];
            else if (k >= 1) Rr[k] = bplus(a[k], Rr[k + 1 < DMAX ? k + 1 : 0], kap, ikap);
        }
    }
    // magnitudes and their adjoints
#pragma unroll(DMAX)
    for (int k = 0; k < DMAX; ++k) {
        if (k < d) {
            float B;
            if (d == 1) B = kEmpty;
            else if (k == 0) B = Rr[1 < DMAX ? 1 : 0];
            else if (k == d - 1) B = F[k - 1 >= 0 ? k - 1 : 0];
            else B = bplus(F[k - 1 >= 0 ? k - 1 : 0], Rr[k + 1 < DMAX ? k + 1 : 0], kap, ikap);
            gE[k] = G[idx[k]];
            const float gtot = gLrow[(size_t)k * Z] + gE[k];  // L_new feeds E (Eq. 9) and the next iteration
            const float gmag = gtot * S * sg[k];
            const bool pos = B > ga;
            acc_a += gmag * fmaxf(B - ga, 0.0f);
            acc_g -= pos ? gmag * al : 0.0f;
            gB[k] = (pos && d > 1) ? gmag * al : 0.0f;
        }
    }
    // through m_k = beta(F_{k-1}, B_{k+1})
#pragma unroll(DMAX)
    for (int k = 0; k < DMAX; ++k) {
        if (k < d && d > 1) {
            if (k == 0) gR[1 < DMAX ? 1 : 0] += gB[k];
            else if (k == d - 1) gF[k - 1 >= 0 ? k - 1 : 0] += gB[k];
            else {
                float dx, dy;
                bplus_grad(F[k - 1 >= 0 ? k - 1 : 0], Rr[k + 1 < DMAX ? k + 1 : 0], ikap, dx, dy);
                gF[k - 1 >= 0 ? k - 1 : 0] += gB[k] * dx;
                gR[k + 1 < DMAX ? k + 1 : 0] += gB[k] * dy;
            }
        }
    }
    // right chain R_k = beta(a_k, R_{k+1}), k = 1 .. d-2, then R_{d-1} = a_{d-1}
#pragma unroll(DMAX)
    for (int k = 1; k < DMAX; ++k) {
        if (k < d) {
            if (k <= d - 2) {
                float dx, dy;
                bplus_grad(a[k], Rr[k + 1 < DMAX ? k + 1 : 0], ikap, dx, dy);
                gA[k] += gR[k] * dx;
                gR[k + 1 < DMAX ? k + 1 : 0] += gR[k] * dy;
            } else if (k == d - 1) {
                gA[k] += gR[k];
            }
        }
    }
    // left chain F_k = beta(F_{k-1}, a_k), k = d-2 .. 1, then F_0 = a_0
#pragma unroll(DMAX)
    for (int kk = 0; kk < DMAX; ++kk) {
        const int k = DMAX - 1 - kk;
        if (k >= 1 && k <= d - 2) {
            float dx, dy;
            bplus_grad(F[k - 1 >= 0 ? k - 1 : 0], a[k], ikap, dx, dy);
            gF[k - 1 >= 0 ? k - 1 : 0] += gF[k] * dx;
            gA[k] += gF[k] * dy;
        }
    }
    if (d > 1) gA[0] += gF[0];
#pragma unroll(DMAX)
    for (int k = 0; k < DMAX; ++k) {
        if (k < d) {
            const float gv = gE[k] + gA[k] * sg[k];  // d|v|/dv = sign(v)
            G[idx[k]] = gv;                           // adjoint of E before the layer
            gLrow[(size_t)k * Z] = -gv;               // adjoint of the old message (Eq. 8)
        }
    }
}

template <int DMAX>
__global__ void __launch_bounds__(512) relaxed_forward_kernel(RelaxArgs A) {
    extern __shared__ __align__(16) float fsm[];
    const int Z = A.Z, n = A.n, T = blockDim.x, FR = T / Z;
    const int tid = threadIdx.x, fl = tid / Z, r = tid - fl * Z;
    float* E_s = fsm;
    int32_t* s_tab = reinterpret_cast<int32_t*>(fsm + (size_t)FR * n);
    const ldpc_dev::Tables TB = ldpc_dev::load_tables(s_tab, A.tab, A.Mb, A.nblk, Z, 1, tid, T);
    const int64_t f = (int64_t)blockIdx.x * FR + fl;
    const bool valid = f < A.batch;
    float* E = E_s + (size_t)fl * n;
    if (valid)
        for (int j = r; j < n; j += Z) E[j] = A.llr[f * n + j];
    __syncthreads();
    const float kap = A.kappa, ikap = 1.0f / A.kappa;
    for (int t = 0; t < A.iters; ++t) {
        if (valid)
            for (int j = r; j < n; j += Z) A.ckE[((int64_t)t * A.batch + f) * n + j] = E[j];
        const float* Lold = t > 0 ? A.ckL + ((int64_t)t * A.batch + f) * A.edges : nullptr;
        float* Lnew = t + 1 < A.iters ? A.ckL + ((int64_t)(t + 1) * A.batch + f) * A.edges : nullptr;
        for (int i = 0; i < A.Mb; ++i) {
            const int d = TB.deg[i], b0 = TB.off[i];
            if (valid && d > 0) {
                const int c = A.cls[i];
                const size_t e0 = (size_t)b0 * Z + r;
                row_forward<DMAX>(E, Lold ? Lold + e0 : nullptr, Lnew ? Lnew + e0 : nullptr, nullptr, TB.et + b0, d,
                                  r, Z, syn_sign(A, f, i * Z + r), A.alpha[t * A.ncls + c], A.gamma[t * A.ncls + c],
                                  kap, ikap);
            }
            __syncthreads();
        }
    }
    if (valid) {
        const int nbytes = (n + 7) / 8;
        float part = 0.0f;
        for (int j = r; j < n; j += Z) {
            const float e = E[j];
            A.ckE[((int64_t)A.iters * A.batch + f) * n + j] = e;
            if (A.bits && A.loss) {
                const float sgn = ((A.bits[f * nbytes + (j >> 3)] >> (j & 7)) & 1) ? -1.0f : 1.0f;
                const float z = -sgn * e;  // BCE with logit e for bit 0: softplus(-(1-2x) e)
                part += fmaxf(z, 0.0f) + log1pf(expf(-fabsf(z)));
            }
        }
        if (A.bits && A.loss) atomicAdd(A.loss, part / ((float)A.batch * (float)n));
    }
}

template <int DMAX>
__global__ void __launch_bounds__(512) relaxed_backward_kernel(RelaxArgs A) {
    extern __shared__ __align__(16) float fsm[];
    const int Z = A.Z, n = A.n, T = blockDim.x, FR = T / Z;
    const int tid = threadIdx.x, fl = tid / Z, r = tid - fl * Z;
    float* E_s = fsm;
    float* G_s = fsm + (size_t)FR * n;
    float* s_acc = G_s + (size_t)FR * n;  // [2 * ncls]
    int32_t* s_tab = reinterpret_cast<int32_t*>(s_acc + 2 * A.ncls);
    const ldpc_dev::Tables TB = ldpc_dev::load_tables(s_tab, A.tab, A.Mb, A.nblk, Z, 1, tid, T);
    const int64_t f = (int64_t)blockIdx.x * FR + fl;
    const bool valid = f < A.batch;
    float* E = E_s + (size_t)fl * n;
    float* G = G_s + (size_t)fl * n;
    const int nbytes = (n + 7) / 8;
    const float kap = A.kappa, ikap = 1.0f / A.kappa;
    if (valid) {
        const float inv = 1.0f / ((float)A.batch * (float)n);
        for (int j = r; j < n; j += Z) {
            const float e = A.ckE[((int64_t)A.iters * A.batch + f) * n + j];
            const float sgn = ((A.bits[f * nbytes + (j >> 3)] >> (j & 7)) & 1) ? -1.0f : 1.0f;
            G[j] = -sgn * sigm(-sgn * e) * inv;  // d softplus(-sgn e) / de
        }
        float* gl = A.gL + f * A.edges;
        for (int64_t e = r; e < A.edges; e += Z) gl[e] = 0.0f;  // the last messages feed nothing
    }
    for (int t = A.iters - 1; t >= 0; --t) {
        if (valid)
            for (int j = r; j < n; j += Z) E[j] = A.ckE[((int64_t)t * A.batch + f) * n + j];
        for (int q = tid; q < 2 * A.ncls; q += T) s_acc[q] = 0.0f;
        __syncthreads();
        const float* Lold = t > 0 ? A.ckL + ((int64_t)t * A.batch + f) * A.edges : nullptr;
        float* Vf = A.V + f * A.edges;
        for (int i = 0; i < A.Mb; ++i) {  // recompute iteration t, keeping L_ji
            const int d = TB.deg[i], b0 = TB.off[i];
            if (valid && d > 0) {
                const int c = A.cls[i];
                const size_t e0 = (size_t)b0 * Z + r;
                row_forward<DMAX>(E, Lold ? Lold + e0 : nullptr, nullptr, Vf + e0, TB.et + b0, d, r, Z,
                                  syn_sign(A, f, i * Z + r), A.alpha[t * A.ncls + c], A.gamma[t * A.ncls + c], kap,
                                  ikap);
            }
            __syncthreads();
        }
        for (int i = A.Mb - 1; i >= 0; --i) {  // reverse the layers
            const int d = TB.deg[i], b0 = TB.off[i];
            if (valid && d > 0) {
                const int c = A.cls[i];
                const size_t e0 = (size_t)b0 * Z + r;
                float acc_a = 0.0f, acc_g = 0.0f;
                row_backward<DMAX>(G, Vf + e0, A.gL + f * A.edges + e0, TB.et + b0, d, r, Z,
                                   syn_sign(A, f, i * Z + r), A.alpha[t * A.ncls + c], A.gamma[t * A.ncls + c], kap,
                                   ikap, acc_a, acc_g);
                atomicAdd(&s_acc[c], acc_a);
                atomicAdd(&s_acc[A.ncls + c], acc_g);
            }
            __syncthreads();
        }
        for (int q = tid; q < A.ncls; q += T) {
            atomicAdd(&A.g_alpha[t * A.ncls + q], s_acc[q]);
            atomicAdd(&A.g_gamma[t * A.ncls + q], s_acc[A.ncls + q]);
        }
        __syncthreads();
    }
    if (valid && A.g_llr)
        for (int j = r; j < n; j += Z) A.g_llr[f * n + j] = G[j];
}

int frames_per_cta(int Z) {
    int fr = 512 / Z;
    return fr < 1 ? 1 : (fr > 4 ? 4 : fr);
}

size_t tab_bytes(const ldpc_code* c) {
    return sizeof(int32_t) * ((size_t)((2 * c->Mb + 1 + 1) & ~1) + 2 * (size_t)c->nblk);
}

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
    const int FR = frames_per_cta(c->Z);
    const size_t smem = sizeof(float) * (size_t)FR * c->n + tab_bytes(c);
    if ((int64_t)smem > ldpc::max_dyn_smem(c->device)) return fail(LDPC_EUNSUPPORTED, "relaxed forward: shared memory");
    RelaxArgs A{c->d_tab, c->Mb, c->nblk, c->Z, c->n, c->m, c->edges, llr, syn, bits, batch, iters, alpha, gamma,
                layer_class, n_classes, kappa, ckE, ckL, loss, nullptr, nullptr, nullptr, nullptr, nullptr};
    const int grid = (batch + FR - 1) / FR;
    auto kern = c->max_deg <= 24 ? relaxed_forward_kernel<24> : relaxed_forward_kernel<32>;
    LDPC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, c->Z * FR, smem, st>>>(A);
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
    const int FR = frames_per_cta(c->Z);
    const size_t smem = sizeof(float) * (2 * (size_t)FR * c->n + 2 * (size_t)n_classes) + tab_bytes(c);
    if ((int64_t)smem > ldpc::max_dyn_smem(c->device))
        return fail(LDPC_EUNSUPPORTED, "relaxed backward: shared memory");
    RelaxArgs A{c->d_tab, c->Mb, c->nblk, c->Z, c->n, c->m, c->edges, nullptr, syn, bits, batch, iters, alpha,
                gamma, layer_class, n_classes, kappa, const_cast<float*>(ckE), const_cast<float*>(ckL), nullptr,
                V, gL, grad_alpha, grad_gamma, grad_llr};
    const int grid = (batch + FR - 1) / FR;
    auto kern = c->max_deg <= 24 ? relaxed_backward_kernel<24> : relaxed_backward_kernel<32>;
    LDPC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, c->Z * FR, smem, st>>>(A);
    ldpc::count_launch();
    LDPC_CUDA_TRY(cudaGetLastError());
    return LDPC_OK;
}

}  // extern "C"
