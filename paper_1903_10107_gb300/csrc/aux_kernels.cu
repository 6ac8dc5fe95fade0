// Channel-LLR quantisation (section 3.1 with the rate adaptation of section
// 4.1), syndrome computation (section 4.1 protocol) and a table probe of the
// byte-lane check-node arithmetic.  The per-frame LLR magnitude is computed
// on the host (ldpc_llr_magnitudes, the host C library's log) and passed to
// the kernels as int8, so the device never evaluates a transcendental whose
// last-ulp rounding could differ from the host's at a half-integer.
#include <math.h>

#include "common.cuh"

namespace {

constexpr int kLlrThreads = 256;

// One thread per 8 positions of one frame (one byte of Bob's packed key).
__global__ void __launch_bounds__(kLlrThreads)
llr_kernel(const uint8_t* __restrict__ bob, const int8_t* __restrict__ llr_mag, const int32_t* __restrict__ rank,
           const int32_t* __restrict__ n_short, const int32_t* __restrict__ n_punct,
           const uint8_t* __restrict__ known, int n, int nbytes, int8_t* __restrict__ out) {
    const int f = blockIdx.y;
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbytes) return;
    int mag = llr_mag[f];
    mag = mag > 127 ? 127 : (mag < -127 ? -127 : mag);
    const int ns = n_short ? n_short[f] : 0;
    const int np = n_punct ? n_punct[f] : 0;
    const uint8_t y = bob[(size_t)f * nbytes + b];
    const uint8_t kn = (known && ns > 0) ? known[(size_t)f * nbytes + b] : 0;
    int8_t* o = out + (size_t)f * n + (size_t)b * 8;
    const int jmax = min(8, n - b * 8);
    uint8_t v[8];
#pragma unroll
    for (int q8 = 0; q8 < 8; q8++) {
        int x = ((y >> q8) & 1) ? -mag : mag;
        if (rank && q8 < jmax) {
            const int rk = rank[b * 8 + q8];
            if (rk < ns) x = ((kn >> q8) & 1) ? -127 : 127;
            else if (rk < ns + np) x = 0;
        }
        v[q8] = (uint8_t)(int8_t)x;
    }
    if (jmax == 8 && (n % 8) == 0) {
        uint2 w;
        w.x = v[0] | (v[1] << 8) | (v[2] << 16) | ((uint32_t)v[3] << 24);
        w.y = v[4] | (v[5] << 8) | (v[6] << 16) | ((uint32_t)v[7] << 24);
        *reinterpret_cast<uint2*>(o) = w;
    } else {
        for (int q8 = 0; q8 < jmax; q8++) o[q8] = (int8_t)v[q8];
    }
}

// One thread per syndrome byte (8 consecutive check rows) of one frame.
__global__ void syndrome_kernel(const int32_t* __restrict__ tab, int Mb, int nblk, int Z, int m, int nbytes_x,
                                int nbytes_s, const uint8_t* __restrict__ bits, uint8_t* __restrict__ syn) {
    extern __shared__ int32_t s_tab[];
    const int words = 2 * Mb + 1 + 2 * nblk;
    for (int i = threadIdx.x; i < words; i += blockDim.x) s_tab[i] = tab[i];
    __syncthreads();
    const int f = blockIdx.y;
    const int sb = blockIdx.x * blockDim.x + threadIdx.x;
    if (sb >= nbytes_s) return;
    const int32_t* deg = s_tab;
    const int32_t* off = s_tab + Mb;
    const int32_t* col = s_tab + 2 * Mb + 1;
    const int32_t* sh = col + nblk;
    const uint8_t* x = bits + (size_t)f * nbytes_x;
    uint32_t out = 0;
    for (int q = 0; q < 8; q++) {
        const int c = sb * 8 + q;
        if (c >= m) break;
        const int i = c / Z, r = c - i * Z;
        uint32_t par = 0;
        for (int k = 0; k < deg[i]; k++) {
            int rr = r + sh[off[i] + k];
            rr -= rr >= Z ? Z : 0;
            const int j = col[off[i] + k] * Z + rr;
            par ^= (x[j >> 3] >> (j & 7)) & 1u;
        }
        out |= par << q;
    }
    syn[(size_t)f * nbytes_s + sb] = (uint8_t)out;
}

__global__ void tau_table_kernel(uint8_t* out) {
    // thread t handles p = t, and q = 4u .. 4u+3 in the four byte lanes
    const int p = blockIdx.x;
    for (int u = threadIdx.x; u < 32; u += blockDim.x) {
        const uint32_t a = (uint32_t)p * lanes::kOnes;
        const uint32_t b = (uint32_t)(4 * u) | ((uint32_t)(4 * u + 1) << 8) | ((uint32_t)(4 * u + 2) << 16) |
                           ((uint32_t)(4 * u + 3) << 24);
        const uint32_t t = lanes::tau(a, b);
        for (int l = 0; l < 4; l++) out[p * 128 + 4 * u + l] = (uint8_t)(t >> (8 * l));
    }
}

}  // namespace

extern "C" {

int ldpc_llr_magnitudes(const double* qber, int batch, double scale, int8_t* mag_out) {
    using ldpc::fail;
    if (batch < 0) return fail(LDPC_EINVAL, "ldpc_llr_magnitudes: negative batch");
    if (batch == 0) return LDPC_OK;
    if (!qber || !mag_out) return fail(LDPC_EINVAL, "ldpc_llr_magnitudes: NULL buffer");
    if (!(scale > 0.0)) return fail(LDPC_EINVAL, "ldpc_llr_magnitudes: bad scale");
    for (int f = 0; f < batch; ++f) {
        const double q = qber[f];
        if (!(q > 0.0 && q < 0.5)) return fail(LDPC_EINVAL, "ldpc_llr_magnitudes: QBER outside (0, 0.5)");
        long r = lround(log((1.0 - q) / q) * scale);  // host libm, round half away from zero
        mag_out[f] = (int8_t)(r > 127 ? 127 : r);
    }
    return LDPC_OK;
}

int ldpc_llr_from_bsc(const ldpc_code* c, const uint8_t* bob_bits, const int8_t* llr_mag, const int32_t* rank,
                      const int32_t* n_short, const int32_t* n_punct, const uint8_t* known, int batch,
                      int8_t* llr_out, void* stream) {
    using ldpc::fail;
    if (!c) return fail(LDPC_EINVAL, "ldpc_llr_from_bsc: NULL code");
    if (batch < 0) return fail(LDPC_EINVAL, "ldpc_llr_from_bsc: negative batch");
    if (batch == 0) return LDPC_OK;
    if (!bob_bits || !llr_mag || !llr_out) return fail(LDPC_EINVAL, "ldpc_llr_from_bsc: NULL buffer");
    if (n_short && !known) return fail(LDPC_EINVAL, "ldpc_llr_from_bsc: shortening needs known values");
    if ((n_short || n_punct) && !rank) return fail(LDPC_EINVAL, "ldpc_llr_from_bsc: counts need a rank table");
    if (batch > 65535) return fail(LDPC_EINVAL, "ldpc_llr_from_bsc: batch above 65535");
    const int nbytes = (c->n + 7) / 8;
    dim3 grid((nbytes + kLlrThreads - 1) / kLlrThreads, batch);
    llr_kernel<<<grid, kLlrThreads, 0, (cudaStream_t)stream>>>(bob_bits, llr_mag, rank, n_short, n_punct, known,
                                                                c->n, nbytes, llr_out);
    ldpc::count_launch();
    LDPC_CUDA_TRY(cudaGetLastError());
    return LDPC_OK;
}

int ldpc_syndrome(const ldpc_code* c, const uint8_t* bits, int batch, uint8_t* syn_out, void* stream) {
    using ldpc::fail;
    if (!c) return fail(LDPC_EINVAL, "ldpc_syndrome: NULL code");
    if (batch < 0 || batch > 65535) return fail(LDPC_EINVAL, "ldpc_syndrome: batch out of range");
    if (batch == 0) return LDPC_OK;
    if (!bits || !syn_out) return fail(LDPC_EINVAL, "ldpc_syndrome: NULL buffer");
    const int nbx = (c->n + 7) / 8, nbs = (c->m + 7) / 8;
    const int threads = 128;
    dim3 grid((nbs + threads - 1) / threads, batch);
    const size_t smem = c->tab_words * sizeof(int32_t);
    syndrome_kernel<<<grid, threads, smem, (cudaStream_t)stream>>>(c->d_tab, c->Mb, c->nblk, c->Z, c->m, nbx, nbs,
                                                                    bits, syn_out);
    ldpc::count_launch();
    LDPC_CUDA_TRY(cudaGetLastError());
    return LDPC_OK;
}

int ldpc_debug_tau_table(uint8_t* out, void* stream) {
    if (!out) return ldpc::fail(LDPC_EINVAL, "ldpc_debug_tau_table: NULL buffer");
    tau_table_kernel<<<128, 32, 0, (cudaStream_t)stream>>>(out);
    ldpc::count_launch();
    LDPC_CUDA_TRY(cudaGetLastError());
    return LDPC_OK;
}

}  // extern "C"
