// Code handles, error reporting and the message scratch arena.
#include <stdio.h>

#include <mutex>

#include "common.cuh"

namespace ldpc {

static thread_local std::string g_last_error;
static std::atomic<int64_t> g_launches{0};

void set_error(const std::string& msg) { g_last_error = msg; }

int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return LDPC_ECUDA;
}

void count_launch(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

int max_dyn_smem(int device) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) return 0;
    return v;
}

int ensure_arena(ldpc_code* c, size_t bytes) {
    if (bytes <= c->arena_bytes) return LDPC_OK;
    if (c->arena) {
        LDPC_CUDA_TRY(cudaDeviceSynchronize());
        cudaFree(c->arena);
        c->arena = nullptr;
        c->arena_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&c->arena, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(LDPC_ENOMEM, std::string("scratch arena of ") + std::to_string(bytes) + " bytes: " +
                                     cudaGetErrorString(e));
    }
    c->arena_bytes = bytes;
    return LDPC_OK;
}

int ensure_io(ldpc_code* c, size_t bytes) {
    if (bytes <= c->io_bytes) return LDPC_OK;
    if (c->io) {
        LDPC_CUDA_TRY(cudaDeviceSynchronize());
        cudaFree(c->io);
        c->io = nullptr;
        c->io_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&c->io, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(LDPC_ENOMEM, std::string("host-buffer staging of ") + std::to_string(bytes) + " bytes: " +
                                     cudaGetErrorString(e));
    }
    c->io_bytes = bytes;
    return LDPC_OK;
}

}  // namespace ldpc

extern "C" {

int ldpc_code_create(const int32_t* base, int Mb, int Nb, int Z, ldpc_code** out) {
    using ldpc::fail;
    if (!base || !out) return fail(LDPC_EINVAL, "ldpc_code_create: NULL pointer");
    *out = nullptr;
    if (Mb <= 0 || Nb <= 0 || Z <= 0) return fail(LDPC_EINVAL, "ldpc_code_create: Mb, Nb and Z must be positive");
    if ((int64_t)Nb * Z > (1 << 24) || (int64_t)Mb * Z > (1 << 24))
        return fail(LDPC_EUNSUPPORTED, "ldpc_code_create: n or m above 2^24");
    ldpc_code* c = new ldpc_code();
    c->Mb = Mb; c->Nb = Nb; c->Z = Z; c->n = Nb * Z; c->m = Mb * Z;
    std::vector<int32_t> deg(Mb), off(Mb + 1), col, sh;
    for (int i = 0; i < Mb; i++) {
        off[i] = (int32_t)col.size();
        for (int k = 0; k < Nb; k++) {
            int s = base[(size_t)i * Nb + k];
            if (s < 0) {
                if (s != -1) { delete c; return fail(LDPC_EINVAL, "ldpc_code_create: negative entry other than -1"); }
                continue;
            }
            if (s >= Z) { delete c; return fail(LDPC_EINVAL, "ldpc_code_create: shift >= Z"); }
            col.push_back(k);
            sh.push_back(s);
        }
        deg[i] = (int32_t)col.size() - off[i];
        if (deg[i] > c->max_deg) c->max_deg = deg[i];
    }
    off[Mb] = (int32_t)col.size();
    c->nblk = (int)col.size();
    c->edges = (int64_t)c->nblk * Z;
    if (c->max_deg > 64) { delete c; return fail(LDPC_EUNSUPPORTED, "ldpc_code_create: row degree above 64"); }
    c->h_tab.reserve(2 * Mb + 1 + 2 * c->nblk);
    c->h_tab.insert(c->h_tab.end(), deg.begin(), deg.end());
    c->h_tab.insert(c->h_tab.end(), off.begin(), off.end());
    c->h_tab.insert(c->h_tab.end(), col.begin(), col.end());
    c->h_tab.insert(c->h_tab.end(), sh.begin(), sh.end());
    c->tab_words = c->h_tab.size();
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_tab, c->tab_words * sizeof(int32_t));
    if (e == cudaSuccess)
        e = cudaMemcpy(c->d_tab, c->h_tab.data(), c->tab_words * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_queue, 256);
    if (e == cudaSuccess) e = cudaMemset(c->d_queue, 0, 256);
    if (e != cudaSuccess) {
        int r = ldpc::cuda_fail(e, "ldpc_code_create: table upload");
        if (c->d_tab) cudaFree(c->d_tab);
        if (c->d_queue) cudaFree(c->d_queue);
        delete c;
        return r;
    }
    *out = c;
    return LDPC_OK;
}

void ldpc_code_destroy(ldpc_code* c) {
    if (!c) return;
    cudaDeviceSynchronize();
    if (c->d_tab) cudaFree(c->d_tab);
    if (c->arena) cudaFree(c->arena);
    if (c->io) cudaFree(c->io);
    if (c->d_queue) cudaFree(c->d_queue);
    delete c;
}

int ldpc_code_info(const ldpc_code* c, int* n, int* m, int64_t* edges, int* max_row_deg) {
    if (!c) return ldpc::fail(LDPC_EINVAL, "ldpc_code_info: NULL code");
    if (n) *n = c->n;
    if (m) *m = c->m;
    if (edges) *edges = c->edges;
    if (max_row_deg) *max_row_deg = c->max_deg;
    return LDPC_OK;
}

int64_t ldpc_launch_count(void) { return ldpc::g_launches.load(); }

const char* ldpc_strerror(int code) {
    switch (code) {
        case LDPC_OK: return "ok";
        case LDPC_EINVAL: return "invalid argument";
        case LDPC_ENOMEM: return "out of device memory";
        case LDPC_ECUDA: return "CUDA error";
        case LDPC_EUNSUPPORTED: return "unsupported shape";
        case LDPC_EKERNEL: return "kernel bound violation";
        default: return "unknown error";
    }
}

const char* ldpc_last_error(void) { return ldpc::g_last_error.c_str(); }

}  // extern "C"
