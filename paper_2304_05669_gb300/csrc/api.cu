// Context, status word and error reporting of the C ABI.
#include <cstdarg>
#include <cstring>

#include "fipt_internal.cuh"

#include <atomic>

namespace {
thread_local char g_err[512] = "";
std::atomic<unsigned long long> g_launches{0};
}

void fipt_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

extern "C" uint64_t fipt_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

fipt_status fipt_set_error(fipt_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

fipt_status fipt_check_cuda(cudaError_t e, const char* what) {
    return fipt_set_error(FIPT_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

bool fipt_aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

extern "C" const char* fipt_last_error(void) { return g_err; }

extern "C" const char* fipt_status_string(fipt_status s) {
    switch (s) {
        case FIPT_OK: return "ok";
        case FIPT_ERR_INVALID_ARG: return "invalid argument";
        case FIPT_ERR_CUDA: return "CUDA error";
        case FIPT_ERR_WORKSPACE: return "workspace too small";
        case FIPT_ERR_BUDGET: return "over memory budget";
        case FIPT_ERR_TIMEOUT: return "timeout";
        case FIPT_ERR_DEVICE_CHECK: return "device check failed";
        case FIPT_ERR_NOT_FOUND: return "not found";
    }
    return "unknown status";
}

extern "C" const char* fipt_version(void) { return "fipt-gb300 sm_103a 1"; }

extern "C" fipt_status fipt_ctx_create(int device, fipt_ctx** out) {
    FIPT_REQUIRE(out, "out is NULL");
    int n = 0;
    FIPT_CUDA(cudaGetDeviceCount(&n));
    FIPT_REQUIRE(device >= 0 && device < n, "device %d not in [0, %d)", device, n);
    FIPT_CUDA(cudaSetDevice(device));
    fipt_ctx* c = new fipt_ctx();
    c->device = device;
    cudaError_t e = cudaMalloc(&c->status, sizeof(int32_t));
    if (e != cudaSuccess) {
        delete c;
        return fipt_check_cuda(e, "cudaMalloc status word");
    }
    e = cudaMemset(c->status, 0, sizeof(int32_t));
    if (e != cudaSuccess) {
        cudaFree(c->status);
        delete c;
        return fipt_check_cuda(e, "cudaMemset status word");
    }
    *out = c;
    return FIPT_OK;
}

extern "C" fipt_status fipt_ctx_destroy(fipt_ctx* c) {
    if (!c) return FIPT_OK;
    cudaSetDevice(c->device);
    cudaFree(c->status);
    delete c;
    return FIPT_OK;
}

extern "C" fipt_status fipt_sync_status(fipt_ctx* c, fipt_stream stream, int32_t* device_code) {
    FIPT_REQUIRE(c, "ctx is NULL");
    FIPT_CUDA(cudaSetDevice(c->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int32_t v = 0;
    FIPT_CUDA(cudaMemcpyAsync(&v, c->status, sizeof(v), cudaMemcpyDeviceToHost, st));
    FIPT_CUDA(cudaMemsetAsync(c->status, 0, sizeof(v), st));
    FIPT_CUDA(cudaStreamSynchronize(st));
    if (device_code) *device_code = v;
    if (v != 0) return fipt_set_error(FIPT_ERR_DEVICE_CHECK, "device status bits 0x%x", v);
    return FIPT_OK;
}
