// meta_noalloc.cu -- meta_cost_and_grad for callers that cannot allocate
// device memory.  The paper has no counterpart: this is a deployment aid.
//
// The scratch the kernels need lives in one file-scope device array of fixed
// size, so the caller passes inputs and outputs only.  Host code cannot use
// the array's name as a device address (in host code it names a host-side
// stand-in), so the entry points look the address up once per device with
// cudaGetSymbolAddress and pass that pointer on as the workspace.
#include <mutex>

#include "meta.h"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[META_NOALLOC_MAX_BYTES];

constexpr int kMaxDevices = 256;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {};

// Device address of the scratch on the current device (set-up, once per
// device, with that device current).
meta_status scratch_of_current_device(void** ptr) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return META_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* a = nullptr;
        if (cudaGetSymbolAddress(&a, g_noalloc_scratch) != cudaSuccess || !a) return META_ERR_CUDA;
        g_noalloc_addr[dev] = a;
    }
    *ptr = g_noalloc_addr[dev];
    return META_OK;
}

}  // namespace

extern "C" meta_status meta_cost_and_grad_noalloc(const meta_problem* prob, const float* I0,
                                                  const float* J, const float* p0,
                                                  const float* mu, const float* rho,
                                                  const float* lambda, double* cost,
                                                  float* grad, void* stream) {
    size_t need = 0;
    meta_status s = meta_workspace_size(prob, &need);
    if (s != META_OK) return s;
    if (need > (size_t)META_NOALLOC_MAX_BYTES) return META_ERR_WORKSPACE;
    void* ptr = nullptr;
    if ((s = scratch_of_current_device(&ptr)) != META_OK) return s;
    // The array keeps the previous call's contents.  Everything the kernels
    // read is written earlier in the same call, except the status word, which
    // must start at zero.
    if (cudaMemsetAsync(ptr, 0, 16, static_cast<cudaStream_t>(stream)) != cudaSuccess)
        return META_ERR_CUDA;
    return meta_cost_and_grad(prob, I0, J, p0, mu, rho, lambda, cost, grad, ptr,
                              (size_t)META_NOALLOC_MAX_BYTES, stream);
}

extern "C" meta_status meta_noalloc_status(int clear, void* stream, unsigned int* fault_bits) {
    if (!fault_bits) return META_ERR_INVALID_ARG;
    void* ptr = nullptr;
    const meta_status s = scratch_of_current_device(&ptr);
    if (s != META_OK) return s;
    return meta_workspace_status(ptr, (size_t)META_NOALLOC_MAX_BYTES, clear, stream, fault_bits);
}

extern "C" meta_status meta_noalloc_selftest_timeout(unsigned long long limit_ns, void* stream) {
    void* ptr = nullptr;
    const meta_status s = scratch_of_current_device(&ptr);
    if (s != META_OK) return s;
    return meta_selftest_timeout(ptr, (size_t)META_NOALLOC_MAX_BYTES, limit_ns, stream);
}
