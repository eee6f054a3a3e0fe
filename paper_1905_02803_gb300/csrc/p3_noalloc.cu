// Allocation-free forward transform: p3_ftran_r2c with its workspace taken
// from a fixed device array compiled into this library instead of from the
// caller.
//
// Who needs it: callers that must not allocate device memory at the point
// where they run a transform -- applications whose device memory is handed
// out by their own pre-sized pool and that forbid libraries from calling
// cudaMalloc, and latency-bound loops where a cudaMalloc/cudaFree pair (which
// can synchronise the device) is not acceptable.  Such a caller still passes
// its own input and output buffers and a plan created beforehand (plan
// creation allocates the plan's small tables once); this call allocates
// nothing.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/p3dfft_gb300.h"
#include "p3_internal.h"

namespace p3 {
// Runs every stage of one direction with the given workspace (p3_plan.cu).
p3_status run_direction(p3_plan plan, int dir, const void* in, void* out, void* ws, void* stream);
size_t plan_workspace(p3_plan plan);
}  // namespace p3

// The scratch array.  Every GPU that loads this library holds it until the
// process exits.  Its contents persist from one call to the next; the
// forward transform writes every workspace element it later reads, so
// nothing needs clearing between calls.
static __device__ __align__(256) unsigned char p3_static_scratch[P3_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch[kMaxDevices];
bool g_ready[kMaxDevices];

// Device address of the scratch array for the current device.  In host code
// the array's name only stands for the device symbol, so the address comes
// from cudaGetSymbolAddress, once per device, with that device current.
p3_status scratch_address(void** out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return P3_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return P3_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ready[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, p3_static_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return P3_ERR_CUDA;
        }
        g_scratch[dev] = p;
        g_ready[dev] = true;
    }
    *out = g_scratch[dev];
    return P3_OK;
}
}  // namespace

extern "C" p3_status p3_ftran_r2c_noalloc(p3_plan plan, const void* in_real, void* out_cplx, void* stream)
{
    if (!plan || !in_real || !out_cplx) return P3_ERR_INVALID;
    if (p3::plan_workspace(plan) > (size_t)P3_NOALLOC_SCRATCH_BYTES) return P3_ERR_UNSUPPORTED;
    void* scratch = nullptr;
    const p3_status st = scratch_address(&scratch);
    if (st != P3_OK) return st;
    return p3::run_direction(plan, 0, in_real, out_cplx, scratch, stream);
}
