// Allocation-free variant of the field scalar product (ov_field_dot).
//
// Some callers cannot allocate device memory at the moment they need a
// reduction: code that runs while a CUDA graph is being captured in global
// mode (cudaMalloc is not allowed then), an application whose memory manager
// owns the whole device and forbids allocations behind its back, or a
// plug-in whose device memory budget is fixed by its host program.
// ov_field_dot keeps its partial sums in a context buffer that it may grow
// with cudaMalloc on first use; this entry point never allocates: its
// partial sums live in one fixed array that is part of the library's device
// image, so every GPU that loads the library holds it until the process exits.
#include <atomic>
#include <mutex>

#include "ctx.h"

namespace {

// One partial sum (double2) per reduction block and right-hand side: at most
// 16 right-hand sides x 1216 blocks (152 SMs x 8), plus 64 entries that hold
// the result on its way to a host output buffer.  311 KB in all.
constexpr int kPartials = 16 * 1216;
constexpr int kResult = 64;
static __device__ __align__(256) double2 g_dot_scratch[kPartials + kResult];

// Device address of g_dot_scratch for each device, looked up once per device.
// In host code the name g_dot_scratch is only a host-side stand-in for the
// symbol, so kernels must be given this address instead.
constexpr int kMaxDevices = 64;
std::atomic<double2*> g_scratch_addr[kMaxDevices];
std::mutex g_setup_mutex;

double2* scratch_for_current_device(int dev)
{
    if (dev < 0 || dev >= kMaxDevices) return nullptr;
    double2* p = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (p) return p;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    p = g_scratch_addr[dev].load(std::memory_order_relaxed);
    if (p) return p;
    void* addr = nullptr;
    if (cudaGetSymbolAddress(&addr, g_dot_scratch) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    p = static_cast<double2*>(addr);
    g_scratch_addr[dev].store(p, std::memory_order_release);
    return p;
}

}  // namespace

using namespace ov;

extern "C" int ov_field_dot_noalloc(const ov_field* x, const ov_field* y, double* out, void* stream)
{
    if (!x || !y || !out || x->owner != y->owner) return OV_EINVAL;
    const FieldDesc& a = x->d;
    const FieldDesc& b = y->d;
    if (a.prec != b.prec || a.nrhs != b.nrhs) return OV_EINVAL;
    ov_ctx* c = x->owner;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return OV_ECUDA;
    }
    if (dev != c->device) return OV_EINVAL;  // fields live on another device
    const int nblk = reduce_blocks(c->g);
    if ((long long)nblk * a.nrhs > kPartials || a.nrhs > kResult) return OV_EINVAL;
    double2* scratch = scratch_for_current_device(dev);
    if (!scratch) return OV_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    // every block writes its own partial, so nothing has to be cleared first
    if (launch_dot(c->g, a, b, scratch, nblk, st) != cudaSuccess) return OV_ECUDA;
    const bool device_out = is_device_ptr(out);
    double* res = device_out ? out : reinterpret_cast<double*>(scratch + kPartials);
    if (launch_finalize(reinterpret_cast<const double*>(scratch), nblk, a.nrhs, 2, res, st) != cudaSuccess)
        return OV_ECUDA;
    if (!device_out) {
        if (cudaMemcpyAsync(out, res, sizeof(double) * 2 * a.nrhs, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return OV_ECUDA;
    }
    return OV_OK;
}
