// stencil_apply_noalloc: the multi-step constant-coefficient sweep for callers that are not
// allowed to allocate device memory.
//
// stencil_apply ping-pongs between `out` and a grid-sized scratch buffer that the plan obtains
// with cudaMalloc on its first multi-step call.  Some callers cannot let that happen: code
// running inside a framework whose caching allocator owns (nearly) all device memory, or
// code that must not pay cudaMalloc's implicit device-wide synchronisation in a
// latency-critical loop.  This entry point takes its scratch from a fixed array that lives
// in the library's own device image instead, so it allocates nothing.
//
// The array (STENCIL_NOALLOC_SCRATCH_BYTES = 16 MiB) exists once per GPU that loads the
// library and stays reserved until the process exits.  Its device address is looked up once
// per device, on the first call made with that device current; make that first call before
// starting any stream capture.  Every call shares the array: two calls whose kernels overlap
// on the GPU (different streams, no ordering between them) race on it.  The scratch needs no
// clearing, since each step writes every cell of its destination before the next step reads it.
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/stencil.h"
#include "internal.h"
#include "plan_internal.h"

namespace {

constexpr size_t kScratchBytes = STENCIL_NOALLOC_SCRATCH_BYTES;
static_assert(kScratchBytes % 256 == 0, "scratch size must keep 256-byte alignment");

// The ping-pong buffer of every allocation-free call on this device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void *g_scratch_addr[kMaxDevices] = {};  // device address of g_noalloc_scratch, per device

// Device address of the scratch array on the current device (looked up once per device).
int scratch_address(void **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return STENCIL_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return STENCIL_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return STENCIL_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return STENCIL_OK;
}

}  // namespace

extern "C" int stencil_apply_noalloc(stencil_handle h, const void *in, void *out, int steps,
                                     void *stream) {
    int rc = gst::check_apply_args(h, in, out, steps);
    if (rc) return rc;
    if (h->kind != STENCIL_CONST) return STENCIL_ERR_BADARG;
    const size_t bytes = (size_t)h->dims[0] * h->dims[1] * h->dims[2] * gst::dtype_size(h->dtype);
    if (bytes > kScratchBytes) return STENCIL_ERR_BADARG;  // grid larger than the fixed scratch
    void *scratch = nullptr;
    rc = scratch_address(&scratch);
    if (rc) return rc;
    // the group schedule of stencil_apply: the last group writes `out`, `in` is never written
    const int fuse = gst::plan_steps_per_launch(*h);
    const int groups = (steps + fuse - 1) / fuse;
    const void *src = in;
    int done = 0;
    for (int g = 0; g < groups; ++g) {
        const int k = (steps - done) < fuse ? (steps - done) : fuse;
        void *dst = ((groups - 1 - g) % 2 == 0) ? out : scratch;
        rc = gst::launch_group_with(*h, h->cf.data(), src, dst, k, (cudaStream_t)stream);
        if (rc) return rc;
        src = dst;
        done += k;
    }
    return STENCIL_OK;
}
