// Device status words: where the kernels of a plan report what they detect (a bounded wait
// that expired) so that the host can read it with stencil_sync_status / wave_sync_status.
//
// The words live in a fixed array in the library's device image, one slot per live plan, so
// that giving a plan its word allocates nothing and needs no GPU at plan time: the slot is
// chosen on the host when the plan is made, its device address is looked up (once per
// device, with that device current) when the plan first launches, and the word is read and
// cleared by a synchronous copy.  Static device memory starts at zero; a slot is cleared
// again before it is handed to the next plan.
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/stencil.h"
#include "internal.h"

namespace gst {

namespace {

constexpr int kMaxDevices = 64;

static __device__ int g_status_words[kStatusSlots];

std::mutex g_mu;
std::vector<int> g_free;  // released slots (cleared)
int g_next = 0;           // slots never handed out start here
int *g_base[kMaxDevices] = {};

int *device_base() {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_base[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_status_words) != cudaSuccess || !p) {
            cudaGetLastError();
            return nullptr;
        }
        g_base[dev] = static_cast<int *>(p);
    }
    return g_base[dev];
}

}  // namespace

int status_acquire() {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_free.empty()) {
        const int s = g_free.back();
        g_free.pop_back();
        return s;
    }
    if (g_next < kStatusSlots) return g_next++;
    return -1;
}

void status_release(int slot, bool used) {
    if (slot < 0) return;
    if (used) {
        // a word the plan's kernels may have set goes back cleared (the caller has
        // synchronised the device)
        const int zero = 0;
        if (cudaMemcpyToSymbol(g_status_words, &zero, sizeof(int), sizeof(int) * slot) !=
            cudaSuccess)
            cudaGetLastError();
    }
    std::lock_guard<std::mutex> lk(g_mu);
    g_free.push_back(slot);
}

int *status_word(int slot) {
    if (slot < 0 || slot >= kStatusSlots) return nullptr;
    int *base = device_base();
    return base ? base + slot : nullptr;
}

int status_take(int slot, cudaStream_t s) {
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return STENCIL_ERR_CUDA;
    }
    if (cudaGetLastError() != cudaSuccess) return STENCIL_ERR_CUDA;
    if (slot < 0) return STENCIL_OK;
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_status_words, sizeof(int), sizeof(int) * slot) !=
        cudaSuccess) {
        cudaGetLastError();
        return STENCIL_ERR_CUDA;
    }
    if (v != 0) {
        const int zero = 0;
        if (cudaMemcpyToSymbol(g_status_words, &zero, sizeof(int), sizeof(int) * slot) !=
            cudaSuccess) {
            cudaGetLastError();
            return STENCIL_ERR_CUDA;
        }
    }
    return v;
}

bool smem_opt_in(const void *kern, size_t smem, bool max_carveout) {
    if (smem <= 48 * 1024) return true;
    struct Entry {
        int dev;
        const void *kern;
        size_t smem;
    };
    static std::mutex mu;
    static std::vector<Entry> done;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    std::lock_guard<std::mutex> lk(mu);
    for (const Entry &e : done)
        if (e.dev == dev && e.kern == kern && e.smem >= smem) return true;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        (max_carveout && cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                              (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess)) {
        cudaGetLastError();
        return false;
    }
    for (Entry &e : done)
        if (e.dev == dev && e.kern == kern) {
            e.smem = smem;
            return true;
        }
    done.push_back({dev, kern, smem});
    return true;
}

}  // namespace gst
