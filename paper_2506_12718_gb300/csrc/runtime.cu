// Device-side runtime state shared by all plans: barrier counters for the
// single-launch convolution kernel and the library's device error word.
//
// Each device gets one pool of kSlots counters (one per 128-byte line) plus an
// error word.  A launch takes the next slot round robin; the counter of a slot
// only grows, and the host remembers its value, so no reset is needed between
// launches.  kSlots launches would have to be in flight at once for two of
// them to share a slot.
#include <mutex>

#include "pac_internal.h"

namespace pac {

namespace {
constexpr int kSlots = 1024;
constexpr int kStride = 32;  // unsigned words per slot (128 bytes)

struct Pool {
    std::mutex mu;
    unsigned* d = nullptr;
    std::vector<unsigned> base;
    unsigned next = 0;
};
Pool g_pool[64];
}  // namespace

static int ensure_pool(int device, Pool& P) {
    if (P.d) return PAC_OK;
    void* d = nullptr;
    const size_t bytes = (size_t)(kSlots + 1) * kStride * sizeof(unsigned);
    cudaError_t e = cudaMalloc(&d, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "barrier pool");
    e = cudaMemset(d, 0, bytes);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaFree(d);
        return cuda_fail(e, "barrier pool init");
    }
    P.d = static_cast<unsigned*>(d);
    P.base.assign(kSlots, 0u);
    (void)device;
    return PAC_OK;
}

int barrier_slot(int device, unsigned** counter, unsigned* base, unsigned arrivals, unsigned** error) {
    if (device < 0 || device >= 64) return fail(PAC_ERR_ARG, "device %d out of range", device);
    Pool& P = g_pool[device];
    std::lock_guard<std::mutex> lk(P.mu);
    if (int rc = ensure_pool(device, P)) return rc;
    const unsigned s = P.next++ % kSlots;
    *counter = P.d + (size_t)s * kStride;
    *base = P.base[s];
    P.base[s] += arrivals;
    *error = P.d + (size_t)kSlots * kStride;
    return PAC_OK;
}

int device_error_word(int device, unsigned** error) {
    if (device < 0 || device >= 64) return fail(PAC_ERR_ARG, "device %d out of range", device);
    Pool& P = g_pool[device];
    std::lock_guard<std::mutex> lk(P.mu);
    if (int rc = ensure_pool(device, P)) return rc;
    *error = P.d + (size_t)kSlots * kStride;
    return PAC_OK;
}

int take_device_error(int device, unsigned* value) {
    *value = 0;
    if (device < 0 || device >= 64) return fail(PAC_ERR_ARG, "device %d out of range", device);
    Pool& P = g_pool[device];
    std::lock_guard<std::mutex> lk(P.mu);
    if (!P.d) return PAC_OK;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "synchronise");
    unsigned* err = P.d + (size_t)kSlots * kStride;
    e = cudaMemcpy(value, err, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && *value) e = cudaMemset(err, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return e == cudaSuccess ? PAC_OK : cuda_fail(e, "read device error word");
}

}  // namespace pac
