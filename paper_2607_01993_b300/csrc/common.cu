// Status reporting and small host-side entry points of libsilh.
#include <cmath>
#include <cstring>
#include <atomic>
#include <mutex>

#include "common.cuh"

namespace silh {

static thread_local char g_last_error[512] = "";
static std::atomic<unsigned long long> g_launches{0};

void count_launches(int nlaunch) { g_launches.fetch_add((unsigned long long)nlaunch); }

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
}

silh_status fail(silh_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return st;
}

bool device_accessible(const void *p) {
    if (p == nullptr) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return true;
    // page-locked host memory counts only when it is mapped at the same address
    return a.type == cudaMemoryTypeHost && a.devicePointer == p;
}

bool sample_accessible(const silh_sample *S) {
    return S != nullptr && device_accessible(S->sizes) && device_accessible(S->offsets) &&
           (S->size == 0 || (device_accessible(S->idx) && device_accessible(S->p)));
}

void ensure_pool_retains(int device) {
    static std::mutex mu;
    static bool done[64] = {false};
    if (device < 0 || device >= 64) return;
    std::lock_guard<std::mutex> lock(mu);
    if (done[device]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    done[device] = true;
}

}  // namespace silh

extern "C" const char *silh_last_error(void) { return silh::g_last_error; }

extern "C" const char *silh_version(void) { return "silh 0.1 (sm_103a)"; }

extern "C" uint64_t silh_kernel_launches(void) { return silh::g_launches.load(); }

extern "C" double silh_t_from_eps(double eps, double delta, int64_t n, int32_t k) {
    if (!(eps > 0.0) || !(delta > 0.0) || n < 1 || k < 1) return NAN;
    return std::ceil((3.0 * 18.0 / (eps * eps)) * std::log(5.0 * (double)n * (double)k / delta));
}
