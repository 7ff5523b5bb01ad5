// Status strings, error text and version of libdect.
#include <cuda_runtime.h>

#include <atomic>
#include <cstring>
#include <string>

#include "dect_internal.cuh"

namespace dect {

static thread_local char g_err[512] = "";
static std::atomic<int64_t> g_launches{0};

void count_launches(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

void set_error(const char *where, cudaError_t e)
{
    std::snprintf(g_err, sizeof(g_err), "%s: %s (%s)", where, cudaGetErrorName(e),
                  cudaGetErrorString(e));
}

void set_error_text(const std::string &s)
{
    std::snprintf(g_err, sizeof(g_err), "%s", s.c_str());
}

}  // namespace dect

extern "C" const char *dect_status_string(dect_status s)
{
    switch (s) {
    case DECT_OK: return "ok";
    case DECT_ERR_INVALID_ARG: return "invalid argument";
    case DECT_ERR_CUDA: return "CUDA error";
    case DECT_ERR_OOM: return "out of device memory";
    case DECT_ERR_TIMEOUT: return "device wait timed out";
    case DECT_ERR_NONFINITE: return "non-finite value";
    case DECT_ERR_NOT_CONVERGED: return "not converged";
    }
    return "unknown status";
}

extern "C" const char *dect_last_error(void) { return dect::g_err; }

extern "C" int dect_version(void) { return 100; }

extern "C" int64_t dect_kernel_launches(void) { return dect::g_launches.load(); }
