// Status strings, error text and version of libdect.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <string>

#include "dect_internal.cuh"

namespace dect {

static thread_local char g_err[512] = "";
static std::atomic<int64_t> g_launches{0};

// readers of the per-translation-unit check words (checked build only)
static CheckReader g_readers[32];
static std::atomic<int> g_nreaders{0};

int register_check_reader(CheckReader r)
{
    const int k = g_nreaders.fetch_add(1);
    if (k < 32) g_readers[k] = r;
    return k;
}

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
    case DECT_ERR_INDEX: return "index check failed";
    }
    return "unknown status";
}

extern "C" const char *dect_last_error(void) { return dect::g_err; }

extern "C" int dect_version(void) { return 100; }

extern "C" int dect_checked_build(void)
{
#ifdef DECT_CHECKED
    return 1;
#else
    return 0;
#endif
}

extern "C" dect_status dect_check_status(void)
{
    if (cudaDeviceSynchronize() != cudaSuccess) {
        dect::set_error("dect_check_status", cudaGetLastError());
        return DECT_ERR_CUDA;
    }
    const int n = std::min(dect::g_nreaders.load(), 32);
    for (int k = 0; k < n; ++k) {
        unsigned long long w = 0;
        cudaError_t e = dect::g_readers[k](&w);
        if (e != cudaSuccess) {
            dect::set_error("dect_check_status", e);
            return DECT_ERR_CUDA;
        }
        if (w) {
            static const char *names[] = {"?", "A x gather", "A^T y gather", "on-the-fly A walk",
                                          "on-the-fly A^T ray", "PLS stencil", "FBP bin", "self-test"};
            const unsigned site = (unsigned)(w >> 48);
            char buf[160];
            std::snprintf(buf, sizeof(buf), "index check failed: %s, index %lld",
                          site < 8 ? names[site] : "?", (long long)(w & 0xffffffffffffull));
            dect::set_error_text(buf);
            return DECT_ERR_INDEX;
        }
    }
    return DECT_OK;
}

extern "C" int64_t dect_kernel_launches(void) { return dect::g_launches.load(); }

// ---------------------------------------------------------------------------
// Self-test of the bounded device wait used by the staged kernels: one block
// waits on an mbarrier that nothing arrives on, for at most `polls` polls,
// and reports whether the wait ran out.  Nothing faults, traps or hangs.
// ---------------------------------------------------------------------------
#include "kernels.cuh"

namespace dect {
namespace {
__global__ void k_wait_selftest(unsigned polls, int *timed_out)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    const bool got = mbar_wait_bounded(&bar, 0u, polls);
    if (__syncthreads_or(!got) && threadIdx.x == 0) *timed_out = 1;
    // complete the phase so the barrier is left balanced
    if (threadIdx.x == 0) mbar_arrive_expect_tx(&bar, 0u);
    __syncthreads();
    mbar_wait_bounded(&bar, 0u, 1u << 20);
}
}  // namespace
}  // namespace dect

namespace dect {
namespace {
// reads a[index] of an 8-element array through an index check
__global__ void k_index_selftest(const float *a, int index, float *out)
{
    int i = index;
    if (!DECT_IDX_OK(i, 8, CHK_SELFTEST)) i = 0;
    *out = a[i];
}
}  // namespace
}  // namespace dect

extern "C" dect_status dect_selftest_index(int index, dect_stream stream)
{
#ifndef DECT_CHECKED
    // without the checks an out-of-range index would be a real access
    if (index < 0 || index >= 8) return DECT_ERR_INVALID_ARG;
#endif
    cudaStream_t s = (cudaStream_t)stream;
    float *d = nullptr;
    DECT_CUDA(cudaMallocAsync((void **)&d, 9 * sizeof(float), s));
    DECT_CUDA(cudaMemsetAsync(d, 0, 9 * sizeof(float), s));
    dect::k_index_selftest<<<1, 1, 0, s>>>(d, index, d + 8);
    DECT_LAUNCH_CHECK();
    dect::count_launches(1);
    DECT_CUDA(cudaFreeAsync(d, s));
    DECT_CUDA(cudaStreamSynchronize(s));
    return dect_check_status();
}

extern "C" dect_status dect_selftest_bounded_wait(unsigned polls, dect_stream stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    int *d = nullptr;
    int h = 0;
    DECT_CUDA(cudaMallocAsync((void **)&d, sizeof(int), s));
    DECT_CUDA(cudaMemsetAsync(d, 0, sizeof(int), s));
    dect::k_wait_selftest<<<1, 64, 0, s>>>(polls, d);
    DECT_LAUNCH_CHECK();
    dect::count_launches(1);
    DECT_CUDA(cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s));
    DECT_CUDA(cudaFreeAsync(d, s));
    DECT_CUDA(cudaStreamSynchronize(s));
    if (h) {
        dect::set_error_text("dect_selftest_bounded_wait: the wait ran out after the poll limit");
        return DECT_ERR_TIMEOUT;
    }
    return DECT_OK;
}
