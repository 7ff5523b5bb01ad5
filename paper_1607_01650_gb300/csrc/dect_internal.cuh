// Internal declarations shared by the translation units of libdect.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>

#include "dect.h"

namespace dect {

constexpr int kSMs = 152;          // GB300: 2 dies x 76 SMs
constexpr int kMaxBatchImages = 32; // images interleaved per ADM pass

// Thread-local text of the last CUDA error (returned by dect_last_error()).
void set_error(const char *where, cudaError_t e);
void set_error_text(const std::string &s);

#define DECT_CUDA(call)                                                         \
    do {                                                                        \
        cudaError_t e_ = (call);                                                \
        if (e_ != cudaSuccess) {                                                \
            ::dect::set_error(#call, e_);                                       \
            return e_ == cudaErrorMemoryAllocation ? DECT_ERR_OOM : DECT_ERR_CUDA; \
        }                                                                       \
    } while (0)

#define DECT_LAUNCH_CHECK() DECT_CUDA(cudaGetLastError())

// Count of kernels launched by the library (dect_kernel_launches()).
void count_launches(int64_t k);

// Packed table entry: .x = pixel (or ray) index, .y = __float_as_int(length in mm).
typedef int2 Entry;

}  // namespace dect

struct dect_plan {
    dect_geometry g;
    int device;
    int n, nv, nb;
    int64_t N, M, nnz;
    int64_t n_grid_aligned;
    int64_t *rowptr;   // [M + 1], ray-major table (CSR of A)
    dect::Entry *ent;  // [nnz]  {pixel, len}
    int64_t *colptr;   // [N + 1], pixel-major table (CSR of A^T)
    dect::Entry *tent; // [nnz]  {ray, len}, rays increasing within a pixel
};

namespace dect {

// Launchers (project.cu).  Planar layout: image b at base + b * N.
cudaError_t launch_project_planar(const dect_plan *p, const float *x, float *y, int batch,
                                  cudaStream_t s);
cudaError_t launch_backproject_planar(const dect_plan *p, const float *y, float *x, int batch,
                                      cudaStream_t s);

}  // namespace dect
