// A x and A^T y on caller-owned planar batches (Eq. (1); the A^T of G_f in Eq. (9)).
#include <cuda_runtime.h>

#include "dect_internal.cuh"
#include "kernels.cuh"

namespace dect {
namespace {

constexpr int kBlock = 256;

template <int NB, int G>
cudaError_t run_rows(const int64_t *ptr, const Entry *ent, int64_t rows, const float *src,
                     int64_t src_stride, float *dst, int64_t dst_stride, int nimg, cudaStream_t s)
{
    if (rows == 0) return cudaSuccess;
    int64_t rpb = kBlock / G;
    int64_t want = (rows + rpb - 1) / rpb;
    int64_t cap = (int64_t)kSMs * 8;
    unsigned grid = (unsigned)(want < cap ? want : cap);
    k_rows_planar<NB, G><<<grid, kBlock, 0, s>>>(ptr, ent, rows, src, src_stride, dst, dst_stride, nimg);
    count_launches(1);
    return cudaGetLastError();
}

// Split a planar batch into chunks of up to 4 images per pass over the table.
template <int GF>
cudaError_t rows_batched(const int64_t *ptr, const Entry *ent, int64_t rows, const float *src,
                         int64_t src_stride, float *dst, int64_t dst_stride, int batch, cudaStream_t s)
{
    int done = 0;
    while (done < batch) {
        int left = batch - done;
        cudaError_t e;
        const float *sp = src + (int64_t)done * src_stride;
        float *dp = dst + (int64_t)done * dst_stride;
        if (left == 1) {
            e = run_rows<1, GF>(ptr, ent, rows, sp, src_stride, dp, dst_stride, 1, s);
            done += 1;
        } else if (left == 2) {
            e = run_rows<2, GF>(ptr, ent, rows, sp, src_stride, dp, dst_stride, 2, s);
            done += 2;
        } else {
            int k = left < 4 ? left : 4;
            e = run_rows<4, GF>(ptr, ent, rows, sp, src_stride, dp, dst_stride, k, s);
            done += k;
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_project_planar(const dect_plan *p, const float *x, float *y, int batch,
                                  cudaStream_t s)
{
    return rows_batched<32>(p->rowptr, p->ent, p->M, x, p->N, y, p->M, batch, s);
}

cudaError_t launch_backproject_planar(const dect_plan *p, const float *y, float *x, int batch,
                                      cudaStream_t s)
{
    return rows_batched<16>(p->colptr, p->tent, p->N, y, p->M, x, p->N, batch, s);
}

}  // namespace dect

using namespace dect;

extern "C" dect_status dect_project(const dect_plan *plan, const float *x, float *y, int batch,
                                    dect_stream stream)
{
    if (!plan || batch < 0) return DECT_ERR_INVALID_ARG;
    if (batch == 0) return DECT_OK;
    if (!x || !y) return DECT_ERR_INVALID_ARG;
    DECT_CUDA(cudaSetDevice(plan->device));
    DECT_CUDA(launch_project_planar(plan, x, y, batch, (cudaStream_t)stream));
    return DECT_OK;
}

extern "C" dect_status dect_backproject(const dect_plan *plan, const float *y, float *x, int batch,
                                        dect_stream stream)
{
    if (!plan || batch < 0) return DECT_ERR_INVALID_ARG;
    if (batch == 0) return DECT_OK;
    if (!x || !y) return DECT_ERR_INVALID_ARG;
    DECT_CUDA(cudaSetDevice(plan->device));
    DECT_CUDA(launch_backproject_planar(plan, y, x, batch, (cudaStream_t)stream));
    return DECT_OK;
}
