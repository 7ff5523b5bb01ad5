// A x and A^T y on caller-owned planar batches (Eq. (1); the A^T of G_f in
// Eq. (9)), through the interleaved table kernels of the ADM: a batch is
// split into passes of up to 64 images; each pass packs its images
// pixel-major ([index][NB], zero-padded to the width NB), streams the table
// once with every entry gathering one contiguous vector of all NB images,
// and unpacks the result to the planar output.
#include <cuda_runtime.h>

#include <algorithm>

#include "dect_internal.cuh"
#include "kernels.cuh"

namespace dect {
namespace {

constexpr int kOpBlock = 1024;  // one block per SM
constexpr int kTile = 8;        // A^T: 8 x 8 pixel tiles, so a tile's sinogram lines stay in one L1

// planar src [nimg][rows] -> interleaved dst [rows][NB] (images >= nimg are 0)
template <int NB>
__global__ void k_to_il(const float *__restrict__ src, float *__restrict__ dst, int64_t rows, int nimg)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= rows * NB) return;
    const int64_t row = t / NB;
    const int img = (int)(t % NB);
    dst[t] = img < nimg ? src[(int64_t)img * rows + row] : 0.f;
}

// interleaved src [rows][NB] -> planar dst [nimg][rows]
template <int NB>
__global__ void k_from_il(const float *__restrict__ src, float *__restrict__ dst, int64_t rows, int nimg)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= rows * NB) return;
    const int64_t row = t / NB;
    const int img = (int)(t % NB);
    if (img < nimg) dst[(int64_t)img * rows + row] = src[t];
}

// dst[row][NB] = sum over the row's entries of len * src[index][NB].  A warp
// per row (G = 32 lanes).  TILED (pixel-major table of an n x n image): the
// block's consecutive rows walk 8 x 8 pixel tiles, so that pixels sharing
// rays share an L1; otherwise rows are taken in order (adjacent rays of a
// view share pixels).  Lanes gather 8 images of an entry at 16 or more
// images (row_dot_w), 4 below (row_dot_g).
template <int NB, bool TILED>
__global__ void __launch_bounds__(kOpBlock) k_rows_il(const int64_t *__restrict__ ptr, const Entry *__restrict__ ent,
                                                      int64_t rows, int n, int nz, const float *__restrict__ src,
                                                      int64_t src_rows, float *__restrict__ dst)
{
    constexpr int G = 32, VW = Batch<NB>::VW, LPE = Batch<NB>::CPB;
    const int lr = threadIdx.x % G, grp = lr / LPE, vl = lr % LPE;
    const int64_t rpb = kOpBlock / G;
    const int tiles_x = (n + kTile - 1) / kTile;
    const int64_t per_slice = (int64_t)tiles_x * tiles_x * kTile * kTile;
    const int64_t vrows = TILED ? per_slice * nz : rows;
    const unsigned long long pol = l2_evict_last_policy();
    for (int64_t v0 = (int64_t)blockIdx.x * rpb; v0 < vrows; v0 += (int64_t)gridDim.x * rpb) {
        const int64_t v = v0 + threadIdx.x / G;
        int64_t row = v;
        bool ok = v < vrows;
        if (TILED && ok) {  // slice k, tile of the slice, pixel of the tile
            const int64_t k = v / per_slice, vs = v % per_slice;
            const int64_t tile = vs / (kTile * kTile);
            const int w = (int)(vs % (kTile * kTile));
            const int i = (int)(tile / tiles_x) * kTile + w / kTile, j = (int)(tile % tiles_x) * kTile + w % kTile;
            ok = i < n && j < n;
            row = (k * n + i) * n + j;
        }
        int64_t b = 0, e = 0;
        if (ok) {
            b = ptr[row];
            e = ptr[row + 1];
        }
        Vec<VW> acc;
        if constexpr (NB >= 16)
            acc = row_dot_w<NB, G, 8, 2>(ent, b, e, lr, src, pol, src_rows, TILED ? CHK_GATHER_AT : CHK_GATHER_A);
        else
            acc = row_dot<NB, G, true>(ent, b, e, src, src_rows, lr, TILED ? CHK_GATHER_AT : CHK_GATHER_A);
        if (ok && grp == 0) st_v<VW>(dst + row * NB + vl * VW, acc);
    }
}

template <int NB>
cudaError_t pass(const int64_t *ptr, const Entry *ent, int64_t rows_in, int64_t rows_out, int n, int nz, bool tiled,
                 const float *src, float *dst, int nimg, float *buf, cudaStream_t s)
{
    float *in_il = buf, *out_il = buf + rows_in * NB;
    const unsigned bi = (unsigned)((rows_in * NB + 255) / 256), bo = (unsigned)((rows_out * NB + 255) / 256);
    k_to_il<NB><<<bi, 256, 0, s>>>(src, in_il, rows_in, nimg);
    if (tiled)
        k_rows_il<NB, true><<<kSMs, kOpBlock, 0, s>>>(ptr, ent, rows_out, n, nz, in_il, rows_in, out_il);
    else
        k_rows_il<NB, false><<<kSMs, kOpBlock, 0, s>>>(ptr, ent, rows_out, n, nz, in_il, rows_in, out_il);
    k_from_il<NB><<<bo, 256, 0, s>>>(out_il, dst, rows_out, nimg);
    count_launches(3);
    return cudaGetLastError();
}

// Passes of up to 64 images over the table (ptr, ent) mapping src rows
// (rows_in per image) to dst rows (rows_out per image).
cudaError_t run_batched(const int64_t *ptr, const Entry *ent, int64_t rows_in, int64_t rows_out, int n, int nz,
                        bool tiled, const float *src, float *dst, int batch, cudaStream_t s)
{
    int width0 = 2;  // widest pass: the next power of two >= min(batch, 64), at least 2
    while (width0 < std::min(batch, kMaxBatchImages)) width0 *= 2;
    float *buf = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&buf, sizeof(float) * (size_t)(rows_in + rows_out) * width0, s);
    if (e != cudaSuccess) return e;
    for (int done = 0; done < batch && e == cudaSuccess;) {
        const int k = std::min(kMaxBatchImages, batch - done);
        const float *sp = src + (int64_t)done * rows_in;
        float *dp = dst + (int64_t)done * rows_out;
        if (k <= 2) e = pass<2>(ptr, ent, rows_in, rows_out, n, nz, tiled, sp, dp, k, buf, s);
        else if (k <= 4) e = pass<4>(ptr, ent, rows_in, rows_out, n, nz, tiled, sp, dp, k, buf, s);
        else if (k <= 8) e = pass<8>(ptr, ent, rows_in, rows_out, n, nz, tiled, sp, dp, k, buf, s);
        else if (k <= 16) e = pass<16>(ptr, ent, rows_in, rows_out, n, nz, tiled, sp, dp, k, buf, s);
        else if (k <= 32) e = pass<32>(ptr, ent, rows_in, rows_out, n, nz, tiled, sp, dp, k, buf, s);
        else e = pass<64>(ptr, ent, rows_in, rows_out, n, nz, tiled, sp, dp, k, buf, s);
        done += k;
    }
    cudaError_t f = cudaFreeAsync(buf, s);
    return e != cudaSuccess ? e : f;
}

}  // namespace

cudaError_t launch_project_planar(const dect_plan *p, const float *x, float *y, int batch, cudaStream_t s)
{
    return run_batched(p->rowptr, p->ent, p->N, p->M, p->n, std::max(p->nz, 1), false, x, y, batch, s);
}

cudaError_t launch_backproject_planar(const dect_plan *p, const float *y, float *x, int batch, cudaStream_t s)
{
    return run_batched(p->colptr, p->tent, p->M, p->N, p->n, std::max(p->nz, 1), true, y, x, batch, s);
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
