// Fan-beam filtered backprojection: the analytic reconstruction the paper
// uses in Sec. 2.4 and Sec. 3, here as an initial image for the ADM
// (dect_adm_tv with warm_start = 1).  Textbook algorithm for an equally
// spaced flat detector over a full 360-degree scan:
//   1. bins moved to a virtual detector through the isocentre,
//      s_b = u_b SOD / SDD, spacing ds = pitch SOD / SDD;
//   2. cosine pre-weight q = p SOD / sqrt(SOD^2 + s_b^2);
//   3. Ram-Lak ramp filter sampled at ds: h(0) = 1 / (4 ds^2), h(k) = 0 for
//      even k != 0, h(k) = -1 / (pi^2 k^2 ds^2) for odd k, qf = ds (q * h);
//   4. back-projection: for pixel P and view v (source S, central-ray
//      direction c, lateral direction e of increasing bin index),
//      L = (P - S).c = SOD + P.c, s = (P.e) SOD / L, and
//      f(P) = sum_v (dtheta / 2) (SOD / L)^2 qf(v, s), linear between bins,
//      0 outside them.
// FP64 filter and per-pixel geometry, FP32 filtered projections and
// back-projection sums; the filter adds each pair of taps from the farthest
// (smallest) to the nearest, the back-projection adds the views in order.
#include <cuda_runtime.h>

#include <cmath>

#include "dect_internal.cuh"

namespace dect {
namespace {

constexpr int kFbpBlock = 256;
constexpr int kFbpImgs = 4;  // images per back-projection thread

struct ViewGeo {
    double cx, cy;  // central-ray direction (source -> isocentre)
    double ex, ey;  // lateral direction (increasing bin index)
};

__global__ void k_fbp_views(dect_geometry g, ViewGeo *vg)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= g.n_views) return;
    const double th = g.start_rad + (double)v * (g.arc_rad / (double)g.n_views);
    const double c = cos(th), s = sin(th);
    vg[v] = ViewGeo{-c, -s, -s, c};
}

// One block per (view, image): cosine weight into shared memory, then the
// ramp filter for every bin, in FP64: the kernel cancels the projections'
// large mean (its taps sum to ~0), which would cost FP32 three digits.
// Shared memory: q[nb] and the odd taps hodd[j] = h(2 j + 1), j < nb / 2 + 1.
__global__ void __launch_bounds__(kFbpBlock) k_fbp_filter(const float *__restrict__ m, float *__restrict__ qf,
                                                       dect_geometry g)
{
    const int nb = g.n_bins, v = blockIdx.x, img = blockIdx.y;
    extern __shared__ double sm[];
    double *q = sm, *hodd = sm + nb;
    const double scale = g.sod_mm / g.sdd_mm;
    const double ds = g.pitch_mm * scale;
    const int64_t row = ((int64_t)img * g.n_views + v) * nb;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        const double u = ((double)b - 0.5 * (double)(nb - 1)) * g.pitch_mm + g.det_offset_mm;
        const double sb = u * scale;
        q[b] = (double)m[row + b] * (g.sod_mm / sqrt(g.sod_mm * g.sod_mm + sb * sb));
    }
    const int nodd = nb / 2 + 1;
    const double pi = 3.14159265358979323846;
    for (int j = threadIdx.x; j < nodd; j += blockDim.x) {
        const double k = 2.0 * j + 1.0;
        hodd[j] = -1.0 / (pi * pi * k * k * ds * ds);
    }
    __syncthreads();
    const double h0 = 1.0 / (4.0 * ds * ds);
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        // taps at odd distances 2 j + 1 on both sides, farthest first
        const int jmax = max(b, nb - 1 - b) / 2;  // 2 jmax + 1 reaches past the farther end
        double acc = 0.0;
        for (int j = jmax; j >= 0; --j) {
            const int d = 2 * j + 1;
            double pair = 0.0;
            if (b - d >= 0) pair += q[b - d];
            if (b + d < nb) pair += q[b + d];
            acc = fma(hodd[j], pair, acc);
        }
        acc = fma(h0, q[b], acc);
        qf[row + b] = (float)(ds * acc);
    }
}

// One thread per pixel and group of kFbpImgs images.
__global__ void __launch_bounds__(kFbpBlock) k_fbp_bp(const float *__restrict__ qf, float *__restrict__ x,
                                                   const ViewGeo *__restrict__ vg, dect_geometry g, int batch)
{
    const int n = g.n, nv = g.n_views, nb = g.n_bins;
    const int64_t N = (int64_t)n * n;
    const int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int img0 = blockIdx.y * kFbpImgs;
    if (pix >= N) return;
    const int i = (int)(pix / n), j = (int)(pix % n);
    // the bin coordinate t reaches n_bins - 1: it is formed in FP64 so that
    // its rounding does not move the interpolation weights
    const double lo = -0.5 * (double)n * g.pixel_mm;
    const double px = lo + ((double)j + 0.5) * g.pixel_mm;  // x: column
    const double py = lo + ((double)i + 0.5) * g.pixel_mm;  // y: row
    const double scale = g.sod_mm / g.sdd_mm;
    const double sod = g.sod_mm;
    const double s0 = (-0.5 * (double)(nb - 1) * g.pitch_mm + g.det_offset_mm) * scale;
    const double inv_ds = 1.0 / (g.pitch_mm * scale);
    const double half_dth = 0.5 * g.arc_rad / (double)nv;
    const double tmax = (double)(nb - 1);
    float acc[kFbpImgs];
#pragma unroll
    for (int k = 0; k < kFbpImgs; ++k) acc[k] = 0.f;
    for (int v = 0; v < nv; ++v) {
        const ViewGeo G = vg[v];
        const double L = sod + px * G.cx + py * G.cy;
        const double r = sod / L;
        const double t = ((px * G.ex + py * G.ey) * r - s0) * inv_ds;
        if (!(t >= 0.0 && t <= tmax)) continue;
        int b0 = (int)floor(t);
        if (b0 > nb - 2) b0 = nb - 2;
        if (!DECT_IDX_OK(b0, nb - 1, CHK_FBP_BIN)) b0 = 0;
        const float w = (float)(t - (double)b0);
        const float wt = (float)(half_dth * r * r);
#pragma unroll
        for (int k = 0; k < kFbpImgs; ++k) {
            const int img = img0 + k;
            if (img < batch) {
                const float *row = qf + ((int64_t)img * nv + v) * nb;
                const float val = fmaf(w, __ldg(row + b0 + 1), (1.f - w) * __ldg(row + b0));
                acc[k] = fmaf(wt, val, acc[k]);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < kFbpImgs; ++k)
        if (img0 + k < batch) x[(int64_t)(img0 + k) * N + pix] = acc[k];
}

}  // namespace
}  // namespace dect

using namespace dect;

extern "C" dect_status dect_fbp(const dect_plan *plan, const float *m, float *x, int batch, dect_stream stream)
{
    if (!plan || batch < 0 || plan->nz > 0) return DECT_ERR_INVALID_ARG;  // fan-beam plans only
    if (batch == 0) return DECT_OK;
    if (!m || !x) return DECT_ERR_INVALID_ARG;
    const dect_geometry &g = plan->g;
    if (std::fabs(g.arc_rad - 6.283185307179586) > 1e-9) {
        set_error_text("dect_fbp: the fan-beam FBP needs a full 360-degree scan (arc_rad = 2 pi)");
        return DECT_ERR_INVALID_ARG;
    }
    if (g.n_bins < 2) {
        set_error_text("dect_fbp: at least 2 detector bins");
        return DECT_ERR_INVALID_ARG;
    }
    const size_t smem = sizeof(double) * ((size_t)g.n_bins + (size_t)(g.n_bins / 2 + 1));
    if (smem > 200 * 1024) {
        set_error_text("dect_fbp: too many detector bins for the shared-memory filter");
        return DECT_ERR_INVALID_ARG;
    }
    DECT_CUDA(cudaSetDevice(plan->device));
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nq = (size_t)batch * g.n_views * g.n_bins;
    float *qf = nullptr;
    ViewGeo *vg = nullptr;
    DECT_CUDA(cudaMallocAsync((void **)&qf, sizeof(float) * nq, s));
    cudaError_t e = cudaMallocAsync((void **)&vg, sizeof(ViewGeo) * g.n_views, s);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fbp_filter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   200 * 1024);
    if (e == cudaSuccess) {
        k_fbp_views<<<(g.n_views + 255) / 256, 256, 0, s>>>(g, vg);
        k_fbp_filter<<<dim3(g.n_views, batch), kFbpBlock, smem, s>>>(m, qf, g);
        const int64_t N = (int64_t)g.n * g.n;
        k_fbp_bp<<<dim3((unsigned)((N + kFbpBlock - 1) / kFbpBlock), (batch + kFbpImgs - 1) / kFbpImgs),
                   kFbpBlock, 0, s>>>(qf, x, vg, g, batch);
        e = cudaGetLastError();
        count_launches(3);
    }
    if (vg) cudaFreeAsync(vg, s);
    cudaFreeAsync(qf, s);
    if (e != cudaSuccess) {
        set_error("dect_fbp", e);
        return e == cudaErrorMemoryAllocation ? DECT_ERR_OOM : DECT_ERR_CUDA;
    }
    return DECT_OK;
}
