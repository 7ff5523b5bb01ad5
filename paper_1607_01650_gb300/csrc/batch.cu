// On-the-fly Siddon projectors and the multi-slice ADM-TV (Eq. (3)-(10))
// over slices of uneven size and view count.
//
// Projector without a stored table.  Element a_ij of A (Eq. (1)) is the
// length of ray i inside pixel j (Siddon's method, ref. [42]: the pieces of
// the ray between consecutive grid-line crossings, each given to the pixel
// that holds it).  Here one device function, `chord`, computes it from the
// ray's parameters and the pixel's four grid lines: with the ray written as
// P + t d (P its point closest to the rotation axis, d its unit direction,
// t in mm), each grid line x = X0 + k px (y likewise) is crossed at
// t = (X0 + k px - P_x) / d_x, and the chord is the overlap of the ray's x
// and y slabs of the pixel.  The forward projector walks each ray through
// the pixels it crosses (the next pixel is the neighbour across the nearer
// of the current pixel's exit lines) and sums chord * x; the adjoint takes
// each pixel, finds for every view the bins whose rays can cross it (the
// detector interval spanned by the pixel's corners seen from the source)
// and sums chord * y.  Both call `chord` with the same operands, so A^T is
// the exact transpose of A (the same FP32 element in both).  A pixel whose
// corner a ray only grazes may be skipped by the walk: its chord is at the
// rounding level.  Crossing parameters are FP32 (t is measured from the
// point nearest the axis, so |t| <= half the image diagonal); the ray and
// view parameters are computed in FP64 and stored in FP32.
//
// The multi-slice ADM also runs on the plans' stored tables instead
// (dect_adm_tv_batch_ex with DECT_PROJ_TABLE): a warp per ray of the
// ray-major table for A, a warp per pixel of the pixel-major table for A^T
// (the row kernels of the single-plan ADM at two channels).
//
// Multi-slice ADM.  Each slice (both energies interleaved, [pixel][2])
// keeps its own state and scalars; one launch per ADM phase covers every
// running slice: a block map assigns blocks to (slice, part), and each
// slice's last block (a ticket per slice) reduces that slice's block
// partials in a fixed order and, in the forward phase, forms the slice's
// step and stopping test in FP64.  Slices whose channels have all stopped
// leave the block map at the next host check.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "dect_internal.cuh"
#include "kernels.cuh"

namespace dect {
namespace {

// ---------------------------------------------------------------------------
// Geometry and the chord of a ray through a pixel
// ---------------------------------------------------------------------------
struct OtfGrid {
    int n;
    float x0;  // first grid line, -n px / 2
    float px;
};

__device__ __forceinline__ float grid_line(const OtfGrid &g, int k) { return __fmaf_rn((float)k, g.px, g.x0); }

// crossing parameter of grid line `line` for a ray through p with 1/d = inv
__device__ __forceinline__ float cross_t(float line, float p, float inv) { return __fmul_rn(__fsub_rn(line, p), inv); }

// Length of the ray (R = (P_x, P_y, d_x, d_y), I = (1/d_x, 1/d_y)) inside
// the pixel bounded by grid lines x = lx0, lx1 and y = ly0, ly1 (values of
// grid_line): the overlap of its two slabs.
__device__ __forceinline__ float chord(float lx0, float lx1, float ly0, float ly1, const float4 &R, const float2 &I)
{
    const float xa = cross_t(lx0, R.x, I.x), xb = cross_t(lx1, R.x, I.x);
    const float ya = cross_t(ly0, R.y, I.y), yb = cross_t(ly1, R.y, I.y);
    const float tmin = fmaxf(fminf(xa, xb), fminf(ya, yb)), tmax = fminf(fmaxf(xa, xb), fmaxf(ya, yb));
    return fmaxf(__fsub_rn(tmax, tmin), 0.f);
}

// sum over the ray's pixels of chord * img[pixel] (two interleaved images).
// The walk is branch-free, so that the 32 rays of a warp advance together,
// and runs in chunks of W steps: each step evaluates the chord of the
// current pixel from its four crossing parameters (the same values `chord`
// computes) and moves across the nearer exit line (both candidate next
// crossings computed, the right one kept); then the chunk's W image loads
// are issued together and summed.  A ray has left the image once a step
// would leave the grid; the rest of its last chunk has zero length.
__device__ float2 ray_sum(const OtfGrid &g, const float4 &R, const float2 &I, const float2 *__restrict__ img)
{
    constexpr int W = 8;
    float2 acc = make_float2(0.f, 0.f);
    const int n = g.n;
    const float x0 = cross_t(grid_line(g, 0), R.x, I.x), xn = cross_t(grid_line(g, n), R.x, I.x);
    const float y0 = cross_t(grid_line(g, 0), R.y, I.y), yn = cross_t(grid_line(g, n), R.y, I.y);
    const float tin = fmaxf(fminf(x0, xn), fminf(y0, yn)), tout = fminf(fmaxf(x0, xn), fmaxf(y0, yn));
    if (!(tin < tout)) return acc;
    // first pixel: the one holding the entry point (a neighbour after
    // rounding is harmless: its chord is ~0 and the walk moves on)
    const float ipx = 1.f / g.px;
    int j = (int)floorf((__fmaf_rn(tin, R.z, R.x) - g.x0) * ipx);
    int i = (int)floorf((__fmaf_rn(tin, R.w, R.y) - g.x0) * ipx);
    j = min(max(j, 0), n - 1);
    i = min(max(i, 0), n - 1);
    const int sj = R.z > 0.f ? 1 : -1, si = R.w > 0.f ? 1 : -1;
    const int oj = sj > 0 ? 1 : 0, oi = si > 0 ? 1 : 0;  // the exit line of a pixel: j + oj, i + oi
    float xa = cross_t(grid_line(g, j), R.x, I.x), xb = cross_t(grid_line(g, j + 1), R.x, I.x);
    float ya = cross_t(grid_line(g, i), R.y, I.y), yb = cross_t(grid_line(g, i + 1), R.y, I.y);
    bool live = true;
    // every step moves i or j one pixel in a fixed direction: the ray leaves
    // within 2n steps
    for (int chunk = 0; chunk <= (2 * n + 2) / W; ++chunk) {
        int64_t idx[W];
        float len[W];
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const float tmin = fmaxf(fminf(xa, xb), fminf(ya, yb)), tmax = fminf(fmaxf(xa, xb), fmaxf(ya, yb));
            len[w] = live ? fmaxf(__fsub_rn(tmax, tmin), 0.f) : 0.f;
            idx[w] = (int64_t)i * n + j;
            const bool xs = fmaxf(xa, xb) < fmaxf(ya, yb);
            const int jn = xs ? j + sj : j, in = xs ? i : i + si;
            const bool stay = live && jn >= 0 && jn < n && in >= 0 && in < n;
            const float nx = cross_t(grid_line(g, jn + oj), R.x, I.x);
            const float ny = cross_t(grid_line(g, in + oi), R.y, I.y);
            const float xa2 = sj > 0 ? xb : nx, xb2 = sj > 0 ? nx : xa;
            const float ya2 = si > 0 ? yb : ny, yb2 = si > 0 ? ny : ya;
            const bool ux = stay && xs, uy = stay && !xs;
            xa = ux ? xa2 : xa;
            xb = ux ? xb2 : xb;
            ya = uy ? ya2 : ya;
            yb = uy ? yb2 : yb;
            j = stay ? jn : j;
            i = stay ? in : i;
            live = stay;
        }
        float2 v[W];
#pragma unroll
        for (int w = 0; w < W; ++w) {
            if (!DECT_IDX_OK(idx[w], (int64_t)n * n, CHK_OTF_WALK)) idx[w] = 0;
            v[w] = __ldg(img + idx[w]);
        }
#pragma unroll
        for (int w = 0; w < W; ++w) {
            acc.x = fmaf(len[w], v[w].x, acc.x);
            acc.y = fmaf(len[w], v[w].y, acc.y);
        }
        if (!live) break;
    }
    return acc;
}

struct OtfGeom {
    OtfGrid g;
    int nv, nb;
    const float4 *ray;   // [nv * nb] (P_x, P_y, d_x, d_y)
    const float2 *inv;   // [nv * nb] (1/d_x, 1/d_y)
    const float4 *view;  // [nv] (S_x, S_y, e_u x, e_u y)
    const float4 *view2; // [nv] (e_w x, e_w y, SDD / pitch, (nb - 1) / 2 - offset / pitch)
};

// sum over the rays crossing pixel (i, j) of chord * sino[ray] (two
// interleaved sinograms), views in order, bins increasing
__device__ float2 pixel_sum(const OtfGeom &G, int i, int j, const float2 *__restrict__ sino)
{
    float2 acc = make_float2(0.f, 0.f);
    const float lx0 = grid_line(G.g, j), lx1 = grid_line(G.g, j + 1);
    const float ly0 = grid_line(G.g, i), ly1 = grid_line(G.g, i + 1);
    for (int v = 0; v < G.nv; ++v) {
        const float4 V = __ldg(G.view + v), W = __ldg(G.view2 + v);
        // detector coordinate (in bins) of the four corners seen from the
        // source: u and w are sums of an x and a y term per corner
        const float ax0 = lx0 - V.x, ax1 = lx1 - V.x, ay0 = ly0 - V.y, ay1 = ly1 - V.y;
        const float ux0 = ax0 * V.z, ux1 = ax1 * V.z, uy0 = ay0 * V.w, uy1 = ay1 * V.w;
        const float wx0 = ax0 * W.x, wx1 = ax1 * W.x, wy0 = ay0 * W.y, wy1 = ay1 * W.y;
        const float b00 = __fdividef(ux0 + uy0, wx0 + wy0), b10 = __fdividef(ux1 + uy0, wx1 + wy0);
        const float b01 = __fdividef(ux0 + uy1, wx0 + wy1), b11 = __fdividef(ux1 + uy1, wx1 + wy1);
        const float lo = fmaf(W.z, fminf(fminf(b00, b10), fminf(b01, b11)), W.w);
        const float hi = fmaf(W.z, fmaxf(fmaxf(b00, b10), fmaxf(b01, b11)), W.w);
        const int b0 = max((int)ceilf(lo - 1e-3f), 0), b1 = min((int)floorf(hi + 1e-3f), G.nb - 1);
        // candidates two at a time, the second one's loads from a valid ray
        // (b0) and its length zeroed when it is past b1
        for (int b = b0; b <= b1; b += 2) {
            int64_t r0 = (int64_t)v * G.nb + b;
            const bool two = b + 1 <= b1;
            int64_t r1 = two ? r0 + 1 : r0;
            if (!DECT_IDX_OK(r0, (int64_t)G.nv * G.nb, CHK_OTF_RAY)) r0 = 0;
            if (!DECT_IDX_OK(r1, (int64_t)G.nv * G.nb, CHK_OTF_RAY)) r1 = 0;
            const float4 R0 = __ldg(G.ray + r0), R1 = __ldg(G.ray + r1);
            const float2 I0 = __ldg(G.inv + r0), I1 = __ldg(G.inv + r1);
            const float2 y0 = __ldg(sino + r0), y1 = __ldg(sino + r1);
            const float l0 = chord(lx0, lx1, ly0, ly1, R0, I0);
            const float l1 = two ? chord(lx0, lx1, ly0, ly1, R1, I1) : 0.f;
            acc.x = fmaf(l0, y0.x, acc.x);
            acc.y = fmaf(l0, y0.y, acc.y);
            acc.x = fmaf(l1, y1.x, acc.x);
            acc.y = fmaf(l1, y1.y, acc.y);
        }
    }
    return acc;
}

OtfGeom otf_geom(const dect_plan *P)
{
    OtfGeom G;
    G.g.n = P->n;
    G.g.px = (float)P->g.pixel_mm;
    G.g.x0 = (float)(-0.5 * P->n * P->g.pixel_mm);
    G.nv = P->nv;
    G.nb = P->nb;
    G.ray = P->otf_ray;
    G.inv = P->otf_inv;
    G.view = P->otf_view;
    G.view2 = P->otf_view2;
    return G;
}

// ---------------------------------------------------------------------------
// Standalone operators on interleaved pairs of images
// ---------------------------------------------------------------------------
constexpr int kOtfBlock = 256;
constexpr int kOtfTile = 16;  // adjoint: 16 x 16 pixel tiles per block

__global__ void __launch_bounds__(kOtfBlock) k_otf_project(OtfGeom G, const float2 *__restrict__ img,
                                                          float2 *__restrict__ out)
{
    const int64_t ray = (int64_t)blockIdx.x * kOtfBlock + threadIdx.x;
    if (ray >= (int64_t)G.nv * G.nb) return;
    out[ray] = ray_sum(G.g, __ldg(G.ray + ray), __ldg(G.inv + ray), img);
}

__device__ __forceinline__ bool tile_pixel(int n, int tile, int &i, int &j)
{
    const int tx = (n + kOtfTile - 1) / kOtfTile;
    i = (tile / tx) * kOtfTile + threadIdx.x / kOtfTile;
    j = (tile % tx) * kOtfTile + threadIdx.x % kOtfTile;
    return i < n && j < n;
}

__global__ void __launch_bounds__(kOtfBlock) k_otf_backproject(OtfGeom G, const float2 *__restrict__ sino,
                                                              float2 *__restrict__ out)
{
    int i, j;
    if (!tile_pixel(G.g.n, blockIdx.x, i, j)) return;
    out[(int64_t)i * G.g.n + j] = pixel_sum(G, i, j, sino);
}

// planar images a, b (b may be null: zeros) -> interleaved pairs, and back
__global__ void k_pair(const float *__restrict__ a, const float *__restrict__ b, float2 *__restrict__ out,
                       int64_t len)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < len) out[t] = make_float2(a[t], b ? b[t] : 0.f);
}
__global__ void k_unpair(const float2 *__restrict__ in, float *__restrict__ a, float *__restrict__ b, int64_t len)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= len) return;
    const float2 v = in[t];
    a[t] = v.x;
    if (b) b[t] = v.y;
}

unsigned blocks_of(int64_t n, int per) { return (unsigned)((n + per - 1) / per); }

cudaError_t otf_operator(const dect_plan *P, const float *src, float *dst, int batch, bool adjoint,
                         cudaStream_t s)
{
    cudaError_t e = otf_setup(P, s);
    if (e != cudaSuccess) return e;
    const int64_t rin = adjoint ? P->M : P->N, rout = adjoint ? P->N : P->M;
    float2 *buf = nullptr;
    e = cudaMallocAsync((void **)&buf, sizeof(float2) * (size_t)(rin + rout), s);
    if (e != cudaSuccess) return e;
    float2 *in = buf, *out = buf + rin;
    const OtfGeom G = otf_geom(P);
    const int tiles = ((P->n + kOtfTile - 1) / kOtfTile) * ((P->n + kOtfTile - 1) / kOtfTile);
    for (int k = 0; k < batch && e == cudaSuccess; k += 2) {
        const bool two = k + 1 < batch;
        k_pair<<<blocks_of(rin, 256), 256, 0, s>>>(src + k * rin, two ? src + (k + 1) * rin : nullptr, in, rin);
        if (adjoint)
            k_otf_backproject<<<tiles, kOtfBlock, 0, s>>>(G, in, out);
        else
            k_otf_project<<<blocks_of(rout, kOtfBlock), kOtfBlock, 0, s>>>(G, in, out);
        k_unpair<<<blocks_of(rout, 256), 256, 0, s>>>(out, dst + k * rout, two ? dst + (k + 1) * rout : nullptr, rout);
        count_launches(3);
        e = cudaGetLastError();
    }
    cudaError_t f = cudaFreeAsync(buf, s);
    return e != cudaSuccess ? e : f;
}

// ---------------------------------------------------------------------------
// Multi-slice ADM
// ---------------------------------------------------------------------------
enum { PH_TV = 0, PH_BWD = 1, PH_FWD = 2, PH_COUNT = 3 };
// stored-table projector: a warp per ray of the ray-major table (A) and per
// pixel of the pixel-major table (A^T, the warps of a block taking turns
// over the block's 16 x 16 tile, whose pixels share sinogram lines in L1)
constexpr int kTabRaysPerBlock = kOtfBlock / 32;
enum { Q_TV = 0, Q_RR = 1, Q_DD = 2, Q_QQ = 3, Q_GG = 4, Q_COUNT = 5 };

struct SliceDesc {
    OtfGeom G;
    int64_t N, M;
    float2 *f[2], *Gr, *lam, *z, *p, *r, *q;  // lam, z, p: [2][N] (two gradient components)
    const float *m;                            // [2][M] measured line integrals (caller's)
    float *x;                                  // [2][N] images (caller's)
    float beta[2];
    int blk0[PH_COUNT], nblk[PH_COUNT];        // this slice's blocks in each phase's launch
    // stored-table projector: the plan's ray-major and pixel-major tables
    const int64_t *rowptr, *colptr;
    const Entry *ent, *tent;
};

struct BatchDev {
    double *alpha, *c_prev, *phi_prev, *rel;  // [S][2]
    double *red;                               // [S][Q_COUNT][2]
    double *part;                              // [max blocks][2][2] block partials
    int *iters, *conv, *active;                // [S][2]
    int *k;                                    // [S] iteration counter
    unsigned *ctr;                             // [S][PH_COUNT + 1] last-block tickets
    int *bad;
};

struct BatchConst {
    float mu, rho, xi;
    double mu_d, rho_d, tol;
    int rule, xi_is_rho, nonneg, joint;
};

// Sum K two-channel values over the block in a fixed order and write the
// block's partial; the last block of the slice (ticket on *ctr) sums the
// slice's partials in block order, hands every thread of that block the
// totals in out[K * 2] (quantity-major) and returns true.
template <int K>
__device__ bool slice_reduce(float (&v)[K][2], double *part, int blk0, int nblk, unsigned *ctr, double *out)
{
    __shared__ double ws[kOtfBlock / 32][K][2];
    __shared__ double tot[K * 2];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < K; ++q)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            float a = v[q][c];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
            if (lane == 0) ws[warp][q][c] = (double)a;
        }
    __syncthreads();
    if (threadIdx.x < 2 * K) {
        const int q = threadIdx.x / 2, c = threadIdx.x % 2;
        double a = 0.0;
        for (int w = 0; w < kOtfBlock / 32; ++w) a += ws[w][q][c];
        part[((size_t)blockIdx.x * K + q) * 2 + c] = a;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ctr, 1u) == (unsigned)nblk - 1;
    __syncthreads();
    if (!last) return false;
    __threadfence();
    // one warp per (quantity, channel): lanes sum fixed strides, then a fixed butterfly
    if (warp < 2 * K) {
        const int q = warp / 2, c = warp % 2;
        double a = 0.0;
        for (int b = lane; b < nblk; b += 32) a += __ldcg(&part[((size_t)(blk0 + b) * K + q) * 2 + c]);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
        if (lane == 0) tot[q * 2 + c] = a;
    }
    if (threadIdx.x == 0) *ctr = 0u;
    __syncthreads();
#pragma unroll
    for (int t = 0; t < K * 2; ++t) out[t] = tot[t];
    return true;
}

__device__ __forceinline__ float step_px(float f, float a, float g, bool clamp)
{
    const float v = fmaf(-a, g, f);
    return clamp && v < 0.f ? 0.f : v;
}

// Start of an iteration for every slice in the map: f^k = f^{k-1} - alpha G
// (projected onto f >= 0 with nonneg), r^k = r^{k-1} - alpha q, the lambda
// step, the z-shrink of Eq. (8) and p = rho (grad f - z) - lambda; TV and
// |r|^2 per channel.  final_pass: only the step and the two norms.
__global__ void __launch_bounds__(kOtfBlock) k_tv_m(const SliceDesc *__restrict__ SD, const int *__restrict__ bmap,
                                                   BatchDev B, BatchConst C, int par, int final_pass)
{
    const int s = bmap[blockIdx.x];
    const SliceDesc &d = SD[s];
    const int n = d.G.g.n, lb = blockIdx.x - d.blk0[PH_TV], nbk = d.nblk[PH_TV];
    const int k = B.k[s];
    const float a0 = (float)B.alpha[2 * s], a1 = (float)B.alpha[2 * s + 1];
    const bool clamp = C.nonneg && k > 0;
    const float inv_rho = 1.0f / C.rho;
    float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
    const float2 *fin = d.f[par];
    float2 *fout = d.f[1 - par];
    const int64_t N = d.N;
    auto upd = [&](int64_t q) {
        const float2 f = fin[q], g = d.Gr[q];
        return make_float2(step_px(f.x, a0, g.x, clamp), step_px(f.y, a1, g.y, clamp));
    };
    int i, j;
    if (tile_pixel(n, lb, i, j)) {
        const int64_t q = (int64_t)i * n + j;
        const float2 fc = upd(q), fu = i > 0 ? upd(q - n) : fc, fl = j > 0 ? upd(q - 1) : fc;
        fout[q] = fc;
        const float d0[2] = {fc.x - fu.x, fc.y - fu.y};  // Eq. (2), 0 on the first row
        const float d1[2] = {fc.x - fl.x, fc.y - fl.y};  // Eq. (2), 0 on the first column
        if (C.joint)
            acc[0][0] += sqrtf(d0[0] * d0[0] + d1[0] * d1[0] + d0[1] * d0[1] + d1[1] * d1[1]);
        else {
            acc[0][0] += sqrtf(d0[0] * d0[0] + d1[0] * d1[0]);
            acc[0][1] += sqrtf(d0[1] * d0[1] + d1[1] * d1[1]);
        }
        if (!final_pass) {
            float l0[2], l1[2], z0[2], z1[2];
            const float2 gc = d.Gr[q], gu = i > 0 ? d.Gr[q - n] : gc, gl = j > 0 ? d.Gr[q - 1] : gc;
            const float gcv[2] = {gc.x, gc.y}, guv[2] = {gu.x, gu.y}, glv[2] = {gl.x, gl.y};
            const float av[2] = {a0, a1};
            const float2 pl0 = (C.xi_is_rho ? d.p : d.lam)[q], pl1 = (C.xi_is_rho ? d.p : d.lam)[N + q];
            const float pl0v[2] = {pl0.x, pl0.y}, pl1v[2] = {pl1.x, pl1.y};
            float2 zo0 = make_float2(0.f, 0.f), zo1 = zo0;
            if (!C.xi_is_rho && k > 0) {
                zo0 = d.z[q];
                zo1 = d.z[N + q];
            }
            const float zo0v[2] = {zo0.x, zo0.y}, zo1v[2] = {zo1.x, zo1.y};
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                if (C.xi_is_rho) {
                    // lambda^k = xi alpha^{k-1} grad G^{k-1} - p^{k-1} (Eq. (7) with xi = rho)
                    l0[c] = 0.f;
                    l1[c] = 0.f;
                    if (k > 0) {
                        const float dg0 = i > 0 ? gcv[c] - guv[c] : 0.f, dg1 = j > 0 ? gcv[c] - glv[c] : 0.f;
                        l0[c] = C.xi * av[c] * dg0 - pl0v[c];
                        l1[c] = C.xi * av[c] * dg1 - pl1v[c];
                    }
                } else {
                    l0[c] = pl0v[c];
                    l1[c] = pl1v[c];
                    if (k > 0) {  // lambda^k = lambda^{k-1} - xi (grad f^k - z^k), Eq. (7)
                        l0[c] -= C.xi * (d0[c] - zo0v[c]);
                        l1[c] -= C.xi * (d1[c] - zo1v[c]);
                    }
                }
            }
            if (C.joint) {
                const float w0 = d0[0] - l0[0] * inv_rho, w1 = d1[0] - l1[0] * inv_rho;
                const float w2 = d0[1] - l0[1] * inv_rho, w3 = d1[1] - l1[1] * inv_rho;
                const float nrm = sqrtf(w0 * w0 + w1 * w1 + w2 * w2 + w3 * w3), sh = nrm - inv_rho;
                const float kk = (sh > 0.f && nrm > 0.f) ? sh / nrm : 0.f;
                z0[0] = kk * w0;
                z1[0] = kk * w1;
                z0[1] = kk * w2;
                z1[1] = kk * w3;
            } else {
#pragma unroll
                for (int c = 0; c < 2; ++c) {  // Eq. (8), w / |w| for the sign of a 2-vector
                    const float w0 = d0[c] - l0[c] * inv_rho, w1 = d1[c] - l1[c] * inv_rho;
                    const float nrm = sqrtf(w0 * w0 + w1 * w1), sh = nrm - inv_rho;
                    const float kk = (sh > 0.f && nrm > 0.f) ? sh / nrm : 0.f;
                    z0[c] = kk * w0;
                    z1[c] = kk * w1;
                }
            }
            float p0[2], p1[2];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                p0[c] = C.rho * (d0[c] - z0[c]) - l0[c];
                p1[c] = C.rho * (d1[c] - z1[c]) - l1[c];
            }
            if (!C.xi_is_rho) {
                d.lam[q] = make_float2(l0[0], l0[1]);
                d.lam[N + q] = make_float2(l1[0], l1[1]);
                d.z[q] = make_float2(z0[0], z0[1]);
                d.z[N + q] = make_float2(z1[0], z1[1]);
            }
            d.p[q] = make_float2(p0[0], p0[1]);
            d.p[N + q] = make_float2(p1[0], p1[1]);
        }
    }
    if (!C.nonneg) {  // r^k = r^{k-1} - alpha q (with the projection r is rebuilt by the forward phase)
        for (int64_t t = (int64_t)lb * kOtfBlock + threadIdx.x; t < d.M; t += (int64_t)nbk * kOtfBlock) {
            float2 rv = d.r[t];
            const float2 qv = d.q[t];
            rv.x = fmaf(-a0, qv.x, rv.x);
            rv.y = fmaf(-a1, qv.y, rv.y);
            d.r[t] = rv;
            acc[1][0] = fmaf(rv.x, rv.x, acc[1][0]);
            acc[1][1] = fmaf(rv.y, rv.y, acc[1][1]);
        }
    }
    double out[4];
    if (slice_reduce<2>(acc, B.part, d.blk0[PH_TV], nbk, B.ctr + s * (PH_COUNT + 1) + PH_TV, out) &&
        threadIdx.x == 0) {
        B.red[(s * Q_COUNT + Q_TV) * 2 + 0] = out[0];
        B.red[(s * Q_COUNT + Q_TV) * 2 + 1] = out[1];
        if (!C.nonneg) {
            B.red[(s * Q_COUNT + Q_RR) * 2 + 0] = out[2];
            B.red[(s * Q_COUNT + Q_RR) * 2 + 1] = out[3];
        }
    }
}

// G = mu A^T r + grad^T p of pixel (i, j), given a = (A^T r)(i, j); adds |G|^2.
__device__ __forceinline__ void bwd_finish(const SliceDesc &d, const BatchConst &C, int i, int j, float2 a,
                                           float (&acc)[1][2])
{
    const int n = d.G.g.n;
    const int64_t q = (int64_t)i * n + j, N = d.N;
    const float2 p0 = d.p[q], p1 = d.p[N + q];
    const float2 pd = i + 1 < n ? d.p[q + n] : make_float2(0.f, 0.f);
    const float2 pr = j + 1 < n ? d.p[N + q + 1] : make_float2(0.f, 0.f);
    float2 g;
    g.x = fmaf(C.mu, a.x, (i > 0 ? p0.x : 0.f) - pd.x + (j > 0 ? p1.x : 0.f) - pr.x);
    g.y = fmaf(C.mu, a.y, (i > 0 ? p0.y : 0.f) - pd.y + (j > 0 ? p1.y : 0.f) - pr.y);
    d.Gr[q] = g;
    acc[0][0] += g.x * g.x;
    acc[0][1] += g.y * g.y;
}

// G = mu A^T r + grad^T p per pixel of the block's 16 x 16 tile; |G|^2 per
// channel.  TABLE: A^T r from the pixel-major table (a warp per pixel, the
// block's warps taking the tile's pixels in turn); otherwise on the fly (a
// thread per pixel).
template <bool TABLE>
__global__ void __launch_bounds__(kOtfBlock) k_bwd_m(const SliceDesc *__restrict__ SD, const int *__restrict__ bmap,
                                                    BatchDev B, BatchConst C)
{
    const int s = bmap[blockIdx.x];
    const SliceDesc &d = SD[s];
    const int n = d.G.g.n, lb = blockIdx.x - d.blk0[PH_BWD];
    float acc[1][2] = {{0.f, 0.f}};
    if constexpr (TABLE) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const int tx = (n + kOtfTile - 1) / kOtfTile;
        const int i0 = (lb / tx) * kOtfTile, j0 = (lb % tx) * kOtfTile;
        for (int k = warp; k < kOtfTile * kOtfTile; k += kOtfBlock / 32) {
            const int i = i0 + k / kOtfTile, j = j0 + k % kOtfTile;
            const bool ok = i < n && j < n;
            int64_t b = 0, e = 0;
            if (ok) {
                b = d.colptr[(int64_t)i * n + j];
                e = d.colptr[(int64_t)i * n + j + 1];
            }
            const Vec<2> a = row_dot<2, 32, true>(d.tent, b, e, reinterpret_cast<const float *>(d.r), d.M, lane,
                                                 CHK_GATHER_AT);
            if (ok && lane == 0) bwd_finish(d, C, i, j, make_float2(a.v[0], a.v[1]), acc);
        }
    } else {
        int i, j;
        if (tile_pixel(n, lb, i, j)) bwd_finish(d, C, i, j, pixel_sum(d.G, i, j, d.r), acc);
    }
    double out[2];
    if (slice_reduce<1>(acc, B.part, d.blk0[PH_BWD], d.nblk[PH_BWD], B.ctr + s * (PH_COUNT + 1) + PH_BWD, out) &&
        threadIdx.x == 0) {
        B.red[(s * Q_COUNT + Q_GG) * 2 + 0] = out[0];
        B.red[(s * Q_COUNT + Q_GG) * 2 + 1] = out[1];
    }
}

// Step and stopping test of slice s in FP64 (its last forward block).
__device__ void slice_finish(int s, const BatchConst &C, const BatchDev &B)
{
    const int k = B.k[s];
    const int span = C.joint ? 2 : 1;
    if (threadIdx.x < 2 && threadIdx.x % span == 0) {
        const int c = threadIdx.x, ch = 2 * s + c;
        auto sum = [&](int qn) {
            double v = B.red[(s * Q_COUNT + qn) * 2 + c];
            if (span == 2) v += B.red[(s * Q_COUNT + qn) * 2 + c + 1];
            return v;
        };
        double alpha = 0.0;
        if (B.active[ch]) {
            const double phi = sum(Q_TV) + 0.5 * C.mu_d * sum(Q_RR);
            if (!isfinite(phi)) atomicOr(B.bad, 1);
            bool stop = false;
            if (k > 0) {
                const double prev = B.phi_prev[ch];
                const double rel = prev > 0.0 ? fabs(phi - prev) / prev : 0.0;
                B.rel[ch] = rel;
                if (C.tol > 0.0 && rel < C.tol) stop = true;
            }
            if (stop) {
                B.active[ch] = 0;
                B.conv[ch] = 1;
                B.iters[ch] = k;
            } else {
                B.phi_prev[ch] = phi;
                const double gg = sum(Q_GG), qq = sum(Q_QQ), dd = sum(Q_DD);
                const double den = C.mu_d * qq + C.rho_d * dd;
                const double cst = den > 0.0 ? gg / den : 0.0;
                alpha = (C.rule == DECT_STEP_CAUCHY || k == 0) ? cst : B.c_prev[ch];
                B.c_prev[ch] = cst;
                B.iters[ch] = k + 1;
            }
        }
        B.alpha[ch] = alpha;
        if (span == 2) {
            B.alpha[ch + 1] = alpha;
            B.active[ch + 1] = B.active[ch];
            B.conv[ch + 1] = B.conv[ch];
            B.iters[ch + 1] = B.iters[ch];
            B.rel[ch + 1] = B.rel[ch];
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) B.k[s] = k + 1;
}

// MODE 1: |grad G|^2 over the slice's pixels, q = A G and |q|^2, then the
// slice's step.  MODE 0: r = A f - beta m.  MODE 2: the same and |r|^2
// (projected f-step).  MODE 3: |A f - beta m|^2 and |r - (A f - beta m)|^2
// (check of the carried residual, into QQ and GG).
// TABLE: q (or A f) from the ray-major table, a warp per ray; otherwise on
// the fly, a thread per ray.
template <int MODE, bool TABLE>
__global__ void __launch_bounds__(kOtfBlock) k_fwd_m(const SliceDesc *__restrict__ SD, const int *__restrict__ bmap,
                                                    BatchDev B, BatchConst C, int fsel)
{
    const int s = bmap[blockIdx.x];
    const SliceDesc &d = SD[s];
    const int n = d.G.g.n, lb = blockIdx.x - d.blk0[PH_FWD], nbk = d.nblk[PH_FWD];
    float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
    if (MODE == 1) {
        for (int64_t t = (int64_t)lb * kOtfBlock + threadIdx.x; t < d.N; t += (int64_t)nbk * kOtfBlock) {
            const int i = (int)(t / n), j = (int)(t % n);
            const float2 gc = d.Gr[t], gu = i > 0 ? d.Gr[t - n] : gc, gl = j > 0 ? d.Gr[t - 1] : gc;
            const float e0 = gc.x - gu.x, e1 = gc.x - gl.x, h0 = gc.y - gu.y, h1 = gc.y - gl.y;
            acc[0][0] += e0 * e0 + e1 * e1;
            acc[0][1] += h0 * h0 + h1 * h1;
        }
    }
    const float2 *src = MODE == 1 ? d.Gr : d.f[fsel];
    int64_t ray;
    float2 v = make_float2(0.f, 0.f);
    bool mine;  // this thread holds the ray's sum
    if constexpr (TABLE) {
        ray = (int64_t)lb * kTabRaysPerBlock + (threadIdx.x >> 5);
        int64_t b = 0, e = 0;
        if (ray < d.M) {
            b = d.rowptr[ray];
            e = d.rowptr[ray + 1];
        }
        const Vec<2> a = row_dot<2, 32, true>(d.ent, b, e, reinterpret_cast<const float *>(src), d.N,
                                             threadIdx.x & 31, CHK_GATHER_A);
        v = make_float2(a.v[0], a.v[1]);
        mine = ray < d.M && (threadIdx.x & 31) == 0;
    } else {
        ray = (int64_t)lb * kOtfBlock + threadIdx.x;
        mine = ray < d.M;
        if (mine) v = ray_sum(d.G.g, __ldg(d.G.ray + ray), __ldg(d.G.inv + ray), src);
    }
    if (mine) {
        if (MODE == 1) {
            d.q[ray] = v;
            acc[1][0] = v.x * v.x;
            acc[1][1] = v.y * v.y;
        } else {
            v.x -= d.beta[0] * d.m[ray];
            v.y -= d.beta[1] * d.m[d.M + ray];
            if (MODE == 0 || MODE == 2) d.r[ray] = v;
            if (MODE >= 2) {
                acc[0][0] = v.x * v.x;
                acc[0][1] = v.y * v.y;
            }
            if (MODE == 3) {
                const float2 rc = d.r[ray];
                acc[1][0] = (rc.x - v.x) * (rc.x - v.x);
                acc[1][1] = (rc.y - v.y) * (rc.y - v.y);
            }
        }
    }
    if (MODE == 0) return;
    double out[4];
    const bool last = slice_reduce<2>(acc, B.part, d.blk0[PH_FWD], nbk, B.ctr + s * (PH_COUNT + 1) + PH_FWD, out);
    if (!last) return;
    if (threadIdx.x == 0) {
        double *r = B.red + s * Q_COUNT * 2;
        if (MODE == 1) {
            r[Q_DD * 2] = out[0], r[Q_DD * 2 + 1] = out[1];
            r[Q_QQ * 2] = out[2], r[Q_QQ * 2 + 1] = out[3];
        } else if (MODE == 2) {
            r[Q_RR * 2] = out[0], r[Q_RR * 2 + 1] = out[1];
        } else {
            r[Q_QQ * 2] = out[0], r[Q_QQ * 2 + 1] = out[1];
            r[Q_GG * 2] = out[2], r[Q_GG * 2 + 1] = out[3];
        }
    }
    if (MODE == 1) {
        __syncthreads();
        slice_finish(s, C, B);
    }
}

// f = beta x (both energies of every slice in the map's TV phase) and back.
__global__ void k_pack_m(const SliceDesc *__restrict__ SD, const int *__restrict__ bmap, int to_state, int fsel)
{
    const int s = bmap[blockIdx.x];
    const SliceDesc &d = SD[s];
    int i, j;
    if (!tile_pixel(d.G.g.n, blockIdx.x - d.blk0[PH_TV], i, j)) return;
    const int64_t q = (int64_t)i * d.G.g.n + j;
    if (to_state)
        d.f[fsel][q] = make_float2(d.beta[0] * d.x[q], d.beta[1] * d.x[d.N + q]);
    else {
        const float2 v = d.f[fsel][q];
        d.x[q] = v.x / d.beta[0];
        d.x[d.N + q] = v.y / d.beta[1];
    }
}

}  // namespace

// Geometry of the on-the-fly projectors, FP64 on the host (the ray and view
// definitions of the plan), stored FP32 on the device.
cudaError_t otf_setup(const dect_plan *P, cudaStream_t s)
{
    if (P->otf_ray) return cudaSuccess;
    const dect_geometry &g = P->g;
    std::vector<float4> ray(P->M), view(P->nv), view2(P->nv);
    std::vector<float2> inv(P->M);
    for (int v = 0; v < P->nv; ++v) {
        const double th = g.start_rad + (double)v * (g.arc_rad / (double)P->nv);
        const double c = std::cos(th), sn = std::sin(th);
        const double sx = g.sod_mm * c, sy = g.sod_mm * sn;
        const double cx = (g.sod_mm - g.sdd_mm) * c, cy = (g.sod_mm - g.sdd_mm) * sn;
        // detector axis e_u = (-sin, cos); central direction e_w = (-cos, -sin)
        view[v] = make_float4((float)sx, (float)sy, (float)-sn, (float)c);
        view2[v] = make_float4((float)-c, (float)-sn, (float)(g.sdd_mm / g.pitch_mm),
                               (float)(0.5 * (double)(P->nb - 1) - g.det_offset_mm / g.pitch_mm));
        for (int b = 0; b < P->nb; ++b) {
            const double u = ((double)b - 0.5 * (double)(P->nb - 1)) * g.pitch_mm + g.det_offset_mm;
            const double ex = cx - u * sn, ey = cy + u * c;  // bin centre
            double dx = ex - sx, dy = ey - sy;
            const double L = std::sqrt(dx * dx + dy * dy);
            dx /= L;
            dy /= L;
            const double t0 = -(sx * dx + sy * dy);  // point of the ray nearest the axis
            const size_t r = (size_t)v * P->nb + b;
            ray[r] = make_float4((float)(sx + t0 * dx), (float)(sy + t0 * dy), (float)dx, (float)dy);
            inv[r] = make_float2((float)(1.0 / dx), (float)(1.0 / dy));
        }
    }
    cudaError_t e = cudaMalloc(&P->otf_ray, sizeof(float4) * P->M);
    if (e == cudaSuccess) e = cudaMalloc(&P->otf_inv, sizeof(float2) * P->M);
    if (e == cudaSuccess) e = cudaMalloc(&P->otf_view, sizeof(float4) * P->nv);
    if (e == cudaSuccess) e = cudaMalloc(&P->otf_view2, sizeof(float4) * P->nv);
    if (e == cudaSuccess) e = cudaMemcpyAsync(P->otf_ray, ray.data(), sizeof(float4) * P->M, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(P->otf_inv, inv.data(), sizeof(float2) * P->M, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(P->otf_view, view.data(), sizeof(float4) * P->nv, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(P->otf_view2, view2.data(), sizeof(float4) * P->nv, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaFree(P->otf_ray);
        cudaFree(P->otf_inv);
        cudaFree(P->otf_view);
        cudaFree(P->otf_view2);
        P->otf_ray = nullptr;
        P->otf_inv = nullptr;
        P->otf_view = P->otf_view2 = nullptr;
    }
    return e;
}

namespace {

// One entry of the multi-slice batch.
struct SliceIn {
    const dect_plan *plan;
    const float *m;
    float *x;
    dect_adm_report *rep;
};

int tiles_of(int n) { return ((n + kOtfTile - 1) / kOtfTile) * ((n + kOtfTile - 1) / kOtfTile); }

// Block maps of the three phases for the slices with `on[s]`; writes each
// slice's first block and block count into its descriptor.  table: the
// forward phase takes a warp per ray.
void build_maps(std::vector<SliceDesc> &desc, const std::vector<char> &on, std::vector<int> (&map)[PH_COUNT],
                bool table)
{
    const int rays_per_block = table ? kTabRaysPerBlock : kOtfBlock;
    for (int ph = 0; ph < PH_COUNT; ++ph) map[ph].clear();
    for (size_t s = 0; s < desc.size(); ++s) {
        SliceDesc &d = desc[s];
        const int nb[PH_COUNT] = {tiles_of(d.G.g.n), tiles_of(d.G.g.n),
                                  (int)((d.M + rays_per_block - 1) / rays_per_block)};
        for (int ph = 0; ph < PH_COUNT; ++ph) {
            d.blk0[ph] = (int)map[ph].size();
            d.nblk[ph] = nb[ph];
            if (on[s]) map[ph].insert(map[ph].end(), nb[ph], (int)s);
        }
    }
}

template <int MODE>
void launch_fwd_m(bool table, int nblk, cudaStream_t st, const SliceDesc *dd, const int *map, const BatchDev &B,
                  const BatchConst &C, int fsel)
{
    if (table)
        k_fwd_m<MODE, true><<<nblk, kOtfBlock, 0, st>>>(dd, map, B, C, fsel);
    else
        k_fwd_m<MODE, false><<<nblk, kOtfBlock, 0, st>>>(dd, map, B, C, fsel);
}

void launch_bwd_m(bool table, int nblk, cudaStream_t st, const SliceDesc *dd, const int *map, const BatchDev &B,
                  const BatchConst &C)
{
    if (table)
        k_bwd_m<true><<<nblk, kOtfBlock, 0, st>>>(dd, map, B, C);
    else
        k_bwd_m<false><<<nblk, kOtfBlock, 0, st>>>(dd, map, B, C);
}

}  // namespace
}  // namespace dect

using namespace dect;

extern "C" dect_status dect_project_otf(const dect_plan *plan, const float *x, float *y, int batch, dect_stream stream)
{
    if (!plan || batch < 0 || plan->nz > 0) return DECT_ERR_INVALID_ARG;
    if (batch == 0) return DECT_OK;
    if (!x || !y) return DECT_ERR_INVALID_ARG;
    DECT_CUDA(cudaSetDevice(plan->device));
    DECT_CUDA(otf_operator(plan, x, y, batch, false, (cudaStream_t)stream));
    return DECT_OK;
}

extern "C" dect_status dect_backproject_otf(const dect_plan *plan, const float *y, float *x, int batch,
                                            dect_stream stream)
{
    if (!plan || batch < 0 || plan->nz > 0) return DECT_ERR_INVALID_ARG;
    if (batch == 0) return DECT_OK;
    if (!x || !y) return DECT_ERR_INVALID_ARG;
    DECT_CUDA(cudaSetDevice(plan->device));
    DECT_CUDA(otf_operator(plan, y, x, batch, true, (cudaStream_t)stream));
    return DECT_OK;
}

extern "C" dect_status dect_adm_tv_batch_ex(const dect_adm_group *groups, int n_groups, const dect_adm_params *prm,
                                            int projector, dect_stream stream)
{
    if (!groups || n_groups < 0 || !prm) return DECT_ERR_INVALID_ARG;
    if (projector != DECT_PROJ_TABLE && projector != DECT_PROJ_OTF) return DECT_ERR_INVALID_ARG;
    const bool table = projector == DECT_PROJ_TABLE;
    if (!(prm->mu > 0) || !(prm->rho > 0) || !(prm->beta[0] > 0) || !(prm->beta[1] > 0) || prm->max_iter < 0 ||
        (prm->step_rule != DECT_STEP_BB1 && prm->step_rule != DECT_STEP_CAUCHY) || !std::isfinite(prm->mu) ||
        !std::isfinite(prm->rho) || !std::isfinite(prm->xi) || !std::isfinite(prm->beta[0]) ||
        !std::isfinite(prm->beta[1]) || prm->check_every < 0 || (prm->nonneg != 0 && prm->nonneg != 1) ||
        (prm->joint_tv != 0 && prm->joint_tv != 1))
        return DECT_ERR_INVALID_ARG;
    std::vector<SliceIn> in;
    int device = -1;
    for (int gi = 0; gi < n_groups; ++gi) {
        const dect_adm_group &G = groups[gi];
        if (!G.plan || G.n_slices < 0 || G.plan->nz > 0) return DECT_ERR_INVALID_ARG;  // fan-beam plans only
        if (G.n_slices > 0 && (!G.m || !G.x)) return DECT_ERR_INVALID_ARG;
        if (device >= 0 && G.plan->device != device) return DECT_ERR_INVALID_ARG;
        device = G.plan->device;
        if (!table && G.plan->n_grid_aligned > 0) {
            set_error_text("dect_adm_tv_batch: a plan has rays along grid lines, where the on-the-fly projector "
                           "and the stored table take different pixels; use dect_adm_tv for that geometry");
            return DECT_ERR_INVALID_ARG;
        }
        for (int i = 0; i < G.n_slices; ++i)
            in.push_back({G.plan, G.m + (int64_t)i * 2 * G.plan->M, G.x + (int64_t)i * 2 * G.plan->N,
                          G.reports ? G.reports + 2 * i : nullptr});
    }
    const int S = (int)in.size();
    if (S == 0) return DECT_OK;
    DECT_CUDA(cudaSetDevice(device));
    cudaStream_t s = (cudaStream_t)stream;
    if (!table)
        for (const SliceIn &q : in) DECT_CUDA(otf_setup(q.plan, s));

    BatchConst C;
    const double xi = prm->xi > 0 ? prm->xi : prm->rho;
    C.mu = (float)prm->mu;
    C.rho = (float)prm->rho;
    C.xi = (float)xi;
    C.mu_d = prm->mu;
    C.rho_d = prm->rho;
    C.tol = prm->rel_obj_tol;
    C.rule = prm->step_rule;
    C.nonneg = prm->nonneg ? 1 : 0;
    C.joint = prm->joint_tv ? 1 : 0;
    C.xi_is_rho = (xi == prm->rho && !C.nonneg) ? 1 : 0;

    // one workspace: per-slice state, then scalars, maps and descriptors
    std::vector<SliceDesc> desc(S);
    std::vector<char> on(S, 1);
    std::vector<int> map[PH_COUNT];
    size_t bytes = 0;
    std::vector<size_t> off(S);
    for (int i = 0; i < S; ++i) {
        off[i] = bytes;
        const int64_t N = in[i].plan->N, M = in[i].plan->M;
        bytes += sizeof(float2) * (size_t)(3 * N + 6 * N + 2 * M);  // f[2], G, lam/z/p (2 components), r, q
        bytes = (bytes + 255) & ~(size_t)255;
    }
    for (int i = 0; i < S; ++i) {
        SliceDesc &d = desc[i];
        d.G = otf_geom(in[i].plan);
        d.N = in[i].plan->N;
        d.M = in[i].plan->M;
        d.m = in[i].m;
        d.x = in[i].x;
        d.beta[0] = (float)prm->beta[0];
        d.beta[1] = (float)prm->beta[1];
        d.rowptr = in[i].plan->rowptr;
        d.colptr = in[i].plan->colptr;
        d.ent = in[i].plan->ent;
        d.tent = in[i].plan->tent;
    }
    build_maps(desc, on, map, table);
    const size_t max_blocks = std::max({map[0].size(), map[1].size(), map[2].size()});
    const size_t o_dbl = bytes;
    bytes += sizeof(double) * ((size_t)S * 2 * 4 + (size_t)S * Q_COUNT * 2 + max_blocks * 2 * 2);
    bytes = (bytes + 255) & ~(size_t)255;
    const size_t o_int = bytes;
    bytes += sizeof(int) * ((size_t)S * 2 * 3 + S + (size_t)S * (PH_COUNT + 1) + 1);
    bytes = (bytes + 255) & ~(size_t)255;
    const size_t o_map = bytes;
    bytes += sizeof(int) * max_blocks * PH_COUNT;
    bytes = (bytes + 255) & ~(size_t)255;
    const size_t o_desc = bytes;
    bytes += sizeof(SliceDesc) * S;
    char *base = nullptr;
    DECT_CUDA(cudaMallocAsync((void **)&base, bytes, s));
    auto fail = [&](cudaError_t e) {
        cudaFreeAsync(base, s);
        set_error("dect_adm_tv_batch", e);
        return e == cudaErrorMemoryAllocation ? DECT_ERR_OOM : DECT_ERR_CUDA;
    };
    cudaError_t e = cudaMemsetAsync(base, 0, bytes, s);
    for (int i = 0; i < S; ++i) {
        SliceDesc &d = desc[i];
        float2 *b = reinterpret_cast<float2 *>(base + off[i]);
        const int64_t N = d.N, M = d.M;
        d.f[0] = b;
        d.f[1] = b + N;
        d.Gr = b + 2 * N;
        d.lam = b + 3 * N;
        d.z = b + 5 * N;
        d.p = b + 7 * N;
        d.r = b + 9 * N;
        d.q = b + 9 * N + M;
    }
    BatchDev B;
    double *dbl = reinterpret_cast<double *>(base + o_dbl);
    B.alpha = dbl;
    B.c_prev = dbl + 2 * S;
    B.phi_prev = dbl + 4 * S;
    B.rel = dbl + 6 * S;
    B.red = dbl + 8 * S;
    B.part = B.red + (size_t)S * Q_COUNT * 2;
    int *ints = reinterpret_cast<int *>(base + o_int);
    B.iters = ints;
    B.conv = ints + 2 * S;
    B.active = ints + 4 * S;
    B.k = ints + 6 * S;
    B.ctr = reinterpret_cast<unsigned *>(ints + 7 * S);
    B.bad = ints + 7 * S + S * (PH_COUNT + 1);
    int *dmap[PH_COUNT];
    for (int ph = 0; ph < PH_COUNT; ++ph) dmap[ph] = reinterpret_cast<int *>(base + o_map) + ph * max_blocks;
    SliceDesc *ddesc = reinterpret_cast<SliceDesc *>(base + o_desc);

    // pinned host staging for the maps, descriptors and flags
    const size_t o_hdesc = (sizeof(int) * max_blocks * PH_COUNT + 63) & ~(size_t)63;
    const size_t o_hact = (o_hdesc + sizeof(SliceDesc) * S + 63) & ~(size_t)63;
    const size_t stage_bytes = o_hact + sizeof(int) * 2 * S;
    char *stage = nullptr;
    if (e == cudaSuccess) e = cudaMallocHost((void **)&stage, stage_bytes);
    if (e != cudaSuccess) {
        if (stage) cudaFreeHost(stage);
        return fail(e);
    }
    int *hmap = reinterpret_cast<int *>(stage);
    SliceDesc *hdesc = reinterpret_cast<SliceDesc *>(stage + o_hdesc);
    int *hact = reinterpret_cast<int *>(stage + o_hact);
    int nblocks[PH_COUNT];
    auto upload_maps = [&]() -> cudaError_t {
        // the previous upload's copies must have read the staging buffer
        cudaError_t er = cudaStreamSynchronize(s);
        for (int ph = 0; ph < PH_COUNT && er == cudaSuccess; ++ph) {
            nblocks[ph] = (int)map[ph].size();
            std::copy(map[ph].begin(), map[ph].end(), hmap + ph * max_blocks);
            if (nblocks[ph] > 0)
                er = cudaMemcpyAsync(dmap[ph], hmap + ph * max_blocks, sizeof(int) * nblocks[ph],
                                     cudaMemcpyHostToDevice, s);
        }
        std::copy(desc.begin(), desc.end(), hdesc);
        if (er == cudaSuccess) er = cudaMemcpyAsync(ddesc, hdesc, sizeof(SliceDesc) * S, cudaMemcpyHostToDevice, s);
        return er;
    };
    for (int i = 0; i < 2 * S; ++i) hact[i] = 1;
    if (e == cudaSuccess) e = cudaMemcpyAsync(B.active, hact, sizeof(int) * 2 * S, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = upload_maps();
    if (e == cudaSuccess && prm->warm_start) {
        k_pack_m<<<nblocks[PH_TV], kOtfBlock, 0, s>>>(ddesc, dmap[PH_TV], 1, 0);
        count_launches(1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {  // r^0 = A f^0 - beta m
        launch_fwd_m<0>(table, nblocks[PH_FWD], s, ddesc, dmap[PH_FWD], B, C, 0);
        count_launches(1);
        e = cudaGetLastError();
    }
    const int K = prm->max_iter;
    const bool use_tol = prm->rel_obj_tol > 0.0;
    int block = use_tol ? (prm->check_every > 0 ? prm->check_every : 10) : 10;
    block = std::max(2, block + (block & 1));
    const int per_iter = C.nonneg ? 4 : 3;
    auto enqueue_iter = [&](int par, cudaStream_t st) {
        k_tv_m<<<nblocks[PH_TV], kOtfBlock, 0, st>>>(ddesc, dmap[PH_TV], B, C, par, 0);
        if (C.nonneg) launch_fwd_m<2>(table, nblocks[PH_FWD], st, ddesc, dmap[PH_FWD], B, C, 1 - par);
        launch_bwd_m(table, nblocks[PH_BWD], st, ddesc, dmap[PH_BWD], B, C);
        launch_fwd_m<1>(table, nblocks[PH_FWD], st, ddesc, dmap[PH_FWD], B, C, 0);
    };
    cudaStream_t cs = nullptr;
    cudaEvent_t ev = nullptr;
    cudaGraphExec_t gx = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    auto make_graph = [&]() -> cudaError_t {
        if (gx) cudaGraphExecDestroy(gx);
        gx = nullptr;
        cudaGraph_t gr = nullptr;
        cudaError_t er = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (er != cudaSuccess) return er;
        for (int it = 0; it < block; ++it) enqueue_iter(it & 1, cs);
        er = cudaStreamEndCapture(cs, &gr);
        if (er == cudaSuccess) er = cudaGraphInstantiate(&gx, gr, 0);
        if (gr) cudaGraphDestroy(gr);
        return er;
    };
    if (e == cudaSuccess) e = cudaEventRecord(ev, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev, 0);
    int done = 0;
    bool graph_stale = true, all_stopped = false;
    while (e == cudaSuccess && done + block <= K) {
        if (graph_stale) {
            e = make_graph();
            graph_stale = false;
            if (e != cudaSuccess) break;
        }
        e = cudaGraphLaunch(gx, cs);
        count_launches((int64_t)per_iter * block);
        done += block;
        if (e != cudaSuccess || !use_tol) continue;
        e = cudaMemcpyAsync(hact, B.active, sizeof(int) * 2 * S, cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
        if (e != cudaSuccess) break;
        int running = 0;
        bool dropped = false;
        for (int i = 0; i < S; ++i) {
            const bool a = hact[2 * i] || hact[2 * i + 1];
            running += a ? 1 : 0;
            if (on[i] && !a) {
                on[i] = 0;
                dropped = true;
            }
        }
        if (running == 0) {
            all_stopped = true;
            break;
        }
        if (dropped && done + block <= K) {
            // stopped slices leave the launches (their state stays as it is)
            build_maps(desc, on, map, table);
            e = cudaStreamSynchronize(cs);
            if (e == cudaSuccess) e = cudaEventRecord(ev, cs);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev, 0);
            if (e == cudaSuccess) e = upload_maps();
            if (e == cudaSuccess) e = cudaEventRecord(ev, s);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev, 0);
            graph_stale = true;
        }
    }
    // remaining iterations one at a time (parity continues from `done`)
    while (e == cudaSuccess && !all_stopped && done < K) {
        enqueue_iter(done & 1, cs);
        count_launches(per_iter);
        ++done;
        e = cudaGetLastError();
    }
    // final step, the objective and the residual check of every slice, then the images
    if (e == cudaSuccess) e = cudaEventRecord(ev, cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev, 0);
    if (e == cudaSuccess) {
        std::fill(on.begin(), on.end(), 1);
        build_maps(desc, on, map, table);
        e = upload_maps();
    }
    const int par = done & 1;
    if (e == cudaSuccess) {
        k_tv_m<<<nblocks[PH_TV], kOtfBlock, 0, s>>>(ddesc, dmap[PH_TV], B, C, par, 1);
        if (C.nonneg) launch_fwd_m<2>(table, nblocks[PH_FWD], s, ddesc, dmap[PH_FWD], B, C, 1 - par);
        launch_fwd_m<3>(table, nblocks[PH_FWD], s, ddesc, dmap[PH_FWD], B, C, 1 - par);
        k_pack_m<<<nblocks[PH_TV], kOtfBlock, 0, s>>>(ddesc, dmap[PH_TV], 0, 1 - par);
        count_launches(C.nonneg ? 4 : 3);
        e = cudaGetLastError();
    }
    std::vector<double> hred((size_t)S * Q_COUNT * 2), hrel(2 * S);
    std::vector<int> hit(2 * S), hconv(2 * S);
    int hbad = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(hred.data(), B.red, sizeof(double) * hred.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hrel.data(), B.rel, sizeof(double) * 2 * S, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hit.data(), B.iters, sizeof(int) * 2 * S, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hconv.data(), B.conv, sizeof(int) * 2 * S, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, B.bad, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (gx) cudaGraphExecDestroy(gx);
    if (ev) cudaEventDestroy(ev);
    if (cs) cudaStreamDestroy(cs);
    cudaFreeHost(stage);
    if (e != cudaSuccess) return fail(e);
    cudaFreeAsync(base, s);
    for (int i = 0; i < S; ++i) {
        if (!in[i].rep) continue;
        for (int c = 0; c < 2; ++c) {
            dect_adm_report &r = in[i].rep[c];
            const double *rd = hred.data() + (size_t)i * Q_COUNT * 2;
            r.iters = K == 0 ? 0 : hit[2 * i + c];
            r.converged = hconv[2 * i + c];
            if (C.joint)
                r.objective = rd[Q_TV * 2] + rd[Q_TV * 2 + 1] + 0.5 * prm->mu * (rd[Q_RR * 2] + rd[Q_RR * 2 + 1]);
            else
                r.objective = rd[Q_TV * 2 + c] + 0.5 * prm->mu * rd[Q_RR * 2 + c];
            r.rel_change = hrel[2 * i + c];
            r.primal_res = std::sqrt(rd[Q_QQ * 2 + c]);
            r.resid_drift = std::sqrt(rd[Q_GG * 2 + c]);
        }
    }
    return (hbad & 1) ? DECT_ERR_NONFINITE : DECT_OK;
}

extern "C" dect_status dect_adm_tv_batch(const dect_adm_group *groups, int n_groups, const dect_adm_params *prm,
                                         dect_stream stream)
{
    return dect_adm_tv_batch_ex(groups, n_groups, prm, DECT_PROJ_OTF, stream);
}
