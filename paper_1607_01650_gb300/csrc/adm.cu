// ADM-TV reconstruction, Eq. (3)-(10) (Sec. 2.2), for a batch of images that
// share one plan.
//
// Each channel c (slice s, energy e) solves min |grad f|_TV + mu/2 |A f - g|^2
// with f = beta_e x, g = beta_e m (Eq. (3)-(4); the TV is taken per channel,
// so the stacked problem separates).  Iteration k of Eq. (10):
//   z^{k+1}      = shrink(grad f^k - lambda^k / rho, 1/rho)           Eq. (8)
//   G^k          = mu A^T r^k + grad^T p,  p = rho(grad f^k - z^{k+1}) - lambda^k
//                  (= mu A^T(A f - g) + rho grad^T(grad f - z) - grad^T lambda, Eq. (9))
//   alpha^k      = exact step c(G^k) = |G|^2 / (mu |A G|^2 + rho |grad G|^2)
//                  (CAUCHY) or the lagged c(G^{k-1}) (BB1)
//   f^{k+1}      = f^k - alpha^k G^k,   r^{k+1} = r^k - alpha^k A G^k  Eq. (9)
//   lambda^{k+1} = lambda^k - xi (grad f^{k+1} - z^{k+1})             Eq. (7)
// The residual r = A f - g is carried by linearity, so an iteration costs one
// A^T (of r) and one A (of G).  The lambda step of iteration k is applied at
// the start of iteration k+1, where grad f^{k+1} is formed anyway.
//
// Layout: up to 64 channels are interleaved pixel-major, f[pixel][NB], so a
// table entry gathers one contiguous vector of all channels.
//
// Kernel sequence per iteration (captured in a CUDA graph):
//   k_tv     f -= alpha G, r -= alpha q, lambda step, z-shrink, p
//                                                        ; |grad f|_TV, |r|^2
//   k_bwd    G = mu A^T r + grad^T p  (pixel-major table) ; |G|^2
//   k_fwd    q = A G  (ray-major table)                  ; |grad G|^2, |q|^2,
//            then the last block forms Phi^k, the stopping test and
//            alpha^k in FP64.
//
// Optional joint TV over the stacked image (both energies of a slice, channels
// 2s and 2s + 1, which one thread always holds together): the TV norm and the
// z-shrink take the 4-vector of both channels' gradients at a pixel, and the
// last block of k_fwd forms one step and one stopping test per slice from
// the sums of the two channels' norms.
//
// Optional projection onto f >= 0 (x in R_+^N, Eq. (1)): k_tv clamps each
// updated pixel, f^{k+1} = max(f^k - alpha^k G^k, 0).  The residual is then
// no longer r - alpha q, so a fourth kernel (k_fwd in mode 2) rebuilds
// r = A f - g after k_tv and reduces |r|^2; and the lambda step needs the
// stored lambda and z (the xi = rho shortcut below assumes the plain step).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <string>
#include <thread>
#include <vector>

#include "dect_internal.cuh"
#include "kernels.cuh"

namespace dect {
namespace {

constexpr int kBlock = 256;
constexpr int kGrid = kSMs * 8;  // fixed grid of every reducing kernel
// k_fwd: 1024-thread blocks, one per SM, so that 32 adjacent rays of a view
// (one warp each) share an L1
constexpr int kFwdBlock = 1024;
constexpr int kFwdGrid = kSMs;

// reduction slots; (TV, RR) and (DD, QQ) are reduced together
enum { R_TV = 0, R_RR = 1, R_DD = 2, R_QQ = 3, R_GG = 4, R_COUNT = 5 };
enum { C_TV = 0, C_BWD = 1, C_FWD = 2, C_RES = 3, C_COUNT = 4 };

struct AdmDev {
    // per-channel scalars
    double *red;       // [R_COUNT][NB] reduction results
    double *part;      // [C_COUNT][2][kGrid][NB] block partials, per kernel
    unsigned *ctr;     // [C_COUNT] last-block counters, then the k_tv tile counter
    double *alpha;     // [NB] step applied by the next k_tv
    double *c_prev;    // [NB]
    double *phi_prev;  // [NB]
    double *rel;       // [NB]
    int *iters;        // [NB]
    int *conv;         // [NB]
    int *active;       // [NB]
    int *slot;         // [NB] caller image (index in the chunk) held by each slot; -1: none
    int *k;            // iteration counter
    int *all_done;     // 1 once no channel is active
    int *bad;          // 1 once a non-finite objective was seen
};

struct AdmConst {
    int n;
    int64_t N, M;
    int xi_is_rho;       // multiplier rebuilt from p (see k_tv)
    int nonneg;          // f-step projected onto f >= 0
    int joint;           // TV over both channels of a slice (channels 2s, 2s + 1)
    float mu, rho, xi;   // FP32 copies for the bulk kernels
    double mu_d, rho_d;  // FP64 for the step and objective
    double tol;
    int rule;
};

template <int NB>
__device__ __forceinline__ double *part_of(const AdmDev &D, int kernel)
{
    return D.part + (size_t)kernel * 2 * kGrid * NB;
}

// z-shrink of Eq. (8) per pixel on the 4-vector of both channels' gradients
// (joint TV over the stacked image).
__device__ __forceinline__ void shrink4(float w0, float w1, float w2, float w3, float t, float &z0,
                                        float &z1, float &z2, float &z3)
{
    float nrm = sqrtf(w0 * w0 + w1 * w1 + w2 * w2 + w3 * w3);
    float s = nrm - t;
    if (s > 0.f && nrm > 0.f) {
        float k = s / nrm;
        z0 = k * w0;
        z1 = k * w1;
        z2 = k * w2;
        z3 = k * w3;
    } else {
        z0 = z1 = z2 = z3 = 0.f;
    }
}

// z-shrink of Eq. (8) per pixel on the 2-vector w (reading: w / |w| for sign).
__device__ __forceinline__ void shrink2(float w0, float w1, float t, float &z0, float &z1)
{
    float nrm = sqrtf(w0 * w0 + w1 * w1);
    float s = nrm - t;
    if (s > 0.f && nrm > 0.f) {
        float k = s / nrm;
        z0 = k * w0;
        z1 = k * w1;
    } else {
        z0 = 0.f;
        z1 = 0.f;
    }
}

// f - a g, projected onto [0, inf) when `clamp` (a NaN stays a NaN, so the
// non-finite-objective check still sees it).
__device__ __forceinline__ float nonneg_step(float f, float a, float g, bool clamp)
{
    const float v = fmaf(-a, g, f);
    return clamp && v < 0.f ? 0.f : v;
}

// ---------------------------------------------------------------------------
// Start of iteration k: apply the previous step (f^k = f^{k-1} - alpha G,
// r^k = r^{k-1} - alpha q; alpha = 0 at k = 0), then the lambda step of the
// previous iteration, the z-shrink and p = rho(grad f - z) - lambda.
// Reduces |grad f^k|_TV and |r^k|^2.  f is double-buffered (f_in -> f_out)
// because the stencil reads neighbours of the updated image.
// final_pass: only the f / r step and the two norms (the result's objective).
// With C.nonneg the updated pixels are clamped at 0 (from k = 1 on: at k = 0
// the step is empty and f^0 is used as given), and r and |r|^2 are left to
// k_fwd in mode 2.
//
// Traversal: blocks claim tiles of W columns x H rows from a counter (the
// last block resets it).  Thread (slot q, vector vl) owns column
// j = j0 - 1 + q of the tile (slot 0 is the column left of the tile:
// computed, never written) and walks down rows i0 - 1 .. i0 + H - 1 (row
// i0 - 1 is only computed).  The updated f and G of the pixel above are the
// thread's own values from the previous row, held in registers; those of the
// pixel to the left come from the neighbouring slot through shared memory
// (double-buffered by row parity: one barrier per row).  Each row's f, G and
// multiplier (p, or lambda) are loaded one row ahead.  Every stored array is
// read and written once, in 16-byte vectors.
// ---------------------------------------------------------------------------
template <int NB>
struct TvShape {
    static constexpr int VW = Batch<NB>::VW, CPB = Batch<NB>::CPB;
    static constexpr int BLK = NB > 32 ? 512 : 256;  // threads per block
    static constexpr int W = BLK / CPB - 1;           // tile columns (+1 halo slot)
    static constexpr int H = 16;                      // tile rows
    static constexpr size_t XS_BYTES = sizeof(float) * 2 * 2 * (W + 1) * NB;
    static constexpr size_t RED_BYTES = sizeof(double) * reduce_smem_doubles<NB, BLK>(2);
    static constexpr size_t SMEM = XS_BYTES > RED_BYTES ? XS_BYTES : RED_BYTES;
};

// r <- r - alpha q over the rays' vectors first, first + stride, ... < rn
// (VW channels each, those of the thread's alpha), adding |r|^2 to acc.
// U vectors' loads are issued together, so the pass is not one load latency
// per vector; the sum runs in the same order as a plain loop.
template <int VW, int U = 4>
__device__ __forceinline__ void r_step(float *__restrict__ r, const float *__restrict__ q, int64_t rn, int64_t first,
                                       int64_t stride, const Vec<VW> &a, Vec<VW> &acc)
{
    for (int64_t t0 = first; t0 < rn; t0 += U * stride) {
        Vec<VW> rv[U], qv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t t = t0 + u * stride;
            if (t < rn) {
                rv[u] = ld_v<VW>(r + t * VW);
                qv[u] = ld_v<VW>(q + t * VW);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t t = t0 + u * stride;
            if (t < rn) {
#pragma unroll
                for (int c = 0; c < VW; ++c) {
                    rv[u].v[c] = fmaf(-a.v[c], qv[u].v[c], rv[u].v[c]);
                    acc.v[c] = fmaf(rv[u].v[c], rv[u].v[c], acc.v[c]);
                }
                st_v<VW>(r + t * VW, rv[u]);
            }
        }
    }
}

// Per-pixel work of the TV step at pixel (i, j), offset o of the thread's
// vector: fc, gc are the stepped f and the G of the pixel, fu, gu those of
// the pixel above and fl, gl those of the pixel to the left (the pixel's own
// on the first row / column); l0, l1 the multiplier rows read for the pixel
// (p^{k-1} with xi = rho, else lambda^{k-1}).  Adds |grad f| (Eq. (2)) to
// acc and, unless final_pass, applies the multiplier step (Eq. (7)), the
// z-shrink (Eq. (8)) and writes p (and, without the xi = rho shortcut,
// lambda and z).  Both TV kernels call it, so they compute the same values.
template <int NB, bool JOINT>
__device__ __forceinline__ void tv_pixel(const Vec<Batch<NB>::VW> &fc, const Vec<Batch<NB>::VW> &gc,
                                         const Vec<Batch<NB>::VW> &fu, const Vec<Batch<NB>::VW> &gu_,
                                         const Vec<Batch<NB>::VW> &fl, const Vec<Batch<NB>::VW> &gl_,
                                         Vec<Batch<NB>::VW> l0, Vec<Batch<NB>::VW> l1, int i, int j, int64_t o,
                                         int64_t sN, const Vec<Batch<NB>::VW> &a, int k, float inv_rho,
                                         const AdmConst &C, int final_pass, float *__restrict__ lam,
                                         float *__restrict__ z, float *__restrict__ p, Vec<Batch<NB>::VW> &acc)
{
    constexpr int VW = Batch<NB>::VW;
    // With xi = rho the multiplier step of Eq. (7) and
    // p^{k-1} = rho(grad f^{k-1} - z^k) - lambda^{k-1} give
    // lambda^k = xi alpha^{k-1} grad G^{k-1} - p^{k-1}: neither lambda nor z
    // has to be stored (l0, l1 carry p^{k-1} then; otherwise lambda^{k-1}).
    Vec<VW> z0, z1;
    if (!final_pass && !C.xi_is_rho && k > 0) {
        z0 = ld_v<VW>(z + o);
        z1 = ld_v<VW>(z + sN + o);
    }
    Vec<VW> p0, p1, d0, d1;
#pragma unroll
    for (int c = 0; c < VW; ++c) {
        d0.v[c] = fc.v[c] - fu.v[c];   // Eq. (2), 0 on the first row
        d1.v[c] = fc.v[c] - fl.v[c];   // Eq. (2), 0 on the first column
    }
    if (JOINT) {  // one norm per slice over both channels (c, c + 1)
#pragma unroll
        for (int c = 0; c < VW; c += 2)
            acc.v[c] += sqrtf(d0.v[c] * d0.v[c] + d1.v[c] * d1.v[c] + d0.v[c + 1] * d0.v[c + 1] +
                              d1.v[c + 1] * d1.v[c + 1]);
    } else {
#pragma unroll
        for (int c = 0; c < VW; ++c) acc.v[c] += sqrtf(d0.v[c] * d0.v[c] + d1.v[c] * d1.v[c]);
    }
    if (!final_pass) {
#pragma unroll
        for (int c = 0; c < VW; ++c) {
            const float g0 = d0.v[c], g1 = d1.v[c];
            float a0, a1;
            if (C.xi_is_rho) {
                a0 = 0.f;
                a1 = 0.f;
                if (k > 0) {
                    const float dg0 = i > 0 ? gc.v[c] - gu_.v[c] : 0.f;
                    const float dg1 = j > 0 ? gc.v[c] - gl_.v[c] : 0.f;
                    a0 = C.xi * a.v[c] * dg0 - l0.v[c];
                    a1 = C.xi * a.v[c] * dg1 - l1.v[c];
                }
            } else {
                a0 = l0.v[c];
                a1 = l1.v[c];
                if (k > 0) {  // lambda^k = lambda^{k-1} - xi (grad f^k - z^k), Eq. (7)
                    a0 -= C.xi * (g0 - z0.v[c]);
                    a1 -= C.xi * (g1 - z1.v[c]);
                }
            }
            l0.v[c] = a0;  // lambda^k
            l1.v[c] = a1;
            if (!JOINT) {
                float s0, s1;
                shrink2(g0 - a0 * inv_rho, g1 - a1 * inv_rho, inv_rho, s0, s1);
                z0.v[c] = s0;
                z1.v[c] = s1;
            }
        }
        if (JOINT) {
#pragma unroll
            for (int c = 0; c < VW; c += 2)
                shrink4(d0.v[c] - l0.v[c] * inv_rho, d1.v[c] - l1.v[c] * inv_rho,
                        d0.v[c + 1] - l0.v[c + 1] * inv_rho, d1.v[c + 1] - l1.v[c + 1] * inv_rho,
                        inv_rho, z0.v[c], z1.v[c], z0.v[c + 1], z1.v[c + 1]);
        }
#pragma unroll
        for (int c = 0; c < VW; ++c) {
            p0.v[c] = C.rho * (d0.v[c] - z0.v[c]) - l0.v[c];
            p1.v[c] = C.rho * (d1.v[c] - z1.v[c]) - l1.v[c];
        }
        if (!C.xi_is_rho) {
            st_v<VW>(lam + o, l0);
            st_v<VW>(lam + sN + o, l1);
            st_v<VW>(z + o, z0);
            st_v<VW>(z + sN + o, z1);
        }
        st_v<VW>(p + o, p0);
        st_v<VW>(p + sN + o, p1);
    }
}

template <int NB, bool JOINT>
__global__ void __launch_bounds__(TvShape<NB>::BLK) k_tv(const float *__restrict__ f_in, float *__restrict__ f_out,
                                                       const float *__restrict__ G, float *__restrict__ lam,
                                                       float *__restrict__ z, float *__restrict__ p,
                                                       float *__restrict__ r, const float *__restrict__ q,
                                                       AdmConst C, AdmDev D, int final_pass)
{
    using S = TvShape<NB>;
    constexpr int VW = S::VW, CPB = S::CPB, W = S::W, H = S::H;
    // row exchange buffer [row parity][f | G][slot][channel]; reused by the final reduction
    __shared__ __align__(16) unsigned char sbuf[S::SMEM];
    float(*xs)[2][W + 1][NB] = reinterpret_cast<float(*)[2][W + 1][NB]>(sbuf);
    const int k = *D.k;
    const float inv_rho = 1.0f / C.rho;
    const bool clamp = C.nonneg && k > 0;
    const int slot = threadIdx.x / CPB, vl = threadIdx.x % CPB;
    const bool in_tile = slot <= W;
    Vec<VW> a;
#pragma unroll
    for (int c = 0; c < VW; ++c) a.v[c] = (float)D.alpha[vl * VW + c];
    Vec<VW> acc[2];
    acc[0].zero();
    acc[1].zero();
    const int64_t sN = C.N * NB;  // component stride of lam, z, p
    const int64_t row = (int64_t)C.n * NB;
    const int tiles_x = (C.n + W - 1) / W, ntiles = tiles_x * ((C.n + H - 1) / H);
    __shared__ int s_tile;
    const float *lsrc = C.xi_is_rho ? p : lam;  // the multiplier rows read per pixel
    const bool need_l = !final_pass;
    for (;;) {
        if (threadIdx.x == 0) s_tile = (int)atomicAdd(D.ctr + C_COUNT, 1u);
        __syncthreads();
        const int tile = s_tile;
        if (tile >= ntiles) break;
        const int j0 = (tile % tiles_x) * W, i0 = (tile / tiles_x) * H;
        const int j = j0 - 1 + slot;
        const bool colok = in_tile && j >= 0 && j < C.n;
        const bool owner = colok && slot > 0;
        const int ibeg = i0 > 0 ? i0 - 1 : 0, iend = min(i0 + H, C.n);
        Vec<VW> fn, gn, ln0, ln1, fup, gup;
        fn.zero();
        gn.zero();
        ln0.zero();
        ln1.zero();
        fup.zero();
        gup.zero();
        if (colok) {
            const int64_t o = ((int64_t)ibeg * C.n + j) * NB + vl * VW;
            fn = ld_v<VW>(f_in + o);
            gn = ld_v<VW>(G + o);
            if (need_l && owner && ibeg >= i0) {
                ln0 = ld_v<VW>(lsrc + o);
                ln1 = ld_v<VW>(lsrc + sN + o);
            }
        }
        for (int i = ibeg; i < iend; ++i) {
            const int par = i & 1;
            const int64_t o = ((int64_t)i * C.n + j) * NB + vl * VW;
            Vec<VW> fc = fn, gc = gn, lc0 = ln0, lc1 = ln1;
            if (colok && i + 1 < iend) {
                fn = ld_v<VW>(f_in + o + row);
                gn = ld_v<VW>(G + o + row);
                if (need_l && owner) {
                    ln0 = ld_v<VW>(lsrc + o + row);
                    ln1 = ld_v<VW>(lsrc + sN + o + row);
                }
            }
#pragma unroll
            for (int c = 0; c < VW; ++c) fc.v[c] = nonneg_step(fc.v[c], a.v[c], gc.v[c], clamp);
            if (in_tile) {
                st_v<VW>(&xs[par][0][slot][vl * VW], fc);
                st_v<VW>(&xs[par][1][slot][vl * VW], gc);
            }
            __syncthreads();
            if (owner && i >= i0) {
                st_v<VW>(f_out + o, fc);
                Vec<VW> fu, gu_, fl, gl_;
                if (i > 0) {
                    fu = fup;
                    gu_ = gup;
                } else {
                    fu = fc;
                    gu_ = gc;
                }
                if (j > 0) {
                    fl = ld_v<VW>(&xs[par][0][slot - 1][vl * VW]);
                    gl_ = ld_v<VW>(&xs[par][1][slot - 1][vl * VW]);
                } else {
                    fl = fc;
                    gl_ = gc;
                }
                tv_pixel<NB, JOINT>(fc, gc, fu, gu_, fl, gl_, lc0, lc1, i, j, o, sN, a, k, inv_rho, C, final_pass,
                                    lam, z, p, acc[0]);
            }
            fup = fc;
            gup = gc;
        }
        __syncthreads();  // the next tile's first row reuses the exchange buffer (and s_tile)
    }
    const int64_t rn = C.nonneg ? 0 : C.M * CPB;  // with the projection r is rebuilt by k_fwd
    r_step<VW>(r, q, rn, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x, a, acc[1]);
    if (reduce_images<NB, 2, S::BLK>(acc, part_of<NB>(D, C_TV), D.red + R_TV * NB, D.ctr + C_TV,
                                     reinterpret_cast<double *>(sbuf)) &&
        threadIdx.x == 0)
        D.ctr[C_COUNT] = 0u;  // every block has left the tile loop: reset the tile counter
}

// ---------------------------------------------------------------------------
// The same TV step with its rows staged by the TMA (TV variant 1).  The
// image is cut into `strips` strips of Wd <= SLOTS - 1 columns; a strip row
// is held together with the column to its left (computed, never written) in
// SLOTS slots of NB floats.  The (strip, row) pairs, strip by strip, are
// split into equal contiguous ranges, one per block, so there is no tile
// counter and no tail of unequal tiles.  The last warp of the block is the
// producer: its lane 0 streams the rows of the block's range -- f, G and the
// two multiplier rows, each one contiguous run of at most SLOTS x NB floats
// -- into a ring of STAGES shared-memory stages with 1-D bulk copies that
// complete on the stage's `full` mbarrier; for the row above the range only
// f and G are copied.  The consumer threads take the rows in order: the
// pixel and its left neighbour from the stage, the pixel above from their
// own registers (the previous row); each consumer warp then releases the
// stage by one arrival on its `empty` mbarrier.  No block-wide barrier per
// row, STAGES rows in flight.  Per pixel the arithmetic is k_tv's (tv_pixel,
// the same f step), so both variants give the same images; only the order
// of the FP32 partial sums of the two norms differs.  Every wait is bounded:
// one that runs out sets bit 1 of *D.bad (DECT_ERR_TIMEOUT), ends the loops
// of the whole block and the producer then waits (bounded) for its copies
// in flight.  Needs 16-byte pixels (NB >= 4) for the copies' alignment.
// ---------------------------------------------------------------------------
template <int NB>
struct TvTmaShape {
    static constexpr int VW = Batch<NB>::VW, CPB = Batch<NB>::CPB;
    static constexpr int BLK = NB > 32 ? 512 : 256;  // consumer threads
    static constexpr int THREADS = BLK + 32;          // + the producer warp
    static constexpr int SLOTS = BLK / CPB;           // a strip's columns + the column to their left
    static constexpr int STAGES = 4;
    static constexpr int RF = SLOTS * NB;             // floats of one array row of a stage
    static constexpr size_t SMEM = sizeof(float) * STAGES * 4 * RF;
    static_assert(NB >= 4, "the bulk copies need 16-byte pixels");
};

constexpr unsigned kTvPolls = 1u << 22;

// wait for phase `parity` of `bar`; false once *fail is set or after
// kTvPolls polls (then *fail is set and the timeout recorded in bit 1 of *bad)
__device__ __forceinline__ bool tv_wait(uint64_t *bar, unsigned parity, volatile int *fail, int *bad)
{
    for (unsigned i = 0; i < kTvPolls; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 255u) == 255u && *fail) return false;
    }
    *fail = 1;
    atomicOr(bad, 2);
    return false;
}

// strip layout of an n x n image for SLOTS slots per strip row
__host__ __device__ inline int tv_strips(int n, int slots) { return (n + slots - 2) / (slots - 1); }

template <int NB, bool JOINT>
__global__ void __launch_bounds__(TvTmaShape<NB>::THREADS) k_tv_tma(
    const float *__restrict__ f_in, float *__restrict__ f_out, const float *__restrict__ G, float *__restrict__ lam,
    float *__restrict__ z, float *__restrict__ p, float *__restrict__ r, const float *__restrict__ q, AdmConst C,
    AdmDev D, int final_pass)
{
    using S = TvTmaShape<NB>;
    constexpr int VW = S::VW, CPB = S::CPB, SLOTS = S::SLOTS, NST = S::STAGES, RF = S::RF;
    extern __shared__ __align__(128) float ring[];  // [stage][f | G | l0 | l1][slot][NB]
    __shared__ __align__(8) uint64_t full[NST], empty[NST];
    __shared__ int fail;
    __shared__ double rsm[reduce_smem_doubles<NB, S::BLK>(2)];
    const int k = *D.k;
    const float inv_rho = 1.0f / C.rho;
    const bool clamp = C.nonneg && k > 0;
    const int vl = threadIdx.x % CPB;
    Vec<VW> a;
#pragma unroll
    for (int c = 0; c < VW; ++c) a.v[c] = (float)D.alpha[vl * VW + c];
    Vec<VW> acc[2];
    acc[0].zero();
    acc[1].zero();
    const int64_t sN = C.N * NB;  // component stride of lam, z, p
    const float *lsrc = C.xi_is_rho ? p : lam;
    const bool need_l = !final_pass;
    const int strips = tv_strips(C.n, SLOTS), Wd = (C.n + strips - 1) / strips;
    const int64_t T = (int64_t)strips * C.n;  // (strip, row) pairs
    const int64_t t0 = T * blockIdx.x / gridDim.x, t1 = T * (blockIdx.x + 1) / gridDim.x;
    const int halo0 = (t1 > t0 && t0 % C.n > 0) ? 1 : 0;  // the row above the range
    const int L = (int)(t1 - t0) + halo0;                  // rows this block streams
    // row `it` of the block: strip s, image row i; `halo`: the row above the range
    auto row_of = [&](int it, int &s, int &i, bool &halo) {
        halo = it < halo0;
        const int64_t t = halo ? t0 : t0 + it - halo0;
        s = (int)(t / C.n);
        i = (int)(t % C.n) - (halo ? 1 : 0);
    };
    if (threadIdx.x == 0) {
        for (int st = 0; st < NST; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], S::BLK / 32);
        }
        fail = 0;
    }
    __syncthreads();
    if (threadIdx.x >= S::BLK) {
        if (threadIdx.x == S::BLK) {  // producer
            int issued = 0;
            for (int it = 0; it < L; ++it) {
                const int st = it % NST;
                if (it >= NST && !tv_wait(&empty[st], ((it / NST) - 1) & 1, &fail, D.bad)) break;
                int s, i;
                bool halo;
                row_of(it, s, i, halo);
                const int jl = s * Wd - 1;  // column of slot 0
                const int c0 = max(jl, 0), c1 = min(s * Wd + Wd - 1, C.n - 1);
                const unsigned bytes = (unsigned)((c1 - c0 + 1) * NB * sizeof(float));
                const bool wl = need_l && !halo;
                mbar_arrive_expect_tx(&full[st], wl ? 4 * bytes : 2 * bytes);
                float *dst = ring + (size_t)st * 4 * RF + (size_t)(c0 - jl) * NB;
                const int64_t go = ((int64_t)i * C.n + c0) * NB;
                bulk_g2s(dst, f_in + go, bytes, &full[st]);
                bulk_g2s(dst + RF, G + go, bytes, &full[st]);
                if (wl) {
                    bulk_g2s(dst + 2 * RF, lsrc + go, bytes, &full[st]);
                    bulk_g2s(dst + 3 * RF, lsrc + sN + go, bytes, &full[st]);
                }
                issued = it + 1;
            }
            // the copies of the last rows must have landed before the block
            // leaves (they have, unless a consumer gave up waiting)
            for (int it = max(issued - NST, 0); it < issued; ++it)
                mbar_wait_bounded(&full[it % NST], (it / NST) & 1, kTvPolls);
        }
    } else {
        const int slot = threadIdx.x / CPB;
        Vec<VW> fup, gup;
        fup.zero();
        gup.zero();
        for (int it = 0; it < L; ++it) {
            const int st = it % NST;
            if (!tv_wait(&full[st], (it / NST) & 1, &fail, D.bad)) break;
            int s, i;
            bool halo;
            row_of(it, s, i, halo);
            const int j = s * Wd - 1 + slot;
            const bool colok = slot <= Wd && j >= 0 && j < C.n;
            const float *sf = ring + (size_t)st * 4 * RF + slot * NB + vl * VW;
            Vec<VW> fc, gc;
            fc.zero();
            gc.zero();
            if (colok) {
                fc = ld_v<VW>(sf);
                gc = ld_v<VW>(sf + RF);
#pragma unroll
                for (int c = 0; c < VW; ++c) fc.v[c] = nonneg_step(fc.v[c], a.v[c], gc.v[c], clamp);
            }
            if (colok && slot > 0 && !halo) {
                const int64_t o = ((int64_t)i * C.n + j) * NB + vl * VW;
                st_v<VW>(f_out + o, fc);
                Vec<VW> fu = fc, gu_ = gc, fl = fc, gl_ = gc, l0, l1;
                if (i > 0) {
                    fu = fup;
                    gu_ = gup;
                }
                if (j > 0) {
                    fl = ld_v<VW>(sf - NB);
                    gl_ = ld_v<VW>(sf - NB + RF);
#pragma unroll
                    for (int c = 0; c < VW; ++c) fl.v[c] = nonneg_step(fl.v[c], a.v[c], gl_.v[c], clamp);
                }
                l0.zero();
                l1.zero();
                if (need_l) {
                    l0 = ld_v<VW>(sf + 2 * RF);
                    l1 = ld_v<VW>(sf + 3 * RF);
                }
                tv_pixel<NB, JOINT>(fc, gc, fu, gu_, fl, gl_, l0, l1, i, j, o, sN, a, k, inv_rho, C, final_pass,
                                    lam, z, p, acc[0]);
            }
            fup = fc;
            gup = gc;
            __syncwarp();
            if ((threadIdx.x & 31) == 0) mbar_arrive(&empty[st]);
        }
    }
    // r pass on the consumer threads only: the reduction below sums the
    // partials of the first BLK threads
    const int64_t rn = C.nonneg || threadIdx.x >= S::BLK ? 0 : C.M * CPB;  // with the projection k_fwd rebuilds r
    r_step<VW>(r, q, rn, (int64_t)blockIdx.x * S::BLK + threadIdx.x, (int64_t)gridDim.x * S::BLK, a, acc[1]);
    reduce_images<NB, 2, S::BLK>(acc, part_of<NB>(D, C_TV), D.red + R_TV * NB, D.ctr + C_TV, rsm);
}

// G = mu A^T r + grad^T p over the pixel-major table.  A block of BLK
// threads takes TW x TH pixel tiles (BLK / G_ pixels at a time), so the
// sinogram lines its pixels gather are shared in L1.
// VWL = 4: lanes gather 4 images of an entry, entries broadcast through a
// per-warp shared-memory slot; VWL = 8 or 16: lanes gather VWL images of an
// entry, R rounds in flight (row_dot_w; NB >= 16 only).
template <int NB, int G_, int TW, int TH, int BLK, int VWL = 4, int R = 2>
__global__ void __launch_bounds__(BLK) k_bwd(const int64_t *__restrict__ colptr,
                                                const Entry *__restrict__ tent,
                                                const float *__restrict__ r, const float *__restrict__ p,
                                                float *__restrict__ G, AdmConst C, AdmDev D)
{
    constexpr int VW = Batch<NB>::VW, LPE = Batch<NB>::CPB;
    constexpr int RPS = BLK / G_;  // pixels per block step
    static_assert((TW * TH) % RPS == 0, "tile split");
    __shared__ double smem[reduce_smem_doubles<NB, BLK>(1)];
    const int lr = threadIdx.x % G_, grp = lr / LPE, vl = lr % LPE;
    const int64_t sN = C.N * NB;
    const int tiles_x = (C.n + TW - 1) / TW;
    const int ntiles = tiles_x * ((C.n + TH - 1) / TH);
    Vec<VW> nrm[1];
    nrm[0].zero();
    const unsigned long long pol = l2_evict_last_policy();
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int ty = tile / tiles_x, tx = tile % tiles_x;
        for (int s0 = 0; s0 < TW * TH; s0 += RPS) {
            const int slot = s0 + threadIdx.x / G_;
            const int i = ty * TH + slot / TW, j = tx * TW + slot % TW;
            const bool ok = i < C.n && j < C.n;
            const int64_t pix = (int64_t)i * C.n + j;
            int64_t b = 0, e = 0;
            if (ok) {
                b = colptr[pix];
                e = colptr[pix + 1];
            }
            Vec<VW> acc;
            if constexpr (VWL > 4 && NB >= 16)
                acc = row_dot_w<NB, G_, VWL, R>(tent, b, e, lr, r, pol, C.M, CHK_GATHER_AT);
            else
                acc = row_dot<NB, G_, true, true>(tent, b, e, r, C.M, lr, CHK_GATHER_AT);
            if (ok && grp == 0) {
                const int64_t o = pix * NB + vl * VW;
                Vec<VW> p0 = ld_v<VW>(p + o), p1 = ld_v<VW>(p + sN + o), pd, pr;
                if (i + 1 < C.n) pd = ld_v<VW>(p + o + (int64_t)C.n * NB); else pd.zero();
                if (j + 1 < C.n) pr = ld_v<VW>(p + sN + o + NB); else pr.zero();
                Vec<VW> out;
#pragma unroll
                for (int c = 0; c < VW; ++c) {
                    float gt = (i > 0 ? p0.v[c] : 0.f) - pd.v[c] + (j > 0 ? p1.v[c] : 0.f) - pr.v[c];
                    out.v[c] = fmaf(C.mu, acc.v[c], gt);
                    nrm[0].v[c] = fmaf(out.v[c], out.v[c], nrm[0].v[c]);
                }
                st_keep<VW>(G + o, out, pol);
            }
        }
    }
    reduce_images<NB, 1, BLK>(nrm, part_of<NB>(D, C_BWD), D.red + R_GG * NB, D.ctr + C_BWD, smem);
}

// G = mu A^T r + grad^T p with everything a tile needs staged in shared
// memory: a block takes kWinTH x kWinTW pixel tiles; per tile, the block
// copies the tile's entries (tile-major table, tile-local ray indices) and,
// per view, the window of sinogram bins the tile meets into shared memory
// with 16-byte cp.async copies, double-buffered so that the copies of the
// next tile overlap the gathers of this one; the tile's pixels then read
// only shared memory.

template <int NB, int G>
__device__ __forceinline__ Vec<Batch<NB>::VW> row_dot_smem(const Entry *sent, int b, int e, int lr,
                                                           const float *win)
{
    constexpr int VW = Batch<NB>::VW, LPE = Batch<NB>::CPB, EG = G / LPE;
    const int grp = lr / LPE, vl = lr % LPE;
    Vec<VW> acc;
    acc.zero();
#pragma unroll 4
    for (int k = b + grp; k < e; k += EG) {
        const Entry t = sent[k];
        const Vec<VW> xv = ld_v<VW>(win + t.x * NB + vl * VW);
        const float w = __int_as_float(t.y);
#pragma unroll
        for (int c = 0; c < VW; ++c) acc.v[c] = fmaf(w, xv.v[c], acc.v[c]);
    }
#pragma unroll
    for (int off = LPE; off < G; off <<= 1)
#pragma unroll
        for (int c = 0; c < VW; ++c) acc.v[c] += __shfl_xor_sync(0xffffffffu, acc.v[c], off);
    return acc;
}

constexpr int kWinBlock = 32 * kWinTP;  // one warp per pixel of a tile
constexpr int kWinWarps = kWinBlock / 32;

struct WinArgs {
    const Entry *tmaj;
    const int64_t *tbase;
    const int *tpo, *wray0, *wcnt, *woff, *wtot;
    int nv, nvp;
    int win_floats;  // floats of one stage's sinogram window
    int ent_max;     // entries of one stage's table part
};

// Data stage st in dynamic shared memory: [window floats][entries]; after the
// two data stages, two descriptor stages of [wray0 | wcnt | woff] x nvp ints.
__device__ __forceinline__ float *win_stage(float *dyn, const WinArgs &A, int st)
{
    return dyn + (size_t)st * (A.win_floats + 2 * A.ent_max);
}
__device__ __forceinline__ int *desc_stage(float *dyn, const WinArgs &A, int st)
{
    return reinterpret_cast<int *>(win_stage(dyn, A, 2)) + (size_t)st * 3 * A.nvp;
}

// Copies of tile `tile`'s view descriptors into descriptor stage ds (16-byte cp.async).
__device__ __forceinline__ void win_copy_desc(const WinArgs &A, float *dyn, int tile, int ds)
{
    int *d = desc_stage(dyn, A, ds);
    const int q = A.nvp / 4;  // 16-byte chunks per array
    const int64_t o = (int64_t)tile * A.nvp;
    for (int c = threadIdx.x; c < 3 * q; c += blockDim.x) {
        const int a = c / q, k = (c % q) * 4;
        const int *src = a == 0 ? A.wray0 : (a == 1 ? A.wcnt : A.woff);
        cp_async16(d + a * A.nvp + k, src + o + k);
    }
}

// Copies of tile `tile`'s entries and sinogram windows into data stage st,
// using the descriptors already in descriptor stage ds; pixel offsets to spo.
template <int NB>
__device__ __forceinline__ void win_copy_data(const WinArgs &A, float *dyn, int (*spo)[kWinTP + 1],
                                              const float *r, int tile, int st, int ds)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float *win = win_stage(dyn, A, st);
    Entry *sent = reinterpret_cast<Entry *>(win + A.win_floats);
    const int64_t e0 = A.tbase[tile], e1 = A.tbase[tile + 1];
    const int nch = (int)((e1 - e0) / 2);
    for (int c = threadIdx.x; c < nch; c += blockDim.x) cp_async16(sent + 2 * c, A.tmaj + e0 + 2 * c);
    const int *d = desc_stage(dyn, A, ds);
    for (int v = warp; v < A.nv; v += kWinWarps) {
        const int ray0 = d[v], cnt = d[A.nvp + v], off = d[2 * A.nvp + v];
        const int nc = cnt * NB / 4;
        const float *src = r + (int64_t)ray0 * NB;
        float *dst = win + (int64_t)off * NB;
        for (int c = lane; c < nc; c += 32) cp_async16(dst + 4 * c, src + 4 * c);
    }
    if (threadIdx.x <= kWinTP) spo[st][threadIdx.x] = A.tpo[(int64_t)tile * (kWinTP + 1) + threadIdx.x];
}

template <int NB>
__global__ void __launch_bounds__(kWinBlock, 1) k_bwd_win(WinArgs A, const float *__restrict__ r,
                                                          const float *__restrict__ p,
                                                          float *__restrict__ G, AdmConst C, AdmDev D)
{
    constexpr int VW = Batch<NB>::VW, LPE = Batch<NB>::CPB;
    constexpr int G_ = 32;
    extern __shared__ __align__(128) float dyn[];
    __shared__ int spo[2][kWinTP + 1];
    __shared__ double smem[reduce_smem_doubles<NB, kWinBlock>(1)];
    const int lr = threadIdx.x & 31, grp = lr / LPE, vl = lr % LPE;
    const int slot = threadIdx.x >> 5;  // pixel of the tile handled by this warp
    const int64_t sN = C.N * NB;
    const int tiles_x = (C.n + kWinTW - 1) / kWinTW;
    const int ntiles = tiles_x * ((C.n + kWinTH - 1) / kWinTH);
    Vec<VW> nrm[1];
    nrm[0].zero();
    // pipeline: at the top of the loop for tile t the group holding
    // (data of t, descriptors of t + 1) is awaited; then the group
    // (descriptors of t + 2, data of t + 1) is issued and overlaps compute(t)
    const int g = gridDim.x;
    int t0 = blockIdx.x;
    if (t0 < ntiles) {
        win_copy_desc(A, dyn, t0, 0);
        cp_async_commit();
        cp_async_wait<0>();
        __syncthreads();
        if (t0 + g < ntiles) win_copy_desc(A, dyn, t0 + g, 1);
        win_copy_data<NB>(A, dyn, spo, r, t0, 0, 0);
        cp_async_commit();
    }
    int it = 0;
    for (int tile = t0; tile < ntiles; tile += g, ++it) {
        const int st = it & 1;
        cp_async_wait<0>();
        __syncthreads();
        const int next = tile + g, next2 = tile + 2 * g;
        if (next2 < ntiles) win_copy_desc(A, dyn, next2, st);        // desc stage of t+2 = t % 2
        if (next < ntiles) win_copy_data<NB>(A, dyn, spo, r, next, st ^ 1, st ^ 1);
        cp_async_commit();
        const int ty = tile / tiles_x, tx = tile % tiles_x;
        const int i = ty * kWinTH + slot / kWinTW, j = tx * kWinTW + slot % kWinTW;
        const bool ok = i < C.n && j < C.n;
        const int64_t pix = (int64_t)i * C.n + j;
        const int64_t o = pix * NB + vl * VW;
        Vec<VW> p0, p1, pd, pr;
        p0.zero(); p1.zero(); pd.zero(); pr.zero();
        if (ok && grp == 0) {
            p0 = ld_v<VW>(p + o);
            p1 = ld_v<VW>(p + sN + o);
            if (i + 1 < C.n) pd = ld_v<VW>(p + o + (int64_t)C.n * NB);
            if (j + 1 < C.n) pr = ld_v<VW>(p + sN + o + NB);
        }
        const float *win = win_stage(dyn, A, st);
        const Entry *sent = reinterpret_cast<const Entry *>(win + A.win_floats);
        const int b = ok ? spo[st][slot] : 0, e = ok ? spo[st][slot + 1] : 0;
        Vec<VW> acc = row_dot_smem<NB, G_>(sent, b, e, lr, win);
        if (ok && grp == 0) {
            Vec<VW> out;
#pragma unroll
            for (int c = 0; c < VW; ++c) {
                float gt = (i > 0 ? p0.v[c] : 0.f) - pd.v[c] + (j > 0 ? p1.v[c] : 0.f) - pr.v[c];
                out.v[c] = fmaf(C.mu, acc.v[c], gt);
                nrm[0].v[c] = fmaf(out.v[c], out.v[c], nrm[0].v[c]);
            }
            st_keep<VW>(G + o, out, l2_evict_last_policy());
        }
        __syncthreads();  // every read of this stage precedes its next copies
    }
    cp_async_wait<0>();
    reduce_images<NB, 1, kWinBlock>(nrm, part_of<NB>(D, C_BWD), D.red + R_GG * NB, D.ctr + C_BWD, smem);
}

// Step size and stopping test, FP64, one thread per channel (last block of k_fwd).
template <int NB>
__device__ void adm_finish(const AdmConst &C, const AdmDev &D)
{
    const int k = *D.k;
    // joint TV: thread 2s decides for the slice (channels 2s, 2s + 1) from
    // the sums of both channels' norms; the odd threads stay idle
    const int span = C.joint ? 2 : 1;
    if (threadIdx.x < NB && threadIdx.x % span == 0) {
        const int b = threadIdx.x;
        auto sum = [&](int slot) {
            double v = D.red[slot * NB + b];
            if (span == 2) v += D.red[slot * NB + b + 1];
            return v;
        };
        double alpha = 0.0;
        if (D.active[b]) {
            const double phi = sum(R_TV) + 0.5 * C.mu_d * sum(R_RR);
            if (!isfinite(phi)) atomicOr(D.bad, 1);
            bool stop = false;
            if (k > 0) {
                const double prev = D.phi_prev[b];
                const double rel = prev > 0.0 ? fabs(phi - prev) / prev : 0.0;
                D.rel[b] = rel;
                if (C.tol > 0.0 && rel < C.tol) stop = true;
            }
            if (stop) {
                D.active[b] = 0;
                D.conv[b] = 1;
                D.iters[b] = k;
            } else {
                D.phi_prev[b] = phi;
                const double gg = sum(R_GG), qq = sum(R_QQ), dd = sum(R_DD);
                const double den = C.mu_d * qq + C.rho_d * dd;
                const double c = den > 0.0 ? gg / den : 0.0;
                alpha = (C.rule == DECT_STEP_CAUCHY || k == 0) ? c : D.c_prev[b];
                D.c_prev[b] = c;
                D.iters[b] = k + 1;
            }
        }
        D.alpha[b] = alpha;
        if (span == 2) {
            D.alpha[b + 1] = alpha;
            D.active[b + 1] = D.active[b];
            D.conv[b + 1] = D.conv[b];
            D.iters[b + 1] = D.iters[b];
            D.rel[b + 1] = D.rel[b];
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int any = 0;
        for (int b = 0; b < NB; ++b) any |= D.active[b];
        *D.all_done = any ? 0 : 1;
        *D.k = k + 1;
    }
}

// MODE 1: |grad G|^2, then q = A G over the ray-major table and |q|^2; the
// last block forms the step.  MODE 0: r = A f - beta m (set-up).  MODE 2:
// r = A f - beta m and |r|^2 into the RR slot (residual of the projected
// f-step, run after k_tv).  MODE 3 (check of the result): the exact
// residual A f - beta m into dst, |A f - beta m|^2 into the QQ slot and
// |r_carried - (A f - beta m)|^2 into the GG slot (r_carried = rc).
// VWL = 4: lanes gather 4 images of an entry (row_dot_g); VWL = 8 or 16:
// lanes gather VWL images of an entry, R rounds in flight (row_dot_w; NB >=
// 16 only).
template <int NB, int G_, int MODE, int VWL = 4, int R = 2, int BLK = kFwdBlock>
__global__ void __launch_bounds__(BLK) k_fwd(const int64_t *__restrict__ rowptr,
                                                const Entry *__restrict__ ent,
                                                const float *__restrict__ src, float *__restrict__ dst,
                                                const float *__restrict__ m_planar,
                                                const float *__restrict__ beta_img, AdmConst C, AdmDev D,
                                                const float *__restrict__ rc = nullptr)
{
    constexpr int VW = Batch<NB>::VW, LPE = Batch<NB>::CPB, CPB = Batch<NB>::CPB;
    __shared__ double smem[reduce_smem_doubles<NB, BLK>(2)];
    const int lr = threadIdx.x % G_, grp = lr / LPE, vl = lr % LPE;
    const int64_t rpb = BLK / G_;
    Vec<VW> nrm[2];
    nrm[0].zero();
    nrm[1].zero();
    const unsigned long long pol = l2_evict_last_policy();
    if (MODE == 1) {
        // |grad G|^2, U pixels' loads issued together (the sum in plain loop order)
        constexpr int U = 2;
        const int64_t row = (int64_t)C.n * NB, tot = C.N * CPB, gs = (int64_t)gridDim.x * blockDim.x;
        for (int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t0 < tot; t0 += U * gs) {
            Vec<VW> gc[U], gu[U], gl[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t t = t0 + u * gs;
                if (t < tot) {
                    const int64_t pix = t / CPB;
                    const int i = (int)(pix / C.n), j = (int)(pix % C.n);
                    const int64_t o = pix * NB + (t % CPB) * VW;
                    gc[u] = ld_gather<VW>(src + o, pol);
                    gu[u] = i > 0 ? ld_gather<VW>(src + o - row, pol) : gc[u];
                    gl[u] = j > 0 ? ld_gather<VW>(src + o - NB, pol) : gc[u];
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (t0 + u * gs < tot) {
#pragma unroll
                    for (int c = 0; c < VW; ++c) {
                        float d0 = gc[u].v[c] - gu[u].v[c], d1 = gc[u].v[c] - gl[u].v[c];
                        nrm[0].v[c] += d0 * d0 + d1 * d1;
                    }
                }
            }
        }
    }
    const int64_t rstep = (int64_t)gridDim.x * rpb;
    for (int64_t row0 = (int64_t)blockIdx.x * rpb; row0 < C.M; row0 += rstep) {
        const int64_t ray = row0 + threadIdx.x / G_;
        int64_t b = 0, e = 0;
        if (ray < C.M) {
            b = rowptr[ray];
            e = rowptr[ray + 1];
        }
        Vec<VW> acc;
        if constexpr (VWL > 4 && NB >= 16)
            acc = row_dot_w<NB, G_, VWL, R>(ent, b, e, lr, src, pol, C.N, CHK_GATHER_A);
        else
            acc = row_dot<NB, G_, true>(ent, b, e, src, C.N, lr, CHK_GATHER_A);
        if (ray < C.M && grp == 0) {
            if (MODE != 1) {
#pragma unroll
                for (int c = 0; c < VW; ++c) {
                    const int img = vl * VW + c;
                    const int im = D.slot[img];
                    float g = im >= 0 ? beta_img[img] * m_planar[(int64_t)im * C.M + ray] : 0.f;
                    acc.v[c] -= g;
                    if (MODE >= 2) nrm[0].v[c] = fmaf(acc.v[c], acc.v[c], nrm[0].v[c]);
                }
                if (MODE == 3) {
                    const Vec<VW> rv = ld_v<VW>(rc + ray * NB + vl * VW);
#pragma unroll
                    for (int c = 0; c < VW; ++c) {
                        const float d = rv.v[c] - acc.v[c];
                        nrm[1].v[c] = fmaf(d, d, nrm[1].v[c]);
                    }
                }
            } else {
#pragma unroll
                for (int c = 0; c < VW; ++c) nrm[1].v[c] = fmaf(acc.v[c], acc.v[c], nrm[1].v[c]);
            }
            st_v<VW>(dst + ray * NB + vl * VW, acc);
        }
    }
    if (MODE == 1) {
        if (reduce_images<NB, 2, BLK>(nrm, part_of<NB>(D, C_FWD), D.red + R_DD * NB, D.ctr + C_FWD, smem))
            adm_finish<NB>(C, D);
    } else if (MODE == 2) {
        Vec<VW> rr[1] = {nrm[0]};
        reduce_images<NB, 1, BLK>(rr, part_of<NB>(D, C_RES), D.red + R_RR * NB, D.ctr + C_RES, smem);
    } else if (MODE == 3) {
        // QQ and GG are adjacent slots: (|A f - beta m|^2, |r_carried - (A f - beta m)|^2)
        static_assert(R_GG == R_QQ + 1, "slot order");
        reduce_images<NB, 2, BLK>(nrm, part_of<NB>(D, C_RES), D.red + R_QQ * NB, D.ctr + C_RES, smem);
    }
}

// Exact residual of the current f (f_cur) against the carried one, for the
// reports: QQ <- |A f - beta m|^2, GG <- |r - (A f - beta m)|^2 (q is
// overwritten; call only where q is no longer needed).


// planar x[img][N] (times beta) -> interleaved f[N][NB]; and back (divided by beta).
template <int NB>
__global__ void k_pack(const float *__restrict__ x, float *__restrict__ f, int64_t N, int nimg,
                       const float *__restrict__ beta_img)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * NB) return;
    int64_t pix = t / NB;
    int img = (int)(t % NB);
    f[t] = img < nimg ? beta_img[img] * x[(int64_t)img * N + pix] : 0.f;
}

// Slots that hold a caller image (and, with only_stopped, whose channel has
// stopped) write it to x[image].
template <int NB>
__global__ void k_unpack(const float *__restrict__ f, float *__restrict__ x, int64_t N,
                         const int *__restrict__ slot, const int *__restrict__ active, int only_stopped,
                         const float *__restrict__ beta_img)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * NB) return;
    int64_t pix = t / NB;
    const int j = (int)(t % NB), img = slot[j];
    if (img >= 0 && !(only_stopped && active[j])) x[(int64_t)img * N + pix] = f[t] / beta_img[j];
}

// Narrowing a batch: slot i of the NB2-wide state takes slot map[i] of the
// NB-wide one (map[i] < 0: an empty slot, zero).
template <int NB, int NB2>
__global__ void k_repack(const float *__restrict__ src, float *__restrict__ dst, int64_t rows,
                         const int *__restrict__ map)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= rows * NB2) return;
    const int64_t row = t / NB2;
    const int i = (int)(t % NB2), j = map[i];
    dst[t] = j >= 0 ? src[row * NB + j] : 0.f;
}

template <int NB, int NB2>
__global__ void k_repack_scalars(AdmDev D, AdmDev D2, const int *__restrict__ map,
                                 const float *__restrict__ beta, float *__restrict__ beta2)
{
    const int i = threadIdx.x;
    if (i < NB2) {
        const int j = map[i];
        const bool on = j >= 0;
        D2.alpha[i] = on ? D.alpha[j] : 0.0;
        D2.c_prev[i] = on ? D.c_prev[j] : 0.0;
        D2.phi_prev[i] = on ? D.phi_prev[j] : 0.0;
        D2.rel[i] = on ? D.rel[j] : 0.0;
        D2.iters[i] = on ? D.iters[j] : 0;
        D2.conv[i] = on ? D.conv[j] : 0;
        D2.active[i] = on ? D.active[j] : 0;
        D2.slot[i] = on ? D.slot[j] : -1;
        beta2[i] = on ? beta[j] : 1.f;
    }
    if (i == 0) {
        *D2.k = *D.k;
        *D2.all_done = 0;
        *D2.bad = *D.bad;
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
template <int NB>
struct Kern {
    static constexpr int GB = NB >= 32 ? 32 : 16;  // lanes per pixel row
    static constexpr int GF = 32;                  // lanes per ray row
};

// A variants (autotuner candidates, one 1024-thread block per SM, a warp
// per ray): 0 lanes gather 4 images of an entry; 1 lanes gather 8 images
// (row_dot_w), four rounds of gathers in flight; 2 as 1 with two rounds.
// Below 16 images only variant 0 exists (the others fall back to it).
constexpr int kFwdVariants = DECT_FWD_VARIANTS;

template <int NB, int MODE>
void launch_fwd(const dect_plan *P, int variant, const float *src, float *dst, const float *m,
                const float *beta, const AdmConst &C, const AdmDev &D, cudaStream_t s,
                const float *rc = nullptr)
{
    constexpr int GF = Kern<NB>::GF;
    switch (NB >= 16 ? variant : 0) {
    case 1:
        k_fwd<NB, GF, MODE, 8, 4, 1024><<<kFwdGrid, 1024, 0, s>>>(P->rowptr, P->ent, src, dst, m, beta, C, D, rc);
        break;
    case 2:
        k_fwd<NB, GF, MODE, 8, 2, 1024><<<kFwdGrid, 1024, 0, s>>>(P->rowptr, P->ent, src, dst, m, beta, C, D, rc);
        break;
    default:
        k_fwd<NB, GF, MODE, 4><<<kFwdGrid, 1024, 0, s>>>(P->rowptr, P->ent, src, dst, m, beta, C, D, rc);
        break;
    }
}

template <int NB>
void launch_residual_check(const dect_plan *P, int variant, const float *f_cur, float *q, const float *r,
                           const float *m, const float *beta, const AdmConst &C, const AdmDev &D,
                           cudaStream_t s)
{
    launch_fwd<NB, 3>(P, variant, f_cur, q, m, beta, C, D, s, r);
    count_launches(1);
}

struct Work {
    float *f[2], *G, *lam, *z, *p, *r, *q, *beta;
    const float *m;  // measured sinograms, planar [nimg][M]
    double *dbl;
    int *ints;
    int *map;         // [NB] slot map while narrowing into this workspace
    unsigned *ctr;
    AdmDev D;
    int win_grid;     // > 0: A^T through shared-memory windows with this grid
    size_t win_smem;  // its dynamic shared memory
    int bwd;          // A^T variant in use
    int fwd;          // A variant in use
    int tv;           // TV-step variant in use (0 k_tv, 1 k_tv_tma)
    int tv_grid;      // blocks of k_tv_tma
};

constexpr size_t kWinSmemMax = 210 * 1024;

// Enable the windowed A^T for this plan and batch width when two stages of
// its window and entries fit in shared memory.
template <int NB>
cudaError_t setup_window(const dect_plan *P, Work &W)
{
    W.win_grid = 0;
    W.win_smem = 0;
    if (P->win_max <= 0) return cudaSuccess;
    const size_t stage = (size_t)P->win_max * NB * sizeof(float) + (size_t)P->tile_ent_max * sizeof(Entry);
    const size_t bytes = 2 * stage + 2 * 3 * sizeof(int) * (size_t)P->nvp;
    if (bytes > kWinSmemMax) return cudaSuccess;
    auto kern = k_bwd_win<NB>;
    // the attribute is per kernel and process-wide: always the same cap, so
    // concurrent calls on plans with different windows cannot race on it
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWinSmemMax);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWinBlock, bytes);
    if (e != cudaSuccess) return e;
    if (per_sm <= 0) return cudaSuccess;
    int grid = kSMs * per_sm;
    if (grid > kGrid) grid = kGrid;
    if (grid > P->win_tiles) grid = P->win_tiles;
    W.win_grid = grid;
    W.win_smem = bytes;
    return cudaSuccess;
}

// A^T variants (autotuner candidates): 0-2 L1-cached gather with 4x4 / 8x8 /
// 16x16 pixel tiles per 256-thread block; 3 shared-memory sinogram windows;
// 4-5 L1-cached gather with one 1024-thread block per SM over tiles of two
// or four block steps (8 x 8 / 16 x 8 pixels at 32 lanes per pixel, 8 x 16 /
// 16 x 16 at 16), whose lines then stay in one L1; 6-7 lanes gather 8
// images of an entry (row_dot_w, NB >= 16 only): 6 with the lanes and tiles
// of 4; 7 with 16 lanes per pixel (two pixels per warp) over 8 x 8 tiles.
constexpr int kBwdVariants = DECT_BWD_VARIANTS;

template <int NB>
void launch_bwd(const dect_plan *P, const Work &W, const AdmConst &C, int variant, cudaStream_t s)
{
    constexpr int GB = Kern<NB>::GB;
    constexpr int RPS1k = 1024 / GB;  // pixels per step of a 1024-thread block
    switch (variant) {
    case 0:
        k_bwd<NB, GB, 4, 4, kBlock><<<kGrid, kBlock, 0, s>>>(P->colptr, P->tent, W.r, W.p, W.G, C, W.D);
        break;
    case 2:
        k_bwd<NB, GB, 16, 16, kBlock><<<kGrid, kBlock, 0, s>>>(P->colptr, P->tent, W.r, W.p, W.G, C, W.D);
        break;
    case 4:
        k_bwd<NB, GB, 8, RPS1k / 4, 1024><<<kSMs, 1024, 0, s>>>(P->colptr, P->tent, W.r, W.p, W.G, C, W.D);
        break;
    case 5:
        k_bwd<NB, GB, 16, RPS1k / 4, 1024><<<kSMs, 1024, 0, s>>>(P->colptr, P->tent, W.r, W.p, W.G, C, W.D);
        break;
    case 6:  // 8 images per lane, the lanes and tiles of variant 4
        if constexpr (NB >= 16)
            k_bwd<NB, GB, 8, RPS1k / 4, 1024, 8, 4><<<kSMs, 1024, 0, s>>>(P->colptr, P->tent, W.r, W.p, W.G, C, W.D);
        break;
    case 7:  // 8 images per lane, 16 lanes per pixel (two pixels per warp), 8 x 8 tiles
        if constexpr (NB >= 16)
            k_bwd<NB, 16, 8, 8, 1024, 8, 4><<<kSMs, 1024, 0, s>>>(P->colptr, P->tent, W.r, W.p, W.G, C, W.D);
        break;
    case 3: {
        WinArgs A{P->tmaj, P->tbase, P->tpo, P->wray0, P->wcnt, P->woff, P->wtot, P->nv, P->nvp,
                  P->win_max * NB, P->tile_ent_max};
        k_bwd_win<NB><<<W.win_grid, kWinBlock, W.win_smem, s>>>(A, W.r, W.p, W.G, C, W.D);
        break;
    }
    default:
        k_bwd<NB, GB, 8, 8, kBlock><<<kGrid, kBlock, 0, s>>>(P->colptr, P->tent, W.r, W.p, W.G, C, W.D);
        break;
    }
}

template <int NB>
constexpr int nb_index()
{
    return NB == 2 ? 0 : NB == 4 ? 1 : NB == 8 ? 2 : NB == 16 ? 3 : NB == 32 ? 4 : 5;
}

// Time every available A^T variant on this workspace (CUDA events, median of
// three launches after one warm-up) and keep the fastest in the plan.  The
// kernels only write G and reduction slots, which the first iteration
// rewrites, so timing them here changes no result.
template <int NB>
cudaError_t tune_bwd(const dect_plan *P, Work &W, const AdmConst &C, cudaStream_t s)
{
    const int idx = nb_index<NB>();
    if (P->bwd_choice[idx] >= 0) {
        W.bwd = P->bwd_choice[idx];
        if (W.bwd == 3 && W.win_grid <= 0) W.bwd = 1;
        if (W.bwd >= 6 && NB < 16) W.bwd = 4;
        return cudaSuccess;
    }
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    int best = 1;
    float best_us = 1e30f;
    for (int v = 0; v < kBwdVariants && e == cudaSuccess; ++v) {
        P->bwd_us[idx][v] = -1.f;
        if (v == 3 && W.win_grid <= 0) continue;
        if (v >= 6 && NB < 16) continue;  // wide-lane variants need 16 images
        launch_bwd<NB>(P, W, C, v, s);
        count_launches(1);
        float t[3];
        for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
            e = cudaEventRecord(a, s);
            launch_bwd<NB>(P, W, C, v, s);
            count_launches(1);
            if (e == cudaSuccess) e = cudaEventRecord(b, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(b);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t[k], a, b);
        }
        if (e != cudaSuccess) break;
        std::sort(t, t + 3);
        const float us = t[1] * 1e3f;
        P->bwd_us[idx][v] = us;
        if (us < best_us) {
            best_us = us;
            best = v;
        }
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    P->bwd_choice[idx] = best;
    W.bwd = best;
    return cudaSuccess;
}

// Time every A variant on the set-up projection r = A f - beta m (CUDA
// events, median of three launches after one warm-up) and keep the fastest
// in the plan.  The caller runs the set-up projection again afterwards with
// the chosen variant (the variants sum in different orders).
template <int NB>
cudaError_t tune_fwd(const dect_plan *P, Work &W, const AdmConst &C, cudaStream_t s)
{
    const int idx = nb_index<NB>();
    if (P->fwd_choice[idx] >= 0) {
        W.fwd = P->fwd_choice[idx];
        return cudaSuccess;
    }
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    int best = 0;
    float best_us = 1e30f;
    for (int v = 0; v < kFwdVariants && e == cudaSuccess; ++v) {
        P->fwd_us[idx][v] = -1.f;
        if (v > 0 && NB < 16) continue;  // only variant 0 below 16 images
        launch_fwd<NB, 0>(P, v, W.f[0], W.r, W.m, W.beta, C, W.D, s);
        count_launches(1);
        float t[3];
        for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
            e = cudaEventRecord(a, s);
            launch_fwd<NB, 0>(P, v, W.f[0], W.r, W.m, W.beta, C, W.D, s);
            count_launches(1);
            if (e == cudaSuccess) e = cudaEventRecord(b, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(b);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t[k], a, b);
        }
        if (e != cudaSuccess) break;
        std::sort(t, t + 3);
        const float us = t[1] * 1e3f;
        P->fwd_us[idx][v] = us;
        if (us < best_us) {
            best_us = us;
            best = v;
        }
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    P->fwd_choice[idx] = best;
    W.fwd = best;
    return cudaSuccess;
}

// TV-step variants (autotuner candidates): 0 k_tv (tiles claimed from a
// counter, rows exchanged through shared memory, one barrier per row); 1
// k_tv_tma (rows streamed by bulk copies into a ring of stages, NB >= 4).
// Both give the same images.
constexpr int kTvVariants = DECT_TV_VARIANTS;

// Prepare k_tv_tma for this width: its shared memory, and the grid (blocks
// that fit on an SM x SMs, at most kGrid, whose partials the reduction holds).
template <int NB>
cudaError_t setup_tv_tma(Work &W)
{
    W.tv_grid = 0;
    if constexpr (NB >= 4) {
        using T = TvTmaShape<NB>;
        cudaError_t e = cudaFuncSetAttribute(k_tv_tma<NB, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)T::SMEM);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_tv_tma<NB, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T::SMEM);
        int per_sm = 0;
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tv_tma<NB, false>, T::THREADS, T::SMEM);
        if (e != cudaSuccess) return e;
        W.tv_grid = std::min(std::max(per_sm, 0) * kSMs, kGrid);
    }
    return cudaSuccess;
}

template <int NB>
void launch_tv(const Work &W, const AdmConst &C, int par, int final_pass, cudaStream_t s);

// Time the TV-step variants (CUDA events, median of three launches after
// one warm-up) and keep the faster in the plan.  Called before the first
// iteration (k = 0, alpha = 0), where the step is idempotent: f[1] = f[0],
// r is unchanged and p (lambda, z) and the two norms are those the first
// iteration computes again, so timing changes no result.
template <int NB>
cudaError_t tune_tv(const dect_plan *P, Work &W, const AdmConst &C, cudaStream_t s)
{
    cudaError_t e = setup_tv_tma<NB>(W);
    if (e != cudaSuccess) return e;
    const int idx = nb_index<NB>();
    const bool tma_ok = NB >= 4 && W.tv_grid > 0;
    if (P->tv_choice[idx] >= 0) {
        W.tv = (P->tv_choice[idx] == 1 && tma_ok) ? 1 : 0;
        return cudaSuccess;
    }
    cudaEvent_t a = nullptr, b = nullptr;
    e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    int best = 0;
    float best_us = 1e30f;
    for (int v = 0; v < kTvVariants && e == cudaSuccess; ++v) {
        P->tv_us[idx][v] = -1.f;
        if (v == 1 && !tma_ok) continue;
        W.tv = v;
        launch_tv<NB>(W, C, 0, 0, s);
        count_launches(1);
        float t[3];
        for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
            e = cudaEventRecord(a, s);
            launch_tv<NB>(W, C, 0, 0, s);
            count_launches(1);
            if (e == cudaSuccess) e = cudaEventRecord(b, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(b);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t[k], a, b);
        }
        if (e != cudaSuccess) break;
        std::sort(t, t + 3);
        const float us = t[1] * 1e3f;
        P->tv_us[idx][v] = us;
        if (us < best_us) {
            best_us = us;
            best = v;
        }
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    P->tv_choice[idx] = best;
    W.tv = best;
    return cudaSuccess;
}

template <int NB>
void launch_tv(const Work &W, const AdmConst &C, int par, int final_pass, cudaStream_t s)
{
    if constexpr (NB >= 4) {
        if (W.tv == 1) {
            using T = TvTmaShape<NB>;
            if (C.joint)
                k_tv_tma<NB, true><<<W.tv_grid, T::THREADS, T::SMEM, s>>>(W.f[par], W.f[1 - par], W.G, W.lam, W.z,
                                                                          W.p, W.r, W.q, C, W.D, final_pass);
            else
                k_tv_tma<NB, false><<<W.tv_grid, T::THREADS, T::SMEM, s>>>(W.f[par], W.f[1 - par], W.G, W.lam, W.z,
                                                                           W.p, W.r, W.q, C, W.D, final_pass);
            return;
        }
    }
    using S = TvShape<NB>;
    const int ntiles = ((C.n + S::W - 1) / S::W) * ((C.n + S::H - 1) / S::H);
    const int grid = std::max(1, std::min(ntiles, kGrid));  // the partials hold kGrid blocks
    if (C.joint)
        k_tv<NB, true><<<grid, S::BLK, 0, s>>>(W.f[par], W.f[1 - par], W.G, W.lam, W.z, W.p, W.r, W.q, C,
                                                W.D, final_pass);
    else
        k_tv<NB, false><<<grid, S::BLK, 0, s>>>(W.f[par], W.f[1 - par], W.G, W.lam, W.z, W.p, W.r, W.q, C,
                                                 W.D, final_pass);
}

// Optional timing events around the two table kernels of one iteration.
struct IterEvents {
    cudaEvent_t b0, b1, f0, f1;
};

// Iteration with f read from f[par] and written to f[1 - par].
template <int NB>
void enqueue_iteration(const dect_plan *P, const Work &W, const AdmConst &C, int par, cudaStream_t s,
                       const IterEvents *ev)
{
    launch_tv<NB>(W, C, par, 0, s);
    if (C.nonneg) launch_fwd<NB, 2>(P, W.fwd, W.f[1 - par], W.r, W.m, W.beta, C, W.D, s);
    if (ev) cudaEventRecordWithFlags(ev->b0, s, cudaEventRecordExternal);
    launch_bwd<NB>(P, W, C, W.bwd, s);
    if (ev) cudaEventRecordWithFlags(ev->b1, s, cudaEventRecordExternal);
    if (ev) cudaEventRecordWithFlags(ev->f0, s, cudaEventRecordExternal);
    launch_fwd<NB, 1>(P, W.fwd, W.G, W.q, nullptr, nullptr, C, W.D, s);
    if (ev) cudaEventRecordWithFlags(ev->f1, s, cudaEventRecordExternal);
}

int kernels_per_iteration(const AdmConst &C) { return C.nonneg ? 4 : 3; }

// Workspace of one batch width: one allocation, laid out once to size and
// then for real, zeroed; the windowed A^T set up for this width.
template <int NB>
cudaError_t alloc_work(const dect_plan *P, Work &W, char **base_out, const float *m, cudaStream_t s)
{
    const int64_t N = P->N, M = P->M;
    const size_t nf = (size_t)N * NB, nr = (size_t)M * NB;
    const size_t ndbl = (size_t)R_COUNT * NB + (size_t)C_COUNT * 2 * kGrid * NB + 4 * NB;
    const size_t nint = 5 * NB + 8;
    auto layout = [&](char *b) -> size_t {
        size_t o = 0;
        auto take = [&](size_t nbytes) { char *p = b ? b + o : nullptr; o = (o + nbytes + 255) & ~(size_t)255; return p; };
        W.f[0] = (float *)take(nf * 4);
        W.f[1] = (float *)take(nf * 4);
        W.G = (float *)take(nf * 4);
        W.lam = (float *)take(2 * nf * 4);
        W.z = (float *)take(2 * nf * 4);
        W.p = (float *)take(2 * nf * 4);
        W.r = (float *)take((nr + 2 * NB) * 4);  // windows may end one ray past M
        W.q = (float *)take(nr * 4);
        W.beta = (float *)take(64 * 4);
        W.dbl = (double *)take(ndbl * 8);
        W.ints = (int *)take(nint * 4);
        W.ctr = (unsigned *)take((C_COUNT + 1) * 4);  // + the k_tv tile counter
        return o;
    };
    const size_t bytes = layout(nullptr);
    char *base = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&base, bytes, s);
    if (e != cudaSuccess) return e;
    *base_out = base;
    layout(base);
    W.m = m;
    AdmDev &D = W.D;
    D.red = W.dbl;
    D.part = D.red + R_COUNT * NB;
    D.alpha = D.part + (size_t)C_COUNT * 2 * kGrid * NB;
    D.c_prev = D.alpha + NB;
    D.phi_prev = D.c_prev + NB;
    D.rel = D.phi_prev + NB;
    D.iters = W.ints;
    D.conv = D.iters + NB;
    D.active = D.conv + NB;
    D.slot = D.active + NB;
    W.map = D.slot + NB;
    D.k = W.map + NB;
    D.all_done = D.k + 1;
    D.bad = D.all_done + 1;
    D.ctr = W.ctr;
    e = cudaMemsetAsync(base, 0, bytes, s);
    if (e == cudaSuccess) e = setup_window<NB>(P, W);
    return e;
}

// Average algorithmic bytes per profiled launch, folded over batch widths.
template <int NB>
void add_profile_bytes(const dect_plan *P, dect_adm_profile *prof, int64_t launches_before)
{
    if (!prof) return;
    const int64_t now = prof->fwd_launches, add = now - launches_before;
    if (now <= 0 || add <= 0) return;
    // A: table + row pointers, G read, q written
    const double fwd = 8.0 * P->nnz + 8.0 * (P->M + 1) + 4.0 * NB * (P->N + P->M);
    // A^T: table + column pointers, r and the two components of p read, G written
    const double bwd = 8.0 * P->nnz + 8.0 * (P->N + 1) + 4.0 * NB * (P->M + 3 * P->N);
    prof->table_bytes_fwd = (int64_t)(((double)prof->table_bytes_fwd * launches_before + fwd * add) / now);
    prof->table_bytes_bwd = (int64_t)(((double)prof->table_bytes_bwd * launches_before + bwd * add) / now);
}

// Report of the caller image held by slot j, from host copies of the
// reduction slots and per-slot counters.
inline void fill_report(dect_adm_report &r, int NB, int j, const AdmConst &C, double mu, int K,
                        const std::vector<double> &hred, const std::vector<double> &hrel,
                        const std::vector<int> &hit, const std::vector<int> &hconv)
{
    r.iters = K == 0 ? 0 : hit[j];
    r.converged = hconv[j];
    if (C.joint) {  // the slice's joint objective, reported on both of its channels
        const int j0 = j & ~1;
        r.objective = hred[R_TV * NB + j0] + hred[R_TV * NB + j0 + 1] +
                      0.5 * mu * (hred[R_RR * NB + j0] + hred[R_RR * NB + j0 + 1]);
    } else {
        r.objective = hred[R_TV * NB + j] + 0.5 * mu * hred[R_RR * NB + j];
    }
    r.rel_change = hrel[j];
    r.primal_res = std::sqrt(hred[R_QQ * NB + j]);
    r.resid_drift = std::sqrt(hred[R_GG * NB + j]);
}

// The iteration loop at batch width NB from iteration done_iters on, with W
// holding the state (freed before return).  With the relative-objective stop,
// once no more than half of the slots hold running channels the batch is
// narrowed: the stopped channels' images and reports are written out (their
// f no longer changes: alpha = 0), the running channels' whole state (f, G,
// lambda, z, p, r, q and the per-channel scalars) is repacked into an
// NB/2-wide workspace, and the loop goes on there with the narrower kernels.
// The iterates are those of the NB-wide run; only the order of the FP64
// cross-block sums follows the new width.
template <int NB>
dect_status iterate(const dect_plan *P, const AdmConst &C, Work W, char *base, float *x,
                    const dect_adm_params *prm, dect_adm_report *rep, dect_adm_profile *prof, cudaStream_t s,
                    int done_iters)
{
    const int64_t N = P->N, tn = N * NB;
    AdmDev &D = W.D;
    const int64_t prof_before = prof ? prof->fwd_launches : 0;
    const int K = prm->max_iter;
    const bool use_tol = prm->rel_obj_tol > 0.0;
    int block = use_tol ? (prm->check_every > 0 ? prm->check_every : 10) : 10;
    block = std::max(2, block + (block & 1));
    cudaStream_t cs = nullptr;
    cudaEvent_t ev = nullptr;
    std::vector<IterEvents> evs;  // [block] for the block graph, then [2] for the single graphs
    cudaGraphExec_t gx_block = nullptr, gx_one[2] = {nullptr, nullptr};
    int *h_flags = nullptr;       // pinned: [0] all_done, [1 .. NB] active
    char *base2 = nullptr;        // the narrowed workspace, once handed on
    cudaError_t err = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (err == cudaSuccess && prof) {
        evs.resize(block + 2);
        for (auto &e : evs) {
            if (err == cudaSuccess) err = cudaEventCreate(&e.b0);
            if (err == cudaSuccess) err = cudaEventCreate(&e.b1);
            if (err == cudaSuccess) err = cudaEventCreate(&e.f0);
            if (err == cudaSuccess) err = cudaEventCreate(&e.f1);
        }
    }
    auto make_graph = [&](int iters, int par0, int ev0, cudaGraphExec_t *out) -> cudaError_t {
        cudaGraph_t gr = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        for (int it = 0; it < iters; ++it)
            // timing events around the middle iteration of the graph only:
            // an event pair per launch costs the iteration a few microseconds
            enqueue_iteration<NB>(P, W, C, (par0 + it) & 1, cs,
                                  prof && it == iters / 2 ? &evs[ev0 + it] : nullptr);
        e = cudaStreamEndCapture(cs, &gr);
        if (e != cudaSuccess) return e;
        e = cudaGraphInstantiate(out, gr, 0);
        cudaGraphDestroy(gr);
        return e;
    };
    // time read-back of the events of a graph of `iters` iterations whose
    // events start at ev0 (those of its middle iteration)
    auto collect = [&](int iters, int ev0) -> cudaError_t {
        if (!prof) return cudaSuccess;
        cudaError_t e = cudaStreamSynchronize(cs);
        for (int it = iters / 2; it == iters / 2 && e == cudaSuccess; ++it) {
            float mb = 0.f, mf = 0.f;
            e = cudaEventElapsedTime(&mb, evs[ev0 + it].b0, evs[ev0 + it].b1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&mf, evs[ev0 + it].f0, evs[ev0 + it].f1);
            prof->bwd_ms_total += mb;
            prof->fwd_ms_total += mf;
            prof->bwd_launches += 1;
            prof->fwd_launches += 1;
        }
        return e;
    };
    // the caller's stream orders the set-up; the capture stream runs the loop
    if (err == cudaSuccess) err = cudaEventRecord(ev, s);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(cs, ev, 0);
    const int remaining = K - done_iters;
    if (err == cudaSuccess && remaining >= block) err = make_graph(block, done_iters & 1, 0, &gx_block);
    if (err == cudaSuccess && remaining % block) {
        err = make_graph(1, 0, block, &gx_one[0]);
        if (err == cudaSuccess) err = make_graph(1, 1, block + 1, &gx_one[1]);
    }
    if (err == cudaSuccess) err = cudaMallocHost((void **)&h_flags, sizeof(int) * (NB + 1));
    if (h_flags) h_flags[0] = 0;
    while (err == cudaSuccess && done_iters + block <= K) {
        err = cudaGraphLaunch(gx_block, cs);
        count_launches((int64_t)kernels_per_iteration(C) * block);
        done_iters += block;
        if (err == cudaSuccess) err = collect(block, 0);
        if (err == cudaSuccess && use_tol) {
            err = cudaMemcpyAsync(h_flags, D.all_done, sizeof(int), cudaMemcpyDeviceToHost, cs);
            if (err == cudaSuccess && NB >= 4)
                err = cudaMemcpyAsync(h_flags + 1, D.active, sizeof(int) * NB, cudaMemcpyDeviceToHost, cs);
            if (err == cudaSuccess) err = cudaStreamSynchronize(cs);
            if (err == cudaSuccess && h_flags[0]) break;
            if constexpr (NB >= 4) {
                int live = 0;
                for (int j = 0; j < NB; ++j) live += h_flags[1 + j] ? 1 : 0;
                if (err == cudaSuccess && live <= NB / 2 && done_iters < K) {
                    // narrow: write out the stopped channels, repack the running ones
                    constexpr int NB2 = NB / 2;
                    const int par = done_iters & 1;
                    std::vector<double> hred(R_COUNT * NB), hrel(NB);
                    std::vector<int> hit(NB), hconv(NB), hslot(NB);
                    if (err == cudaSuccess) {
                        k_unpack<NB><<<(unsigned)((tn + 255) / 256), 256, 0, cs>>>(W.f[par], x, N, D.slot, D.active, 1,
                                                                                   W.beta);
                        err = cudaGetLastError();
                        count_launches(1);
                    }
                    std::vector<int> map(NB2, -1);
                    for (int j = 0, i = 0; j < NB; ++j)
                        if (h_flags[1 + j]) map[i++] = j;  // running channels, in order (pairs stay pairs)
                    Work W2;
                    err = alloc_work<NB2>(P, W2, &base2, W.m, cs);
                    if (err == cudaSuccess) {
                        W2.bwd = 1;
                        W2.fwd = 0;
                        // time the A and A^T variants on the empty workspace, before the state arrives
                        W2.tv = 0;
                        err = tune_bwd<NB2>(P, W2, C, cs);
                        if (err == cudaSuccess) err = tune_fwd<NB2>(P, W2, C, cs);
                        if (err == cudaSuccess) err = tune_tv<NB2>(P, W2, C, cs);
                    }
                    if (err == cudaSuccess)
                        err = cudaMemcpyAsync(W2.map, map.data(), sizeof(int) * NB2, cudaMemcpyHostToDevice, cs);
                    if (err == cudaSuccess) {
                        auto rp = [&](const float *src, float *dst, int64_t rows) {
                            const int64_t t = rows * NB2;
                            k_repack<NB, NB2><<<(unsigned)((t + 255) / 256), 256, 0, cs>>>(src, dst, rows, W2.map);
                        };
                        rp(W.f[par], W2.f[par], N);
                        rp(W.G, W2.G, N);
                        rp(W.lam, W2.lam, 2 * N);
                        rp(W.z, W2.z, 2 * N);
                        rp(W.p, W2.p, 2 * N);
                        rp(W.r, W2.r, P->M);
                        rp(W.q, W2.q, P->M);
                        k_repack_scalars<NB, NB2><<<1, 64, 0, cs>>>(D, W2.D, W2.map, W.beta, W2.beta);
                        err = cudaGetLastError();
                        count_launches(8);
                    }
                    // the state has moved: check the stopped channels' carried
                    // residual against A f - beta m (q and the QQ / GG slots of
                    // this workspace are free now), then write their reports
                    if (err == cudaSuccess) {
                        launch_residual_check<NB>(P, W.fwd, W.f[par], W.q, W.r, W.m, W.beta, C, D, cs);
                        err = cudaGetLastError();
                    }
                    if (err == cudaSuccess) err = cudaMemcpyAsync(hred.data(), D.red, sizeof(double) * R_COUNT * NB, cudaMemcpyDeviceToHost, cs);
                    if (err == cudaSuccess) err = cudaMemcpyAsync(hrel.data(), D.rel, sizeof(double) * NB, cudaMemcpyDeviceToHost, cs);
                    if (err == cudaSuccess) err = cudaMemcpyAsync(hit.data(), D.iters, sizeof(int) * NB, cudaMemcpyDeviceToHost, cs);
                    if (err == cudaSuccess) err = cudaMemcpyAsync(hconv.data(), D.conv, sizeof(int) * NB, cudaMemcpyDeviceToHost, cs);
                    if (err == cudaSuccess) err = cudaMemcpyAsync(hslot.data(), D.slot, sizeof(int) * NB, cudaMemcpyDeviceToHost, cs);
                    if (err == cudaSuccess) err = cudaStreamSynchronize(cs);
                    if (err == cudaSuccess && rep)
                        for (int j = 0; j < NB; ++j)
                            if (hslot[j] >= 0 && !h_flags[1 + j])
                                fill_report(rep[hslot[j]], NB, j, C, prm->mu, K, hred, hrel, hit, hconv);
                    // the state now lives in the narrowed workspace
                    if (err == cudaSuccess) err = cudaEventRecord(ev, cs);
                    if (err == cudaSuccess) err = cudaStreamWaitEvent(s, ev, 0);
                    if (err == cudaSuccess) {
                        // release this phase, then continue at NB2
                        add_profile_bytes<NB>(P, prof, prof_before);
                        cudaFreeAsync(base, s);
                        base = nullptr;
                        if (gx_block) cudaGraphExecDestroy(gx_block);
                        if (gx_one[0]) cudaGraphExecDestroy(gx_one[0]);
                        if (gx_one[1]) cudaGraphExecDestroy(gx_one[1]);
                        gx_block = gx_one[0] = gx_one[1] = nullptr;
                        cudaStreamSynchronize(cs);
                        for (auto &e : evs) {
                            cudaEventDestroy(e.b0); cudaEventDestroy(e.b1);
                            cudaEventDestroy(e.f0); cudaEventDestroy(e.f1);
                        }
                        evs.clear();
                        cudaFreeHost(h_flags);
                        h_flags = nullptr;
                        cudaEventDestroy(ev);
                        cudaStreamDestroy(cs);
                        return iterate<NB2>(P, C, W2, base2, x, prm, rep, prof, s, done_iters);
                    }
                    break;
                }
            }
        }
    }
    bool finished = use_tol && err == cudaSuccess && h_flags && h_flags[0];
    while (err == cudaSuccess && !finished && done_iters < K) {
        const int par = done_iters & 1;
        err = cudaGraphLaunch(gx_one[par], cs);
        count_launches(kernels_per_iteration(C));
        ++done_iters;
        if (err == cudaSuccess) err = collect(1, block + par);
    }
    // final step f^K = f^{K-1} - alpha G and the objective at the result
    const int par = done_iters & 1;
    if (err == cudaSuccess) {
        launch_tv<NB>(W, C, par, 1, cs);
        if (C.nonneg) launch_fwd<NB, 2>(P, W.fwd, W.f[1 - par], W.r, W.m, W.beta, C, D, cs);
        k_unpack<NB><<<(unsigned)((tn + 255) / 256), 256, 0, cs>>>(W.f[1 - par], x, N, D.slot, D.active, 0,
                                                                   W.beta);
        count_launches(C.nonneg ? 3 : 2);
        launch_residual_check<NB>(P, W.fwd, W.f[1 - par], W.q, W.r, W.m, W.beta, C, D, cs);
        err = cudaGetLastError();
    }
    if (err == cudaSuccess) err = cudaEventRecord(ev, cs);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(s, ev, 0);
    add_profile_bytes<NB>(P, prof, prof_before);

    std::vector<double> hred(R_COUNT * NB), hrel(NB);
    std::vector<int> hit(NB), hconv(NB), hslot(NB);
    int hbad = 0;
    if (err == cudaSuccess) err = cudaMemcpyAsync(hred.data(), D.red, sizeof(double) * R_COUNT * NB, cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaMemcpyAsync(hrel.data(), D.rel, sizeof(double) * NB, cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaMemcpyAsync(hit.data(), D.iters, sizeof(int) * NB, cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaMemcpyAsync(hconv.data(), D.conv, sizeof(int) * NB, cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaMemcpyAsync(hslot.data(), D.slot, sizeof(int) * NB, cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaMemcpyAsync(&hbad, D.bad, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (base) cudaFreeAsync(base, s);
    if (base2) cudaFreeAsync(base2, s);  // a narrowing that failed half-way
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    if (gx_block) cudaGraphExecDestroy(gx_block);
    if (gx_one[0]) cudaGraphExecDestroy(gx_one[0]);
    if (gx_one[1]) cudaGraphExecDestroy(gx_one[1]);
    if (h_flags) cudaFreeHost(h_flags);
    for (auto &e : evs) {
        cudaEventDestroy(e.b0); cudaEventDestroy(e.b1);
        cudaEventDestroy(e.f0); cudaEventDestroy(e.f1);
    }
    if (ev) cudaEventDestroy(ev);
    if (cs) cudaStreamDestroy(cs);
    if (err != cudaSuccess) {
        set_error("dect_adm_tv", err);
        return err == cudaErrorMemoryAllocation ? DECT_ERR_OOM : DECT_ERR_CUDA;
    }
    if (rep)
        for (int j = 0; j < NB; ++j)
            if (hslot[j] >= 0) fill_report(rep[hslot[j]], NB, j, C, prm->mu, K, hred, hrel, hit, hconv);
    if (hbad & 2) {
        set_error_text("dect_adm_tv: a bounded wait of the TV step ran out");
        return DECT_ERR_TIMEOUT;
    }
    return (hbad & 1) ? DECT_ERR_NONFINITE : DECT_OK;
}

AdmConst adm_const(const dect_plan *P, const dect_adm_params *prm)
{
    AdmConst C;
    C.n = P->n;
    C.N = P->N;
    C.M = P->M;
    C.mu = (float)prm->mu;
    C.rho = (float)prm->rho;
    double xi = prm->xi > 0 ? prm->xi : prm->rho;
    C.xi = (float)xi;
    C.nonneg = prm->nonneg ? 1 : 0;
    C.joint = prm->joint_tv ? 1 : 0;
    C.xi_is_rho = (xi == prm->rho && !C.nonneg) ? 1 : 0;
    C.mu_d = prm->mu;
    C.rho_d = prm->rho;
    C.tol = prm->rel_obj_tol;
    C.rule = prm->step_rule;
    return C;
}

// Autotune the A, A^T and TV-step variants of width NB and of every width a
// batch of NB can narrow to, each on an empty workspace (as a narrowing does
// before the state arrives), so that chunks run side by side later find
// their choices made and no timing sees another chunk's kernels.  m: a
// sinogram of the plan (read by the set-up projection only).
template <int NB>
cudaError_t pretune(const dect_plan *P, const float *m, const AdmConst &C, cudaStream_t s)
{
    const int idx = nb_index<NB>();
    cudaError_t e = cudaSuccess;
    if (P->bwd_choice[idx] < 0 || P->fwd_choice[idx] < 0 || P->tv_choice[idx] < 0) {
        Work W;
        char *base = nullptr;
        e = alloc_work<NB>(P, W, &base, m, s);
        W.bwd = 1;
        W.fwd = 0;
        W.tv = 0;
        if (e == cudaSuccess) e = tune_bwd<NB>(P, W, C, s);
        if (e == cudaSuccess) e = tune_fwd<NB>(P, W, C, s);
        if (e == cudaSuccess) e = tune_tv<NB>(P, W, C, s);
        if (base) cudaFreeAsync(base, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if constexpr (NB > 2) {
        if (e == cudaSuccess) e = pretune<NB / 2>(P, m, C, s);
    }
    return e;
}

template <int NB>
dect_status run_chunk(const dect_plan *P, const float *m, float *x, int nimg,
                      const dect_adm_params *prm, const float *beta_host, dect_adm_report *rep,
                      dect_adm_profile *prof, cudaStream_t s)
{
    const int64_t N = P->N;
    const AdmConst C = adm_const(P, prm);

    Work W;
    char *base = nullptr;
    cudaError_t e = alloc_work<NB>(P, W, &base, m, s);
    if (e != cudaSuccess) {
        if (base) cudaFreeAsync(base, s);
        set_error("dect_adm_tv", e);
        return e == cudaErrorMemoryAllocation ? DECT_ERR_OOM : DECT_ERR_CUDA;
    }
    AdmDev &D = W.D;
    std::vector<float> hbeta(64, 1.f);
    std::vector<int> hact(NB, 0), hslot(NB, -1);
    for (int b = 0; b < nimg; ++b) {
        hbeta[b] = beta_host[b];
        hact[b] = 1;
        hslot[b] = b;
    }
    // zero state (the workspace is cleared); G = q = 0 and alpha = 0 make the
    // first step of k_tv a no-op
    auto fail = [&](cudaError_t err) {
        cudaFreeAsync(base, s);
        set_error("dect_adm_tv", err);
        return err == cudaErrorMemoryAllocation ? DECT_ERR_OOM : DECT_ERR_CUDA;
    };
    if ((e = cudaMemcpyAsync(W.beta, hbeta.data(), 64 * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpyAsync(D.active, hact.data(), NB * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpyAsync(D.slot, hslot.data(), NB * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess) return fail(e);
    const int64_t tn = N * NB;
    if (prm->warm_start) {
        k_pack<NB><<<(unsigned)((tn + 255) / 256), 256, 0, s>>>(x, W.f[0], N, nimg, W.beta);
        count_launches(1);
    }
    // r^0 = A f^0 - beta m, with the A variant the autotuner keeps
    W.fwd = 0;
    if ((e = tune_fwd<NB>(P, W, C, s)) != cudaSuccess) return fail(e);
    launch_fwd<NB, 0>(P, W.fwd, W.f[0], W.r, m, W.beta, C, D, s);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
    W.bwd = 1;
    if ((e = tune_bwd<NB>(P, W, C, s)) != cudaSuccess) return fail(e);
    W.tv = 0;
    if ((e = tune_tv<NB>(P, W, C, s)) != cudaSuccess) return fail(e);
    // (hbeta, hact and hslot are pageable: their copies have read them by now)
    return iterate<NB>(P, C, W, base, x, prm, rep, prof, s, 0);
}

}  // namespace
}  // namespace dect

using namespace dect;

extern "C" dect_status dect_adm_tv_ex(const dect_plan *plan, const float *m, float *x, int n_slices,
                                      const dect_adm_params *prm, dect_adm_report *reports,
                                      dect_adm_profile *prof, dect_stream stream)
{
    if (!plan || !prm || n_slices < 0 || plan->nz > 0) return DECT_ERR_INVALID_ARG;  // fan-beam plans only
    if (n_slices == 0) return DECT_OK;
    if (!m || !x) return DECT_ERR_INVALID_ARG;
    if (!(prm->mu > 0) || !(prm->rho > 0) || !(prm->beta[0] > 0) || !(prm->beta[1] > 0) ||
        prm->max_iter < 0 || (prm->step_rule != DECT_STEP_BB1 && prm->step_rule != DECT_STEP_CAUCHY) ||
        !std::isfinite(prm->mu) || !std::isfinite(prm->rho) || !std::isfinite(prm->xi) ||
        !std::isfinite(prm->beta[0]) || !std::isfinite(prm->beta[1]) || prm->check_every < 0 ||
        (prm->nonneg != 0 && prm->nonneg != 1) || (prm->joint_tv != 0 && prm->joint_tv != 1))
        return DECT_ERR_INVALID_ARG;
    DECT_CUDA(cudaSetDevice(plan->device));
    cudaStream_t s = (cudaStream_t)stream;
    if (prof) {
        prof->fwd_ms_total = prof->bwd_ms_total = 0.0;
        prof->table_bytes_fwd = prof->table_bytes_bwd = 0;
        prof->fwd_launches = prof->bwd_launches = 0;
    }
    const int total = 2 * n_slices;
    const int nchunks = (total + kMaxBatchImages - 1) / kMaxBatchImages;
    // one chunk of up to kMaxBatchImages channels (32 slices) on stream st
    auto run_one = [&](int ci, cudaStream_t st, dect_adm_profile *pf) -> dect_status {
        const int c0 = ci * kMaxBatchImages;
        const int nimg = std::min(kMaxBatchImages, total - c0);
        std::vector<float> beta(nimg);
        for (int b = 0; b < nimg; ++b) beta[b] = (float)prm->beta[(c0 + b) % 2];
        const float *mc = m + (int64_t)c0 * plan->M;
        float *xc = x + (int64_t)c0 * plan->N;
        dect_adm_report *rc = reports ? reports + c0 : nullptr;
        if (nimg <= 2) return run_chunk<2>(plan, mc, xc, nimg, prm, beta.data(), rc, pf, st);
        if (nimg <= 4) return run_chunk<4>(plan, mc, xc, nimg, prm, beta.data(), rc, pf, st);
        if (nimg <= 8) return run_chunk<8>(plan, mc, xc, nimg, prm, beta.data(), rc, pf, st);
        if (nimg <= 16) return run_chunk<16>(plan, mc, xc, nimg, prm, beta.data(), rc, pf, st);
        if (nimg <= 32) return run_chunk<32>(plan, mc, xc, nimg, prm, beta.data(), rc, pf, st);
        return run_chunk<64>(plan, mc, xc, nimg, prm, beta.data(), rc, pf, st);
    };
    if (nchunks == 1) return run_one(0, s, prof);

    // Several chunks: two at a time, each from its own host thread on its
    // own stream, so that one chunk's kernels fill the SMs another leaves
    // idle (the tail of each launch, the narrowed end of each chunk).  Every
    // width is autotuned first; chunks share no data, so each gives the
    // result it gives alone.
    {
        cudaError_t e = pretune<kMaxBatchImages>(plan, m, adm_const(plan, prm), s);
        if (e != cudaSuccess) {
            set_error("dect_adm_tv", e);
            return e == cudaErrorMemoryAllocation ? DECT_ERR_OOM : DECT_ERR_CUDA;
        }
    }
    cudaEvent_t start = nullptr;
    DECT_CUDA(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
    DECT_CUDA(cudaEventRecord(start, s));
    std::vector<dect_status> status(nchunks, DECT_OK);
    std::vector<dect_adm_profile> profs(nchunks, dect_adm_profile{});
    std::vector<std::string> errs(nchunks);
    std::vector<cudaEvent_t> done(nchunks, nullptr);
    std::atomic<int> next{0};
    auto work = [&]() {
        cudaSetDevice(plan->device);
        cudaStream_t ws = nullptr;
        if (cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) != cudaSuccess) {
            for (int c; (c = next.fetch_add(1)) < nchunks;) status[c] = DECT_ERR_CUDA;
            return;
        }
        for (int c; (c = next.fetch_add(1)) < nchunks;) {
            if (cudaStreamWaitEvent(ws, start, 0) != cudaSuccess) {
                status[c] = DECT_ERR_CUDA;
                continue;
            }
            status[c] = run_one(c, ws, prof ? &profs[c] : nullptr);
            if (status[c] != DECT_OK) errs[c] = dect_last_error();
            cudaEvent_t ev = nullptr;
            if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess &&
                cudaEventRecord(ev, ws) == cudaSuccess)
                done[c] = ev;
        }
        cudaStreamSynchronize(ws);
        cudaStreamDestroy(ws);
    };
    std::thread second(work);
    work();
    second.join();
    dect_status worst = DECT_OK;
    for (int c = 0; c < nchunks; ++c) {
        if (done[c]) {
            cudaStreamWaitEvent(s, done[c], 0);
            cudaEventDestroy(done[c]);
        }
        if (status[c] == DECT_ERR_NONFINITE) {
            if (worst == DECT_OK) worst = status[c];
        } else if (status[c] != DECT_OK && (worst == DECT_OK || worst == DECT_ERR_NONFINITE)) {
            worst = status[c];
            set_error_text(errs[c]);
        }
        if (prof) {
            const dect_adm_profile &q = profs[c];
            const int64_t n0 = prof->fwd_launches, n1 = n0 + q.fwd_launches;
            if (n1 > 0) {
                prof->table_bytes_fwd = (int64_t)(((double)prof->table_bytes_fwd * n0 +
                                                   (double)q.table_bytes_fwd * q.fwd_launches) / n1);
                prof->table_bytes_bwd = (int64_t)(((double)prof->table_bytes_bwd * n0 +
                                                   (double)q.table_bytes_bwd * q.fwd_launches) / n1);
            }
            prof->fwd_ms_total += q.fwd_ms_total;
            prof->bwd_ms_total += q.bwd_ms_total;
            prof->fwd_launches = n1;
            prof->bwd_launches += q.bwd_launches;
        }
    }
    cudaEventDestroy(start);
    return worst;
}

extern "C" dect_status dect_adm_tv(const dect_plan *plan, const float *m, float *x, int n_slices,
                                   const dect_adm_params *prm, dect_adm_report *reports,
                                   dect_stream stream)
{
    return dect_adm_tv_ex(plan, m, x, n_slices, prm, reports, nullptr, stream);
}

extern "C" dect_status dect_adm_tv_groups(const dect_adm_group *groups, int n_groups,
                                          const dect_adm_params *prm, int workers, dect_stream stream)
{
    if (!groups || n_groups < 0 || !prm || workers < 0) return DECT_ERR_INVALID_ARG;
    if (n_groups == 0) return DECT_OK;
    for (int i = 0; i < n_groups; ++i) {
        if (!groups[i].plan || groups[i].n_slices < 0 || groups[i].plan->nz > 0) return DECT_ERR_INVALID_ARG;
        for (int j = 0; j < i; ++j)
            if (groups[j].plan == groups[i].plan) return DECT_ERR_INVALID_ARG;  // plans must differ
    }
    const int device = groups[0].plan->device;
    for (int i = 1; i < n_groups; ++i)
        if (groups[i].plan->device != device) return DECT_ERR_INVALID_ARG;
    DECT_CUDA(cudaSetDevice(device));
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t start = nullptr;
    DECT_CUDA(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
    DECT_CUDA(cudaEventRecord(start, s));
    const int nw = workers > 0 ? std::min(workers, n_groups) : std::min(n_groups, 8);
    std::vector<dect_status> status(n_groups, DECT_OK);
    std::vector<cudaEvent_t> done(n_groups, nullptr);
    std::atomic<int> next{0};
    auto work = [&]() {
        cudaSetDevice(device);
        cudaStream_t ws = nullptr;
        if (cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) != cudaSuccess) {
            for (int g; (g = next.fetch_add(1)) < n_groups;) status[g] = DECT_ERR_CUDA;
            return;
        }
        for (int g; (g = next.fetch_add(1)) < n_groups;) {
            if (cudaStreamWaitEvent(ws, start, 0) != cudaSuccess) {
                status[g] = DECT_ERR_CUDA;
                continue;
            }
            const dect_adm_group &G = groups[g];
            status[g] = dect_adm_tv(G.plan, G.m, G.x, G.n_slices, prm, G.reports, (dect_stream)ws);
            cudaEvent_t e = nullptr;
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess &&
                cudaEventRecord(e, ws) == cudaSuccess)
                done[g] = e;
        }
        cudaStreamSynchronize(ws);
        cudaStreamDestroy(ws);
    };
    std::vector<std::thread> pool;
    for (int w = 1; w < nw; ++w) pool.emplace_back(work);
    work();
    for (auto &t : pool) t.join();
    dect_status first = DECT_OK;
    for (int g = 0; g < n_groups; ++g) {
        if (done[g]) {
            cudaStreamWaitEvent(s, done[g], 0);
            cudaEventDestroy(done[g]);
        }
        if (first == DECT_OK && status[g] != DECT_OK) first = status[g];
    }
    cudaEventDestroy(start);
    DECT_CUDA(cudaStreamSynchronize(s));
    return first;
}
