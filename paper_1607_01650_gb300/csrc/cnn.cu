// CNN warm start: a small encoder-decoder that maps a short ADM
// reconstruction to an estimate of the converged one, from which ADM then
// continues.  Not part of the paper's method; the learned part of the
// workload.  Network (3x3 convolutions with bias, ReLU after each):
//
//   a1 = conv(x/s, 1->32)   e1 = conv(a1, 32->32)                 H x W
//   p1 = avgpool2(e1)  a3 = conv(p1, 32->64)   e2 = conv(a3, 64->64)
//   p2 = avgpool2(e2)  a5 = conv(p2, 64->128)  bt = conv(a5, 128->128)
//   c2 = [up2(bt), e2] a7 = conv(c2, 192->64)  d2 = conv(a7, 64->64)
//   c1 = [up2(d2), e1] a9 = conv(c1, 96->32)   d1 = conv(a9, 32->32)
//   out = x + s (Wh . d1 + bh)                                    (1x1 head)
//
// Activations are NHWC BF16 (channel counts padded to multiples of 32; the
// input has 32 channels of which only the first is non-zero); the 3x3
// convolutions are implicit GEMMs on the 5th-generation tensor cores
// (tcgen05.mma, BF16 inputs, FP32 accumulation in tensor memory, operands
// staged by TMA): k_conv_tc for the forward pass and the input gradients
// (the same kernel with the weights flipped and transposed), k_wgrad_tc for
// the weight gradients, whose per-block partials are added in a fixed order.
// The warp-level mma.sync kernels (k_conv, k_wgrad) remain as a second,
// selectable path.  Master weights, gradients and the Adam state are FP32.  Parameter vector layout (shared with the host):
// per layer W[Cout][Cin][3][3] then b[Cout]; then the head Wh[32], bh.
#include <cuda.h>  // CUtensorMap and its enums (the encoder is fetched from the driver at run time)
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cudaTypedefs.h>  // PFN_cuTensorMapEncodeTiled_v12000

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "dect_internal.cuh"
#include "kernels.cuh"

typedef __nv_bfloat16 bf16;

namespace dect {
namespace {

constexpr int kLayers = 10;
constexpr int kCin[kLayers] = {1, 32, 32, 64, 64, 128, 192, 64, 96, 32};
constexpr int kCout[kLayers] = {32, 32, 64, 64, 128, 128, 64, 64, 32, 32};

int cin_pad(int l) { return kCin[l] < 32 ? 32 : kCin[l]; }

int64_t num_params()
{
    int64_t n = 0;
    for (int l = 0; l < kLayers; ++l) n += (int64_t)kCout[l] * kCin[l] * 9 + kCout[l];
    return n + 33;
}

// ---------------------------------------------------------------------------
// PTX helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp16_zfill(void *smem, const void *gmem, bool valid)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(smem)), "l"(gmem),
                 "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

__device__ __forceinline__ void ldsm_x4(unsigned (&r)[4], const void *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(unsigned (&r)[4], const void *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Elementwise pieces move 8 channels (16 bytes) per thread; channel counts,
// row strides and view offsets are multiples of 8.
struct B8 {
    float v[8];
};
__device__ __forceinline__ B8 ld8(const bf16 *p)
{
    const uint4 u = *reinterpret_cast<const uint4 *>(p);
    const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u);
    B8 r;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 f = __bfloat1622float2(h[i]);
        r.v[2 * i] = f.x;
        r.v[2 * i + 1] = f.y;
    }
    return r;
}
__device__ __forceinline__ void st8(bf16 *p, const B8 &r)
{
    uint4 u;
    __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(&u);
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(r.v[2 * i], r.v[2 * i + 1]);
    *reinterpret_cast<uint4 *>(p) = u;
}

// ---------------------------------------------------------------------------
// 3x3 convolution, implicit GEMM: Y[p][co] = sum over (tap, ci) of
// X[p + off(tap)][ci] * Wt[co][tap][ci] (+ bias, ReLU, mask).  Block tile 64
// pixels x BN output channels, K chunks of 32 (one tap, 32 input channels),
// cp.async double buffering with zero fill outside the image.
// Requires Cin % 32 == 0 and Cout % BN == 0.
// ---------------------------------------------------------------------------
struct ConvArgs {
    const bf16 *X;
    int ldx, Cin;
    const bf16 *Wt;     // [Cout][9][Cin]
    const float *bias;  // [Cout] or null
    bf16 *Y;
    int ldy, Cout;
    const bf16 *mask;   // optional: Y *= (mask[p][co] > 0)
    int ldm;
    int relu;
    int B, H, W;
};

template <int BN>
__global__ void __launch_bounds__(128) k_conv(ConvArgs a)
{
    constexpr int BM = 64, BK = 32, LDS = BK + 8;  // padded rows: 80 bytes
    constexpr int WN = BN / 2, NT = WN / 8;        // 2 x 2 warps, warp tile 32 x WN
    __shared__ __align__(16) bf16 sA[2][BM][LDS];
    __shared__ __align__(16) bf16 sB[2][BN][LDS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 1, wn = warp & 1;
    const int P = a.B * a.H * a.W;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int nk = 9 * a.Cin / BK;

    // each thread always loads the same two A rows: decompose their pixels once
    int rh[2], rw[2];
    const bf16 *rbase[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int c = tid + u * 128, row = c >> 2, q = c & 3;
        const int p = m0 + row;
        if (p < P) {
            const int b = p / (a.H * a.W), hw = p % (a.H * a.W);
            rh[u] = hw / a.W;
            rw[u] = hw % a.W;
            rbase[u] = a.X + ((int64_t)(b * a.H + rh[u]) * a.W + rw[u]) * a.ldx + q * 8;
        } else {
            rh[u] = -100000;  // never inside the image
            rw[u] = 0;
            rbase[u] = a.X;
        }
    }
    auto load = [&](int kc, int st) {
        const int k = kc * BK, tap = k / a.Cin, ci0 = k % a.Cin;
        const int kh = tap / 3 - 1, kw = tap % 3 - 1;
        const int64_t shift = ((int64_t)kh * a.W + kw) * a.ldx + ci0;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int c = tid + u * 128, row = c >> 2, q = c & 3;
            const int hh = rh[u] + kh, ww = rw[u] + kw;
            const bool ok = hh >= 0 && hh < a.H && ww >= 0 && ww < a.W;
            cp16_zfill(&sA[st][row][q * 8], ok ? rbase[u] + shift : a.X, ok);
        }
        for (int c = tid; c < BN * 4; c += 128) {
            const int row = c >> 2, q = c & 3;
            const bf16 *src = a.Wt + ((int64_t)(n0 + row) * 9 + tap) * a.Cin + ci0 + q * 8;
            cp16_zfill(&sB[st][row][q * 8], src, true);
        }
        cp_commit();
    };

    float acc[2][NT][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < NT; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;

    load(0, 0);
    for (int kc = 0; kc < nk; ++kc) {
        if (kc + 1 < nk) {
            load(kc + 1, (kc + 1) & 1);
            cp_wait<1>();
        } else {
            cp_wait<0>();
        }
        __syncthreads();
        const int st = kc & 1;
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            unsigned af[2][4];
#pragma unroll
            for (int i = 0; i < 2; ++i)
                ldsm_x4(af[i], &sA[st][wm * 32 + i * 16 + (lane & 15)][kk + (lane >> 4) * 8]);
#pragma unroll
            for (int j = 0; j < NT; j += 2) {
                unsigned bfr[4];
                ldsm_x4(bfr, &sB[st][wn * WN + j * 8 + (lane & 7) + (lane >> 4) * 8][kk + ((lane >> 3) & 1) * 8]);
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    mma_bf16(acc[i][j], af[i], bfr[0], bfr[1]);
                    mma_bf16(acc[i][j + 1], af[i], bfr[2], bfr[3]);
                }
            }
        }
        __syncthreads();
    }
    const int g = lane >> 2, t4 = lane & 3;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < NT; ++j)
#pragma unroll
            for (int hlf = 0; hlf < 2; ++hlf) {
                const int p = m0 + wm * 32 + i * 16 + g + hlf * 8;
                const int co = n0 + wn * WN + j * 8 + 2 * t4;
                if (p >= P) continue;
                float v0 = acc[i][j][hlf * 2], v1 = acc[i][j][hlf * 2 + 1];
                if (a.bias) {
                    v0 += a.bias[co];
                    v1 += a.bias[co + 1];
                }
                if (a.relu) {
                    v0 = fmaxf(v0, 0.f);
                    v1 = fmaxf(v1, 0.f);
                }
                if (a.mask) {
                    const bf16 *mk = a.mask + (int64_t)p * a.ldm + co;
                    if (!(__bfloat162float(mk[0]) > 0.f)) v0 = 0.f;
                    if (!(__bfloat162float(mk[1]) > 0.f)) v1 = 0.f;
                }
                *reinterpret_cast<__nv_bfloat162 *>(a.Y + (int64_t)p * a.ldy + co) = __floats2bfloat162_rn(v0, v1);
            }
}

// ---------------------------------------------------------------------------
// 3x3 convolution on the 5th-generation tensor cores (tcgen05), the same
// implicit GEMM as k_conv.  Persistent and warp-specialised: one block per
// SM (two where shared memory allows) walks output tiles of 128 pixels (an
// 8 x 16 patch of one image) x BN output channels.
//   * The block's BN x 9 x Cin weights are loaded once by TMA and stay in
//     shared memory when they fit (STREAM = false); otherwise each stage of
//     the ring carries its chunk's BN x 9 x 32 weights with the pixels
//     (STREAM = true), so that BN can be the whole layer: a tcgen05.mma of
//     M = 128 costs about as much at N = 32 or 64 as at N = 128.
//   * For each chunk of 32 input channels the tensor-memory accelerator (TMA)
//     copies three column-shifted halo patches (10 x 16 pixels at x offsets
//     -1, 0, +1, rows -1 .. +8, zero-filled outside the image).  The A
//     operand of tap (dy, dx) is then the shifted copy dx started dy + 1
//     rows in: 8 contiguous rows of 16 pixels, so each of the 9 taps is two
//     tcgen05.mma (K = 16 each) with no data movement of its own.
//   * The FP32 accumulator lives in tensor memory (TMEM, lane = pixel,
//     column = channel), double-buffered so that the epilogue of one tile
//     overlaps the MMAs of the next.
// Warp 0 issues the TMA copies, warp 1 the MMAs, warps 2-5 run the
// epilogue (tcgen05.ld of 16 columns, bias, ReLU, mask, BF16 store); warp
// w reads TMEM lanes 32 (w % 4) .. + 31.  mbarriers hand over the stages:
// a_full (TMA -> MMA), a_empty (MMA done reading -> TMA), acc_full (last
// MMA of a tile -> epilogue), acc_empty (epilogue -> MMA).  Operands are
// K-major with 64-byte rows in the 64-byte swizzle.  Every wait is bounded:
// a role whose wait runs out raises a shared flag that ends the others'
// loops; the block then records the timeout in *err, lets its copies and
// MMAs in flight complete (bounded waits), frees its TMEM and returns.
// Requires Cin % 32 == 0 and Cout % BN == 0.
// ---------------------------------------------------------------------------
constexpr int kTcTH = 8, kTcTW = 16;                    // output pixels per tile: 8 rows x 16
constexpr int kTcBK = 32;                               // input channels per chunk (64-byte rows)
constexpr int kTcRowBytes = kTcTW * kTcBK * 2;          // one image row of a copy: 1 KB
constexpr int kTcCopy = (kTcTH + 2) * kTcRowBytes;      // one shifted halo copy: 10 KB
constexpr int kTcAStage = 3 * kTcCopy;                  // the three copies of a chunk
constexpr int kTcMaxStages = 8;                        // depth of the A ring: as deep as shared memory allows
constexpr int kTcThreads = 320;                         // producer, MMA issuer, 8 epilogue warps
constexpr int kTcSmemMax = 227 * 1024;                  // opt-in shared memory per block
constexpr int kTcWeightMax = 108 * 1024;                // leaves room for at least 3 A stages
constexpr unsigned kTcPolls = 1u << 22;

// shared memory of k_conv_tc: resident weights, ring, barriers, bias
__host__ __device__ constexpr int tc_weight_bytes(int Cin, int BN) { return (Cin / kTcBK) * 9 * BN * kTcBK * 2; }
__host__ __device__ constexpr int tc_wslice_bytes(int BN) { return 9 * BN * kTcBK * 2; }  // one chunk's weights
__host__ __device__ constexpr int tc_stage_bytes(int BN, bool stream, bool dxn)
{
    return (dxn ? kTcCopy : kTcAStage) + (stream ? tc_wslice_bytes(BN) : 0);
}
// tensor-memory columns of a block: two accumulators of BN (or 3 BN) columns,
// rounded up to a power of two
__host__ __device__ constexpr unsigned tc_tmem_cols(int BN, bool dxn)
{
    return (dxn ? 6 : 2) * BN <= 64 ? 64u : (dxn ? 6 : 2) * BN <= 128 ? 128u : (dxn ? 6 : 2) * BN <= 256 ? 256u : 512u;
}
__host__ __device__ constexpr int tc_fixed_bytes(int Cin, int BN, bool stream)
{
    return 1024 /* alignment slack */ + (stream ? 0 : tc_weight_bytes(Cin, BN)) + 32 * 8 /* barriers */ +
           BN * 4 /* bias */;
}

// wait for phase `parity`, giving up after kTcPolls polls or once *fail is set
__device__ __forceinline__ bool tc_wait(uint64_t *bar, unsigned parity, volatile int *fail)
{
    for (unsigned i = 0; i < kTcPolls; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 255u) == 255u && *fail) return false;
    }
    return false;
}

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];\n" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int c0, int c1, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];\n" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tc_alloc(uint32_t *slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// D (TMEM) (+)= A (smem) x B (smem)^T with K = 16; accumulate = 0 overwrites D.
__device__ __forceinline__ void tc_mma(uint32_t taddr, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(taddr),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// arrive on `bar` once every tcgen05 operation this thread issued has completed
__device__ __forceinline__ void tc_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane (no wait)
__device__ __forceinline__ void tc_ld16_nowait(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major operand with 64-byte rows in
// the 64-byte swizzle (the layout TMA writes with CU_TENSOR_MAP_SWIZZLE_64B):
// start address >> 4 (bits 0-13), leading offset 16 B (unused by this
// layout, bits 16-29), 512 B between 8-row groups (bits 32-45), descriptor
// version 1 (bit 46), base offset 0, swizzle mode 4 = 64 B (bits 61-63).
// The tile must start on a 512-byte boundary; +2 in the low word moves the
// start 32 bytes along K (the second K = 16 step of a 64-byte row).
__device__ __forceinline__ uint64_t sw64_desc(const void *tile)
{
    const uint32_t a = smem_u32(tile);
    return (uint64_t)((a >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}

// Instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 (bits
// 17-22), M >> 4 (bits 24-28).
__host__ __device__ constexpr uint32_t tc_idesc(int m, int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

template <int BN, bool STREAM, bool DXN>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_conv_tc(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmW, ConvArgs a,
              int tiles_x, int tiles_y, int nstage, int cps, int w3d, unsigned *err)
{
    static_assert(BN % 32 == 0 && BN >= 32 && BN <= 128, "output channels per block: 32 .. 128, a multiple of 32");
    static_assert(!DXN || BN <= 64, "with the taps folded into N, N = 3 BN <= 192");
    constexpr int AW = DXN ? 3 * BN : BN;  // accumulator columns of one tile
    constexpr uint32_t TM_COLS = tc_tmem_cols(BN, DXN);  // two accumulators
    constexpr uint32_t idesc = tc_idesc(kTcTH * kTcTW, AW);
    constexpr int OW = DXN ? kTcTW - 2 : kTcTW;  // output columns per tile
    extern __shared__ unsigned char smraw[];
    unsigned char *sm =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
    constexpr int CHUNK = tc_stage_bytes(BN, STREAM, DXN);  // one chunk of 32 input channels
    const int STAGE = cps * CHUNK;                          // a stage: cps chunks of the same tile
    constexpr int ACOPY = DXN ? kTcCopy : kTcAStage;  // the pixel part of a stage
    const int nck = a.Cin / kTcBK;
    const int wbytes = STREAM ? 0 : tc_weight_bytes(a.Cin, BN);
    unsigned char *sW = sm, *sA = sm + wbytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sA + nstage * STAGE);
    uint64_t *wbar = bars, *a_full = bars + 1, *a_empty = bars + 1 + kTcMaxStages;
    uint64_t *acc_full = bars + 1 + 2 * kTcMaxStages, *acc_empty = acc_full + 2, *mma_done = acc_empty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mma_done + 1);
    float *s_bias = reinterpret_cast<float *>(bars + 32);
    __shared__ volatile int s_fail;
    __shared__ int s_consumed;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int per_img = tiles_x * tiles_y, ntiles = a.B * per_img;
    const int n0 = blockIdx.y * BN;

    if (threadIdx.x == 0) {
        mbar_init(wbar, 1);
        for (int s = 0; s < nstage; ++s) {
            mbar_init(a_full + s, 1);
            mbar_init(a_empty + s, 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(acc_full + s, 1);
            mbar_init(acc_empty + s, 8);
        }
        mbar_init(mma_done, 1);
        s_fail = 0;
        s_consumed = 0;
    }
    if (threadIdx.x < BN) s_bias[threadIdx.x] = a.bias ? a.bias[n0 + threadIdx.x] : 0.f;
    if (warp == 0) tc_alloc(tmem_slot, TM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    int issued = 0;  // A chunks issued (producer thread)
    if (warp == 0) {
        if (lane == 0) {
            // resident weights (none when they stream: the barrier's phase
            // then completes at once)
            mbar_arrive_expect_tx(wbar, (unsigned)wbytes);
            if (!STREAM)
                for (int c = 0; c < nck; ++c)
                    for (int tap = 0; tap < 9; ++tap)
                        tma_load_2d(sW + (c * 9 + tap) * BN * kTcBK * 2, &tmW, tap * a.Cin + c * kTcBK, n0, wbar);
            int n = 0, s = 0, u = 0;  // chunk count, its stage and the stage's use
            for (int t = blockIdx.x; t < ntiles && !s_fail; t += gridDim.x) {
                const int b = t / per_img, r = t % per_img;
                const int y0 = (r / tiles_x) * kTcTH, x0 = (r % tiles_x) * OW - (DXN ? 1 : 0);
                for (int c0 = 0; c0 < nck; c0 += cps, ++n, s = (s + 1 == nstage) ? 0 : s + 1, u += (s == 0)) {
                    if (u > 0 && !tc_wait(a_empty + s, (u - 1) & 1, &s_fail)) {
                        s_fail = 1;
                        break;
                    }
                    mbar_arrive_expect_tx(a_full + s, (unsigned)STAGE);
                    for (int c = c0; c < c0 + cps; ++c) {
                    unsigned char *dst = sA + s * STAGE + (c - c0) * CHUNK;
                    if (DXN) {
                        tma_load_4d(dst, &tmX, c * kTcBK, x0, y0 - 1, b, a_full + s);
                    } else {
#pragma unroll
                        for (int d = 0; d < 3; ++d)
                            tma_load_4d(dst + d * kTcCopy, &tmX, c * kTcBK, x0 + d - 1, y0 - 1, b, a_full + s);
                    }
                    if (STREAM) {
                        if (w3d) {  // one box {32 channels, BN rows, 9 taps}
                            tma_load_3d(dst + ACOPY, &tmW, c * kTcBK, n0, 0, a_full + s);
                        } else {
#pragma unroll
                            for (int tap = 0; tap < 9; ++tap)
                                tma_load_2d(dst + ACOPY + tap * BN * kTcBK * 2, &tmW, tap * a.Cin + c * kTcBK, n0,
                                            a_full + s);
                        }
                    }
                    }
                    issued = n + 1;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // descriptors of the ring's first stage and of the first weight
            // slice; every other operand is a constant offset from these
            const uint64_t a_desc0 = sw64_desc(sA), w_desc0 = sw64_desc(sW);
            int n = 0, j = 0, s = 0, u = 0;  // chunk count, its stage and the stage's use
            bool ok = tc_wait(wbar, 0, &s_fail);
            for (int t = blockIdx.x; ok && t < ntiles; t += gridDim.x, ++j) {
                const int acc = j & 1, ua = j >> 1;
                if (ua > 0 && !tc_wait(acc_empty + acc, (ua - 1) & 1, &s_fail)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(acc * AW);
                for (int c0 = 0; c0 < nck; c0 += cps, ++n, s = (s + 1 == nstage) ? 0 : s + 1, u += (s == 0)) {
                    if (!tc_wait(a_full + s, u & 1, &s_fail)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    for (int c = c0; c < c0 + cps; ++c) {
                    // (start address >> 4) sits in the low bits and never carries
                    const uint64_t ad0 = a_desc0 + (uint64_t)((s * STAGE + (c - c0) * CHUNK) >> 4);
                    const uint64_t bd0 = STREAM ? ad0 + (uint64_t)(ACOPY >> 4)
                                                : w_desc0 + (uint64_t)((c * tc_wslice_bytes(BN)) >> 4);
                    if (DXN) {
                        // row shift dy: the copy dy rows in; B = the three taps
                        // (dy, -1 .. +1), 3 BN consecutive weight rows
#pragma unroll
                        for (int dy = 0; dy < 3; ++dy) {
                            const uint64_t ad = ad0 + (uint64_t)((dy * kTcRowBytes) >> 4);
                            const uint64_t bd = bd0 + (uint64_t)((dy * 3 * BN * kTcBK * 2) >> 4);
                            tc_mma(d, ad, bd, idesc, (c | dy) ? 1u : 0u);
                            tc_mma(d, ad + 2, bd + 2, idesc, 1u);
                        }
                    } else {
#pragma unroll
                        for (int tap = 0; tap < 9; ++tap) {
                            const uint64_t ad =
                                ad0 + (uint64_t)(((tap % 3) * kTcCopy + (tap / 3) * kTcRowBytes) >> 4);
                            const uint64_t bd = bd0 + (uint64_t)((tap * BN * kTcBK * 2) >> 4);
                            tc_mma(d, ad, bd, idesc, (c | tap) ? 1u : 0u);
                            tc_mma(d, ad + 2, bd + 2, idesc, 1u);
                        }
                    }
                    }
                    tc_commit(a_empty + s);
                    s_consumed = n + 1;
                }
                if (!ok) break;
                tc_commit(acc_full + acc);
            }
            if (!ok) s_fail = 1;
            tc_commit(mma_done);
        }
    } else {
        // epilogue warps 2 .. 9: warp w reads TMEM lanes 32 (w % 4) .. + 31 and
        // takes half (w - 2) / 4 of the block's BN channels
        const int q = warp & 3;
        const int m = q * 32 + lane;
        constexpr int HALF = BN / 2;
        const int cbeg = ((warp - 2) >> 2) * HALF;
        int j = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++j) {
            const int acc = j & 1, ua = j >> 1;
            const bool ok = tc_wait(acc_full + acc, ua & 1, &s_fail);
            if (!__all_sync(0xffffffffu, ok)) {
                s_fail = 1;
                break;
            }
            tc_fence_after();
            const int b = t / per_img, r = t % per_img;
            const int xm = m % kTcTW;
            const int y = (r / tiles_x) * kTcTH + m / kTcTW, x = (r % tiles_x) * OW - (DXN ? 1 : 0) + xm;
            // with folded taps the first and last column of the patch are halo
            const bool in = y < a.H && x < a.W && (!DXN || (xm >= 1 && xm <= kTcTW - 2));
            const int64_t p = ((int64_t)b * a.H + y) * a.W + x;
            const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * AW);
            // all of the warp's columns are loaded before one wait: NP pieces
            // of 16 columns (three blocks of them with folded taps)
            constexpr int NP = HALF / 16, NB3 = DXN ? 3 : 1;
            uint32_t rv[NB3][NP][16];
#pragma unroll
            for (int k = 0; k < NB3; ++k)
#pragma unroll
                for (int j = 0; j < NP; ++j) tc_ld16_nowait(trow + (uint32_t)(k * BN + cbeg + 16 * j), rv[k][j]);
            tc_wait_ld();
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                float v[16];
                if (DXN) {
                    // Y[x] = D[x - 1][tap dx = -1] + D[x][dx = 0] + D[x + 1][dx = +1]:
                    // the neighbours are lanes m -+ 1 of the same 16-pixel row
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        v[i] = __shfl_up_sync(0xffffffffu, __uint_as_float(rv[0][j][i]), 1) +
                               __uint_as_float(rv[DXN ? 1 : 0][j][i]) +
                               __shfl_down_sync(0xffffffffu, __uint_as_float(rv[DXN ? 2 : 0][j][i]), 1);
                } else {
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(rv[0][j][i]);
                }
                if (!in) continue;
                const int c0 = cbeg + 16 * j, co = n0 + c0;
#pragma unroll
                for (int g = 0; g < 2; ++g) {
                    B8 mk, o;
                    if (a.mask) mk = ld8(a.mask + p * a.ldm + co + 8 * g);
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        float rvl = v[8 * g + i] + s_bias[c0 + 8 * g + i];
                        if (a.relu) rvl = fmaxf(rvl, 0.f);
                        if (a.mask && !(mk.v[i] > 0.f)) rvl = 0.f;
                        o.v[i] = rvl;
                    }
                    st8(a.Y + p * a.ldy + co + 8 * g, o);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acc_empty + acc);
        }
    }
    __syncwarp();
    __syncthreads();
    if (threadIdx.x == 0) {
        // the MMAs issued have completed once mma_done fires; copies still in
        // flight after a failure land before the block's shared memory goes
        const bool mma_ok = mbar_wait_bounded(mma_done, 0, kTcPolls);
        if (s_fail || !mma_ok) {
            atomicOr(err, 1u);
            mbar_wait_bounded(wbar, 0, kTcPolls);
            for (int n = s_consumed; n < issued; ++n)
                mbar_wait_bounded(a_full + n % nstage, (n / nstage) & 1, kTcPolls);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tc_dealloc(tmem, TM_COLS);
}

// ---------------------------------------------------------------------------
// Weight gradient, split-K implicit GEMM: for one tap and tile of (co, ci),
// part[split][co][tap][ci] = sum over the split's pixels p of
// dY[p][co] * X[p + off(tap)][ci].  Both operands are staged [pixel][channel]
// and read with transposing ldmatrix.
// ---------------------------------------------------------------------------
struct WgradArgs {
    const bf16 *dY;
    int ldd, Cout;
    const bf16 *X;
    int ldx, Cin;
    float *part;  // [splits][Cout][9][Cin]
    int B, H, W, pps;
};

__global__ void __launch_bounds__(128) k_wgrad(WgradArgs a)
{
    constexpr int BM = 32, BN = 32, BK = 32, LDA = BM + 8, LDB = BN + 8;
    __shared__ __align__(16) bf16 sD[2][BK][LDA];
    __shared__ __align__(16) bf16 sX[2][BK][LDB];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 1, wn = warp & 1;  // warp tile 16 (co) x 16 (ci)
    const int P = a.B * a.H * a.W;
    const int split = blockIdx.x;
    const int tiles_ci = a.Cin / BN;
    const int tap = blockIdx.y / tiles_ci, ci0 = (blockIdx.y % tiles_ci) * BN;
    const int co0 = blockIdx.z * BM;
    const int kh = tap / 3, kw = tap % 3;
    const int p_begin = split * a.pps, p_end = min(P, p_begin + a.pps);
    const int nk = (p_end - p_begin + BK - 1) / BK;

    auto load = [&](int kc, int st) {
        const int pb = p_begin + kc * BK;
        {
            const int c = tid;  // 32 pixels x 4 chunks of 8 co
            const int row = c >> 2, q = c & 3;
            const int p = pb + row;
            const bool ok = p < p_end;
            const bf16 *src = ok ? a.dY + (int64_t)p * a.ldd + co0 + q * 8 : a.dY;
            cp16_zfill(&sD[st][row][q * 8], src, ok);
        }
        {
            const int c = tid;
            const int row = c >> 2, q = c & 3;
            const int p = pb + row;
            bool ok = p < p_end;
            const bf16 *src = a.X;
            if (ok) {
                const int b = p / (a.H * a.W), hw = p % (a.H * a.W), h = hw / a.W, w = hw % a.W;
                const int hh = h + kh - 1, ww = w + kw - 1;
                ok = hh >= 0 && hh < a.H && ww >= 0 && ww < a.W;
                if (ok) src = a.X + ((int64_t)(b * a.H + hh) * a.W + ww) * a.ldx + ci0 + q * 8;
            }
            cp16_zfill(&sX[st][row][q * 8], src, ok);
        }
        cp_commit();
    };

    float acc[2][4];
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[j][r] = 0.f;
    if (nk > 0) load(0, 0);
    for (int kc = 0; kc < nk; ++kc) {
        if (kc + 1 < nk) {
            load(kc + 1, (kc + 1) & 1);
            cp_wait<1>();
        } else {
            cp_wait<0>();
        }
        __syncthreads();
        const int st = kc & 1;
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            unsigned af[4], bfr[4];
            // A (co x pixel) from sD[pixel][co]: transposed 8x8 blocks
            ldsm_x4_t(af, &sD[st][kk + (lane & 7) + (lane >> 4) * 8][wm * 16 + ((lane >> 3) & 1) * 8]);
            // B (pixel x ci) from sX[pixel][ci]: transposed 8x8 blocks
            ldsm_x4_t(bfr, &sX[st][kk + (lane & 7) + ((lane >> 3) & 1) * 8][wn * 16 + (lane >> 4) * 8]);
            mma_bf16(acc[0], af, bfr[0], bfr[1]);
            mma_bf16(acc[1], af, bfr[2], bfr[3]);
        }
        __syncthreads();
    }
    const int g = lane >> 2, t4 = lane & 3;
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int hlf = 0; hlf < 2; ++hlf) {
            const int co = co0 + wm * 16 + g + hlf * 8;
            const int ci = ci0 + wn * 16 + j * 8 + 2 * t4;
            float *dst = a.part + (((int64_t)split * a.Cout + co) * 9 + tap) * a.Cin + ci;
            dst[0] = acc[j][hlf * 2];
            dst[1] = acc[j][hlf * 2 + 1];
        }
}

// dW (flat layout [Cout][Cin_real][3][3]) = sum over the splits of
// part[split][co][tap][ci], in a fixed order: a block takes 32 consecutive
// elements e = (co * 9 + tap) * Cin_pad + ci (coalesced reads) and 8 slices
// of the splits (slice j sums splits j, j + 8, ...); the slices are then
// added in slice order.
__global__ void __launch_bounds__(256) k_wgrad_reduce(const float *part, int splits, int Cout, int Cin_pad,
                                                      int Cin_real, float *dW)
{
    __shared__ double red[8][32];
    const int64_t n = (int64_t)Cout * 9 * Cin_pad;
    const int64_t e = (int64_t)blockIdx.x * 32 + (threadIdx.x & 31);
    const int j = threadIdx.x >> 5;
    double acc = 0.0;
    if (e < n)
        for (int k = j; k < splits; k += 8) acc += part[(int64_t)k * n + e];
    red[j][threadIdx.x & 31] = acc;
    __syncthreads();
    if (threadIdx.x < 32 && e < n) {
        double t = 0.0;
        for (int jj = 0; jj < 8; ++jj) t += red[jj][threadIdx.x];
        const int ci = (int)(e % Cin_pad);
        const int64_t r = e / Cin_pad;
        const int tap = (int)(r % 9), co = (int)(r / 9);
        if (ci < Cin_real) dW[((int64_t)co * Cin_real + ci) * 9 + tap] = (float)t;
    }
}

// ---------------------------------------------------------------------------
// Weight gradient on the tensor cores (tcgen05):
//   dW[co][tap][ci] = sum over pixels p of X[p + off(tap)][ci] * dY[p][co]
// as D[m][n] = sum over k of A[m][k] B[n][k] with k = pixel, n = co and m a
// row of a "slot" (tap, 32 input channels): an MMA of M = 128 covers a
// group of four slots.  Both operands are read in their NHWC layout, i.e.
// MN-major (the 32 channels of a pixel contiguous): TMA copies, per tile of
// 8 x 16 pixels, one box {32 channels, 16, 8} of X shifted by each slot's
// tap (zero outside the image) and the Cout / 32 boxes of dY; in the 64-byte
// swizzle an atom is 32 channels x 8 pixels, atoms along M (or N) are one
// box apart (LBO) and groups of 8 pixels 512 bytes apart (SBO); a K = 16
// step is one image row of the tile (+1 KB).  A persistent block keeps its
// groups' accumulators (FP32, G x Cout columns) in tensor memory over all
// its tiles and writes them once as a partial; the partials are then added
// in block order (k_wgrad_tc_reduce).  Roles and bounded waits as in
// k_conv_tc: warp 0 TMA, warp 1 MMA, warps 2-5 read the accumulators.
// ---------------------------------------------------------------------------
constexpr int kWgR = 8;                               // image rows per tile (K = 128 pixels)
constexpr int kWgBox = kWgR * kTcTW * kTcBK * 2;      // one box {32 channels, 16, 8}: 8 KB
constexpr int kWgMaxStages = 4;
constexpr int kWgThreads = 192;

struct WgTcArgs {
    int Cin, Cout, B, H, W;
    int ncb;      // Cin / 32: slots per tap
    int ngroups;  // ceil(9 ncb / 4)
};

__host__ __device__ constexpr int wg_stage_bytes(int G, int N) { return (4 * G + N / 32) * kWgBox; }

// MN-major operand in the 64-byte swizzle: atoms of 32 elements x 8 rows,
// `lbo` bytes between atoms along M (or N), 512 bytes between 8-row groups
__device__ __forceinline__ uint64_t sw64_mn_desc(const void *tile, uint32_t lbo)
{
    const uint32_t a = smem_u32(tile);
    return (uint64_t)((a >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)(512 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}

// kind::f16 instruction descriptor with both operands MN-major (bits 15, 16)
__host__ __device__ constexpr uint32_t tc_idesc_mn(int m, int n) { return tc_idesc(m, n) | (1u << 15) | (1u << 16); }

template <int N>
__global__ void __launch_bounds__(kWgThreads, 1)
    k_wgrad_tc(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmD, WgTcArgs a,
               int G, int nstage, float *part, unsigned *err)
{
    static_assert(N == 32 || N == 64 || N == 128, "Cout of a forward layer");
    constexpr uint32_t idesc = tc_idesc_mn(128, N);
    extern __shared__ unsigned char smraw[];
    unsigned char *sm =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
    const int STAGE = wg_stage_bytes(G, N);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + nstage * STAGE);
    uint64_t *full = bars, *empty = bars + kWgMaxStages, *done = bars + 2 * kWgMaxStages;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    __shared__ volatile int s_fail;
    __shared__ int s_consumed;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_x = (a.W + kTcTW - 1) / kTcTW, tiles_y = (a.H + kWgR - 1) / kWgR;
    const int per_img = tiles_x * tiles_y, ntiles = a.B * per_img;
    // blockIdx.x: the group set (the blocks sharing a tile are launched side
    // by side, so that they read its pixels from L2 at about the same time);
    // blockIdx.y: the block's share of the tiles
    const int g0 = blockIdx.x * G, gn = min(G, a.ngroups - g0);
    const int nslot = 9 * a.ncb;
    uint32_t tm_cols = 32;
    while (tm_cols < (uint32_t)(G * N)) tm_cols *= 2;

    if (threadIdx.x == 0) {
        for (int q = 0; q < nstage; ++q) {
            mbar_init(full + q, 1);
            mbar_init(empty + q, 1);
        }
        mbar_init(done, 1);
        s_fail = 0;
        s_consumed = 0;
    }
    if (warp == 0) tc_alloc(tmem_slot, tm_cols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    int issued = 0;
    if (warp == 0) {
        if (lane == 0) {
            // boxes per tile: the valid slots of the block's groups, then dY
            int nvalid = 0;
            for (int k = 0; k < 4 * gn; ++k) nvalid += (g0 * 4 + k) < nslot;
            const unsigned bytes = (unsigned)((nvalid + N / 32) * kWgBox);
            int n = 0, st = 0, u = 0;
            for (int t = blockIdx.y; t < ntiles && !s_fail; t += gridDim.y, ++n) {
                if (u > 0 && !tc_wait(empty + st, (u - 1) & 1, &s_fail)) {
                    s_fail = 1;
                    break;
                }
                const int b = t / per_img, r = t % per_img;
                const int y0 = (r / tiles_x) * kWgR, x0 = (r % tiles_x) * kTcTW;
                unsigned char *dst = sm + st * STAGE;
                mbar_arrive_expect_tx(full + st, bytes);
                for (int k = 0; k < 4 * gn; ++k) {
                    const int sidx = g0 * 4 + k;
                    if (sidx >= nslot) break;
                    const int tap = sidx / a.ncb, cb = sidx % a.ncb;
                    tma_load_4d(dst + k * kWgBox, &tmX, cb * kTcBK, x0 + tap % 3 - 1, y0 + tap / 3 - 1, b, full + st);
                }
#pragma unroll
                for (int j = 0; j < N / 32; ++j)
                    tma_load_4d(dst + (4 * G + j) * kWgBox, &tmD, j * kTcBK, x0, y0, b, full + st);
                issued = n + 1;
                if (++st == nstage) {
                    st = 0;
                    ++u;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int n = 0, st = 0, u = 0;
            bool ok = true;
            for (int t = blockIdx.y; t < ntiles; t += gridDim.y, ++n) {
                if (!tc_wait(full + st, u & 1, &s_fail)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const unsigned char *base = sm + st * STAGE;
                const uint64_t bd0 = sw64_mn_desc(base + 4 * G * kWgBox, kWgBox);
                for (int gi = 0; gi < gn; ++gi) {
                    const uint64_t ad0 = sw64_mn_desc(base + gi * 4 * kWgBox, kWgBox);
#pragma unroll
                    for (int i = 0; i < kWgR; ++i)  // one image row (16 pixels) per K step: +1 KB
                        tc_mma(tmem + (uint32_t)(gi * N), ad0 + (uint64_t)(i * 64), bd0 + (uint64_t)(i * 64), idesc,
                               (n | i) ? 1u : 0u);
                }
                tc_commit(empty + st);
                s_consumed = n + 1;
                if (++st == nstage) {
                    st = 0;
                    ++u;
                }
            }
            if (!ok) s_fail = 1;
            tc_commit(done);
        }
    } else {
        // accumulators -> partial: part[block y][group][row][co], row = slot-in-group * 32 + channel
        const int q = warp & 3;
        const bool ok = tc_wait(done, 0, &s_fail);
        if (__all_sync(0xffffffffu, ok)) {
            tc_fence_after();
            for (int gi = 0; gi < gn; ++gi) {
                float *dst = part + (((int64_t)blockIdx.y * a.ngroups + g0 + gi) * 128 + q * 32 + lane) * N;
#pragma unroll 1
                for (int c0 = 0; c0 < N; c0 += 16) {
                    uint32_t v[16];
                    tc_ld16_nowait(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(gi * N + c0), v);
                    tc_wait_ld();
#pragma unroll
                    for (int i = 0; i < 16; i += 4)
                        *reinterpret_cast<float4 *>(dst + c0 + i) =
                            make_float4(__uint_as_float(v[i]), __uint_as_float(v[i + 1]), __uint_as_float(v[i + 2]),
                                        __uint_as_float(v[i + 3]));
                }
            }
        } else {
            s_fail = 1;
        }
    }
    __syncwarp();
    __syncthreads();
    if (threadIdx.x == 0) {
        const bool mma_ok = mbar_wait_bounded(done, 0, kTcPolls);
        if (s_fail || !mma_ok) {
            atomicOr(err, 1u);
            for (int n = s_consumed; n < issued; ++n)
                mbar_wait_bounded(full + n % nstage, (n / nstage) & 1, kTcPolls);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tc_dealloc(tmem, tm_cols);
}

// dW (flat [Cout][Cin_real][3][3]) = sum over blocks k of part[k][g][row][co]
// (fixed order), row = (slot % 4) * 32 + channel, slot = tap * ncb + ci / 32.
__global__ void k_wgrad_tc_reduce(const float *part, int nparts, int ngroups, int N, int ncb, int Cin_real,
                                  float *dW)
{
    const int64_t n = (int64_t)ngroups * 128 * N;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int co = (int)(e % N);
        const int64_t rr = e / N;
        const int row = (int)(rr % 128), g = (int)(rr / 128);
        const int sidx = g * 4 + row / 32, ci = (sidx % ncb) * 32 + row % 32, tap = sidx / ncb;
        if (sidx >= 9 * ncb || ci >= Cin_real) continue;
        double acc = 0.0;
        for (int k = 0; k < nparts; ++k) acc += part[(int64_t)k * n + e];
        dW[((int64_t)co * Cin_real + ci) * 9 + tap] = (float)acc;
    }
}

// Per-channel sums of a [P][ld] BF16 tensor over pixels: one block per range
// of pps pixels; thread t sums channels 8 (t % (C/8)) .. +7 over the pixels
// p0 + t / (C/8), + 256 / (C/8), ...; then a fixed-order reduction in shared
// memory.  part[block][C].
__global__ void k_chansum(const bf16 *Y, int ld, int C, int P, int pps, float *part)
{
    __shared__ float red[256][8];
    const int C8 = C / 8, lanes = 256 / C8;  // C8 divides 256 for C in {32, 64, 128}
    const int cg = threadIdx.x % C8, pr = threadIdx.x / C8;
    const int p0 = blockIdx.x * pps, p1 = min(P, p0 + pps);
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (pr < lanes)
        for (int p = p0 + pr; p < p1; p += lanes) {
            const B8 v = ld8(Y + (int64_t)p * ld + cg * 8);
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[k] += v.v[k];
        }
#pragma unroll
    for (int k = 0; k < 8; ++k) red[threadIdx.x][k] = acc[k];
    __syncthreads();
    if (threadIdx.x < C) {
        const int g = threadIdx.x / 8, k = threadIdx.x % 8;
        float s = 0.f;
        for (int r = 0; r < lanes; ++r) s += red[r * C8 + g][k];
        part[(int64_t)blockIdx.x * C + threadIdx.x] = s;
    }
}

// out[c] = sum over k of part[k][c] (k < nblk), fixed order: one block per
// column; thread t sums k = t, t + 256, ...; then a fixed tree.
__global__ void __launch_bounds__(256) k_sum_cols(const float *part, int nblk, int width, float *out)
{
    __shared__ double red[256];
    const int c = blockIdx.x;
    double acc = 0.0;
    for (int k = threadIdx.x; k < nblk; k += 256) acc += part[(int64_t)k * width + c];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = (float)red[0];
}

// ---------------------------------------------------------------------------
// Elementwise pieces
// ---------------------------------------------------------------------------
// network input: channel 0 = x / s, channels 1 .. 31 zero (the first layer's
// padded input); grid-stride, as its grid is capped (grid_for)
__global__ void k_in_prep(const float *x, int P, float inv_s, bf16 *xin)
{
    const int64_t n = (int64_t)P * 32;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int p = (int)(i / 32), c = (int)(i % 32);
        xin[i] = __float2bfloat16(c == 0 ? x[p] * inv_s : 0.f);
    }
}

// dst (H/2 x W/2) = 2x2 average of src (H x W), C channels
__global__ void k_pool(const bf16 *src, int lds, bf16 *dst, int ldd, int C, int B, int H, int W)
{
    const int H2 = H / 2, W2 = W / 2, C8 = C / 8;
    const int n = B * H2 * W2 * C8;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int c = (i % C8) * 8, q = i / C8;
        const int b = q / (H2 * W2), hw = q % (H2 * W2), h = hw / W2, w = hw % W2;
        const int64_t s0 = ((int64_t)(b * H + 2 * h) * W + 2 * w) * lds + c;
        const B8 x0 = ld8(src + s0), x1 = ld8(src + s0 + lds), x2 = ld8(src + s0 + (int64_t)W * lds),
                 x3 = ld8(src + s0 + (int64_t)W * lds + lds);
        B8 r;
#pragma unroll
        for (int k = 0; k < 8; ++k) r.v[k] = 0.25f * (x0.v[k] + x1.v[k] + x2.v[k] + x3.v[k]);
        st8(dst + (int64_t)q * ldd + c, r);
    }
}

// dst (2H x 2W) = nearest up-sampling of src (H x W)
__global__ void k_up(const bf16 *src, int lds, bf16 *dst, int ldd, int C, int B, int H, int W)
{
    const int H2 = 2 * H, W2 = 2 * W, C8 = C / 8;
    const int n = B * H2 * W2 * C8;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int c = (i % C8) * 8, q = i / C8;
        const int b = q / (H2 * W2), hw = q % (H2 * W2), h = hw / W2, w = hw % W2;
        *reinterpret_cast<uint4 *>(dst + (int64_t)q * ldd + c) =
            *reinterpret_cast<const uint4 *>(src + ((int64_t)(b * H + h / 2) * W + w / 2) * lds + c);
    }
}

// d(src) of the up-sampling (sum of the 2x2 children) times (x > 0): H x W output
__global__ void k_up_back_mask(const bf16 *dy, int ldy, const bf16 *x, int ldx, bf16 *dx, int ldd, int C,
                               int B, int H, int W)
{
    const int C8 = C / 8, n = B * H * W * C8, W2 = 2 * W;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int c = (i % C8) * 8, q = i / C8;
        const int b = q / (H * W), hw = q % (H * W), h = hw / W, w = hw % W;
        const int64_t s0 = ((int64_t)(b * 2 * H + 2 * h) * W2 + 2 * w) * ldy + c;
        const B8 y0 = ld8(dy + s0), y1 = ld8(dy + s0 + ldy), y2 = ld8(dy + s0 + (int64_t)W2 * ldy),
                 y3 = ld8(dy + s0 + (int64_t)W2 * ldy + ldy), xm = ld8(x + (int64_t)q * ldx + c);
        B8 r;
#pragma unroll
        for (int k = 0; k < 8; ++k) r.v[k] = xm.v[k] > 0.f ? y0.v[k] + y1.v[k] + y2.v[k] + y3.v[k] : 0.f;
        st8(dx + (int64_t)q * ldd + c, r);
    }
}

// de = (dskip + pool_back(dp)) * (e > 0) at H x W
__global__ void k_pool_back_mask(const bf16 *dskip, int lds, const bf16 *dp, int ldp, const bf16 *e, int lde,
                                 bf16 *de, int ldd, int C, int B, int H, int W)
{
    const int C8 = C / 8, n = B * H * W * C8, H2 = H / 2, W2 = W / 2;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int c = (i % C8) * 8, q = i / C8;
        const int b = q / (H * W), hw = q % (H * W), h = hw / W, w = hw % W;
        const B8 sk = ld8(dskip + (int64_t)q * lds + c),
                 pp = ld8(dp + ((int64_t)(b * H2 + h / 2) * W2 + w / 2) * ldp + c), em = ld8(e + (int64_t)q * lde + c);
        B8 r;
#pragma unroll
        for (int k = 0; k < 8; ++k) r.v[k] = em.v[k] > 0.f ? sk.v[k] + 0.25f * pp.v[k] : 0.f;
        st8(de + (int64_t)q * ldd + c, r);
    }
}

// out = x + s (Wh . d1 + bh); per-block partial sums of (out - t)^2 when t given
__global__ void k_head(const bf16 *d1, const float *Wh, const float *bh, const float *x, float s, int P,
                       float *out, const float *t, float *lpart)
{
    __shared__ float red[256];
    float l = 0.f;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
        float h = *bh;
        const bf16 *row = d1 + (int64_t)p * 32;
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const B8 v = ld8(row + 8 * g);
#pragma unroll
            for (int c = 0; c < 8; ++c) h = fmaf(Wh[8 * g + c], v.v[c], h);
        }
        const float o = x[p] + s * h;
        if (out) out[p] = o;
        if (t) {
            const float e = o - t[p];
            l += e * e;
        }
    }
    if (!lpart) return;
    red[threadIdx.x] = l;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) lpart[blockIdx.x] = red[0];
}

// Head backward: dh = s * 2 (out - t) / P; dd1 = dh Wh * (d1 > 0);
// partials of dWh[c] = sum dh d1[c] and dbh = sum dh per block.
__global__ void k_head_back(const bf16 *d1, const float *Wh, const float *out, const float *t, float s, int P,
                            bf16 *dd1, float *part /*[blocks][33]*/)
{
    __shared__ float red[33][256];
    float acc[33];
#pragma unroll
    for (int c = 0; c < 33; ++c) acc[c] = 0.f;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
        const float dh = s * 2.f * (out[p] - t[p]) / (float)P;
        const bf16 *row = d1 + (int64_t)p * 32;
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const B8 v = ld8(row + 8 * g);
            B8 o;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                acc[8 * g + c] = fmaf(dh, v.v[c], acc[8 * g + c]);
                o.v[c] = v.v[c] > 0.f ? dh * Wh[8 * g + c] : 0.f;
            }
            st8(dd1 + (int64_t)p * 32 + 8 * g, o);
        }
        acc[32] += dh;
    }
#pragma unroll
    for (int c = 0; c < 33; ++c) red[c][threadIdx.x] = acc[c];
    __syncthreads();
    if (threadIdx.x < 33) {
        float sum = 0.f;
        for (int k = 0; k < (int)blockDim.x; ++k) sum += red[threadIdx.x][k];
        part[blockIdx.x * 33 + threadIdx.x] = sum;
    }
}


// FP32 flat layer weights -> BF16 [Cout][9][Cin_pad] (forward) and
// [Cin][9][Cout] flipped (input gradient).
__global__ void k_wprep(const float *w, int Cout, int Cin, int Cin_pad, bf16 *wf, bf16 *wt)
{
    const int64_t n = (int64_t)Cout * Cin_pad * 9;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int co = (int)(i / (9 * Cin_pad)), r = (int)(i % (9 * Cin_pad));
        const int tap = r / Cin_pad, ci = r % Cin_pad;
        const float v = ci < Cin ? w[((int64_t)co * Cin + ci) * 9 + tap] : 0.f;
        wf[i] = __float2bfloat16(v);
        if (wt && ci < Cin) wt[((int64_t)ci * 9 + (8 - tap)) * Cout + co] = __float2bfloat16(v);
    }
}

__global__ void k_adam(float *p, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

unsigned grid_for(int64_t n) { return (unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)kSMs * 16); }

}  // namespace
}  // namespace dect

using namespace dect;

struct dect_cnn {
    int device;
    int max_p;  // max batch * H * W
    float *prm, *grad, *m, *v;  // FP32 [num_params]
    int64_t np;
    int64_t off_w[kLayers], off_b[kLayers], off_h;
    bf16 *wf[kLayers], *wt[kLayers];
    // activations (NHWC BF16): full res
    bf16 *xin, *a1, *e1, *c1, *a9, *d1;
    // half res
    bf16 *p1, *a3, *c2, *a7, *d2;
    // quarter res
    bf16 *p2, *a5, *bt;
    // gradients
    bf16 *g_full_a, *g_full_b, *g_c1, *g_half_a, *g_half_b, *g_c2, *g_q_a, *g_q_b;
    float *out, *wpart, *cpart, *hpart;
    size_t wpart_elems;
    int steps;  // Adam step count
    int conv_path;  // DECT_CNN_CONV_TCGEN05 or DECT_CNN_CONV_MMA_SYNC
    int conv_blocks_per_sm;  // k_conv_tc: 1 or 2 resident blocks per SM
    unsigned *err;  // device word: bit 0 = a bounded wait of k_conv_tc ran out
};

namespace {

bool alloc(void **p, size_t bytes) { return cudaMalloc(p, bytes) == cudaSuccess; }

// cuTensorMapEncodeTiled, fetched from the driver once (no link to libcuda)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// Launch plan of k_conv_tc for one layer: output channels per block (the
// whole layer up to 128; 96 for 192), weights resident when they fit in
// kTcWeightMax, else streamed with the pixels; the deepest ring that fits,
// with two blocks per SM when asked for and each keeps two stages or more.
struct TcPlan {
    int bn = 0, nstage = 0, per_sm = 1, smem = 0, cps = 1;
    bool stream = false, dxn = false;
};

TcPlan tc_plan(int Cin, int Cout, int blocks_per_sm)
{
    TcPlan p;
    if (Cin % kTcBK || Cout % 32) return p;
    const int bn = Cout <= 128 ? Cout : (Cout % 128 == 0 ? 128 : 96);
    if (Cout % bn) return p;
    // up to 64 output channels the three taps of a row go into N (3 BN)
    p.dxn = bn <= 64;
    p.stream = tc_weight_bytes(Cin, bn) > kTcWeightMax;
    const int chunk = tc_stage_bytes(bn, p.stream, p.dxn), fixed = tc_fixed_bytes(Cin, bn, p.stream);
    const int nck = Cin / kTcBK;
    // Chunks per stage: the most of a tile's chunks (a divisor of Cin / 32)
    // that leave the ring `min_st` stages in `budget` bytes.
    auto pick = [&](int budget, int min_st, int &cps, int &nst) {
        for (int c = nck; c >= 1; --c)
            if (nck % c == 0 && (budget - fixed) / (c * chunk) >= min_st) {
                cps = c;
                nst = std::min(kTcMaxStages, (budget - fixed) / (c * chunk));
                return true;
            }
        return false;
    };
    // two blocks per SM (each in half the SM's shared memory, at least two
    // stages) when asked for; otherwise, or when that does not fit, one block
    // with at least three stages (two if nothing more fits).  A block holding
    // all 512 tensor-memory columns must have its SM alone.
    const bool two = blocks_per_sm == 2 && tc_tmem_cols(bn, p.dxn) <= 256 &&
                     pick((228 * 1024) / 2 - 1024, 2, p.cps, p.nstage);
    if (two)
        p.per_sm = 2;
    else if (!pick(kTcSmemMax, 3, p.cps, p.nstage))
        pick(kTcSmemMax, 2, p.cps, p.nstage);
    const int stage = p.cps * chunk;
    if (p.nstage < 2) return TcPlan();
    p.bn = bn;
    p.smem = fixed + p.nstage * stage;
    // one block per SM: more than half of the SM's shared memory
    if (p.per_sm == 1) p.smem = std::max(p.smem, 116 * 1024);
    return p;
}

template <int BN, bool STREAM, bool DXN>
dect_status launch_conv_tc(const dect_cnn *n, const ConvArgs &a, const TcPlan &plan, cudaStream_t s)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) {
        set_error_text("k_conv_tc: cuTensorMapEncodeTiled is not available from the driver");
        return DECT_ERR_CUDA;
    }
    // X: NHWC view, 4-D {channel, x, y, image}; the box is one shifted halo copy
    CUtensorMap tx, tw;
    const cuuint64_t xdim[4] = {(cuuint64_t)a.Cin, (cuuint64_t)a.W, (cuuint64_t)a.H, (cuuint64_t)a.B};
    const cuuint64_t xstr[3] = {(cuuint64_t)a.ldx * 2, (cuuint64_t)a.W * a.ldx * 2, (cuuint64_t)a.H * a.W * a.ldx * 2};
    const cuuint32_t xbox[4] = {(cuuint32_t)kTcBK, (cuuint32_t)kTcTW, (cuuint32_t)(kTcTH + 2), 1u};
    const cuuint32_t ones[4] = {1u, 1u, 1u, 1u};
    CUresult r = enc(&tx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16 *>(a.X), xdim, xstr, xbox, ones,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    // Wt [Cout][9][Cin].  Streamed: one 3-D box {32 channels, BN rows, 9 taps}
    // per chunk (the tap stride Cin is smaller than the row stride 9 Cin), or,
    // if the driver does not take that map, boxes of BN rows x 32 channels of
    // one tap in a 2-D view [Cout][9 Cin] (the resident weights use those).
    int w3d = 0;
    if (r == CUDA_SUCCESS && STREAM) {
        const cuuint64_t wdim3[3] = {(cuuint64_t)a.Cin, (cuuint64_t)a.Cout, 9};
        const cuuint64_t wstr3[2] = {(cuuint64_t)9 * a.Cin * 2, (cuuint64_t)a.Cin * 2};
        const cuuint32_t wbox3[3] = {(cuuint32_t)kTcBK, (cuuint32_t)BN, 9u};
        w3d = enc(&tw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<bf16 *>(a.Wt), wdim3, wstr3, wbox3, ones,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    }
    const cuuint64_t wdim[2] = {(cuuint64_t)9 * a.Cin, (cuuint64_t)a.Cout};
    const cuuint64_t wstr[1] = {(cuuint64_t)9 * a.Cin * 2};
    const cuuint32_t wbox[2] = {(cuuint32_t)kTcBK, (cuuint32_t)BN};
    if (r == CUDA_SUCCESS && !w3d)
        r = enc(&tw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16 *>(a.Wt), wdim, wstr, wbox, ones,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error_text("k_conv_tc: cuTensorMapEncodeTiled failed with CUresult " + std::to_string((int)r));
        return DECT_ERR_CUDA;
    }
    // Every block takes more than a third of the SM's shared memory, so at
    // most two share an SM and their tensor memory (at most 256 columns
    // each) always fits in its 512.
    DECT_CUDA(
        cudaFuncSetAttribute(k_conv_tc<BN, STREAM, DXN>, cudaFuncAttributeMaxDynamicSharedMemorySize, plan.smem));
    constexpr int OW = DXN ? kTcTW - 2 : kTcTW;  // output columns per tile
    const int tiles_x = (a.W + OW - 1) / OW, tiles_y = (a.H + kTcTH - 1) / kTcTH;
    const int ntiles = a.B * tiles_x * tiles_y, ny = a.Cout / BN;
    const int gx = std::max(1, std::min(ntiles, (kSMs * plan.per_sm + ny - 1) / ny));
    k_conv_tc<BN, STREAM, DXN><<<dim3(gx, ny), kTcThreads, plan.smem, s>>>(tx, tw, a, tiles_x, tiles_y, plan.nstage,
                                                                            plan.cps, w3d, n->err);
    return DECT_OK;
}

dect_status conv(const dect_cnn *n, const bf16 *X, int ldx, int Cin, const bf16 *Wt, const float *bias, bf16 *Y,
                 int ldy, int Cout, const bf16 *mask, int ldm, bool relu, int B, int H, int W, cudaStream_t s)
{
    ConvArgs a{X, ldx, Cin, Wt, bias, Y, ldy, Cout, mask, ldm, relu ? 1 : 0, B, H, W};
    const int P = B * H * W;
    if (n->conv_path == DECT_CNN_CONV_TCGEN05) {
        dect_status st = DECT_ERR_INVALID_ARG;
        const TcPlan pl = tc_plan(Cin, Cout, n->conv_blocks_per_sm);
        switch (pl.bn * 2 + (pl.stream ? 1 : 0)) {
        case 256: st = launch_conv_tc<128, false, false>(n, a, pl, s); break;
        case 257: st = launch_conv_tc<128, true, false>(n, a, pl, s); break;
        case 192: st = launch_conv_tc<96, false, false>(n, a, pl, s); break;
        case 193: st = launch_conv_tc<96, true, false>(n, a, pl, s); break;
        case 128: st = launch_conv_tc<64, false, true>(n, a, pl, s); break;
        case 129: st = launch_conv_tc<64, true, true>(n, a, pl, s); break;
        case 64: st = launch_conv_tc<32, false, true>(n, a, pl, s); break;
        case 65: st = launch_conv_tc<32, true, true>(n, a, pl, s); break;
        default: set_error_text("k_conv_tc: no launch plan fits this layer");
        }
        if (st != DECT_OK) return st;
    } else if (Cout % 64 == 0) {
        dim3 g((P + 63) / 64, Cout / 64);
        k_conv<64><<<g, 128, 0, s>>>(a);
    } else {
        dim3 g((P + 63) / 64, Cout / 32);
        k_conv<32><<<g, 128, 0, s>>>(a);
    }
    count_launches(1);
    (void)n;
    DECT_CUDA(cudaGetLastError());
    return DECT_OK;
}

// NHWC BF16 view {C channels, W, H, B} (row stride ld) with boxes of
// 32 channels x 16 x `rows` pixels in the 64-byte swizzle
CUresult encode_nhwc(PFN_cuTensorMapEncodeTiled_v12000 enc, CUtensorMap *m, const bf16 *p, int C, int ld, int B,
                     int H, int W, int rows)
{
    const cuuint64_t dim[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
    const cuuint64_t str[3] = {(cuuint64_t)ld * 2, (cuuint64_t)W * ld * 2, (cuuint64_t)H * W * ld * 2};
    const cuuint32_t box[4] = {(cuuint32_t)kTcBK, (cuuint32_t)kTcTW, (cuuint32_t)rows, 1u};
    const cuuint32_t ones[4] = {1u, 1u, 1u, 1u};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16 *>(p), dim, str, box, ones,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

// Weight gradient of layer l on the tensor cores (k_wgrad_tc + its reduce).
template <int N>
dect_status wgrad_tc(dect_cnn *n, int l, const bf16 *dY, int ldd, const bf16 *X, int ldx, int B, int H, int W,
                     cudaStream_t s)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) {
        set_error_text("k_wgrad_tc: cuTensorMapEncodeTiled is not available from the driver");
        return DECT_ERR_CUDA;
    }
    const int Cinp = cin_pad(l);
    WgTcArgs a{Cinp, N, B, H, W, Cinp / kTcBK, (9 * (Cinp / kTcBK) + 3) / 4};
    // groups of four slots per block: as many as two stages of the ring allow
    const int G = std::min(N == 32 ? 3 : 2, a.ngroups);
    const int stage = wg_stage_bytes(G, N);
    const int nstage = std::min(kWgMaxStages, (kTcSmemMax - 1024 - 256 - kWgBox) / stage);
    if (nstage < 2) {
        set_error_text("k_wgrad_tc: no ring of two stages fits");
        return DECT_ERR_INVALID_ARG;
    }
    // (plus one box of slack after the barriers: no operand address, under
    // either stride of its descriptor, can leave the block's shared memory)
    const int smem = 1024 + nstage * stage + 256 + kWgBox;
    CUtensorMap tx, td;
    CUresult r = encode_nhwc(enc, &tx, X, Cinp, ldx, B, H, W, kWgR);
    if (r == CUDA_SUCCESS) r = encode_nhwc(enc, &td, dY, N, ldd, B, H, W, kWgR);
    if (r != CUDA_SUCCESS) {
        set_error_text("k_wgrad_tc: cuTensorMapEncodeTiled failed with CUresult " + std::to_string((int)r));
        return DECT_ERR_CUDA;
    }
    const int gy = (a.ngroups + G - 1) / G;
    const int ntiles = B * ((W + kTcTW - 1) / kTcTW) * ((H + kWgR - 1) / kWgR);
    const int gx = std::max(1, std::min(ntiles, kSMs / gy));
    if ((int64_t)gx * a.ngroups * 128 * N > (int64_t)n->wpart_elems) {
        set_error_text("k_wgrad_tc: partials exceed the scratch buffer");
        return DECT_ERR_INVALID_ARG;
    }
    DECT_CUDA(cudaFuncSetAttribute(k_wgrad_tc<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    k_wgrad_tc<N><<<dim3(gy, gx), kWgThreads, smem, s>>>(tx, td, a, G, nstage, n->wpart, n->err);
    k_wgrad_tc_reduce<<<grid_for((int64_t)a.ngroups * 128 * N), 256, 0, s>>>(n->wpart, gx, a.ngroups, N, a.ncb,
                                                                            kCin[l], n->grad + n->off_w[l]);
    count_launches(2);
    return DECT_OK;
}

dect_status wgrad(dect_cnn *n, int l, const bf16 *dY, int ldd, const bf16 *X, int ldx, int B, int H, int W,
                  cudaStream_t s)
{
    const int Cout = kCout[l], Cinp = cin_pad(l), P = B * H * W;
    if (n->conv_path == DECT_CNN_CONV_TCGEN05) {
        dect_status st = DECT_ERR_INVALID_ARG;
        switch (Cout) {
        case 32: st = wgrad_tc<32>(n, l, dY, ldd, X, ldx, B, H, W, s); break;
        case 64: st = wgrad_tc<64>(n, l, dY, ldd, X, ldx, B, H, W, s); break;
        case 128: st = wgrad_tc<128>(n, l, dY, ldd, X, ldx, B, H, W, s); break;
        default: set_error_text("k_wgrad_tc: unsupported output channel count");
        }
        if (st != DECT_OK) return st;
        const int cpps = 4096, csplits = (P + cpps - 1) / cpps;
        k_chansum<<<csplits, 256, 0, s>>>(dY, ldd, Cout, P, cpps, n->cpart);
        k_sum_cols<<<Cout, 256, 0, s>>>(n->cpart, csplits, Cout, n->grad + n->off_b[l]);
        count_launches(2);
        DECT_CUDA(cudaGetLastError());
        return DECT_OK;
    }
    const int tiles = 9 * (Cinp / 32) * (Cout / 32);
    int pps = 2048;
    while ((int64_t)((P + pps - 1) / pps) * Cout * 9 * Cinp > (int64_t)n->wpart_elems) pps *= 2;
    const int splits = (P + pps - 1) / pps;
    WgradArgs a{dY, ldd, Cout, X, ldx, Cinp, n->wpart, B, H, W, pps};
    dim3 g(splits, 9 * (Cinp / 32), Cout / 32);
    (void)tiles;
    k_wgrad<<<g, 128, 0, s>>>(a);
    k_wgrad_reduce<<<(unsigned)(((int64_t)Cout * 9 * Cinp + 31) / 32), 256, 0, s>>>(n->wpart, splits, Cout, Cinp, kCin[l],
                                                                        n->grad + n->off_w[l]);
    const int cpps = 4096, csplits = (P + cpps - 1) / cpps;
    k_chansum<<<csplits, 256, 0, s>>>(dY, ldd, Cout, P, cpps, n->cpart);
    k_sum_cols<<<Cout, 256, 0, s>>>(n->cpart, csplits, Cout, n->grad + n->off_b[l]);
    count_launches(4);
    DECT_CUDA(cudaGetLastError());
    return DECT_OK;
}

dect_status forward(dect_cnn *n, const float *x, int B, int H, int W, float scale, cudaStream_t s)
{
    const int P = B * H * W, H2 = H / 2, W2 = W / 2, H4 = H / 4, W4 = W / 4;
    const int P2 = B * H2 * W2, P4 = B * H4 * W4;
    for (int l = 0; l < kLayers; ++l) {
        k_wprep<<<grid_for((int64_t)kCout[l] * cin_pad(l) * 9), 256, 0, s>>>(
            n->prm + n->off_w[l], kCout[l], kCin[l], cin_pad(l), n->wf[l], n->wt[l]);
        count_launches(1);
    }
    k_in_prep<<<grid_for((int64_t)P * 32), 256, 0, s>>>(x, P, 1.f / scale, n->xin);
    count_launches(1);
    const float *b = n->prm;
    dect_status st;
#define CONV(...) if ((st = conv(n, __VA_ARGS__)) != DECT_OK) return st
    CONV(n->xin, 32, 32, n->wf[0], b + n->off_b[0], n->a1, 32, 32, nullptr, 0, true, B, H, W, s);
    CONV(n->a1, 32, 32, n->wf[1], b + n->off_b[1], n->c1 + 64, 96, 32, nullptr, 0, true, B, H, W, s);  // e1
    k_pool<<<grid_for((int64_t)P2 * 4), 256, 0, s>>>(n->c1 + 64, 96, n->p1, 32, 32, B, H, W);
    CONV(n->p1, 32, 32, n->wf[2], b + n->off_b[2], n->a3, 64, 64, nullptr, 0, true, B, H2, W2, s);
    CONV(n->a3, 64, 64, n->wf[3], b + n->off_b[3], n->c2 + 128, 192, 64, nullptr, 0, true, B, H2, W2, s);  // e2
    k_pool<<<grid_for((int64_t)P4 * 8), 256, 0, s>>>(n->c2 + 128, 192, n->p2, 64, 64, B, H2, W2);
    CONV(n->p2, 64, 64, n->wf[4], b + n->off_b[4], n->a5, 128, 128, nullptr, 0, true, B, H4, W4, s);
    CONV(n->a5, 128, 128, n->wf[5], b + n->off_b[5], n->bt, 128, 128, nullptr, 0, true, B, H4, W4, s);
    k_up<<<grid_for((int64_t)P2 * 16), 256, 0, s>>>(n->bt, 128, n->c2, 192, 128, B, H4, W4);
    CONV(n->c2, 192, 192, n->wf[6], b + n->off_b[6], n->a7, 64, 64, nullptr, 0, true, B, H2, W2, s);
    CONV(n->a7, 64, 64, n->wf[7], b + n->off_b[7], n->d2, 64, 64, nullptr, 0, true, B, H2, W2, s);
    k_up<<<grid_for((int64_t)P * 8), 256, 0, s>>>(n->d2, 64, n->c1, 96, 64, B, H2, W2);
    CONV(n->c1, 96, 96, n->wf[8], b + n->off_b[8], n->a9, 32, 32, nullptr, 0, true, B, H, W, s);
    CONV(n->a9, 32, 32, n->wf[9], b + n->off_b[9], n->d1, 32, 32, nullptr, 0, true, B, H, W, s);
#undef CONV
    count_launches(3);
    DECT_CUDA(cudaGetLastError());
    return DECT_OK;
}

bool shape_ok(const dect_cnn *n, int B, int H, int W)
{
    return n && B >= 1 && H >= 4 && W >= 4 && H % 4 == 0 && W % 4 == 0 && (int64_t)B * H * W <= n->max_p;
}

}  // namespace

extern "C" int64_t dect_cnn_num_params(void) { return num_params(); }

extern "C" dect_status dect_cnn_create(int device, int max_pixels, dect_cnn **out)
{
    if (!out || max_pixels < 16) return DECT_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    DECT_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return DECT_ERR_INVALID_ARG;
    DECT_CUDA(cudaSetDevice(device));
    dect_cnn *n = new dect_cnn();
    std::memset(n, 0, sizeof(*n));
    n->device = device;
    n->max_p = max_pixels;
    n->conv_blocks_per_sm = 2;
    n->np = num_params();
    int64_t o = 0;
    for (int l = 0; l < kLayers; ++l) {
        n->off_w[l] = o;
        o += (int64_t)kCout[l] * kCin[l] * 9;
        n->off_b[l] = o;
        o += kCout[l];
    }
    n->off_h = o;
    const size_t P = (size_t)max_pixels, P2 = P / 4 + 1, P4 = P / 16 + 1;
    bool ok = alloc((void **)&n->prm, 4 * n->np) && alloc((void **)&n->grad, 4 * n->np) &&
              alloc((void **)&n->m, 4 * n->np) && alloc((void **)&n->v, 4 * n->np);
    for (int l = 0; l < kLayers && ok; ++l) {
        ok = alloc((void **)&n->wf[l], 2 * (size_t)kCout[l] * 9 * cin_pad(l)) &&
             alloc((void **)&n->wt[l], 2 * (size_t)kCin[l] * 9 * kCout[l] + 64);
    }
    auto A = [&](bf16 **p, size_t elems) { if (ok) ok = alloc((void **)p, 2 * elems + 64); };
    A(&n->xin, P * 32); A(&n->a1, P * 32); A(&n->e1, 16); A(&n->c1, P * 96); A(&n->a9, P * 32); A(&n->d1, P * 32);
    A(&n->p1, P2 * 32); A(&n->a3, P2 * 64); A(&n->c2, P2 * 192); A(&n->a7, P2 * 64); A(&n->d2, P2 * 64);
    A(&n->p2, P4 * 64); A(&n->a5, P4 * 128); A(&n->bt, P4 * 128);
    A(&n->g_full_a, P * 32); A(&n->g_full_b, P * 32); A(&n->g_c1, P * 96);
    A(&n->g_half_a, P2 * 64); A(&n->g_half_b, P2 * 64); A(&n->g_c2, P2 * 192);
    A(&n->g_q_a, P4 * 128); A(&n->g_q_b, P4 * 128);
    n->wpart_elems = (size_t)64 << 20;  // 256 MB of FP32 split-K partials at most
    if (ok) ok = alloc((void **)&n->out, 4 * P) && alloc((void **)&n->wpart, 4 * n->wpart_elems) &&
                 alloc((void **)&n->cpart, 4 * ((P / 4096 + 2) * 192)) && alloc((void **)&n->hpart, 4 * 4096 * 33);
    if (ok) ok = alloc((void **)&n->err, sizeof(unsigned));
    if (ok) ok = cudaMemset(n->m, 0, 4 * n->np) == cudaSuccess && cudaMemset(n->v, 0, 4 * n->np) == cudaSuccess &&
                 cudaMemset(n->prm, 0, 4 * n->np) == cudaSuccess && cudaMemset(n->err, 0, sizeof(unsigned)) == cudaSuccess;
    if (!ok) {
        dect_cnn_destroy(n);
        return DECT_ERR_OOM;
    }
    *out = n;
    return DECT_OK;
}

extern "C" dect_status dect_cnn_destroy(dect_cnn *n)
{
    if (!n) return DECT_OK;
    cudaSetDevice(n->device);
    cudaDeviceSynchronize();
    void *ptrs[] = {n->prm, n->grad, n->m, n->v, n->xin, n->a1, n->e1, n->c1, n->a9, n->d1, n->p1, n->a3,
                    n->c2, n->a7, n->d2, n->p2, n->a5, n->bt, n->g_full_a, n->g_full_b, n->g_c1, n->g_half_a,
                    n->g_half_b, n->g_c2, n->g_q_a, n->g_q_b, n->out, n->wpart, n->cpart, n->hpart, n->err};
    for (void *p : ptrs) cudaFree(p);
    for (int l = 0; l < kLayers; ++l) {
        cudaFree(n->wf[l]);
        cudaFree(n->wt[l]);
    }
    delete n;
    return DECT_OK;
}

extern "C" dect_status dect_cnn_set_params(dect_cnn *n, const float *params)
{
    if (!n || !params) return DECT_ERR_INVALID_ARG;
    DECT_CUDA(cudaSetDevice(n->device));
    DECT_CUDA(cudaMemcpy(n->prm, params, 4 * n->np, cudaMemcpyHostToDevice));
    DECT_CUDA(cudaMemset(n->m, 0, 4 * n->np));
    DECT_CUDA(cudaMemset(n->v, 0, 4 * n->np));
    n->steps = 0;
    return DECT_OK;
}

extern "C" dect_status dect_cnn_get_params(const dect_cnn *n, float *params)
{
    if (!n || !params) return DECT_ERR_INVALID_ARG;
    DECT_CUDA(cudaSetDevice(n->device));
    DECT_CUDA(cudaMemcpy(params, n->prm, 4 * n->np, cudaMemcpyDeviceToHost));
    return DECT_OK;
}

extern "C" dect_status dect_cnn_forward(dect_cnn *n, const float *x, float *out, int batch, int h, int w,
                                        float scale, dect_stream stream)
{
    if (!shape_ok(n, batch, h, w) || !x || !out || !(scale > 0)) return DECT_ERR_INVALID_ARG;
    DECT_CUDA(cudaSetDevice(n->device));
    cudaStream_t s = (cudaStream_t)stream;
    dect_status st = forward(n, x, batch, h, w, scale, s);
    if (st != DECT_OK) return st;
    const int P = batch * h * w;
    k_head<<<grid_for(P), 256, 0, s>>>(n->d1, n->prm + n->off_h, n->prm + n->off_h + 32, x, scale, P, out,
                                      nullptr, nullptr);
    count_launches(1);
    DECT_LAUNCH_CHECK();
    return DECT_OK;
}

extern "C" dect_status dect_cnn_loss_grad(dect_cnn *n, const float *x, const float *target, int batch, int h,
                                          int w, float scale, float *loss, float *grad_host, dect_stream stream)
{
    if (!shape_ok(n, batch, h, w) || !x || !target || !(scale > 0)) return DECT_ERR_INVALID_ARG;
    DECT_CUDA(cudaSetDevice(n->device));
    cudaStream_t s = (cudaStream_t)stream;
    dect_status st = forward(n, x, batch, h, w, scale, s);
    if (st != DECT_OK) return st;
    const int B = batch, H = h, W = w, H2 = H / 2, W2 = W / 2, H4 = H / 4, W4 = W / 4;
    const int P = B * H * W, P2 = B * H2 * W2, P4 = B * H4 * W4;
    const int hb = (int)std::min<int64_t>((P + 255) / 256, 4096);
    k_head<<<hb, 256, 0, s>>>(n->d1, n->prm + n->off_h, n->prm + n->off_h + 32, x, scale, P, n->out, target,
                              n->hpart);
    k_sum_cols<<<1, 256, 0, s>>>(n->hpart, hb, 1, n->cpart);  // loss * P in cpart[0]
    float lsum = 0.f;
    DECT_CUDA(cudaMemcpyAsync(&lsum, n->cpart, 4, cudaMemcpyDeviceToHost, s));
    // head backward
    k_head_back<<<hb, 256, 0, s>>>(n->d1, n->prm + n->off_h, n->out, target, scale, P, n->g_full_a, n->hpart);
    k_sum_cols<<<33, 256, 0, s>>>(n->hpart, hb, 33, n->grad + n->off_h);
    count_launches(4);
    // conv10: input a9, output grad g_full_a (dd1, masked)
    if ((st = wgrad(n, 9, n->g_full_a, 32, n->a9, 32, B, H, W, s)) != DECT_OK) return st;
    if ((st = conv(n, n->g_full_a, 32, 32, n->wt[9], nullptr, n->g_full_b, 32, 32, n->a9, 32, false, B, H, W, s)) != DECT_OK) return st;  // da9
    if ((st = wgrad(n, 8, n->g_full_b, 32, n->c1, 96, B, H, W, s)) != DECT_OK) return st;
    if ((st = conv(n, n->g_full_b, 32, 32, n->wt[8], nullptr, n->g_c1, 96, 96, nullptr, 0, false, B, H, W, s)) != DECT_OK) return st;  // dc1
    k_up_back_mask<<<grid_for((int64_t)P2 * 8), 256, 0, s>>>(n->g_c1, 96, n->d2, 64, n->g_half_a, 64, 64, B, H2, W2);  // dd2
    if ((st = wgrad(n, 7, n->g_half_a, 64, n->a7, 64, B, H2, W2, s)) != DECT_OK) return st;
    if ((st = conv(n, n->g_half_a, 64, 64, n->wt[7], nullptr, n->g_half_b, 64, 64, n->a7, 64, false, B, H2, W2, s)) != DECT_OK) return st;  // da7
    if ((st = wgrad(n, 6, n->g_half_b, 64, n->c2, 192, B, H2, W2, s)) != DECT_OK) return st;
    if ((st = conv(n, n->g_half_b, 64, 64, n->wt[6], nullptr, n->g_c2, 192, 192, nullptr, 0, false, B, H2, W2, s)) != DECT_OK) return st;  // dc2
    k_up_back_mask<<<grid_for((int64_t)P4 * 16), 256, 0, s>>>(n->g_c2, 192, n->bt, 128, n->g_q_a, 128, 128, B, H4, W4);  // dbt
    if ((st = wgrad(n, 5, n->g_q_a, 128, n->a5, 128, B, H4, W4, s)) != DECT_OK) return st;
    if ((st = conv(n, n->g_q_a, 128, 128, n->wt[5], nullptr, n->g_q_b, 128, 128, n->a5, 128, false, B, H4, W4, s)) != DECT_OK) return st;  // da5
    if ((st = wgrad(n, 4, n->g_q_b, 128, n->p2, 64, B, H4, W4, s)) != DECT_OK) return st;
    if ((st = conv(n, n->g_q_b, 128, 128, n->wt[4], nullptr, n->g_q_a, 64, 64, nullptr, 0, false, B, H4, W4, s)) != DECT_OK) return st;  // dp2
    k_pool_back_mask<<<grid_for((int64_t)P2 * 8), 256, 0, s>>>(n->g_c2 + 128, 192, n->g_q_a, 64, n->c2 + 128, 192,
                                                               n->g_half_a, 64, 64, B, H2, W2);  // de2
    if ((st = wgrad(n, 3, n->g_half_a, 64, n->a3, 64, B, H2, W2, s)) != DECT_OK) return st;
    if ((st = conv(n, n->g_half_a, 64, 64, n->wt[3], nullptr, n->g_half_b, 64, 64, n->a3, 64, false, B, H2, W2, s)) != DECT_OK) return st;  // da3
    if ((st = wgrad(n, 2, n->g_half_b, 64, n->p1, 32, B, H2, W2, s)) != DECT_OK) return st;
    if ((st = conv(n, n->g_half_b, 64, 64, n->wt[2], nullptr, n->g_half_a, 32, 32, nullptr, 0, false, B, H2, W2, s)) != DECT_OK) return st;  // dp1
    k_pool_back_mask<<<grid_for((int64_t)P * 4), 256, 0, s>>>(n->g_c1 + 64, 96, n->g_half_a, 32, n->c1 + 64, 96,
                                                              n->g_full_a, 32, 32, B, H, W);  // de1
    if ((st = wgrad(n, 1, n->g_full_a, 32, n->a1, 32, B, H, W, s)) != DECT_OK) return st;
    if ((st = conv(n, n->g_full_a, 32, 32, n->wt[1], nullptr, n->g_full_b, 32, 32, n->a1, 32, false, B, H, W, s)) != DECT_OK) return st;  // da1
    if ((st = wgrad(n, 0, n->g_full_b, 32, n->xin, 32, B, H, W, s)) != DECT_OK) return st;
    count_launches(3);
    DECT_LAUNCH_CHECK();
    DECT_CUDA(cudaStreamSynchronize(s));
    if ((st = dect_cnn_check(n)) != DECT_OK) return st;
    if (loss) *loss = lsum / (float)P;
    if (grad_host) DECT_CUDA(cudaMemcpy(grad_host, n->grad, 4 * n->np, cudaMemcpyDeviceToHost));
    return DECT_OK;
}

extern "C" dect_status dect_cnn_adam_step(dect_cnn *n, float lr, float beta1, float beta2, float eps,
                                          dect_stream stream)
{
    if (!n || !(lr > 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0))
        return DECT_ERR_INVALID_ARG;
    DECT_CUDA(cudaSetDevice(n->device));
    n->steps += 1;
    const float c1 = 1.f - std::pow(beta1, (float)n->steps), c2 = 1.f - std::pow(beta2, (float)n->steps);
    k_adam<<<grid_for(n->np), 256, 0, (cudaStream_t)stream>>>(n->prm, n->grad, n->m, n->v, n->np, lr, beta1, beta2,
                                                             eps, c1, c2);
    count_launches(1);
    DECT_LAUNCH_CHECK();
    return DECT_OK;
}

extern "C" dect_status dect_cnn_set_conv_path(dect_cnn *n, int path)
{
    if (!n || (path != DECT_CNN_CONV_TCGEN05 && path != DECT_CNN_CONV_MMA_SYNC)) return DECT_ERR_INVALID_ARG;
    n->conv_path = path;
    return DECT_OK;
}

extern "C" int dect_cnn_get_conv_path(const dect_cnn *n) { return n ? n->conv_path : -1; }

extern "C" dect_status dect_cnn_set_conv_tuning(dect_cnn *n, int blocks_per_sm)
{
    if (!n || (blocks_per_sm != 1 && blocks_per_sm != 2)) return DECT_ERR_INVALID_ARG;
    n->conv_blocks_per_sm = blocks_per_sm;
    return DECT_OK;
}

extern "C" dect_status dect_cnn_check(dect_cnn *n)
{
    if (!n) return DECT_ERR_INVALID_ARG;
    DECT_CUDA(cudaSetDevice(n->device));
    DECT_CUDA(cudaDeviceSynchronize());
    unsigned h = 0;
    DECT_CUDA(cudaMemcpy(&h, n->err, sizeof(h), cudaMemcpyDeviceToHost));
    if (h) {
        DECT_CUDA(cudaMemset(n->err, 0, sizeof(unsigned)));
        set_error_text("k_conv_tc: a bounded wait ran out (the convolution's output is not valid)");
        return DECT_ERR_TIMEOUT;
    }
    return DECT_OK;
}
