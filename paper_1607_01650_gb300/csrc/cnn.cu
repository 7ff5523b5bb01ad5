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
// convolutions are implicit GEMMs on the tensor cores (mma.sync m16n8k16,
// BF16 inputs, FP32 accumulation).  Input gradients use the same kernel with
// the weights flipped and transposed; weight gradients are a split-K
// implicit GEMM reduced in a fixed order.  Master weights, gradients and the
// Adam state are FP32.  Parameter vector layout (shared with the host):
// per layer W[Cout][Cin][3][3] then b[Cout]; then the head Wh[32], bh.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "dect_internal.cuh"

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
__device__ __forceinline__ unsigned su32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp16_zfill(void *smem, const void *gmem, bool valid)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(su32(smem)), "l"(gmem),
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
                 : "r"(su32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(unsigned (&r)[4], const void *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(su32(p)));
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

// dW (flat layout [Cout][Cin_real][3][3]) = sum over splits, in order.
__global__ void k_wgrad_reduce(const float *part, int splits, int Cout, int Cin_pad, int Cin_real, float *dW)
{
    const int64_t n = (int64_t)Cout * Cin_real * 9;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int co = (int)(i / (Cin_real * 9)), r = (int)(i % (Cin_real * 9));
        const int ci = r / 9, tap = r % 9;
        double s = 0.0;
        for (int k = 0; k < splits; ++k) s += part[(((int64_t)k * Cout + co) * 9 + tap) * Cin_pad + ci];
        dW[i] = (float)s;
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

__global__ void k_chansum_reduce(const float *part, int splits, int C, float *out)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    double s = 0.0;
    for (int k = 0; k < splits; ++k) s += part[(int64_t)k * C + c];
    out[c] = (float)s;
}

// ---------------------------------------------------------------------------
// Elementwise pieces
// ---------------------------------------------------------------------------
__global__ void k_in_prep(const float *x, int P, float inv_s, bf16 *xin)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)P * 32) return;
    const int p = (int)(i / 32), c = (int)(i % 32);
    xin[i] = __float2bfloat16(c == 0 ? x[p] * inv_s : 0.f);
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
        for (int c = 0; c < 32; ++c) h = fmaf(Wh[c], __bfloat162float(row[c]), h);
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
        for (int c = 0; c < 32; ++c) {
            const float v = __bfloat162float(row[c]);
            acc[c] = fmaf(dh, v, acc[c]);
            dd1[(int64_t)p * 32 + c] = __float2bfloat16(v > 0.f ? dh * Wh[c] : 0.f);
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

__global__ void k_sum_parts(const float *part, int nblk, int width, float *out)
{
    const int c = threadIdx.x;
    if (c >= width) return;
    double s = 0.0;
    for (int k = 0; k < nblk; ++k) s += part[k * width + c];
    out[c] = (float)s;
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
};

namespace {

bool alloc(void **p, size_t bytes) { return cudaMalloc(p, bytes) == cudaSuccess; }

dect_status conv(const dect_cnn *n, const bf16 *X, int ldx, int Cin, const bf16 *Wt, const float *bias, bf16 *Y,
                 int ldy, int Cout, const bf16 *mask, int ldm, bool relu, int B, int H, int W, cudaStream_t s)
{
    ConvArgs a{X, ldx, Cin, Wt, bias, Y, ldy, Cout, mask, ldm, relu ? 1 : 0, B, H, W};
    const int P = B * H * W;
    if (Cout % 64 == 0) {
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

dect_status wgrad(dect_cnn *n, int l, const bf16 *dY, int ldd, const bf16 *X, int ldx, int B, int H, int W,
                  cudaStream_t s)
{
    const int Cout = kCout[l], Cinp = cin_pad(l), P = B * H * W;
    const int tiles = 9 * (Cinp / 32) * (Cout / 32);
    int pps = 2048;
    while ((int64_t)((P + pps - 1) / pps) * Cout * 9 * Cinp > (int64_t)n->wpart_elems) pps *= 2;
    const int splits = (P + pps - 1) / pps;
    WgradArgs a{dY, ldd, Cout, X, ldx, Cinp, n->wpart, B, H, W, pps};
    dim3 g(splits, 9 * (Cinp / 32), Cout / 32);
    (void)tiles;
    k_wgrad<<<g, 128, 0, s>>>(a);
    k_wgrad_reduce<<<grid_for((int64_t)Cout * kCin[l] * 9), 256, 0, s>>>(n->wpart, splits, Cout, Cinp, kCin[l],
                                                                        n->grad + n->off_w[l]);
    const int cpps = 4096, csplits = (P + cpps - 1) / cpps;
    k_chansum<<<csplits, 256, 0, s>>>(dY, ldd, Cout, P, cpps, n->cpart);
    k_chansum_reduce<<<1, 128, 0, s>>>(n->cpart, csplits, Cout, n->grad + n->off_b[l]);
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
    if (ok) ok = cudaMemset(n->m, 0, 4 * n->np) == cudaSuccess && cudaMemset(n->v, 0, 4 * n->np) == cudaSuccess &&
                 cudaMemset(n->prm, 0, 4 * n->np) == cudaSuccess;
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
                    n->g_half_b, n->g_c2, n->g_q_a, n->g_q_b, n->out, n->wpart, n->cpart, n->hpart};
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
    k_sum_parts<<<1, 64, 0, s>>>(n->hpart, hb, 1, n->cpart);  // loss * P in cpart[0]
    float lsum = 0.f;
    DECT_CUDA(cudaMemcpyAsync(&lsum, n->cpart, 4, cudaMemcpyDeviceToHost, s));
    // head backward
    k_head_back<<<hb, 256, 0, s>>>(n->d1, n->prm + n->off_h, n->out, target, scale, P, n->g_full_a, n->hpart);
    k_sum_parts<<<1, 64, 0, s>>>(n->hpart, hb, 33, n->grad + n->off_h);
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
