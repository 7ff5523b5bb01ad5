// PLS image-domain decomposition, Eq. (11)-(15) (Sec. 2.3).
//
//   d   = D^{-1} x per pixel, D = [[eta_1H, eta_2H], [eta_1L, eta_2L]]     Eq. (11)-(12)
//         (closed-form 2x2 inverse in FP64)
//   e_ik= edge_eps if pixel i or k is an edge, else 1                     Eq. (14)
//         (edge: 3x3 Prewitt magnitude of x_h or x_l over its maximum > tau)
//   (I + gamma L_e) u_m = d_m,  (L_e u)_i = sum_{k in N_i} e_ik (u_i - u_k)
//         -- Eq. (15) with Hessian R = 2 L_e -- by Jacobi-preconditioned CG
//         from u = d, FP32 vectors, FP64 scalars.
//
// Vectors: v = 2 s + m (slice s, material m) at u + v N (the [slice][2][n][n]
// layout of the input and output); the CG runs
// all vectors of the batch in lockstep with per-vector step sizes and stop
// flags.  The edge decision is taken in FP32 (the precision of the
// reconstructed images; the paper fixes none for it): it can differ from the
// FP64 decision only at pixels whose normalised magnitude lies within FP32
// rounding of the threshold.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "dect_internal.cuh"

namespace dect {
namespace {

constexpr int kBlock = 256;

struct PlsDev {
    // scalars per vector
    double *red;      // [3][nvec] results of the last reduction
    double *part;     // [gx * nvec * 3] block partials
    unsigned *ctr;    // [2] last-block counters
    double *alpha, *beta, *rz, *bnorm, *relres;  // [nvec]
    int *iters, *done, *it;                      // [nvec], [nvec], [1]
    int *all_done;
    int *maxbits;     // [2 * nslices] float bits of max Prewitt magnitude
};

struct PlsConst {
    int n, nz;   // nz = 1: 2-D images (4 neighbours); nz > 1: volumes (6 neighbours)
    int64_t N;
    int nvec;
    float gamma, eps;
    double tol;
};

// FP32 warp sums, FP64 across warps and blocks (fixed order).  The block
// that finishes last writes out[y * K + k] (y = blockIdx.y) and returns true.
template <int K>
__device__ bool reduce_planar(const float (&v)[K], double *part, double *out, unsigned *counter)
{
    __shared__ double smem[(kBlock / 32) * K];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float w[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        w[k] = v[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) w[k] += __shfl_xor_sync(0xffffffffu, w[k], off);
    }
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) smem[warp * K + k] = (double)w[k];
    __syncthreads();
    const unsigned gx = gridDim.x, gy = gridDim.y;
    if (threadIdx.x < K) {
        double s = 0.0;
        for (int q = 0; q < nw; ++q) s += smem[q * K + threadIdx.x];
        part[((size_t)blockIdx.y * gx + blockIdx.x) * K + threadIdx.x] = s;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gx * gy - 1);
    __syncthreads();
    if (!last) return false;
    __threadfence();
    for (unsigned t = threadIdx.x; t < gy * K; t += blockDim.x) {
        const unsigned y = t / K, k = t % K;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        unsigned b = 0;
        for (; b + 4 <= gx; b += 4) {
            s0 += __ldcg(&part[((size_t)y * gx + b) * K + k]);
            s1 += __ldcg(&part[((size_t)y * gx + b + 1) * K + k]);
            s2 += __ldcg(&part[((size_t)y * gx + b + 2) * K + k]);
            s3 += __ldcg(&part[((size_t)y * gx + b + 3) * K + k]);
        }
        for (; b < gx; ++b) s0 += __ldcg(&part[((size_t)y * gx + b) * K + k]);
        out[t] = (s0 + s1) + (s2 + s3);
    }
    if (threadIdx.x == 0) *counter = 0u;
    __syncthreads();
    return true;
}

__device__ __forceinline__ int clampi(int a, int lo, int hi) { return a < lo ? lo : (a > hi ? hi : a); }

// Prewitt magnitude, FP32, explicit rounding (same order of operations as
// the decision rule states).
__device__ __forceinline__ float prewitt_at(const float *__restrict__ x, int n, int i, int j)
{
    const int jl = clampi(j - 1, 0, n - 1), jr = clampi(j + 1, 0, n - 1);
    const int iu = clampi(i - 1, 0, n - 1), id = clampi(i + 1, 0, n - 1);
    float gx = 0.f, gy = 0.f;
#pragma unroll
    for (int t = -1; t <= 1; ++t) {
        const int ii = clampi(i + t, 0, n - 1), jj = clampi(j + t, 0, n - 1);
        gx = __fadd_rn(gx, __fsub_rn(x[(int64_t)ii * n + jr], x[(int64_t)ii * n + jl]));
        gy = __fadd_rn(gy, __fsub_rn(x[(int64_t)id * n + jj], x[(int64_t)iu * n + jj]));
    }
    return __fsqrt_rn(__fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy)));
}

// 3-D Prewitt magnitude (volumes of nz > 1 slices), FP32, each component
// summed in the order of the two outer offsets s, t = -1, 0, 1.
__device__ __forceinline__ float prewitt3_at(const float *__restrict__ x, int n, int nz, int k, int i, int j)
{
    auto X = [&](int kk, int ii, int jj) {
        return x[((int64_t)clampi(kk, 0, nz - 1) * n + clampi(ii, 0, n - 1)) * n + clampi(jj, 0, n - 1)];
    };
    float gx = 0.f, gy = 0.f, gz = 0.f;
    for (int a = -1; a <= 1; ++a)
        for (int b = -1; b <= 1; ++b) {
            gx = __fadd_rn(gx, __fsub_rn(X(k + a, i + b, j + 1), X(k + a, i + b, j - 1)));
            gy = __fadd_rn(gy, __fsub_rn(X(k + a, i + 1, j + b), X(k + a, i - 1, j + b)));
            gz = __fadd_rn(gz, __fsub_rn(X(k + 1, i + a, j + b), X(k - 1, i + a, j + b)));
        }
    return __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy)), __fmul_rn(gz, gz)));
}

// d = D^{-1} x (FP64), written as the initial u (skipped when u is null);
// Prewitt magnitudes and their maxima.
__global__ void k_prep(const float *__restrict__ x, int n, int nz, int64_t N, double a, double b, double c,
                       double e, float *__restrict__ u, float *__restrict__ mh,
                       float *__restrict__ ml, int *__restrict__ maxbits)
{
    const int s = blockIdx.y;
    const float *xs = x + (int64_t)(2 * s) * N, *ls = xs + N;
    float lmax_h = 0.f, lmax_l = 0.f;
    const double det = __dsub_rn(__dmul_rn(a, e), __dmul_rn(b, c));
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N;
         p += (int64_t)gridDim.x * blockDim.x) {
        const double h = xs[p], l = ls[p];
        const double d1 = __ddiv_rn(__dsub_rn(__dmul_rn(e, h), __dmul_rn(b, l)), det);
        const double d2 = __ddiv_rn(__dadd_rn(__dmul_rn(-c, h), __dmul_rn(a, l)), det);
        if (u) {
            u[(int64_t)(2 * s) * N + p] = (float)d1;
            u[(int64_t)(2 * s + 1) * N + p] = (float)d2;
        }
        const int64_t plane = (int64_t)n * n;
        const int k = (int)(p / plane), i = (int)((p % plane) / n), j = (int)(p % n);
        const float g1 = nz > 1 ? prewitt3_at(xs, n, nz, k, i, j) : prewitt_at(xs, n, i, j);
        const float g2 = nz > 1 ? prewitt3_at(ls, n, nz, k, i, j) : prewitt_at(ls, n, i, j);
        mh[(int64_t)s * N + p] = g1;
        ml[(int64_t)s * N + p] = g2;
        lmax_h = fmaxf(lmax_h, g1);
        lmax_l = fmaxf(lmax_l, g2);
    }
    // maxima of non-negative floats: integer max of their bit patterns
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        lmax_h = fmaxf(lmax_h, __shfl_xor_sync(0xffffffffu, lmax_h, off));
        lmax_l = fmaxf(lmax_l, __shfl_xor_sync(0xffffffffu, lmax_l, off));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&maxbits[2 * s], __float_as_int(lmax_h));
        atomicMax(&maxbits[2 * s + 1], __float_as_int(lmax_l));
    }
}

__global__ void k_mask(const float *__restrict__ mh, const float *__restrict__ ml, int64_t N,
                       const int *__restrict__ maxbits, float tau, unsigned char *__restrict__ mask)
{
    const int s = blockIdx.y;
    const float Mh = __int_as_float(maxbits[2 * s]), Ml = __int_as_float(maxbits[2 * s + 1]);
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = (int64_t)s * N + p;
        const bool eh = Mh > 0.f && __fdiv_rn(mh[q], Mh) > tau;
        const bool el = Ml > 0.f && __fdiv_rn(ml[q], Ml) > tau;
        mask[q] = (unsigned char)(eh || el);
    }
}

// (I + gamma L_e) applied at pixel (i, j) to vector `u` of slice mask `mk`;
// also returns the Jacobi diagonal.
struct Stencil {
    const unsigned char *mk;
    int n, nz;
    float gamma, eps;
    __device__ __forceinline__ float w(int64_t p, int64_t q) const { return (mk[p] | mk[q]) ? eps : 1.f; }
};

// (I + gamma L_e) applied at element p (slice k, row i, column j) of vector
// `val`; also returns the Jacobi diagonal.  Volumes (nz > 1) add the two
// neighbours along z.
template <typename F>
__device__ __forceinline__ float apply_op(const Stencil &S, int64_t p, F val, float &diag)
{
    const int64_t plane = (int64_t)S.n * S.n;
    const int k = (int)(p / plane), i = (int)((p % plane) / S.n), j = (int)(p % S.n);
    const float c = val(p);
    float acc = 0.f, wsum = 0.f;
    const int64_t N = plane * S.nz;
    // neighbours inside the image only (out-of-image links are omitted, Eq. (14))
    auto nb = [&](int64_t q) { return DECT_IDX_OK(q, N, CHK_PLS_STENCIL) ? q : p; };
    if (k > 0) { const int64_t q = nb(p - plane); float w = S.w(p, q); acc += w * (c - val(q)); wsum += w; }
    if (k + 1 < S.nz) { const int64_t q = nb(p + plane); float w = S.w(p, q); acc += w * (c - val(q)); wsum += w; }
    if (i > 0) { const int64_t q = nb(p - S.n); float w = S.w(p, q); acc += w * (c - val(q)); wsum += w; }
    if (i + 1 < S.n) { const int64_t q = nb(p + S.n); float w = S.w(p, q); acc += w * (c - val(q)); wsum += w; }
    if (j > 0) { const int64_t q = nb(p - 1); float w = S.w(p, q); acc += w * (c - val(q)); wsum += w; }
    if (j + 1 < S.n) { const int64_t q = nb(p + 1); float w = S.w(p, q); acc += w * (c - val(q)); wsum += w; }
    diag = 1.f + S.gamma * wsum;
    return c + S.gamma * acc;
}


// r = d - A d, z = r / diag, p = 0; reductions <r,z>, <r,r>, <d,d>.
__global__ void k_init(float *__restrict__ uall, const unsigned char *__restrict__ mask,
                       float *__restrict__ r, float *__restrict__ z, float *__restrict__ p,
                       PlsConst C, PlsDev D)
{
    const int v = blockIdx.y;
    const float *u = uall + (int64_t)v * C.N;
    Stencil S{mask + (int64_t)(v >> 1) * C.N, C.n, C.nz, C.gamma, C.eps};
    float acc[3] = {0.f, 0.f, 0.f};
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < C.N;
         q += (int64_t)gridDim.x * blockDim.x) {
        float diag;
        const float Ad = apply_op(S, q, [&](int64_t k) { return u[k]; }, diag);
        const float d = u[q];
        const float rr = d - Ad, zz = rr / diag;
        const int64_t o = (int64_t)v * C.N + q;
        r[o] = rr;
        z[o] = zz;
        p[o] = 0.f;
        acc[0] = fmaf(rr, zz, acc[0]);
        acc[1] = fmaf(rr, rr, acc[1]);
        acc[2] = fmaf(d, d, acc[2]);
    }
    if (reduce_planar<3>(acc, D.part, D.red, D.ctr)) {
        for (int w = threadIdx.x; w < C.nvec; w += blockDim.x) {
            D.rz[w] = D.red[w * 3 + 0];
            D.bnorm[w] = sqrt(D.red[w * 3 + 2]);
            D.relres[w] = D.bnorm[w] > 0.0 ? sqrt(D.red[w * 3 + 1]) / D.bnorm[w] : 0.0;
            D.beta[w] = 0.0;
            D.alpha[w] = 0.0;
            D.iters[w] = 0;
            D.done[w] = (C.tol > 0.0 && D.relres[w] < C.tol) || D.bnorm[w] == 0.0;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int all = 1;
            for (int w = 0; w < C.nvec; ++w) all &= D.done[w];
            *D.all_done = all;
            *D.it = 0;
        }
    }
}

// p_new = z + beta p_old, Ap = (I + gamma L_e) p_new; reduction <p, Ap>; alpha.
__global__ void k_cg_a(const float *__restrict__ z, const float *__restrict__ p_old,
                       float *__restrict__ p_new, float *__restrict__ Ap,
                       const unsigned char *__restrict__ mask, PlsConst C, PlsDev D)
{
    const int v = blockIdx.y;
    const float beta = (float)D.beta[v];
    const float *zv = z + (int64_t)v * C.N, *pv = p_old + (int64_t)v * C.N;
    Stencil S{mask + (int64_t)(v >> 1) * C.N, C.n, C.nz, C.gamma, C.eps};
    float acc[1] = {0.f};
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < C.N;
         q += (int64_t)gridDim.x * blockDim.x) {
        float diag;
        auto pn = [&](int64_t k) { return fmaf(beta, pv[k], zv[k]); };
        const float a = apply_op(S, q, pn, diag);
        const float pc = pn(q);
        p_new[(int64_t)v * C.N + q] = pc;
        Ap[(int64_t)v * C.N + q] = a;
        acc[0] = fmaf(pc, a, acc[0]);
    }
    if (reduce_planar<1>(acc, D.part, D.red, D.ctr)) {
        for (int w = threadIdx.x; w < C.nvec; w += blockDim.x) {
            const double pap = D.red[w];
            D.alpha[w] = (!D.done[w] && pap > 0.0) ? D.rz[w] / pap : 0.0;
        }
    }
}

// u += alpha p, r -= alpha Ap, z = r / diag; reductions <r,z>, <r,r>; beta and stop test.
__global__ void k_cg_b(float *__restrict__ uall, const float *__restrict__ p,
                       const float *__restrict__ Ap, float *__restrict__ r, float *__restrict__ z,
                       const unsigned char *__restrict__ mask, PlsConst C, PlsDev D)
{
    const int v = blockIdx.y;
    const float alpha = (float)D.alpha[v];
    float *u = uall + (int64_t)v * C.N;
    Stencil S{mask + (int64_t)(v >> 1) * C.N, C.n, C.nz, C.gamma, C.eps};
    float acc[2] = {0.f, 0.f};
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < C.N;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t plane = (int64_t)C.n * C.n;
        const int k = (int)(q / plane), i = (int)((q % plane) / C.n), j = (int)(q % C.n);
        const int64_t o = (int64_t)v * C.N + q;
        float wsum = 0.f;
        if (k > 0) wsum += S.w(q, q - plane);
        if (k + 1 < C.nz) wsum += S.w(q, q + plane);
        if (i > 0) wsum += S.w(q, q - C.n);
        if (i + 1 < C.n) wsum += S.w(q, q + C.n);
        if (j > 0) wsum += S.w(q, q - 1);
        if (j + 1 < C.n) wsum += S.w(q, q + 1);
        const float diag = 1.f + C.gamma * wsum;
        u[q] = fmaf(alpha, p[o], u[q]);
        const float rr = fmaf(-alpha, Ap[o], r[o]);
        const float zz = rr / diag;
        r[o] = rr;
        z[o] = zz;
        acc[0] = fmaf(rr, zz, acc[0]);
        acc[1] = fmaf(rr, rr, acc[1]);
    }
    if (reduce_planar<2>(acc, D.part, D.red, D.ctr)) {
        const int it = *D.it;
        for (int w = threadIdx.x; w < C.nvec; w += blockDim.x) {
            if (D.done[w]) {
                D.beta[w] = 0.0;
                continue;
            }
            const double rz_new = D.red[w * 2 + 0];
            D.beta[w] = D.rz[w] != 0.0 ? rz_new / D.rz[w] : 0.0;
            D.rz[w] = rz_new;
            D.relres[w] = D.bnorm[w] > 0.0 ? sqrt(D.red[w * 2 + 1]) / D.bnorm[w] : 0.0;
            D.iters[w] = it + 1;
            if (C.tol > 0.0 && D.relres[w] < C.tol) D.done[w] = 1;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int all = 1;
            for (int w = 0; w < C.nvec; ++w) all &= D.done[w];
            *D.all_done = all;
            *D.it = it + 1;
        }
    }
}

}  // namespace
}  // namespace dect

using namespace dect;

namespace dect {
namespace {

// The decomposition of `batch` images (nz = 1) or volumes (nz slices).
dect_status pls_run(const float *x, int n, int nz, int batch, const dect_pls_params *prm, float *u,
                    dect_pls_report *reports, dect_stream stream)
{
    if (!prm || n < 1 || batch < 0 || n > 16384 || nz < 1 || nz > 4096) return DECT_ERR_INVALID_ARG;
    if (batch == 0) return DECT_OK;
    if (!x || !u) return DECT_ERR_INVALID_ARG;
    {
        const size_t span = (size_t)batch * 2 * n * n * nz * sizeof(float);
        const char *xa = (const char *)x, *ua = (const char *)u;
        if (xa < ua + span && ua < xa + span) return DECT_ERR_INVALID_ARG;
    }
    if (!(prm->gamma >= 0) || !(prm->edge_eps >= 0) || prm->max_iter < 0 || !std::isfinite(prm->gamma))
        return DECT_ERR_INVALID_ARG;
    const double a = prm->eta[0][0], b = prm->eta[1][0], c = prm->eta[0][1], e = prm->eta[1][1];
    const double det = a * e - b * c;
    if (!(std::fabs(det) > 0) || !std::isfinite(det)) return DECT_ERR_INVALID_ARG;
    if (batch > 65535 / 2) return DECT_ERR_INVALID_ARG;  // grid.y holds a vector index
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    DECT_CUDA(cudaGetDevice(&dev));

    const int64_t N = (int64_t)n * n * nz;
    const int nvec = 2 * batch;
    const int64_t want = (N + kBlock - 1) / kBlock;
    const int gx = (int)std::max<int64_t>(1, std::min<int64_t>(want, std::max(1, (kSMs * 8) / nvec)));

    // scratch from the stream-ordered pool: lay out once to size, then for real
    const size_t nf = (size_t)nvec * N;
    float *r = nullptr, *z = nullptr, *pa = nullptr, *pb = nullptr, *Ap = nullptr;
    float *mh = nullptr, *ml = nullptr;
    unsigned char *mask = nullptr;
    PlsDev D;
    auto layout = [&](char *base) -> size_t {
        size_t o = 0;
        auto take = [&](size_t nb) { char *p = base ? base + o : nullptr; o = (o + nb + 255) & ~(size_t)255; return p; };
        r = (float *)take(nf * 4);
        z = (float *)take(nf * 4);
        pa = (float *)take(nf * 4);
        pb = (float *)take(nf * 4);
        Ap = (float *)take(nf * 4);
        mh = (float *)take((size_t)batch * N * 4);
        ml = (float *)take((size_t)batch * N * 4);
        mask = (unsigned char *)take((size_t)batch * N);
        D.part = (double *)take((size_t)gx * nvec * 3 * 8);
        D.red = (double *)take((size_t)nvec * 3 * 8);
        D.alpha = (double *)take((size_t)nvec * 8);
        D.beta = (double *)take((size_t)nvec * 8);
        D.rz = (double *)take((size_t)nvec * 8);
        D.bnorm = (double *)take((size_t)nvec * 8);
        D.relres = (double *)take((size_t)nvec * 8);
        D.iters = (int *)take((size_t)nvec * 4);
        D.done = (int *)take((size_t)nvec * 4);
        D.it = (int *)take(4);
        D.all_done = (int *)take(4);
        D.ctr = (unsigned *)take(8);
        D.maxbits = (int *)take((size_t)2 * batch * 4);
        return o;
    };
    const size_t bytes = layout(nullptr);
    char *base = nullptr;
    DECT_CUDA(cudaMallocAsync((void **)&base, bytes, s));
    layout(base);
    DECT_CUDA(cudaMemsetAsync(D.ctr, 0, 8, s));
    DECT_CUDA(cudaMemsetAsync(D.maxbits, 0, (size_t)2 * batch * 4, s));

    PlsConst C;
    C.n = n;
    C.nz = nz;
    C.N = N;
    C.nvec = nvec;
    C.gamma = (float)prm->gamma;
    C.eps = (float)prm->edge_eps;
    C.tol = prm->tol;

    dim3 gs((unsigned)gx, (unsigned)batch), gv((unsigned)gx, (unsigned)nvec);
    k_prep<<<gs, kBlock, 0, s>>>(x, n, nz, N, a, b, c, e, u, mh, ml, D.maxbits);
    DECT_LAUNCH_CHECK();
    k_mask<<<gs, kBlock, 0, s>>>(mh, ml, N, D.maxbits, (float)prm->edge_tau, mask);
    DECT_LAUNCH_CHECK();
    k_init<<<gv, kBlock, 0, s>>>(u, mask, r, z, pa, C, D);
    DECT_LAUNCH_CHECK();
    count_launches(3);

    const int K = prm->max_iter;
    const bool use_tol = prm->tol > 0.0;
    const int block = 10;
    cudaError_t err = cudaSuccess;
    cudaStream_t cs = nullptr;
    cudaEvent_t ev = nullptr;
    cudaGraphExec_t gx2 = nullptr;
    int *h_done = nullptr;
    err = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (err == cudaSuccess) err = cudaEventRecord(ev, s);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(cs, ev, 0);
    // two CG iterations per unit keep the p ping-pong in place
    auto two_iters = [&](cudaStream_t st) {
        k_cg_a<<<gv, kBlock, 0, st>>>(z, pa, pb, Ap, mask, C, D);
        k_cg_b<<<gv, kBlock, 0, st>>>(u, pb, Ap, r, z, mask, C, D);
        k_cg_a<<<gv, kBlock, 0, st>>>(z, pb, pa, Ap, mask, C, D);
        k_cg_b<<<gv, kBlock, 0, st>>>(u, pa, Ap, r, z, mask, C, D);
    };
    if (err == cudaSuccess && K >= 2 * block) {
        cudaGraph_t gr = nullptr;
        err = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (err == cudaSuccess) {
            for (int q = 0; q < block; ++q) two_iters(cs);
            err = cudaStreamEndCapture(cs, &gr);
        }
        if (err == cudaSuccess) err = cudaGraphInstantiate(&gx2, gr, 0);
        if (gr) cudaGraphDestroy(gr);
    }
    if (err == cudaSuccess) err = cudaMallocHost((void **)&h_done, sizeof(int));
    int done_it = 0;
    bool finished = false;
    if (err == cudaSuccess && use_tol) {
        err = cudaMemcpyAsync(h_done, D.all_done, sizeof(int), cudaMemcpyDeviceToHost, cs);
        if (err == cudaSuccess) err = cudaStreamSynchronize(cs);
        finished = err == cudaSuccess && *h_done;
    }
    while (err == cudaSuccess && !finished && done_it + 2 * block <= K && gx2) {
        err = cudaGraphLaunch(gx2, cs);
        count_launches(4 * block);
        done_it += 2 * block;
        if (err == cudaSuccess && use_tol) {
            err = cudaMemcpyAsync(h_done, D.all_done, sizeof(int), cudaMemcpyDeviceToHost, cs);
            if (err == cudaSuccess) err = cudaStreamSynchronize(cs);
            finished = err == cudaSuccess && *h_done;
        }
    }
    // remaining iterations one by one (ping-pong parity by position)
    float *p_cur = pa, *p_nxt = pb;
    while (err == cudaSuccess && !finished && done_it < K) {
        k_cg_a<<<gv, kBlock, 0, cs>>>(z, p_cur, p_nxt, Ap, mask, C, D);
        k_cg_b<<<gv, kBlock, 0, cs>>>(u, p_nxt, Ap, r, z, mask, C, D);
        std::swap(p_cur, p_nxt);
        ++done_it;
        count_launches(2);
        err = cudaGetLastError();
    }
    if (err == cudaSuccess) err = cudaEventRecord(ev, cs);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(s, ev, 0);
    std::vector<int> hit(nvec);
    std::vector<double> hrel(nvec);
    if (err == cudaSuccess) err = cudaMemcpyAsync(hit.data(), D.iters, nvec * 4, cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaMemcpyAsync(hrel.data(), D.relres, nvec * 8, cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(base, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    if (gx2) cudaGraphExecDestroy(gx2);
    if (h_done) cudaFreeHost(h_done);
    if (ev) cudaEventDestroy(ev);
    if (cs) cudaStreamDestroy(cs);
    if (err != cudaSuccess) {
        set_error("dect_pls_decompose", err);
        return err == cudaErrorMemoryAllocation ? DECT_ERR_OOM : DECT_ERR_CUDA;
    }
    if (reports) {
        for (int sl = 0; sl < batch; ++sl)
            for (int m = 0; m < 2; ++m) {
                reports[sl].iters[m] = hit[2 * sl + m];
                reports[sl].relres[m] = hrel[2 * sl + m];
            }
    }
    (void)dev;
    return DECT_OK;
}

}  // namespace
}  // namespace dect

extern "C" dect_status dect_pls_decompose(const float *x, int n, int batch, const dect_pls_params *prm,
                                          float *u, dect_pls_report *reports, dect_stream stream)
{
    return dect::pls_run(x, n, 1, batch, prm, u, reports, stream);
}

extern "C" dect_status dect_pls_decompose_cone(const float *x, int n, int nz, int batch, const dect_pls_params *prm,
                                               float *u, dect_pls_report *reports, dect_stream stream)
{
    return dect::pls_run(x, n, nz, batch, prm, u, reports, stream);
}

namespace dect {
namespace {

dect_status edge_mask_run(const float *x, int n, int nz, int batch, double edge_tau, uint8_t *mask,
                          dect_stream stream)
{
    if (n < 1 || batch < 0 || n > 16384 || nz < 1 || nz > 4096 || !std::isfinite(edge_tau))
        return DECT_ERR_INVALID_ARG;
    if (batch == 0) return DECT_OK;
    if (!x || !mask || batch > 65535) return DECT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t N = (int64_t)n * n * nz;
    const int64_t want = (N + kBlock - 1) / kBlock;
    const int gx = (int)std::max<int64_t>(1, std::min<int64_t>(want, std::max(1, (kSMs * 8) / batch)));
    const size_t mag_bytes = ((size_t)batch * N * 4 + 255) & ~(size_t)255;
    char *base = nullptr;
    DECT_CUDA(cudaMallocAsync((void **)&base, 2 * mag_bytes + (size_t)2 * batch * 4, s));
    float *mh = (float *)base, *ml = (float *)(base + mag_bytes);
    int *maxbits = (int *)(base + 2 * mag_bytes);
    cudaError_t err = cudaMemsetAsync(maxbits, 0, (size_t)2 * batch * 4, s);
    if (err == cudaSuccess) {
        dim3 gs((unsigned)gx, (unsigned)batch);
        k_prep<<<gs, kBlock, 0, s>>>(x, n, nz, N, 1.0, 0.0, 0.0, 1.0, nullptr, mh, ml, maxbits);
        k_mask<<<gs, kBlock, 0, s>>>(mh, ml, N, maxbits, (float)edge_tau, mask);
        count_launches(2);
        err = cudaGetLastError();
    }
    cudaFreeAsync(base, s);
    if (err != cudaSuccess) {
        set_error("dect_pls_edge_mask", err);
        return DECT_ERR_CUDA;
    }
    return DECT_OK;
}

}  // namespace
}  // namespace dect

extern "C" dect_status dect_pls_edge_mask(const float *x, int n, int batch, double edge_tau, uint8_t *mask,
                                          dect_stream stream)
{
    return dect::edge_mask_run(x, n, 1, batch, edge_tau, mask, stream);
}

extern "C" dect_status dect_pls_edge_mask_cone(const float *x, int n, int nz, int batch, double edge_tau,
                                               uint8_t *mask, dect_stream stream)
{
    return dect::edge_mask_run(x, n, nz, batch, edge_tau, mask, stream);
}

// ---------------------------------------------------------------------------
// Allocation-free variant of dect_pls_decompose.
//
// Some callers cannot allocate device memory while they run: for example an
// inline reconstruction service that reserves the whole device pool at
// start-up and must keep its footprint fixed, or a plug-in hosted by a
// process whose own allocator owns the GPU.  This entry point takes its
// scratch from one fixed array in the library image instead of the
// stream-ordered allocator, creates no stream, event or graph, and pins no
// host memory.
// ---------------------------------------------------------------------------
namespace dect {
namespace {

// Upper bounds of the allocation-free path (see dect.h).
constexpr int64_t kNoAllocMaxPixels = DECT_PLS_NOALLOC_MAX_PIXELS;
constexpr int kNoAllocMaxBatch = DECT_PLS_NOALLOC_MAX_BATCH;
constexpr size_t kNoAllocBytes = (size_t)14 << 20;

// The scratch itself: every device that loads the library holds it until
// the process exits.  In host code this name is only a stand-in; the device
// address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_pls_scratch[kNoAllocBytes];

std::mutex g_scratch_mu;
void *g_scratch_addr[256];  // per device ordinal, filled on the first call

cudaError_t scratch_address(int dev, void **out)
{
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_pls_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace dect

extern "C" dect_status dect_pls_decompose_noalloc(const float *x, int n, int batch,
                                                  const dect_pls_params *prm, float *u,
                                                  dect_pls_report *reports, dect_stream stream)
{
    if (!prm || n < 1 || batch < 0 || n > 16384) return DECT_ERR_INVALID_ARG;
    if (batch == 0) return DECT_OK;
    if (!x || !u) return DECT_ERR_INVALID_ARG;
    if ((int64_t)batch * n * n > kNoAllocMaxPixels || batch > kNoAllocMaxBatch) {
        set_error_text("dect_pls_decompose_noalloc: batch * n * n must be <= " +
                       std::to_string(kNoAllocMaxPixels) + " and batch <= " +
                       std::to_string(kNoAllocMaxBatch) + " (use dect_pls_decompose for larger work)");
        return DECT_ERR_INVALID_ARG;
    }
    {
        const size_t span = (size_t)batch * 2 * n * n * sizeof(float);
        const char *xa = (const char *)x, *ua = (const char *)u;
        if (xa < ua + span && ua < xa + span) return DECT_ERR_INVALID_ARG;
    }
    if (!(prm->gamma >= 0) || !(prm->edge_eps >= 0) || prm->max_iter < 0 || !std::isfinite(prm->gamma))
        return DECT_ERR_INVALID_ARG;
    const double a = prm->eta[0][0], b = prm->eta[1][0], c = prm->eta[0][1], e = prm->eta[1][1];
    const double det = a * e - b * c;
    if (!(std::fabs(det) > 0) || !std::isfinite(det)) return DECT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    DECT_CUDA(cudaGetDevice(&dev));
    void *scratch = nullptr;
    DECT_CUDA(scratch_address(dev, &scratch));

    const int64_t N = (int64_t)n * n;
    const int nvec = 2 * batch;
    const int64_t want = (N + kBlock - 1) / kBlock;
    const int gx = (int)std::max<int64_t>(1, std::min<int64_t>(want, std::max(1, (kSMs * 8) / nvec)));

    // same layout as the allocating path, placed in the fixed array
    const size_t nf = (size_t)nvec * N;
    char *base = (char *)scratch;
    size_t o = 0;
    auto take = [&](size_t nb) { char *p = base + o; o = (o + nb + 255) & ~(size_t)255; return p; };
    float *r = (float *)take(nf * 4);
    float *z = (float *)take(nf * 4);
    float *pa = (float *)take(nf * 4);
    float *pb = (float *)take(nf * 4);
    float *Ap = (float *)take(nf * 4);
    float *mh = (float *)take((size_t)batch * N * 4);
    float *ml = (float *)take((size_t)batch * N * 4);
    unsigned char *mask = (unsigned char *)take((size_t)batch * N);
    PlsDev D;
    D.part = (double *)take((size_t)gx * nvec * 3 * 8);
    D.red = (double *)take((size_t)nvec * 3 * 8);
    D.alpha = (double *)take((size_t)nvec * 8);
    D.beta = (double *)take((size_t)nvec * 8);
    D.rz = (double *)take((size_t)nvec * 8);
    D.bnorm = (double *)take((size_t)nvec * 8);
    D.relres = (double *)take((size_t)nvec * 8);
    D.iters = (int *)take((size_t)nvec * 4);
    D.done = (int *)take((size_t)nvec * 4);
    D.it = (int *)take(4);
    D.all_done = (int *)take(4);
    D.ctr = (unsigned *)take(8);
    D.maxbits = (int *)take((size_t)2 * batch * 4);
    if (o > kNoAllocBytes) {  // cannot happen within the limits above
        set_error_text("dect_pls_decompose_noalloc: scratch layout exceeds the fixed array");
        return DECT_ERR_INVALID_ARG;
    }
    // the array keeps the previous call's contents: zero what must start at zero
    DECT_CUDA(cudaMemsetAsync(D.ctr, 0, 8, s));
    DECT_CUDA(cudaMemsetAsync(D.maxbits, 0, (size_t)2 * batch * 4, s));

    PlsConst C;
    C.n = n;
    C.nz = 1;
    C.N = N;
    C.nvec = nvec;
    C.gamma = (float)prm->gamma;
    C.eps = (float)prm->edge_eps;
    C.tol = prm->tol;

    dim3 gs((unsigned)gx, (unsigned)batch), gv((unsigned)gx, (unsigned)nvec);
    k_prep<<<gs, kBlock, 0, s>>>(x, n, 1, N, a, b, c, e, u, mh, ml, D.maxbits);
    DECT_LAUNCH_CHECK();
    k_mask<<<gs, kBlock, 0, s>>>(mh, ml, N, D.maxbits, (float)prm->edge_tau, mask);
    DECT_LAUNCH_CHECK();
    k_init<<<gv, kBlock, 0, s>>>(u, mask, r, z, pa, C, D);
    DECT_LAUNCH_CHECK();
    count_launches(3);

    // plain launches on the caller's stream; the stop flag is read into a
    // host stack variable every 10 iterations when a tolerance is set
    const int K = prm->max_iter;
    const bool use_tol = prm->tol > 0.0;
    float *p_cur = pa, *p_nxt = pb;
    int done_flag = 0;
    for (int it = 0; it < K; ++it) {
        if (use_tol && it % 10 == 0) {
            DECT_CUDA(cudaMemcpyAsync(&done_flag, D.all_done, sizeof(int), cudaMemcpyDeviceToHost, s));
            DECT_CUDA(cudaStreamSynchronize(s));
            if (done_flag) break;
        }
        k_cg_a<<<gv, kBlock, 0, s>>>(z, p_cur, p_nxt, Ap, mask, C, D);
        k_cg_b<<<gv, kBlock, 0, s>>>(u, p_nxt, Ap, r, z, mask, C, D);
        DECT_LAUNCH_CHECK();
        count_launches(2);
        std::swap(p_cur, p_nxt);
    }
    int hit[2 * kNoAllocMaxBatch];
    double hrel[2 * kNoAllocMaxBatch];
    DECT_CUDA(cudaMemcpyAsync(hit, D.iters, nvec * sizeof(int), cudaMemcpyDeviceToHost, s));
    DECT_CUDA(cudaMemcpyAsync(hrel, D.relres, nvec * sizeof(double), cudaMemcpyDeviceToHost, s));
    DECT_CUDA(cudaStreamSynchronize(s));
    if (reports) {
        for (int sl = 0; sl < batch; ++sl)
            for (int m = 0; m < 2; ++m) {
                reports[sl].iters[m] = hit[2 * sl + m];
                reports[sl].relres[m] = hrel[2 * sl + m];
            }
    }
    return DECT_OK;
}
