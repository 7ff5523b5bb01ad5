// Device building blocks shared by the operator and ADM translation units:
// the row kernels that stream a table of A (ray-major for A x, pixel-major
// for A^T y), and the deterministic per-image FP64 reduction.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dect_internal.cuh"

namespace dect {

// ---------------------------------------------------------------------------
// Image batches.  NB images are processed together.  In the interleaved
// layout ("IL") pixel j of image b sits at base[j * NB + b]; in the planar
// layout at base[b * stride + j].  A thread moves VW consecutive images.
// ---------------------------------------------------------------------------
template <int NB>
struct Batch {
    static constexpr int VW = NB >= 4 ? 4 : NB;  // floats per vector
    static constexpr int CPB = NB / VW;          // vectors per pixel
};

template <int VW>
struct Vec {
    float v[VW];
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int c = 0; c < VW; ++c) v[c] = 0.f;
    }
};

template <int VW>
__device__ __forceinline__ Vec<VW> ld_il(const float *__restrict__ p)
{
    Vec<VW> r;
    if constexpr (VW == 4) {
        float4 t = __ldg(reinterpret_cast<const float4 *>(p));
        r.v[0] = t.x; r.v[1] = t.y; r.v[2] = t.z; r.v[3] = t.w;
    } else if constexpr (VW == 2) {
        float2 t = __ldg(reinterpret_cast<const float2 *>(p));
        r.v[0] = t.x; r.v[1] = t.y;
    } else {
        r.v[0] = __ldg(p);
    }
    return r;
}

// Gather of read-only data that other rows of the same launch will gather
// again: kept in L1 and in L2 with evict-last priority, so that the streamed
// table entries (evict-first) are the lines that make room.
__device__ __forceinline__ unsigned long long l2_evict_last_policy()
{
    unsigned long long pol;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

template <int VW>
__device__ __forceinline__ Vec<VW> ld_gather(const float *__restrict__ p, unsigned long long pol)
{
    Vec<VW> r;
    if constexpr (VW == 4) {
        asm("ld.global.nc.L1::evict_last.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
            : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3])
            : "l"(p), "l"(pol));
    } else if constexpr (VW == 2) {
        asm("ld.global.nc.L1::evict_last.L2::cache_hint.v2.f32 {%0,%1}, [%2], %3;"
            : "=f"(r.v[0]), "=f"(r.v[1])
            : "l"(p), "l"(pol));
    } else {
        asm("ld.global.nc.L1::evict_last.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(r.v[0]) : "l"(p), "l"(pol));
    }
    return r;
}

// plain (coherent) load, for data written earlier in the same kernel sequence
template <int VW>
__device__ __forceinline__ Vec<VW> ld_v(const float *p)
{
    Vec<VW> r;
    if constexpr (VW == 4) {
        float4 t = *reinterpret_cast<const float4 *>(p);
        r.v[0] = t.x; r.v[1] = t.y; r.v[2] = t.z; r.v[3] = t.w;
    } else if constexpr (VW == 2) {
        float2 t = *reinterpret_cast<const float2 *>(p);
        r.v[0] = t.x; r.v[1] = t.y;
    } else {
        r.v[0] = *p;
    }
    return r;
}

template <int VW>
__device__ __forceinline__ void st_v(float *p, const Vec<VW> &a)
{
    if constexpr (VW == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(a.v[0], a.v[1], a.v[2], a.v[3]);
    } else if constexpr (VW == 2) {
        *reinterpret_cast<float2 *>(p) = make_float2(a.v[0], a.v[1]);
    } else {
        *p = a.v[0];
    }
}

// Store of data that the next kernels read again (G: gathered by A G, read
// by the TV step): written to L2 with evict-last priority, so that it stays
// there while the table streams (evict-first) pass through.
template <int VW>
__device__ __forceinline__ void st_keep(float *p, const Vec<VW> &a, unsigned long long pol)
{
    if constexpr (VW == 4) {
        asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1,%2,%3,%4}, %5;" ::"l"(p), "f"(a.v[0]), "f"(a.v[1]),
                     "f"(a.v[2]), "f"(a.v[3]), "l"(pol)
                     : "memory");
    } else if constexpr (VW == 2) {
        asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1,%2}, %3;" ::"l"(p), "f"(a.v[0]), "f"(a.v[1]), "l"(pol)
                     : "memory");
    } else {
        asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(a.v[0]), "l"(pol) : "memory");
    }
}

__device__ __forceinline__ Entry ld_entry(const Entry *p)
{
    // table entries are read once per pass: stream them past L1
    return __ldcs(p);
}

// ---------------------------------------------------------------------------
// Deterministic per-image reduction of K quantities at once: every thread
// holds K vectors of VW partial values for images (lane % CPB) * VW + c.
// Values are summed in FP32 inside a warp and in FP64 across warps and
// blocks, always in the same order: the warps of a block add into RED_SLOTS
// shared slots in rounds of RED_SLOTS warps, then the slots are added.  The
// block that finishes last writes the grid totals to out[k][img] and
// returns true (in every thread of that block); `counter` is reset for the
// next launch.  Blocks have BLOCK threads; smem must hold
// reduce_smem_doubles<NB, BLOCK>(K) doubles (kept small: the table kernels
// need the L1 that shared memory would take); part holds K * gridDim.x * NB
// doubles.
// ---------------------------------------------------------------------------
template <int BLOCK>
__host__ __device__ constexpr int red_slots()
{
    return (BLOCK / 32) % 8 == 0 ? 8 : BLOCK / 32;
}

template <int NB, int BLOCK>
__host__ __device__ constexpr int red_split()
{
    return BLOCK / NB < 8 ? BLOCK / NB : 8;
}

template <int NB, int BLOCK = 256>
__host__ __device__ constexpr int reduce_smem_doubles(int K)
{
    return K * (red_slots<BLOCK>() > red_split<NB, BLOCK>() ? red_slots<BLOCK>() : red_split<NB, BLOCK>()) * NB;
}

template <int NB, int K, int BLOCK = 256>
__device__ __forceinline__ bool reduce_images(Vec<Batch<NB>::VW> (&v)[K], double *__restrict__ part,
                                              double *__restrict__ out, unsigned *counter,
                                              double *smem)
{
    constexpr int VW = Batch<NB>::VW, CPB = Batch<NB>::CPB;
    constexpr int NW = BLOCK / 32, SL = red_slots<BLOCK>(), SPLIT = red_split<NB, BLOCK>();
    static_assert(NW % SL == 0 && BLOCK % NB == 0, "reduce_images: block shape");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t pstride = (size_t)gridDim.x * NB;
#pragma unroll
    for (int q = 0; q < K; ++q)
#pragma unroll
        for (int off = CPB; off < 32; off <<= 1)
#pragma unroll
            for (int c = 0; c < VW; ++c) v[q].v[c] += __shfl_xor_sync(0xffffffffu, v[q].v[c], off);
#pragma unroll 1
    for (int rnd = 0; rnd < NW / SL; ++rnd) {
        if (warp / SL == rnd && lane < CPB)
#pragma unroll
            for (int q = 0; q < K; ++q)
#pragma unroll
                for (int c = 0; c < VW; ++c) {
                    double &d = smem[(q * SL + warp % SL) * NB + lane * VW + c];
                    d = (rnd == 0 ? 0.0 : d) + (double)v[q].v[c];
                }
        __syncthreads();
    }
    if (threadIdx.x < K * NB) {
        const int q = threadIdx.x / NB, img = threadIdx.x % NB;
        double s = 0.0;
        for (int w = 0; w < SL; ++w) s += smem[(q * SL + w) * NB + img];
        part[q * pstride + (size_t)blockIdx.x * NB + img] = s;
    }
    __threadfence();
    __syncthreads();
    __shared__ bool last;
    if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!last) return false;
    __threadfence();
    // grid total: SPLIT threads per image each sum a fixed stride of the block
    // partials, then one thread per image adds the SPLIT sub-sums in order
    const int img = threadIdx.x % NB, sub = threadIdx.x / NB;
    double sv[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
        sv[q] = 0.0;
        if (sub < SPLIT) {
#pragma unroll 4
            for (unsigned b = sub; b < gridDim.x; b += SPLIT) sv[q] += __ldcg(&part[q * pstride + (size_t)b * NB + img]);
        }
    }
    __syncthreads();  // smem is reused below
    if (sub < SPLIT)
#pragma unroll
        for (int q = 0; q < K; ++q) smem[(q * SPLIT + sub) * NB + img] = sv[q];
    __syncthreads();
    if (threadIdx.x < K * NB) {
        const int q = threadIdx.x / NB, im = threadIdx.x % NB;
        double t = 0.0;
        for (int u = 0; u < SPLIT; ++u) t += smem[(q * SPLIT + u) * NB + im];
        out[q * NB + im] = t;
    }
    if (threadIdx.x == 0) *counter = 0u;
    __syncthreads();
    return true;
}

// ---------------------------------------------------------------------------
// Row kernel core: one row (a ray of the ray-major table or a pixel of the
// pixel-major table) is handled by G lanes.  The G lanes load the row's
// entries cooperatively, G at a time (coalesced, streamed past L1), one batch
// ahead of use, so a table entry's DRAM latency overlaps the gathers of the
// previous batch.  Inside a batch, entry j is broadcast (by shuffle, or with
// SBC through a per-warp shared-memory slot, 8 KB per block, when a lane
// holds one entry per batch) to the LPE = CPB lanes that gather its VW-wide
// vectors of the NB images; the
// batch's EG = G / LPE entry groups give every lane LPE independent gathers.
// Groups are summed by a fixed xor-butterfly: the result is bitwise
// reproducible.  After the call, the lanes with group == 0 hold the row's sums.
// Every lane of the warp must call it (rows past the end pass b = e).
// ---------------------------------------------------------------------------
template <int NB, int G, typename Gather, bool SBC = false>
__device__ __forceinline__ Vec<Batch<NB>::VW> row_dot_g(const Entry *__restrict__ ent, int64_t b,
                                                        int64_t e, int lr, Gather gather)
{
    constexpr int VW = Batch<NB>::VW, LPE = Batch<NB>::CPB, EG = G / LPE;
    constexpr int U = LPE >= 4 ? 1 : 4 / LPE;  // batches in flight per step
    static_assert(G % LPE == 0 && G <= 32, "bad row split");
    const int grp = lr / LPE, vl = lr % LPE;
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned gbase = lane & ~(unsigned)(G - 1);  // first lane of this row group
    Vec<VW> acc;
    acc.zero();
    Entry cur[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int64_t k = b + u * G + lr;
        cur[u] = k < e ? ld_entry(ent + k) : make_int2(0, 0);
    }
    // the loop runs in lockstep over the warp (its shuffles need every lane):
    // rows shorter than the warp's longest see padded entries
    const unsigned maxlen = __reduce_max_sync(0xffffffffu, (unsigned)(e - b));
    for (int64_t base = b; base < b + (int64_t)maxlen; base += U * G) {
        Entry nxt[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t k = base + (U + u) * G + lr;
            nxt[u] = k < e ? ld_entry(ent + k) : make_int2(0, 0);
        }
        if constexpr (SBC && U == 1) {
            // one batch per warp: broadcast through shared memory, one 8-byte
            // load per round instead of two shuffles
            __shared__ Entry s_ent[32][32];  // per-warp entry batch
            __syncwarp();
            s_ent[warp][lane] = cur[0];
            __syncwarp();
#pragma unroll
            for (int j = 0; j < G / EG; ++j) {
                const Entry en = s_ent[warp][gbase + j * EG + grp];
                // padded entries carry w = 0 and index 0: a valid address, no contribution
                const Vec<VW> xv = gather(en.x, vl);
                const float w = __int_as_float(en.y);
#pragma unroll
                for (int c = 0; c < VW; ++c) acc.v[c] = fmaf(w, xv.v[c], acc.v[c]);
            }
        } else {
            // rounds in groups of R: R entries broadcast, then R independent
            // gathers in flight, then their multiply-adds
            constexpr int NR = G / EG, R = NR < 8 ? NR : 8;
            static_assert(NR <= 8 || NR % 8 == 0, "rounds must split into groups of 8");
#pragma unroll
            for (int u = 0; u < U; ++u) {
#pragma unroll
                for (int j0 = 0; j0 < NR; j0 += R) {
                    int pix[R];
                    float w[R];
                    Vec<VW> xv[R];
#pragma unroll
                    for (int j = 0; j < R; ++j) {
                        const unsigned srcl = gbase + (j0 + j) * EG + grp;
                        pix[j] = __shfl_sync(0xffffffffu, cur[u].x, srcl);
                        w[j] = __int_as_float(__shfl_sync(0xffffffffu, cur[u].y, srcl));
                    }
#pragma unroll
                    for (int j = 0; j < R; ++j) xv[j] = gather(pix[j], vl);
#pragma unroll
                    for (int j = 0; j < R; ++j)
#pragma unroll
                        for (int c = 0; c < VW; ++c) acc.v[c] = fmaf(w[j], xv[j].v[c], acc.v[c]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) cur[u] = nxt[u];
    }
#pragma unroll
    for (int off = LPE; off < G; off <<= 1)
#pragma unroll
        for (int c = 0; c < VW; ++c) acc.v[c] += __shfl_xor_sync(0xffffffffu, acc.v[c], off);
    return acc;
}

// ---------------------------------------------------------------------------
// Row kernel core, wide-lane form: a lane gathers VWL = 8 or 16 images of an
// entry (VWL / 4 loads of 16 bytes) instead of 4; NB = 16, 32 or 64.  The
// time of the table kernels goes into returning loaded data to registers:
// every entry returns its NB x 4 bytes of image data plus its 8-byte
// (index, length) to each lane that gathers a part of it, and LPW = NB / VWL
// lanes share an entry here instead of NB / 4.  Load i of lane vl covers
// images 4 (i LPW + vl) .. + 3, so the LPW lanes of an entry read 16 LPW
// contiguous bytes per load (with VWL = 8 at 64 images: one whole 128-byte
// line of the entry per load, as many lines per warp-wide load as the
// 4-image form).  Entries are loaded as in row_dot_g (G at a time,
// coalesced, one batch ahead) and broadcast by shuffles; EG = G / LPW entry
// groups take the batch's entries in rounds, R rounds' gathers in flight.
// Groups are summed by a fixed xor-butterfly.  The result is returned in the
// layout of row_dot_g: lane lr holds images 4 (lr % CPB) .. + 3 (every group
// holds the full sums, and lane lr's own wide vector covers those images at
// block (lr % CPB) / LPW).  Every lane of the warp must call it.
// ---------------------------------------------------------------------------
template <int NB, int G, int VWL, int R>
__device__ __forceinline__ Vec<4> row_dot_w(const Entry *__restrict__ ent, int64_t b, int64_t e, int lr,
                                            const float *__restrict__ src, unsigned long long pol,
                                            int64_t rows, unsigned site)
{
    static_assert((NB == 16 || NB == 32 || NB == 64) && (VWL == 8 || VWL == 16) && VWL <= NB,
                  "wide row core: 16, 32 or 64 images, 8 or 16 per lane");
    constexpr int NV = VWL / 4, LPW = NB / VWL, EG = G / LPW, NR = G / EG, CPB = NB / 4;
    constexpr int RR = NR < R ? NR : R;
    static_assert(G % LPW == 0 && G <= 32 && NR % RR == 0, "bad row split");
    const int grp = lr / LPW, vl = lr % LPW;
    const unsigned lane = threadIdx.x & 31;
    const unsigned gbase = lane & ~(unsigned)(G - 1);
    float acc[VWL];
#pragma unroll
    for (int k = 0; k < VWL; ++k) acc[k] = 0.f;
    Entry cur = b + lr < e ? ld_entry(ent + b + lr) : make_int2(0, 0);
    const unsigned maxlen = __reduce_max_sync(0xffffffffu, (unsigned)(e - b));
    for (int64_t base = b; base < b + (int64_t)maxlen; base += G) {
        const int64_t kn = base + G + lr;
        const Entry nxt = kn < e ? ld_entry(ent + kn) : make_int2(0, 0);
#pragma unroll
        for (int j0 = 0; j0 < NR; j0 += RR) {
            int pix[RR];
            float w[RR];
#pragma unroll
            for (int j = 0; j < RR; ++j) {
                const unsigned srcl = gbase + (j0 + j) * EG + grp;
                pix[j] = __shfl_sync(0xffffffffu, cur.x, srcl);
                w[j] = __int_as_float(__shfl_sync(0xffffffffu, cur.y, srcl));
                if (!DECT_IDX_OK(pix[j], rows, site)) pix[j] = 0;
            }
            Vec<4> xv[RR][NV];
#pragma unroll
            for (int j = 0; j < RR; ++j)
#pragma unroll
                for (int i = 0; i < NV; ++i)
                    xv[j][i] = ld_gather<4>(src + (int64_t)pix[j] * NB + 4 * (i * LPW + vl), pol);
#pragma unroll
            for (int j = 0; j < RR; ++j)
#pragma unroll
                for (int i = 0; i < NV; ++i)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[4 * i + c] = fmaf(w[j], xv[j][i].v[c], acc[4 * i + c]);
        }
        cur = nxt;
    }
#pragma unroll
    for (int off = LPW; off < G; off <<= 1)
#pragma unroll
        for (int k = 0; k < VWL; ++k) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], off);
    const int q = (lr % CPB) / LPW;
    Vec<4> out;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        float v = acc[c];
#pragma unroll
        for (int i = 1; i < NV; ++i) v = q == i ? acc[4 * i + c] : v;
        out.v[c] = v;
    }
    return out;
}

// Gathers of one VW-wide vector of the NB images at index `pix`.
template <int NB>
struct GatherIL {  // interleaved [index][NB] in global memory, `rows` indices
    const float *src;
    int64_t rows;
    unsigned site;
    unsigned long long pol = l2_evict_last_policy();
    __device__ __forceinline__ Vec<Batch<NB>::VW> operator()(int pix, int vl) const
    {
        if (!DECT_IDX_OK(pix, rows, site)) pix = 0;
        return ld_gather<Batch<NB>::VW>(src + (int64_t)pix * NB + vl * Batch<NB>::VW, pol);
    }
};
// src holds `rows` interleaved rows; site: the check site of its gathers.
template <int NB, int G, bool IL, bool SBC = false>
__device__ __forceinline__ Vec<Batch<NB>::VW> row_dot(const Entry *__restrict__ ent, int64_t b, int64_t e,
                                                      const float *__restrict__ src, int64_t rows, int lr,
                                                      unsigned site)
{
    static_assert(IL, "only the interleaved layout is gathered");
    return row_dot_g<NB, G, GatherIL<NB>, SBC>(ent, b, e, lr, GatherIL<NB>{src, rows, site});
}

}  // namespace dect

namespace dect {

// ---------------------------------------------------------------------------
// mbarrier helpers.  Every wait is bounded: after `limit` failed polls the
// caller gets false and records the timeout instead of spinning forever.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

// 1-D bulk copy (TMA) of `bytes` bytes from global memory into this block's
// shared memory, counted on `bar` as transaction bytes.  Both addresses must
// be 16-byte aligned and `bytes` a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Wait for phase `parity` of `bar`; false after `limit` unsuccessful polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity, unsigned limit)
{
    for (unsigned i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

}  // namespace dect

namespace dect {

// Ampere-style asynchronous 16-byte global -> shared copies (L2 only).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

}  // namespace dect
