// Plan: the Siddon system matrix A of Eq. (1) (Sec. 2.1; Siddon's method,
// ref. [42]) built on the device, stored ray-major for A x and pixel-major
// for the gather form of A^T y.
//
// Ray geometry (Fig. 1): view v at angle t_v = start + v * (arc / nv), source
// SOD (cos t, sin t), flat detector centred at (SOD - SDD)(cos t, sin t) with
// axis (-sin t, cos t), bin b at u_b = (b - (nb - 1) / 2) pitch + offset.
// The end points are computed on the host in FP64 (host libm); the walk runs
// on the device in FP64 with explicitly rounded operations (no FMA
// contraction), so every crossing parameter is the correctly rounded value of
// (plane - S) / d.
//
// Tie rule: a piece of the ray between two consecutive distinct crossing
// parameters belongs to the pixel holding the piece's midpoint,
// col = floor((x_mid - x_lo) / px); pieces of zero length are dropped, and
// consecutive pieces in the same pixel form one element of A.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "dect_internal.cuh"

namespace dect {
namespace {

__device__ constexpr double kInf = __builtin_huge_val();

// Ray end points, FP64: (Sx, Sy, Dx, Dy).
struct RayPts {
    double sx, sy, dx_, dy_;
};

struct Grid {
    int n;
    double px;
    double lo;   // -(n/2) px, the first grid line
};

__device__ __forceinline__ double plane_at(const Grid &g, int k)
{
    return __dadd_rn(g.lo, __dmul_rn((double)k, g.px));
}

__device__ __forceinline__ double cross_param(double plane, double s, double d)
{
    return __ddiv_rn(__dsub_rn(plane, s), d);
}

// One axis of the walk: the grid lines of this axis crossed by the ray in
// increasing parameter order.
struct AxisWalk {
    int k;        // index of the next grid line
    int step;     // +1 or -1
    double next;  // its crossing parameter, +inf when none is left
};

__device__ __forceinline__ void axis_init(AxisWalk &w, const Grid &g, double s, double d,
                                          double amin, double amax)
{
    w.next = kInf;
    w.step = 0;
    w.k = 0;
    if (d == 0.0) return;
    // estimate the line index at the entry point, then settle it exactly on
    // the first line whose parameter is > amin
    double pos = __dadd_rn(s, __dmul_rn(amin, d));
    int k = (int)floor(__ddiv_rn(__dsub_rn(pos, g.lo), g.px));
    if (d > 0.0) {
        w.step = 1;
        if (k < 0) k = 0;
        if (k > g.n) k = g.n;
        while (k <= g.n && cross_param(plane_at(g, k), s, d) <= amin) ++k;
        while (k - 1 >= 0 && cross_param(plane_at(g, k - 1), s, d) > amin) --k;
    } else {
        w.step = -1;
        k += 1;
        if (k < 0) k = 0;
        if (k > g.n) k = g.n;
        while (k >= 0 && cross_param(plane_at(g, k), s, d) <= amin) --k;
        while (k + 1 <= g.n && cross_param(plane_at(g, k + 1), s, d) > amin) ++k;
    }
    w.k = k;
    if (k >= 0 && k <= g.n) {
        double t = cross_param(plane_at(g, k), s, d);
        if (t < amax) w.next = t;
    }
}

__device__ __forceinline__ void axis_advance(AxisWalk &w, const Grid &g, double s, double d,
                                             double amax)
{
    w.k += w.step;
    w.next = kInf;
    if (w.k >= 0 && w.k <= g.n) {
        double t = cross_param(plane_at(g, w.k), s, d);
        if (t < amax) w.next = t;
    }
}

// Walk one ray.  Writes entries when `out` is non-null; returns the count.
__device__ int siddon_walk(const RayPts &r, const Grid &g, Entry *out, int *grid_aligned)
{
    const double dx = __dsub_rn(r.dx_, r.sx);
    const double dy = __dsub_rn(r.dy_, r.sy);
    const double L = __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
    const double hi = __dadd_rn(g.lo, __dmul_rn((double)g.n, g.px));

    if (grid_aligned) {
        // a ray that runs (within 1e-9 mm) along a grid line
        int al = 0;
        if (fabs(dx) <= 1e-12 * L) {
            double f = (r.sx - g.lo) / g.px;
            if (fabs(f - rint(f)) * g.px < 1e-9) al = 1;
        }
        if (fabs(dy) <= 1e-12 * L) {
            double f = (r.sy - g.lo) / g.px;
            if (fabs(f - rint(f)) * g.px < 1e-9) al = 1;
        }
        *grid_aligned = al;
    }

    double amin = 0.0, amax = 1.0;
    if (dx != 0.0) {
        double t0 = cross_param(g.lo, r.sx, dx), t1 = cross_param(hi, r.sx, dx);
        amin = fmax(amin, fmin(t0, t1));
        amax = fmin(amax, fmax(t0, t1));
    } else if (!(r.sx >= g.lo && r.sx < hi)) {
        return 0;
    }
    if (dy != 0.0) {
        double t0 = cross_param(g.lo, r.sy, dy), t1 = cross_param(hi, r.sy, dy);
        amin = fmax(amin, fmin(t0, t1));
        amax = fmin(amax, fmax(t0, t1));
    } else if (!(r.sy >= g.lo && r.sy < hi)) {
        return 0;
    }
    if (!(amin < amax)) return 0;

    AxisWalk wx, wy;
    axis_init(wx, g, r.sx, dx, amin, amax);
    axis_init(wy, g, r.sy, dy, amin, amax);

    // One element per (ray, pixel): pieces that the midpoint rule gives to the
    // pixel of the previous piece (a crossing within rounding of a grid
    // corner) are added to it, in walk order, before the single FP32 rounding.
    int cnt = 0;
    int pend_pix = -1;
    double pend_len = 0.0;
    double cur = amin;
    // at most 2(n+1) crossings plus the exit
    for (int guard = 0; guard < 2 * g.n + 4; ++guard) {
        double a1 = fmin(fmin(wx.next, wy.next), amax);
        if (a1 > cur) {
            double mid = __dmul_rn(0.5, __dadd_rn(cur, a1));
            double xm = __dadd_rn(r.sx, __dmul_rn(mid, dx));
            double ym = __dadd_rn(r.sy, __dmul_rn(mid, dy));
            int col = (int)floor(__ddiv_rn(__dsub_rn(xm, g.lo), g.px));
            int row = (int)floor(__ddiv_rn(__dsub_rn(ym, g.lo), g.px));
            if (col >= 0 && col < g.n && row >= 0 && row < g.n) {
                const int pix = row * g.n + col;
                const double seg = __dmul_rn(__dsub_rn(a1, cur), L);
                if (pix == pend_pix) {
                    pend_len = __dadd_rn(pend_len, seg);
                } else {
                    if (pend_pix >= 0) {
                        if (out) out[cnt] = make_int2(pend_pix, __float_as_int(__double2float_rn(pend_len)));
                        ++cnt;
                    }
                    pend_pix = pix;
                    pend_len = seg;
                }
            }
        }
        if (a1 >= amax) break;
        if (wx.next == a1) axis_advance(wx, g, r.sx, dx, amax);
        if (wy.next == a1) axis_advance(wy, g, r.sy, dy, amax);
        cur = a1;
    }
    if (pend_pix >= 0) {
        if (out) out[cnt] = make_int2(pend_pix, __float_as_int(__double2float_rn(pend_len)));
        ++cnt;
    }
    return cnt;
}

__global__ void k_siddon_count(const RayPts *__restrict__ rays, int64_t M, Grid g,
                               int64_t *__restrict__ counts, unsigned long long *aligned)
{
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= M) return;
    int al = 0;
    counts[r] = siddon_walk(rays[r], g, nullptr, &al);
    if (al) atomicAdd(aligned, 1ull);
}

__global__ void k_siddon_fill(const RayPts *__restrict__ rays, int64_t M, Grid g,
                              const int64_t *__restrict__ rowptr, Entry *__restrict__ ent)
{
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= M) return;
    siddon_walk(rays[r], g, ent + rowptr[r], nullptr);
}

// ---------------------------------------------------------------------------
// Cone-beam walk (3-D Siddon): the same rule with a third axis.  The volume
// is n x n x nz voxels, index (kz n + row) n + col; gxy is the grid of x and
// y, gz the grid of z.
// ---------------------------------------------------------------------------
struct RayPts3 {
    double sx, sy, sz, dx_, dy_, dz_;
};

__device__ int siddon_walk3(const RayPts3 &r, const Grid &gxy, const Grid &gz, Entry *out)
{
    const double dx = __dsub_rn(r.dx_, r.sx), dy = __dsub_rn(r.dy_, r.sy), dz = __dsub_rn(r.dz_, r.sz);
    const double L = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
    const double s[3] = {r.sx, r.sy, r.sz}, d[3] = {dx, dy, dz};
    const Grid *gs[3] = {&gxy, &gxy, &gz};
    double amin = 0.0, amax = 1.0;
    for (int a = 0; a < 3; ++a) {
        const Grid &g = *gs[a];
        const double hi = __dadd_rn(g.lo, __dmul_rn((double)g.n, g.px));
        if (d[a] != 0.0) {
            const double t0 = cross_param(g.lo, s[a], d[a]), t1 = cross_param(hi, s[a], d[a]);
            amin = fmax(amin, fmin(t0, t1));
            amax = fmin(amax, fmax(t0, t1));
        } else if (!(s[a] >= g.lo && s[a] < hi)) {
            return 0;
        }
    }
    if (!(amin < amax)) return 0;
    AxisWalk w[3];
    for (int a = 0; a < 3; ++a) axis_init(w[a], *gs[a], s[a], d[a], amin, amax);
    const int n = gxy.n, nz = gz.n;
    int cnt = 0, pend = -1;
    double pend_len = 0.0, cur = amin;
    for (int guard = 0; guard < 2 * n + nz + 6; ++guard) {
        const double a1 = fmin(fmin(fmin(w[0].next, w[1].next), w[2].next), amax);
        if (a1 > cur) {
            const double mid = __dmul_rn(0.5, __dadd_rn(cur, a1));
            int idx[3];
            for (int a = 0; a < 3; ++a) {
                const double pos = __dadd_rn(s[a], __dmul_rn(mid, d[a]));
                idx[a] = (int)floor(__ddiv_rn(__dsub_rn(pos, gs[a]->lo), gs[a]->px));
            }
            if (idx[0] >= 0 && idx[0] < n && idx[1] >= 0 && idx[1] < n && idx[2] >= 0 && idx[2] < nz) {
                const int vox = (idx[2] * n + idx[1]) * n + idx[0];
                const double seg = __dmul_rn(__dsub_rn(a1, cur), L);
                if (vox == pend) {
                    pend_len = __dadd_rn(pend_len, seg);
                } else {
                    if (pend >= 0) {
                        if (out) out[cnt] = make_int2(pend, __float_as_int(__double2float_rn(pend_len)));
                        ++cnt;
                    }
                    pend = vox;
                    pend_len = seg;
                }
            }
        }
        if (a1 >= amax) break;
        for (int a = 0; a < 3; ++a)
            if (w[a].next == a1) axis_advance(w[a], *gs[a], s[a], d[a], amax);
        cur = a1;
    }
    if (pend >= 0) {
        if (out) out[cnt] = make_int2(pend, __float_as_int(__double2float_rn(pend_len)));
        ++cnt;
    }
    return cnt;
}

__global__ void k_siddon3_count(const RayPts3 *__restrict__ rays, int64_t M, Grid gxy, Grid gz,
                                int64_t *__restrict__ counts)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < M) counts[r] = siddon_walk3(rays[r], gxy, gz, nullptr);
}

__global__ void k_siddon3_fill(const RayPts3 *__restrict__ rays, int64_t M, Grid gxy, Grid gz,
                               const int64_t *__restrict__ rowptr, Entry *__restrict__ ent)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < M) siddon_walk3(rays[r], gxy, gz, ent + rowptr[r]);
}

// ---------------------------------------------------------------------------
// Exclusive scan of int64 counts (in place into out[0..n], out[n] = total).
// ---------------------------------------------------------------------------
constexpr int kScanBlock = 1024;

__global__ void k_scan_block(const int64_t *__restrict__ in, int64_t n, int64_t *__restrict__ out,
                             int64_t *__restrict__ block_sums)
{
    __shared__ int64_t s[kScanBlock];
    int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    int64_t v = (i < n) ? in[i] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < kScanBlock; off <<= 1) {
        int64_t t = (threadIdx.x >= (unsigned)off) ? s[threadIdx.x - off] : 0;
        __syncthreads();
        s[threadIdx.x] += t;
        __syncthreads();
    }
    if (i < n) out[i] = s[threadIdx.x] - v;  // exclusive
    if (threadIdx.x == kScanBlock - 1) block_sums[blockIdx.x] = s[threadIdx.x];
}

__global__ void k_scan_add(int64_t *__restrict__ out, int64_t n, const int64_t *__restrict__ offs)
{
    int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    if (i < n) out[i] += offs[blockIdx.x];
}

__global__ void k_set_last(int64_t *out, int64_t n, const int64_t *in_last, const int64_t *cnt_last)
{
    out[n] = *in_last + *cnt_last;
}

// out[0..n-1] = exclusive scan of in, out[n] = sum.  in and out may not alias.
cudaError_t scan_exclusive(const int64_t *in, int64_t n, int64_t *out, cudaStream_t s)
{
    if (n == 0) {
        return cudaMemsetAsync(out, 0, sizeof(int64_t), s);
    }
    int64_t nblk = (n + kScanBlock - 1) / kScanBlock;
    int64_t *sums = nullptr, *offs = nullptr;
    cudaError_t e = cudaMallocAsync(&sums, sizeof(int64_t) * nblk, s);
    if (e != cudaSuccess) return e;
    e = cudaMallocAsync(&offs, sizeof(int64_t) * (nblk + 1), s);
    if (e != cudaSuccess) return e;
    k_scan_block<<<(unsigned)nblk, kScanBlock, 0, s>>>(in, n, out, sums);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (nblk > 1) {
        e = scan_exclusive(sums, nblk, offs, s);
        if (e != cudaSuccess) return e;
        k_scan_add<<<(unsigned)nblk, kScanBlock, 0, s>>>(out, n, offs);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    k_set_last<<<1, 1, 0, s>>>(out, n, out + (n - 1), in + (n - 1));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    cudaFreeAsync(sums, s);
    cudaFreeAsync(offs, s);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Pixel-major transpose of the table.
// ---------------------------------------------------------------------------
__global__ void k_col_count(const Entry *__restrict__ ent, int64_t nnz, int *__restrict__ cnt)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz;
         k += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[ent[k].x], 1);
}

__global__ void k_int_to_i64(const int *__restrict__ a, int64_t n, int64_t *__restrict__ b)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = a[i];
}

// Scatter every entry into its pixel's segment (order inside a segment is
// arbitrary here and fixed by k_col_sort).
__global__ void k_col_scatter(const int64_t *__restrict__ rowptr, const Entry *__restrict__ ent,
                              int64_t M, const int64_t *__restrict__ colptr,
                              int *__restrict__ cursor, Entry *__restrict__ tmp)
{
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= M) return;
    for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k) {
        Entry e = ent[k];
        int slot = atomicAdd(&cursor[e.x], 1);
        tmp[colptr[e.x] + slot] = make_int2((int)r, e.y);
    }
}

// One warp per pixel: rank sort of the segment by ray index (a ray meets a
// pixel at most once, so ranks are unique and the order is deterministic).
__global__ void k_col_sort(const int64_t *__restrict__ colptr, int64_t N,
                           const Entry *__restrict__ tmp, Entry *__restrict__ tent)
{
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (warp >= N) return;
    int64_t b = colptr[warp], e = colptr[warp + 1];
    int len = (int)(e - b);
    for (int i = lane; i < len; i += 32) {
        Entry mine = tmp[b + i];
        int rank = 0;
        for (int j = 0; j < len; ++j) rank += (tmp[b + j].x < mine.x);
        tent[b + rank] = mine;
    }
}

// Per-tile sinogram windows for the shared-memory A^T (one block per tile):
// per view the range of bins that the tile's pixels meet, widened to an even
// start and an even count (16-byte aligned copies for any batch of >= 2
// images); prefix offsets; and the tile-local index of every entry.
__global__ void k_win_build(const int64_t *__restrict__ colptr, const Entry *__restrict__ tent, int n,
                            int nv, int nvp, int nb, int *__restrict__ wray0, int *__restrict__ wcnt,
                            int *__restrict__ woff, int *__restrict__ wtot,
                            Entry *__restrict__ tlocal, int *__restrict__ wmax)
{
    extern __shared__ int sw[];  // [2 * nv]
    int *lo = sw, *hi = sw + nv;
    const int tiles_x = (n + kWinTW - 1) / kWinTW;
    const int tile = blockIdx.x, ty = tile / tiles_x, tx = tile % tiles_x;
    for (int v = threadIdx.x; v < nv; v += blockDim.x) {
        lo[v] = 0x7fffffff;
        hi[v] = -1;
    }
    __syncthreads();
    for (int s = 0; s < kWinTH * kWinTW; ++s) {
        const int i = ty * kWinTH + s / kWinTW, j = tx * kWinTW + s % kWinTW;
        if (i >= n || j >= n) continue;
        const int64_t pix = (int64_t)i * n + j;
        for (int64_t k = colptr[pix] + threadIdx.x; k < colptr[pix + 1]; k += blockDim.x) {
            const int ray = tent[k].x, v = ray / nb;
            atomicMin(&lo[v], ray);
            atomicMax(&hi[v], ray);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int off = 0;
        for (int v = 0; v < nv; ++v) {
            int start = 0, cnt = 0;
            if (hi[v] >= 0) {
                start = lo[v] & ~1;
                cnt = ((hi[v] + 2) & ~1) - start;
            }
            wray0[(int64_t)tile * nvp + v] = start;
            wcnt[(int64_t)tile * nvp + v] = cnt;
            woff[(int64_t)tile * nvp + v] = off;
            lo[v] = start;
            hi[v] = off;
            off += cnt;
        }
        for (int v = nv; v < nvp; ++v) {
            wray0[(int64_t)tile * nvp + v] = 0;
            wcnt[(int64_t)tile * nvp + v] = 0;
            woff[(int64_t)tile * nvp + v] = off;
        }
        wtot[tile] = off;
        atomicMax(wmax, off);
    }
    __syncthreads();
    for (int s = 0; s < kWinTH * kWinTW; ++s) {
        const int i = ty * kWinTH + s / kWinTW, j = tx * kWinTW + s % kWinTW;
        if (i >= n || j >= n) continue;
        const int64_t pix = (int64_t)i * n + j;
        for (int64_t k = colptr[pix] + threadIdx.x; k < colptr[pix + 1]; k += blockDim.x) {
            const Entry t = tent[k];
            const int v = t.x / nb;
            tlocal[k] = make_int2(hi[v] + (t.x - lo[v]), t.y);
        }
    }
}

// Entries of each tile, padded to an even count.
__global__ void k_tile_count(const int64_t *__restrict__ colptr, int n, int ntiles,
                             int64_t *__restrict__ cnt)
{
    const int tile = blockIdx.x * blockDim.x + threadIdx.x;
    if (tile >= ntiles) return;
    const int tiles_x = (n + kWinTW - 1) / kWinTW, ty = tile / tiles_x, tx = tile % tiles_x;
    int64_t c = 0;
    for (int s = 0; s < kWinTP; ++s) {
        const int i = ty * kWinTH + s / kWinTW, j = tx * kWinTW + s % kWinTW;
        if (i < n && j < n) {
            const int64_t pix = (int64_t)i * n + j;
            c += colptr[pix + 1] - colptr[pix];
        }
    }
    cnt[tile] = (c + 1) & ~(int64_t)1;
}

// Copy each tile's tile-local entries to their tile-major place (one block per tile).
__global__ void k_tile_fill(const int64_t *__restrict__ colptr, const Entry *__restrict__ tlocal, int n,
                            const int64_t *__restrict__ tbase, int *__restrict__ tpo,
                            Entry *__restrict__ tmaj, int *__restrict__ emax)
{
    const int tile = blockIdx.x;
    const int tiles_x = (n + kWinTW - 1) / kWinTW, ty = tile / tiles_x, tx = tile % tiles_x;
    __shared__ int off[kWinTP + 1];
    if (threadIdx.x == 0) {
        int o = 0;
        for (int s = 0; s < kWinTP; ++s) {
            off[s] = o;
            const int i = ty * kWinTH + s / kWinTW, j = tx * kWinTW + s % kWinTW;
            if (i < n && j < n) {
                const int64_t pix = (int64_t)i * n + j;
                o += (int)(colptr[pix + 1] - colptr[pix]);
            }
        }
        off[kWinTP] = o;
        for (int s = 0; s <= kWinTP; ++s) tpo[(int64_t)tile * (kWinTP + 1) + s] = off[s];
        if (o & 1) tmaj[tbase[tile] + o] = make_int2(0, 0);
        atomicMax(emax, (int)(tbase[tile + 1] - tbase[tile]));
    }
    __syncthreads();
    for (int s = 0; s < kWinTP; ++s) {
        const int i = ty * kWinTH + s / kWinTW, j = tx * kWinTW + s % kWinTW;
        if (i >= n || j >= n) continue;
        const int64_t pix = (int64_t)i * n + j;
        const int64_t b = colptr[pix], len = colptr[pix + 1] - b;
        for (int64_t k = threadIdx.x; k < len; k += blockDim.x) tmaj[tbase[tile] + off[s] + k] = tlocal[b + k];
    }
}

bool geometry_ok(const dect_geometry *g)
{
    if (!g) return false;
    if (g->n < 1 || g->n > 8192 || g->n_views < 1 || g->n_bins < 1) return false;
    if (!(g->pixel_mm > 0) || !(g->pitch_mm > 0) || !(g->arc_rad > 0)) return false;
    if (!std::isfinite(g->pixel_mm) || !std::isfinite(g->pitch_mm) || !std::isfinite(g->sod_mm) ||
        !std::isfinite(g->sdd_mm) || !std::isfinite(g->start_rad) || !std::isfinite(g->arc_rad) ||
        !std::isfinite(g->det_offset_mm))
        return false;
    double half_diag = 0.5 * g->n * g->pixel_mm * std::sqrt(2.0);
    if (!(g->sod_mm > half_diag) || !(g->sdd_mm > g->sod_mm)) return false;
    if ((int64_t)g->n_views * g->n_bins > (int64_t)1 << 30) return false;
    return true;
}

}  // namespace

}  // namespace dect

using namespace dect;

extern "C" dect_status dect_plan_create(const dect_geometry *geom, int device, dect_stream stream,
                                        dect_plan **out)
{
    if (!out || !geometry_ok(geom)) return DECT_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    DECT_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return DECT_ERR_INVALID_ARG;
    DECT_CUDA(cudaSetDevice(device));
    cudaStream_t s = (cudaStream_t)stream;

    dect_plan *p = new dect_plan();
    std::memset(p, 0, sizeof(*p));
    p->g = *geom;
    p->device = device;
    p->n = geom->n;
    p->nv = geom->n_views;
    p->nb = geom->n_bins;
    p->N = (int64_t)p->n * p->n;
    p->M = (int64_t)p->nv * p->nb;
    for (int k = 0; k < 6; ++k) p->bwd_choice[k] = p->fwd_choice[k] = p->tv_choice[k] = -1;

    // ray end points on the host, FP64 (see file header)
    std::vector<RayPts> h(p->M);
    for (int v = 0; v < p->nv; ++v) {
        double th = geom->start_rad + (double)v * (geom->arc_rad / (double)p->nv);
        double c = std::cos(th), sn = std::sin(th);
        double sx = geom->sod_mm * c, sy = geom->sod_mm * sn;
        double cx = (geom->sod_mm - geom->sdd_mm) * c, cy = (geom->sod_mm - geom->sdd_mm) * sn;
        for (int b = 0; b < p->nb; ++b) {
            double u = ((double)b - 0.5 * (double)(p->nb - 1)) * geom->pitch_mm + geom->det_offset_mm;
            RayPts r;
            r.sx = sx;
            r.sy = sy;
            r.dx_ = cx - u * sn;
            r.dy_ = cy + u * c;
            h[(size_t)v * p->nb + b] = r;
        }
    }
    Grid g;
    g.n = p->n;
    g.px = geom->pixel_mm;
    g.lo = -0.5 * (double)p->n * geom->pixel_mm;

    RayPts *d_rays = nullptr;
    int64_t *d_cnt = nullptr;
    unsigned long long *d_al = nullptr;
    int *d_ccnt = nullptr, *d_cursor = nullptr;
    int64_t *d_ccnt64 = nullptr;
    Entry *d_tmp = nullptr;
    dect_status st = DECT_OK;
    auto fail = [&](dect_status code) {
        cudaStreamSynchronize(s);
        cudaFree(d_rays); cudaFree(d_cnt); cudaFree(d_al); cudaFree(d_ccnt);
        cudaFree(d_cursor); cudaFree(d_ccnt64); cudaFree(d_tmp);
        cudaFree(p->rowptr); cudaFree(p->ent); cudaFree(p->colptr); cudaFree(p->tent);
        cudaFree(p->wray0); cudaFree(p->wcnt); cudaFree(p->woff); cudaFree(p->wtot); cudaFree(p->tlocal);
        cudaFree(p->tmaj); cudaFree(p->tbase); cudaFree(p->tpo);
        delete p;
        return code;
    };
#define PLAN_CUDA(call)                                                            \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            set_error(#call, e_);                                                  \
            return fail(e_ == cudaErrorMemoryAllocation ? DECT_ERR_OOM : DECT_ERR_CUDA); \
        }                                                                          \
    } while (0)

    PLAN_CUDA(cudaMalloc(&d_rays, sizeof(RayPts) * p->M));
    PLAN_CUDA(cudaMemcpyAsync(d_rays, h.data(), sizeof(RayPts) * p->M, cudaMemcpyHostToDevice, s));
    PLAN_CUDA(cudaMalloc(&d_cnt, sizeof(int64_t) * p->M));
    PLAN_CUDA(cudaMalloc(&d_al, sizeof(unsigned long long)));
    PLAN_CUDA(cudaMemsetAsync(d_al, 0, sizeof(unsigned long long), s));
    PLAN_CUDA(cudaMalloc(&p->rowptr, sizeof(int64_t) * (p->M + 1)));
    const int T = 128;
    k_siddon_count<<<(unsigned)((p->M + T - 1) / T), T, 0, s>>>(d_rays, p->M, g, d_cnt, d_al);
    PLAN_CUDA(cudaGetLastError());
    PLAN_CUDA(scan_exclusive(d_cnt, p->M, p->rowptr, s));
    int64_t nnz = 0;
    unsigned long long al = 0;
    PLAN_CUDA(cudaMemcpyAsync(&nnz, p->rowptr + p->M, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    PLAN_CUDA(cudaMemcpyAsync(&al, d_al, sizeof(al), cudaMemcpyDeviceToHost, s));
    PLAN_CUDA(cudaStreamSynchronize(s));
    p->nnz = nnz;
    p->n_grid_aligned = (int64_t)al;
    if (nnz >= ((int64_t)1 << 31)) return fail(DECT_ERR_INVALID_ARG);

    // padding after the last row: the row kernels copy whole 16-byte pairs
    // and whole batches, which may run past a row's end
    size_t ne = (size_t)(nnz > 0 ? nnz : 1) + kTablePad;
    PLAN_CUDA(cudaMalloc(&p->ent, sizeof(Entry) * ne));
    PLAN_CUDA(cudaMemsetAsync(p->ent, 0, sizeof(Entry) * ne, s));
    k_siddon_fill<<<(unsigned)((p->M + T - 1) / T), T, 0, s>>>(d_rays, p->M, g, p->rowptr, p->ent);
    PLAN_CUDA(cudaGetLastError());

    // pixel-major transpose
    PLAN_CUDA(cudaMalloc(&d_ccnt, sizeof(int) * p->N));
    PLAN_CUDA(cudaMalloc(&d_cursor, sizeof(int) * p->N));
    PLAN_CUDA(cudaMalloc(&d_ccnt64, sizeof(int64_t) * p->N));
    PLAN_CUDA(cudaMalloc(&p->colptr, sizeof(int64_t) * (p->N + 1)));
    PLAN_CUDA(cudaMalloc(&d_tmp, sizeof(Entry) * ne));
    PLAN_CUDA(cudaMalloc(&p->tent, sizeof(Entry) * ne));
    PLAN_CUDA(cudaMemsetAsync(p->tent, 0, sizeof(Entry) * ne, s));
    PLAN_CUDA(cudaMemsetAsync(d_ccnt, 0, sizeof(int) * p->N, s));
    PLAN_CUDA(cudaMemsetAsync(d_cursor, 0, sizeof(int) * p->N, s));
    if (nnz > 0) {
        k_col_count<<<kSMs * 8, 256, 0, s>>>(p->ent, nnz, d_ccnt);
        PLAN_CUDA(cudaGetLastError());
    }
    k_int_to_i64<<<(unsigned)((p->N + 255) / 256), 256, 0, s>>>(d_ccnt, p->N, d_ccnt64);
    PLAN_CUDA(cudaGetLastError());
    PLAN_CUDA(scan_exclusive(d_ccnt64, p->N, p->colptr, s));
    if (nnz > 0) {
        k_col_scatter<<<(unsigned)((p->M + T - 1) / T), T, 0, s>>>(p->rowptr, p->ent, p->M, p->colptr,
                                                                   d_cursor, d_tmp);
        PLAN_CUDA(cudaGetLastError());
        int64_t threads = p->N * 32;
        k_col_sort<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(p->colptr, p->N, d_tmp, p->tent);
        PLAN_CUDA(cudaGetLastError());
    }
    // shared-memory windows of the tiled A^T
    if (p->nv <= kWinMaxViews && nnz > 0) {
        const int tiles_x = (p->n + kWinTW - 1) / kWinTW, tiles_y = (p->n + kWinTH - 1) / kWinTH;
        p->win_tiles = tiles_x * tiles_y;
        p->nvp = (p->nv + 3) & ~3;
        const size_t tv = (size_t)p->win_tiles * p->nvp;
        PLAN_CUDA(cudaMalloc(&p->wray0, sizeof(int) * tv));
        PLAN_CUDA(cudaMalloc(&p->wcnt, sizeof(int) * tv));
        PLAN_CUDA(cudaMalloc(&p->woff, sizeof(int) * tv));
        PLAN_CUDA(cudaMalloc(&p->wtot, sizeof(int) * p->win_tiles));
        PLAN_CUDA(cudaMalloc(&p->tlocal, sizeof(Entry) * ne));
        PLAN_CUDA(cudaMemsetAsync(p->tlocal, 0, sizeof(Entry) * ne, s));
        int *d_wmax = d_ccnt;  // reuse a scratch int
        PLAN_CUDA(cudaMemsetAsync(d_wmax, 0, sizeof(int), s));
        const size_t sm = sizeof(int) * 2 * p->nv;
        if (sm > 48 * 1024)
            PLAN_CUDA(cudaFuncSetAttribute(k_win_build, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_win_build<<<p->win_tiles, 256, sm, s>>>(p->colptr, p->tent, p->n, p->nv, p->nvp, p->nb, p->wray0, p->wcnt,
                                                   p->woff, p->wtot, p->tlocal, d_wmax);
        PLAN_CUDA(cudaGetLastError());
        int wmax = 0;
        PLAN_CUDA(cudaMemcpyAsync(&wmax, d_wmax, sizeof(int), cudaMemcpyDeviceToHost, s));
        PLAN_CUDA(cudaStreamSynchronize(s));
        // tile-major copy of the tile-local entries
        const int nt = p->win_tiles;
        PLAN_CUDA(cudaMalloc(&p->tbase, sizeof(int64_t) * (nt + 1)));
        PLAN_CUDA(cudaMalloc(&p->tpo, sizeof(int) * (size_t)nt * (kWinTP + 1)));
        int64_t *d_tcnt = nullptr;
        PLAN_CUDA(cudaMalloc(&d_tcnt, sizeof(int64_t) * nt));
        k_tile_count<<<(nt + 255) / 256, 256, 0, s>>>(p->colptr, p->n, nt, d_tcnt);
        PLAN_CUDA(cudaGetLastError());
        PLAN_CUDA(scan_exclusive(d_tcnt, nt, p->tbase, s));
        int64_t tot = 0;
        PLAN_CUDA(cudaMemcpyAsync(&tot, p->tbase + nt, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        PLAN_CUDA(cudaStreamSynchronize(s));
        cudaFree(d_tcnt);
        PLAN_CUDA(cudaMalloc(&p->tmaj, sizeof(Entry) * (size_t)(tot + kTablePad)));
        PLAN_CUDA(cudaMemsetAsync(p->tmaj, 0, sizeof(Entry) * (size_t)(tot + kTablePad), s));
        PLAN_CUDA(cudaMemsetAsync(d_wmax, 0, sizeof(int), s));
        k_tile_fill<<<nt, 256, 0, s>>>(p->colptr, p->tlocal, p->n, p->tbase, p->tpo, p->tmaj, d_wmax);
        PLAN_CUDA(cudaGetLastError());
        int emax = 0;
        PLAN_CUDA(cudaMemcpyAsync(&emax, d_wmax, sizeof(int), cudaMemcpyDeviceToHost, s));
        PLAN_CUDA(cudaStreamSynchronize(s));
        p->tile_ent_max = emax;
        p->win_max = wmax;
    }
    PLAN_CUDA(cudaStreamSynchronize(s));
    cudaFree(d_rays); cudaFree(d_cnt); cudaFree(d_al); cudaFree(d_ccnt);
    cudaFree(d_cursor); cudaFree(d_ccnt64); cudaFree(d_tmp);
#undef PLAN_CUDA
    (void)st;
    *out = p;
    return DECT_OK;
}

namespace {

bool cone_ok(const dect_cone_geometry *g)
{
    if (!g) return false;
    if (g->n < 1 || g->n > 4096 || g->nz < 1 || g->nz > 4096 || g->n_views < 1 || g->n_rows < 1 ||
        g->n_cols < 1)
        return false;
    const double vals[] = {g->pixel_mm, g->slice_mm, g->pitch_u_mm, g->pitch_v_mm, g->sod_mm, g->sdd_mm,
                           g->start_rad, g->arc_rad, g->offset_u_mm, g->offset_v_mm};
    for (double v : vals)
        if (!std::isfinite(v)) return false;
    if (!(g->pixel_mm > 0) || !(g->slice_mm > 0) || !(g->pitch_u_mm > 0) || !(g->pitch_v_mm > 0) ||
        !(g->arc_rad > 0))
        return false;
    const double half_diag = 0.5 * g->n * g->pixel_mm * std::sqrt(2.0);
    if (!(g->sod_mm > half_diag) || !(g->sdd_mm > g->sod_mm)) return false;
    if ((int64_t)g->n_views * g->n_rows * g->n_cols > (int64_t)1 << 30) return false;
    if ((int64_t)g->n * g->n * g->nz > (int64_t)1 << 30) return false;
    return true;
}

}  // namespace

extern "C" dect_status dect_plan_create_cone(const dect_cone_geometry *geom, int device, dect_stream stream,
                                             dect_plan **out)
{
    if (!out || !cone_ok(geom)) return DECT_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    DECT_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return DECT_ERR_INVALID_ARG;
    DECT_CUDA(cudaSetDevice(device));
    cudaStream_t s = (cudaStream_t)stream;

    dect_plan *p = new dect_plan();
    std::memset(p, 0, sizeof(*p));
    // the fan-beam fields that describe the in-plane geometry
    p->g.n = geom->n;
    p->g.pixel_mm = geom->pixel_mm;
    p->g.n_views = geom->n_views;
    p->g.n_bins = geom->n_cols;
    p->g.pitch_mm = geom->pitch_u_mm;
    p->g.sod_mm = geom->sod_mm;
    p->g.sdd_mm = geom->sdd_mm;
    p->g.start_rad = geom->start_rad;
    p->g.arc_rad = geom->arc_rad;
    p->g.det_offset_mm = geom->offset_u_mm;
    p->cone = *geom;
    p->device = device;
    p->n = geom->n;
    p->nz = geom->nz;
    p->nv = geom->n_views;
    p->nr = geom->n_rows;
    p->nb = geom->n_cols;
    p->N = (int64_t)geom->n * geom->n * geom->nz;
    p->M = (int64_t)geom->n_views * geom->n_rows * geom->n_cols;
    for (int k = 0; k < 6; ++k) p->bwd_choice[k] = p->fwd_choice[k] = p->tv_choice[k] = -1;

    // ray end points on the host, FP64 (ray (v, r, c) -> (v nr + r) nc + c)
    std::vector<RayPts3> h(p->M);
    for (int v = 0; v < p->nv; ++v) {
        const double th = geom->start_rad + (double)v * (geom->arc_rad / (double)p->nv);
        const double c = std::cos(th), sn = std::sin(th);
        const double sx = geom->sod_mm * c, sy = geom->sod_mm * sn;
        const double cx = (geom->sod_mm - geom->sdd_mm) * c, cy = (geom->sod_mm - geom->sdd_mm) * sn;
        for (int r = 0; r < p->nr; ++r) {
            const double z = ((double)r - 0.5 * (double)(p->nr - 1)) * geom->pitch_v_mm + geom->offset_v_mm;
            for (int b = 0; b < p->nb; ++b) {
                const double u = ((double)b - 0.5 * (double)(p->nb - 1)) * geom->pitch_u_mm + geom->offset_u_mm;
                RayPts3 q;
                q.sx = sx;
                q.sy = sy;
                q.sz = 0.0;
                q.dx_ = cx - u * sn;
                q.dy_ = cy + u * c;
                q.dz_ = z;
                h[((size_t)v * p->nr + r) * p->nb + b] = q;
            }
        }
    }
    Grid gxy, gz;
    gxy.n = p->n;
    gxy.px = geom->pixel_mm;
    gxy.lo = -0.5 * (double)p->n * geom->pixel_mm;
    gz.n = p->nz;
    gz.px = geom->slice_mm;
    gz.lo = -0.5 * (double)p->nz * geom->slice_mm;

    RayPts3 *d_rays = nullptr;
    int64_t *d_cnt = nullptr, *d_ccnt64 = nullptr;
    int *d_ccnt = nullptr, *d_cursor = nullptr;
    Entry *d_tmp = nullptr;
    auto fail = [&](dect_status code) {
        cudaStreamSynchronize(s);
        cudaFree(d_rays); cudaFree(d_cnt); cudaFree(d_ccnt); cudaFree(d_cursor); cudaFree(d_ccnt64); cudaFree(d_tmp);
        cudaFree(p->rowptr); cudaFree(p->ent); cudaFree(p->colptr); cudaFree(p->tent);
        delete p;
        return code;
    };
#define PLAN_CUDA(call)                                                            \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            set_error(#call, e_);                                                  \
            return fail(e_ == cudaErrorMemoryAllocation ? DECT_ERR_OOM : DECT_ERR_CUDA); \
        }                                                                          \
    } while (0)
    // rays within 1e-9 mm of running along a grid plane (the midpoint rule
    // then gives them to the + side)
    for (size_t k = 0; k < h.size(); ++k) {
        const RayPts3 &q = h[k];
        const double d[3] = {q.dx_ - q.sx, q.dy_ - q.sy, q.dz_ - q.sz}, o[3] = {q.sx, q.sy, q.sz};
        const double L = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        const Grid *gg[3] = {&gxy, &gxy, &gz};
        for (int a = 0; a < 3; ++a)
            if (std::fabs(d[a]) <= 1e-12 * L) {
                const double f = (o[a] - gg[a]->lo) / gg[a]->px;
                if (std::fabs(f - std::rint(f)) * gg[a]->px < 1e-9) {
                    ++p->n_grid_aligned;
                    break;
                }
            }
    }
    PLAN_CUDA(cudaMalloc(&d_rays, sizeof(RayPts3) * p->M));
    PLAN_CUDA(cudaMemcpyAsync(d_rays, h.data(), sizeof(RayPts3) * p->M, cudaMemcpyHostToDevice, s));
    PLAN_CUDA(cudaMalloc(&d_cnt, sizeof(int64_t) * p->M));
    PLAN_CUDA(cudaMalloc(&p->rowptr, sizeof(int64_t) * (p->M + 1)));
    const int T = 128;
    k_siddon3_count<<<(unsigned)((p->M + T - 1) / T), T, 0, s>>>(d_rays, p->M, gxy, gz, d_cnt);
    PLAN_CUDA(cudaGetLastError());
    PLAN_CUDA(scan_exclusive(d_cnt, p->M, p->rowptr, s));
    int64_t nnz = 0;
    PLAN_CUDA(cudaMemcpyAsync(&nnz, p->rowptr + p->M, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    PLAN_CUDA(cudaStreamSynchronize(s));
    p->nnz = nnz;
    if (nnz >= ((int64_t)1 << 31)) return fail(DECT_ERR_INVALID_ARG);
    const size_t ne = (size_t)(nnz > 0 ? nnz : 1) + kTablePad;
    PLAN_CUDA(cudaMalloc(&p->ent, sizeof(Entry) * ne));
    PLAN_CUDA(cudaMemsetAsync(p->ent, 0, sizeof(Entry) * ne, s));
    k_siddon3_fill<<<(unsigned)((p->M + T - 1) / T), T, 0, s>>>(d_rays, p->M, gxy, gz, p->rowptr, p->ent);
    PLAN_CUDA(cudaGetLastError());
    // voxel-major transpose (rays increasing inside a voxel)
    PLAN_CUDA(cudaMalloc(&d_ccnt, sizeof(int) * p->N));
    PLAN_CUDA(cudaMalloc(&d_cursor, sizeof(int) * p->N));
    PLAN_CUDA(cudaMalloc(&d_ccnt64, sizeof(int64_t) * p->N));
    PLAN_CUDA(cudaMalloc(&p->colptr, sizeof(int64_t) * (p->N + 1)));
    PLAN_CUDA(cudaMalloc(&d_tmp, sizeof(Entry) * ne));
    PLAN_CUDA(cudaMalloc(&p->tent, sizeof(Entry) * ne));
    PLAN_CUDA(cudaMemsetAsync(p->tent, 0, sizeof(Entry) * ne, s));
    PLAN_CUDA(cudaMemsetAsync(d_ccnt, 0, sizeof(int) * p->N, s));
    PLAN_CUDA(cudaMemsetAsync(d_cursor, 0, sizeof(int) * p->N, s));
    if (nnz > 0) {
        k_col_count<<<kSMs * 8, 256, 0, s>>>(p->ent, nnz, d_ccnt);
        PLAN_CUDA(cudaGetLastError());
    }
    k_int_to_i64<<<(unsigned)((p->N + 255) / 256), 256, 0, s>>>(d_ccnt, p->N, d_ccnt64);
    PLAN_CUDA(cudaGetLastError());
    PLAN_CUDA(scan_exclusive(d_ccnt64, p->N, p->colptr, s));
    if (nnz > 0) {
        k_col_scatter<<<(unsigned)((p->M + T - 1) / T), T, 0, s>>>(p->rowptr, p->ent, p->M, p->colptr, d_cursor,
                                                                   d_tmp);
        PLAN_CUDA(cudaGetLastError());
        const int64_t threads = p->N * 32;
        k_col_sort<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(p->colptr, p->N, d_tmp, p->tent);
        PLAN_CUDA(cudaGetLastError());
    }
    PLAN_CUDA(cudaStreamSynchronize(s));
    cudaFree(d_rays); cudaFree(d_cnt); cudaFree(d_ccnt); cudaFree(d_cursor); cudaFree(d_ccnt64); cudaFree(d_tmp);
#undef PLAN_CUDA
    *out = p;
    return DECT_OK;
}

extern "C" dect_status dect_plan_destroy(dect_plan *p)
{
    if (!p) return DECT_OK;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(p->device);
    cudaDeviceSynchronize();
    cudaFree(p->rowptr);
    cudaFree(p->ent);
    cudaFree(p->colptr);
    cudaFree(p->tent);
    cudaFree(p->otf_ray);
    cudaFree(p->otf_inv);
    cudaFree(p->otf_view);
    cudaFree(p->otf_view2);
    cudaFree(p->wray0);
    cudaFree(p->wcnt);
    cudaFree(p->woff);
    cudaFree(p->wtot);
    cudaFree(p->tlocal);
    cudaFree(p->tmaj);
    cudaFree(p->tbase);
    cudaFree(p->tpo);
    cudaSetDevice(cur);
    delete p;
    return DECT_OK;
}

extern "C" dect_status dect_plan_get_info(const dect_plan *p, dect_plan_info *info)
{
    if (!p || !info) return DECT_ERR_INVALID_ARG;
    info->n_pixels = p->N;
    info->n_rays = p->M;
    info->nnz = p->nnz;
    info->table_bytes = (int64_t)sizeof(Entry) * 2 * p->nnz + (int64_t)sizeof(int64_t) * (p->M + p->N + 2);
    info->n_grid_aligned = p->n_grid_aligned;
    return DECT_OK;
}

extern "C" dect_status dect_plan_copy_table(const dect_plan *p, int64_t *rowptr, int32_t *pix,
                                            float *len, dect_stream stream)
{
    if (!p) return DECT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    DECT_CUDA(cudaSetDevice(p->device));
    if (rowptr)
        DECT_CUDA(cudaMemcpyAsync(rowptr, p->rowptr, sizeof(int64_t) * (p->M + 1),
                                  cudaMemcpyDeviceToHost, s));
    if ((pix || len) && p->nnz > 0) {
        std::vector<Entry> h((size_t)p->nnz);
        DECT_CUDA(cudaMemcpyAsync(h.data(), p->ent, sizeof(Entry) * p->nnz, cudaMemcpyDeviceToHost, s));
        DECT_CUDA(cudaStreamSynchronize(s));
        for (int64_t k = 0; k < p->nnz; ++k) {
            if (pix) pix[k] = h[k].x;
            if (len) {
                float f;
                std::memcpy(&f, &h[k].y, sizeof(float));
                len[k] = f;
            }
        }
    }
    DECT_CUDA(cudaStreamSynchronize(s));
    return DECT_OK;
}

namespace {

int width_index(int images)
{
    switch (images) {
    case 2: return 0;
    case 4: return 1;
    case 8: return 2;
    case 16: return 3;
    case 32: return 4;
    case 64: return 5;
    default: return -1;
    }
}

}  // namespace

extern "C" dect_status dect_plan_get_tuning(const dect_plan *p, int images, int *choice,
                                            float us[DECT_BWD_VARIANTS])
{
    if (!p || !choice || !us) return DECT_ERR_INVALID_ARG;
    const int idx = width_index(images);
    if (idx < 0) return DECT_ERR_INVALID_ARG;
    *choice = p->bwd_choice[idx];
    for (int v = 0; v < DECT_BWD_VARIANTS; ++v) us[v] = p->bwd_choice[idx] >= 0 ? p->bwd_us[idx][v] : -1.f;
    return DECT_OK;
}

extern "C" dect_status dect_plan_set_tuning(dect_plan *p, int images, int choice)
{
    if (!p || choice < -1 || choice >= DECT_BWD_VARIANTS) return DECT_ERR_INVALID_ARG;
    const int idx = width_index(images);
    if (idx < 0) return DECT_ERR_INVALID_ARG;
    p->bwd_choice[idx] = choice;
    for (int v = 0; v < DECT_BWD_VARIANTS; ++v) p->bwd_us[idx][v] = -1.f;
    return DECT_OK;
}

extern "C" dect_status dect_plan_get_fwd_tuning(const dect_plan *p, int images, int *choice,
                                                float us[DECT_FWD_VARIANTS])
{
    if (!p || !choice || !us) return DECT_ERR_INVALID_ARG;
    const int idx = width_index(images);
    if (idx < 0) return DECT_ERR_INVALID_ARG;
    *choice = p->fwd_choice[idx];
    for (int v = 0; v < DECT_FWD_VARIANTS; ++v) us[v] = p->fwd_choice[idx] >= 0 ? p->fwd_us[idx][v] : -1.f;
    return DECT_OK;
}

extern "C" dect_status dect_plan_set_fwd_tuning(dect_plan *p, int images, int choice)
{
    if (!p || choice < -1 || choice >= DECT_FWD_VARIANTS) return DECT_ERR_INVALID_ARG;
    const int idx = width_index(images);
    if (idx < 0) return DECT_ERR_INVALID_ARG;
    p->fwd_choice[idx] = choice;
    for (int v = 0; v < DECT_FWD_VARIANTS; ++v) p->fwd_us[idx][v] = -1.f;
    return DECT_OK;
}

extern "C" dect_status dect_plan_get_tv_tuning(const dect_plan *p, int images, int *choice,
                                               float us[DECT_TV_VARIANTS])
{
    if (!p || !choice || !us) return DECT_ERR_INVALID_ARG;
    const int idx = width_index(images);
    if (idx < 0) return DECT_ERR_INVALID_ARG;
    *choice = p->tv_choice[idx];
    for (int v = 0; v < DECT_TV_VARIANTS; ++v) us[v] = p->tv_choice[idx] >= 0 ? p->tv_us[idx][v] : -1.f;
    return DECT_OK;
}

extern "C" dect_status dect_plan_set_tv_tuning(dect_plan *p, int images, int choice)
{
    if (!p || choice < -1 || choice >= DECT_TV_VARIANTS) return DECT_ERR_INVALID_ARG;
    const int idx = width_index(images);
    if (idx < 0) return DECT_ERR_INVALID_ARG;
    p->tv_choice[idx] = choice;
    for (int v = 0; v < DECT_TV_VARIANTS; ++v) p->tv_us[idx][v] = -1.f;
    return DECT_OK;
}
