// Internal declarations shared by the translation units of libdect.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>

#include "dect.h"

namespace dect {

constexpr int kSMs = 152;          // GB300: 2 dies x 76 SMs
constexpr int kMaxBatchImages = 64; // images interleaved per ADM pass
constexpr int kTablePad = 512;      // zero entries after the last row of each table
// A^T with shared-memory sinogram windows: pixel tiles of kWinTH x kWinTW
constexpr int kWinTH = 4, kWinTW = 4;
constexpr int kWinTP = kWinTH * kWinTW;
constexpr int kWinMaxViews = 4096;

// Thread-local text of the last CUDA error (returned by dect_last_error()).
void set_error(const char *where, cudaError_t e);
void set_error_text(const std::string &s);

#define DECT_CUDA(call)                                                         \
    do {                                                                        \
        cudaError_t e_ = (call);                                                \
        if (e_ != cudaSuccess) {                                                \
            ::dect::set_error(#call, e_);                                       \
            return e_ == cudaErrorMemoryAllocation ? DECT_ERR_OOM : DECT_ERR_CUDA; \
        }                                                                       \
    } while (0)

#define DECT_LAUNCH_CHECK() DECT_CUDA(cudaGetLastError())

// Count of kernels launched by the library (dect_kernel_launches()).
void count_launches(int64_t k);

// Packed table entry: .x = pixel (or ray) index, .y = __float_as_int(length in mm).
typedef int2 Entry;

// ---------------------------------------------------------------------------
// Index checks of the checked build (compiled with -DDECT_CHECKED).  A
// checked access whose index falls outside [0, bound) is not made: the
// caller substitutes a safe index, and the first such failure of the
// process (site code << 48 | index) is recorded in this translation unit's
// device word, which dect_check_status() reads and clears.  Without
// DECT_CHECKED the checks compile to nothing.
// ---------------------------------------------------------------------------
enum CheckSite : unsigned {
    CHK_GATHER_A = 1,     // A x: image index from the ray-major table
    CHK_GATHER_AT = 2,    // A^T y: ray index from the pixel-major table
    CHK_OTF_WALK = 3,     // on-the-fly A: pixel of the walk
    CHK_OTF_RAY = 4,      // on-the-fly A^T: candidate ray
    CHK_PLS_STENCIL = 5,  // PLS: neighbour of the 5-point stencil
    CHK_FBP_BIN = 6,      // FBP: interpolation bin
    CHK_SELFTEST = 7      // dect_selftest_index
};

typedef cudaError_t (*CheckReader)(unsigned long long *word);
// register a translation unit's reader (called by static initialisers)
int register_check_reader(CheckReader r);

#ifdef DECT_CHECKED
static __device__ unsigned long long g_check_word;

static cudaError_t read_check_word(unsigned long long *w)
{
    cudaError_t e = cudaMemcpyFromSymbol(w, g_check_word, sizeof(*w));
    const unsigned long long zero = 0ull;
    if (e == cudaSuccess && *w) e = cudaMemcpyToSymbol(g_check_word, &zero, sizeof(zero));
    return e;
}
static const int g_check_reader_registered = register_check_reader(read_check_word);

__device__ __forceinline__ bool check_index(int64_t i, int64_t bound, unsigned site)
{
    if (i >= 0 && i < bound) return true;
    atomicCAS(&g_check_word, 0ull, ((unsigned long long)site << 48) | ((unsigned long long)i & 0xffffffffffffull));
    return false;
}
#define DECT_IDX_OK(i, bound, site) ::dect::check_index((int64_t)(i), (int64_t)(bound), (site))
#else
#define DECT_IDX_OK(i, bound, site) true
#endif

}  // namespace dect

struct dect_plan {
    dect_geometry g;
    dect_cone_geometry cone;  // cone-beam plans (nz > 1 or nr > 1; zero otherwise)
    int device;
    int n, nv, nb;
    int nz, nr;               // cone-beam: slices and detector rows (0 for fan-beam plans)
    int64_t N, M, nnz;
    int64_t n_grid_aligned;
    int64_t *rowptr;   // [M + 1], ray-major table (CSR of A)
    dect::Entry *ent;  // [nnz]  {pixel, len}
    int64_t *colptr;   // [N + 1], pixel-major table (CSR of A^T)
    dect::Entry *tent; // [nnz]  {ray, len}, rays increasing within a pixel
    // Per pixel tile (kWinTH x kWinTW) and view: the window of the tile's rays,
    // [wray0, wray0 + wcnt) (even start and count), placed at woff in the
    // tile's shared-memory window of wtot rays; tlocal = tent with the ray
    // replaced by its index in the tile's window.  win_max = max wtot
    // (0 when the windowed A^T is not available for this geometry).
    int win_tiles;
    int win_max;
    int nvp;                   // descriptor stride per tile: nv rounded up to 4
    int *wray0, *wcnt, *woff;  // [win_tiles * nvp]
    int *wtot;                 // [win_tiles]
    dect::Entry *tlocal;       // [nnz + pad]
    // The same entries tile-major: tile t's pixels (row-major inside the tile)
    // at tmaj[tbase[t] .. tbase[t + 1]) (even offsets, zero-padded to an even
    // count); pixel s of tile t at tpo[t * (kWinTP + 1) + s] relative to
    // tbase[t].  tile_ent_max = max entries of a tile.
    dect::Entry *tmaj;
    int64_t *tbase;            // [win_tiles + 1]
    int *tpo;                  // [win_tiles * (kWinTP + 1)]
    int tile_ent_max;
    // Autotuner cache: chosen A^T variant per ADM batch width (index log2(NB) - 1),
    // -1 until the first ADM call with that width has timed the candidates.
    mutable int bwd_choice[6];
    mutable float bwd_us[6][DECT_BWD_VARIANTS];
    // The same for the A variant (k_fwd).
    mutable int fwd_choice[6];
    mutable float fwd_us[6][DECT_FWD_VARIANTS];
    // The same for the TV step (k_tv or k_tv_tma).
    mutable int tv_choice[6];
    mutable float tv_us[6][DECT_TV_VARIANTS];
    // On-the-fly projector geometry (built on first use, see batch.cu): per
    // ray the point closest to the rotation axis and the unit direction
    // (otf_ray), the reciprocals of the direction (otf_inv); per view the
    // source and the detector frame (otf_view, otf_view2).  FP64 computed,
    // FP32 stored.
    mutable float4 *otf_ray;
    mutable float2 *otf_inv;
    mutable float4 *otf_view, *otf_view2;
};

namespace dect {

// Launchers (project.cu).  Planar layout: image b at base + b * N.
cudaError_t launch_project_planar(const dect_plan *p, const float *x, float *y, int batch,
                                  cudaStream_t s);
cudaError_t launch_backproject_planar(const dect_plan *p, const float *y, float *x, int batch,
                                      cudaStream_t s);

// On-the-fly projector geometry of a plan (batch.cu): built and cached on the
// first call; synchronises `s` then.
cudaError_t otf_setup(const dect_plan *p, cudaStream_t s);

}  // namespace dect
