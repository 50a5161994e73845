// Internal declarations shared by the CUDA translation units of libcmcg.
//
// Grid: nodes j = ix + sx (iy + sy iz), x fastest, sx = nx + 1 etc.  2D grids use nz = 0,
// sz = 1.  Lumped weights W_j = h^d prod_a w(j_a) with w = 1/2 on the two end nodes of an
// axis; the unscaled mirror Laplacian Lt(y)_j = sum_a (2 y_j - y_{j-e_a} - y_{j+e_a})
// (2nd order) or sum_a (5/2 y_j - 4/3 (y_{j-e_a} + y_{j+e_a}) + 1/12 (y_{j-2e_a} + y_{j+2e_a}))
// (4th order) with even reflection at the faces; K = W Lt / h^2 (Sec. 4.1/4.3 mass lumping
// on a Cartesian grid).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "cmcg.h"

namespace cmcg {

struct Geom {
    int dim;
    int nx, ny, nz;       // intervals (nz = 0 in 2D)
    int sx, sy, sz;       // nodes per axis
    long long np;         // nodes
    double h;
    unsigned abc;         // bit f set: face f (-x,+x,-y,+y,-z,+z) is absorbing
};

__host__ __device__ __forceinline__ long long node(const Geom& g, int ix, int iy, int iz) {
    return (long long)ix + (long long)g.sx * ((long long)iy + (long long)g.sy * iz);
}

// Number of absorbing faces through a node.  beta = (dt/2) M^-1 B = nb c dt / h = nb sqrt(kappa).
__device__ __forceinline__ int num_abc(const Geom& g, int ix, int iy, int iz) {
    int nb = 0;
    nb += (ix == 0) & (int)(g.abc & 1u);
    nb += (ix == g.nx) & (int)((g.abc >> 1) & 1u);
    nb += (iy == 0) & (int)((g.abc >> 2) & 1u);
    nb += (iy == g.ny) & (int)((g.abc >> 3) & 1u);
    if (g.dim == 3) {
        nb += (iz == 0) & (int)((g.abc >> 4) & 1u);
        nb += (iz == g.nz) & (int)((g.abc >> 5) & 1u);
    }
    return nb;
}

// Lumped volume weight W_j.
__device__ __forceinline__ double weight(const Geom& g, int ix, int iy, int iz) {
    double w = (g.dim == 3) ? g.h * g.h * g.h : g.h * g.h;
    if (ix == 0 || ix == g.nx) w *= 0.5;
    if (iy == 0 || iy == g.ny) w *= 0.5;
    if (g.dim == 3 && (iz == 0 || iz == g.nz)) w *= 0.5;
    return w;
}

// Offsets of the mirror / even-reflection neighbours along one axis of stride s.
__device__ __forceinline__ long long off_m1(int i, long long s) { return i > 0 ? -s : s; }
__device__ __forceinline__ long long off_p1(int i, int n, long long s) { return i < n ? s : -s; }
__device__ __forceinline__ long long off_m2(int i, long long s) {
    int k = i - 2;
    k = k < 0 ? -k : k;
    return (long long)(k - i) * s;
}
__device__ __forceinline__ long long off_p2(int i, int n, long long s) {
    int k = i + 2;
    k = k > n ? 2 * n - k : k;
    return (long long)(k - i) * s;
}

// ---- compiled-in bounds checks --------------------------------------------------------
// The checked build (libcmcg_checked.so, compiled with -DCMCG_CHECKED) tests, in the kernels
// that derive node indices from their launch coordinates, that every index a thread will touch
// lies inside its arrays.  A thread that fails records the check site and the offending index
// in its translation unit's error word and skips its accesses (it is treated as outside the
// grid); cmcg_check_status reads and clears the words.  In the normal build the checks compile
// to `true` and the words do not exist.
#ifdef CMCG_CHECKED
namespace {
__device__ unsigned long long g_check_count;
__device__ long long g_check_site;
__device__ long long g_check_index;
}  // namespace
__device__ __forceinline__ bool check_range(long long lo, long long hi, long long n, int site) {
    if (lo >= 0 && hi < n && lo <= hi) return true;
    if (atomicAdd(&g_check_count, 1ull) == 0ull) {
        g_check_site = site;
        g_check_index = lo < 0 ? lo : hi;
    }
    return false;
}
// Reads (count, site, index) of this translation unit's word into out[0..2] and clears it.
#define CMCG_CHECK_TU(name)                                                                   \
    void check_read_##name(long long* out) {                                                  \
        unsigned long long c = 0;                                                             \
        long long si = -1, ix = 0;                                                            \
        cudaMemcpyFromSymbol(&c, g_check_count, sizeof(c));                                   \
        cudaMemcpyFromSymbol(&si, g_check_site, sizeof(si));                                  \
        cudaMemcpyFromSymbol(&ix, g_check_index, sizeof(ix));                                 \
        const unsigned long long zero = 0;                                                    \
        cudaMemcpyToSymbol(g_check_count, &zero, sizeof(zero));                               \
        out[0] = (long long)c;                                                                \
        out[1] = c ? si : -1;                                                                 \
        out[2] = c ? ix : 0;                                                                  \
    }
#define CMCG_RANGE_OK(lo, hi, n, site) ::cmcg::check_range((lo), (hi), (n), (site))
#else
#define CMCG_CHECK_TU(name)                \
    void check_read_##name(long long* out) { \
        out[0] = 0;                          \
        out[1] = -1;                         \
        out[2] = 0;                          \
    }
#define CMCG_RANGE_OK(lo, hi, n, site) true
#endif

// Check sites (the kernel families that test their index ranges).
enum CheckSite {
    kSiteColumn = 1,     // column-marching kernels of wave.cu (steps, period ends, source)
    kSiteVector = 2,     // the float4 step (flat chunks)
    kSiteBatch = 3,      // a work item of the batched step kernel
    kSitePairGlobal = 4, // two-step kernel: a column's node or plane
    kSitePairShared = 5, // two-step kernel: a shared-memory neighbour
    kSiteMultigrid = 6,  // column-marching multigrid kernels of riesz.cu
};

// Does the index range of a column-marching thread lie inside the grid: node (ix, iy, iz) for
// z0 <= iz < z1 and its mirror neighbours up to `radius` nodes away along each axis?
__device__ __forceinline__ bool column_in_range(const Geom& g, int ix, int iy, int z0, int z1, int radius, int site) {
#ifdef CMCG_CHECKED
    if (z0 >= z1) return true;  // no planes: nothing is touched
    if (ix < 0 || ix > g.nx || iy < 0 || iy > g.ny || z0 < 0 || z1 > g.sz)
        return check_range(-1, -1, 0, site);
    const long long sY = g.sx, sZ = (long long)g.sx * g.sy;
    long long dmin = 0, dmax = 0;  // in-plane offsets
    auto take = [&](long long d) {
        dmin = d < dmin ? d : dmin;
        dmax = d > dmax ? d : dmax;
    };
    take(off_m1(ix, 1));
    take(off_p1(ix, g.nx, 1));
    take(off_m1(iy, sY));
    take(off_p1(iy, g.ny, sY));
    if (radius >= 2) {
        take(off_m2(ix, 1));
        take(off_p2(ix, g.nx, 1));
        take(off_m2(iy, sY));
        take(off_p2(iy, g.ny, sY));
    }
    long long zlo = 0, zhi = 0;  // z offsets at the first and the last plane
    if (g.dim == 3) {
        zlo = off_m1(z0, sZ);
        zlo = off_p1(z0, g.nz, sZ) < zlo ? off_p1(z0, g.nz, sZ) : zlo;
        zhi = off_p1(z1 - 1, g.nz, sZ);
        zhi = off_m1(z1 - 1, sZ) > zhi ? off_m1(z1 - 1, sZ) : zhi;
        if (radius >= 2) {
            zlo = off_m2(z0, sZ) < zlo ? off_m2(z0, sZ) : zlo;
            zhi = off_p2(z1 - 1, g.nz, sZ) > zhi ? off_p2(z1 - 1, g.nz, sZ) : zhi;
        }
        zlo = zlo < 0 ? zlo : 0;
        zhi = zhi > 0 ? zhi : 0;
    }
    const long long lo = node(g, ix, iy, z0) + (dmin < zlo ? dmin : zlo);
    const long long hi = node(g, ix, iy, z1 - 1) + (dmax > zhi ? dmax : zhi);
    return check_range(lo, hi, g.np, site);
#else
    (void)g, (void)ix, (void)iy, (void)z0, (void)z1, (void)radius, (void)site;
    return true;
#endif
}

// Unscaled Laplacian Lt(f) at node j for a value functor f(index) -> R.
template <int ORDER, typename R, typename F>
__device__ __forceinline__ R lap_t(const Geom& g, F f, long long j, int ix, int iy, int iz) {
    const R c = f(j);
    const long long sX = 1, sY = g.sx, sZ = (long long)g.sx * g.sy;
    if (ORDER == 2) {
        R acc = f(j + off_m1(ix, sX)) + f(j + off_p1(ix, g.nx, sX));
        acc += f(j + off_m1(iy, sY)) + f(j + off_p1(iy, g.ny, sY));
        R diag = R(4) * c;
        if (g.dim == 3) {
            acc += f(j + off_m1(iz, sZ)) + f(j + off_p1(iz, g.nz, sZ));
            diag = R(6) * c;
        }
        return diag - acc;
    } else {
        const R c1 = R(4) / R(3), c2 = R(1) / R(12);
        R a1 = f(j + off_m1(ix, sX)) + f(j + off_p1(ix, g.nx, sX));
        R a2 = f(j + off_m2(ix, sX)) + f(j + off_p2(ix, g.nx, sX));
        a1 += f(j + off_m1(iy, sY)) + f(j + off_p1(iy, g.ny, sY));
        a2 += f(j + off_m2(iy, sY)) + f(j + off_p2(iy, g.ny, sY));
        R diag = R(5) * c;
        if (g.dim == 3) {
            a1 += f(j + off_m1(iz, sZ)) + f(j + off_p1(iz, g.nz, sZ));
            a2 += f(j + off_m2(iz, sZ)) + f(j + off_p2(iz, g.nz, sZ));
            diag = R(7.5) * c;
        }
        return diag - c1 * a1 + c2 * a2;
    }
}

// Unscaled 7-point Laplacian of f along a thread's z-column, with the z-neighbours carried in
// registers from plane to plane (mirror at the z faces).  Same sum, in the same order, as
// lap_t<2> ((x- + x+) + (y- + y+)) + (z- + z+), so the results are bitwise equal.
template <typename T, typename F>
struct ColumnLap7 {
    F f;
    long long sZ, oxm, oxp, oym, oyp;
    int nz;
    T below, here, above;  // f at iz - 1, iz, iz + 1 (mirrored at the faces)
    __device__ __forceinline__ void start(long long j, int iz) {
        here = f(j);
        below = f(j + (iz > 0 ? -sZ : sZ));
        above = f(j + (iz < nz ? sZ : -sZ));
    }
    __device__ __forceinline__ T lap(long long j) const {
        T acc = f(j + oxm) + f(j + oxp);
        acc += f(j + oym) + f(j + oyp);
        acc += below + above;
        return T(6) * here - acc;
    }
    // move to plane iz + 1 (node j + sZ); valid while iz + 1 <= nz
    __device__ __forceinline__ void advance(long long j, int iz) {
        below = here;
        here = above;
        above = f(j + sZ + (iz + 1 < nz ? sZ : -sZ));
    }
};

template <typename T, typename F>
__device__ __forceinline__ ColumnLap7<T, F> column_lap(const Geom& g, F f, int ix, int iy) {
    ColumnLap7<T, F> c;
    c.f = f;
    c.sZ = (long long)g.sx * g.sy;
    c.oxm = off_m1(ix, 1);
    c.oxp = off_p1(ix, g.nx, 1);
    c.oym = off_m1(iy, g.sx);
    c.oyp = off_p1(iy, g.ny, g.sx);
    c.nz = g.nz;
    return c;
}

// ---- deterministic block reductions -------------------------------------------------
// Each block reduces NV doubles; thread 0 stores them in partials[k * gridDim.x + block].
// The last block to finish (atomic ticket) sums the partials in a fixed order and writes
// the totals to out[0..NV).  The result does not depend on block scheduling.
constexpr int kRedThreads = 256;

template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* smem /* NV*32 */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x * blockDim.y * blockDim.z + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) smem[k * 32 + warp] = x;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double x = lane < nwarps ? smem[k * 32 + lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            v[k] = x;
        }
    }
    __syncthreads();
}

// Returns true in (all threads of) the last block, whose v then holds the grand totals.
template <int NV>
__device__ __forceinline__ bool grid_sum(double (&v)[NV], double* partials, unsigned* ticket) {
    __shared__ double smem[NV * 32];
    __shared__ bool last;
    // linear thread id within the block
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthreads = blockDim.x * blockDim.y * blockDim.z;
    const long long nblocks = (long long)gridDim.x * gridDim.y * gridDim.z;
    const long long bid = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
    // block_sum expects a 1D-like warp layout; tid-based lanes
    {
        const int lane = tid & 31, warp = tid >> 5;
        const int nwarps = (nthreads + 31) >> 5;
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double x = v[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if (lane == 0) smem[k * 32 + warp] = x;
        }
        __syncthreads();
        if (tid == 0) {
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                double s = 0.0;
                for (int w = 0; w < nwarps; ++w) s += smem[k * 32 + w];
                partials[k * nblocks + bid] = s;
            }
            __threadfence();
            unsigned t = atomicAdd(ticket, 1u);
            last = (t == (unsigned)(nblocks - 1));
        }
        __syncthreads();
    }
    if (!last) return false;
    __threadfence();
    // fixed-order final sum over partials
    {
        const int lane = tid & 31, warp = tid >> 5;
        const int nwarps = (nthreads + 31) >> 5;
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double x = 0.0;
            for (long long b = tid; b < nblocks; b += nthreads) x += __ldcg(&partials[k * nblocks + b]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if (lane == 0) smem[k * 32 + warp] = x;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = 0.0;
            for (int w = 0; w < nwarps; ++w) s += smem[k * 32 + w];
            v[k] = s;
        }
        if (tid == 0) *ticket = 0u;
    }
    return true;
}

// Compensated (Kahan) FP32 running sum: a thread's partial sum of FP32 products without
// FP64 arithmetic (GB300 issues FP64 at 1/64 of the FP32 rate); converted to double once.
struct KahanF {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x) {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// Device scalar slots of the CG recurrences (double sc[]).
enum Slot {
    SC_GAMMA = 0,    // gamma = r . rhat = ||r||_E^2
    SC_GAMMA0,       // gamma at step (4)
    SC_GD,           // ghat . d = (g~, d)_E
    SC_GAMMA_NEW,
    SC_ALPHA,
    SC_BETA,
    SC_REL,          // sqrt(gamma / gamma0)
    SC_J,            // energy functional of the last forward period
    SC_GSUM,         // sum of ghat0 (range projection of the singular Riesz problem)
    SC_STATUS,       // 0 ok, 1 non-finite / non-positive CG scalar
    // Riesz PCG
    SC_P_BB,         // ||b||^2
    SC_P_RZ,         // r . z
    SC_P_PAP,        // p . Ap
    SC_P_RR,         // r . r
    SC_P_ZAP,        // z . Ap
    SC_P_ALPHA,
    SC_P_BETA,
    SC_P_BSUM,       // sum(rhs) for the projection
    SC_P_XW,         // sum(W x) for the mean removal
    // recovery
    SC_R0, SC_R1, SC_R2, SC_R3, SC_R4, SC_R5, SC_R6, SC_R7,
    SC_DEVERR,       // nonzero: a kernel's bounded wait ran out (the CMCG status code it reports)
    SC_COUNT
};

constexpr int kMaxBlocksReduce = 152 * 8;
constexpr int kNumTickets = 8;

}  // namespace cmcg
