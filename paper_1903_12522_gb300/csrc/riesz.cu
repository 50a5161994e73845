// Riesz map of Eq. CMCG_PRECONDITIONIER: K s = rhs with K = W (-Lap_h) (the discrete
// (grad s, grad phi)), solved matrix-free on the GPU.  The paper solves this SPD,
// omega-independent problem with a two-level Schwarz method (Sec. 4.4); here it is FP64
// flexible PCG whose preconditioner is one geometric multigrid V-cycle in FP32:
//   - vertex-centred coarsening n -> n/2 (co-located nodes), rediscretised K on each level,
//     Dirichlet mask taken from the co-located fine node;
//   - damped Jacobi smoothing, residual restriction by the transpose of (bi/tri)linear
//     interpolation, prolongation by that interpolation;
//   - the coarsest level solved by Jacobi sweeps inside one thread block.
#include <math.h>

#include "common.cuh"
#include "kernels.h"

namespace cmcg {

namespace {

constexpr int kT = 256;
constexpr int kCoarseMax = 4096;

inline unsigned vec_blocks(long long n) {
    long long b = (n + kT - 1) / kT;
    if (b > kMaxBlocksReduce) b = kMaxBlocksReduce;
    if (b < 1) b = 1;
    return (unsigned)b;
}

inline unsigned node_blocks(long long n) { return (unsigned)((n + kT - 1) / kT); }

// Node coordinates (node counts stay below 2^31, so 32-bit division suffices).
__device__ __forceinline__ void coords(const Geom& g, long long j, int& ix, int& iy, int& iz) {
    const unsigned u = (unsigned)j;
    const unsigned t = u / (unsigned)g.sx;
    ix = (int)(u - t * (unsigned)g.sx);
    iz = (int)(t / (unsigned)g.sy);
    iy = (int)(t - (unsigned)iz * (unsigned)g.sy);
}

template <typename R>
struct LdM {  // masked load: Dirichlet nodes read as 0
    const R* __restrict__ p;
    const unsigned char* __restrict__ m;
    __device__ __forceinline__ R operator()(long long i) const { return (m && m[i]) ? R(0) : p[i]; }
};

// ---- multigrid (FP32) ---------------------------------------------------------------------
__global__ void __launch_bounds__(kT) k_jacobi(Geom g, const unsigned char* __restrict__ mask,
                                               const float* __restrict__ xin, float* __restrict__ xout,
                                               const float* __restrict__ b, float omega, int zero_init) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= g.np) return;
    if (mask && mask[j]) {
        xout[j] = 0.f;
        return;
    }
    int ix, iy, iz;
    coords(g, j, ix, iy, iz);
    const float W = (float)weight(g, ix, iy, iz);
    const float h2 = (float)(g.h * g.h);
    const float twod = (float)(2 * g.dim);
    if (zero_init) {
        xout[j] = omega * h2 * b[j] / (twod * W);
    } else {
        LdM<float> f{xin, mask};
        const float L = lap_t<2, float>(g, f, j, ix, iy, iz);
        xout[j] = xin[j] + omega * (h2 * b[j] / W - L) / twod;
    }
}

__global__ void __launch_bounds__(kT) k_residual(Geom g, const unsigned char* __restrict__ mask,
                                                 const float* __restrict__ x, const float* __restrict__ b,
                                                 float* __restrict__ r) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= g.np) return;
    if (mask && mask[j]) {
        r[j] = 0.f;
        return;
    }
    int ix, iy, iz;
    coords(g, j, ix, iy, iz);
    const float W = (float)weight(g, ix, iy, iz);
    const float ih2 = (float)(1.0 / (g.h * g.h));
    LdM<float> f{x, mask};
    r[j] = b[j] - W * ih2 * lap_t<2, float>(g, f, j, ix, iy, iz);
}

// b_c[J] = sum over fine nodes i with |i - 2J|_inf <= 1 of prod_a (1 or 1/2) r_f[i].
__global__ void __launch_bounds__(kT) k_restrict(Geom gf, const float* __restrict__ rf, Geom gc,
                                                 const unsigned char* __restrict__ maskc, float* __restrict__ bc) {
    const long long J = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (J >= gc.np) return;
    if (maskc && maskc[J]) {
        bc[J] = 0.f;
        return;
    }
    int jx, jy, jz;
    coords(gc, J, jx, jy, jz);
    const int cx = 2 * jx, cy = 2 * jy, cz = 2 * jz;
    float acc = 0.f;
    const int zlo = gf.dim == 3 ? -1 : 0, zhi = gf.dim == 3 ? 1 : 0;
    for (int dz = zlo; dz <= zhi; ++dz) {
        const int fz = cz + dz;
        if (fz < 0 || fz > gf.nz) continue;
        const float wz = dz == 0 ? 1.f : 0.5f;
        for (int dy = -1; dy <= 1; ++dy) {
            const int fy = cy + dy;
            if (fy < 0 || fy > gf.ny) continue;
            const float wy = dy == 0 ? 1.f : 0.5f;
            for (int dx = -1; dx <= 1; ++dx) {
                const int fx = cx + dx;
                if (fx < 0 || fx > gf.nx) continue;
                const float wx = dx == 0 ? 1.f : 0.5f;
                acc += wx * wy * wz * rf[node(gf, fx, fy, fz)];
            }
        }
    }
    bc[J] = acc;
}

// x_f[i] += interpolated x_c.
__global__ void __launch_bounds__(kT) k_prolong_add(Geom gc, const float* __restrict__ xc, Geom gf,
                                                    const unsigned char* __restrict__ maskf, float* __restrict__ xf) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= gf.np) return;
    if (maskf && maskf[i]) return;
    int ix, iy, iz;
    coords(gf, i, ix, iy, iz);
    const int x0 = ix >> 1, x1 = (ix + 1) >> 1;
    const int y0 = iy >> 1, y1 = (iy + 1) >> 1;
    const int z0 = iz >> 1, z1 = (iz + 1) >> 1;
    float v;
    if (gf.dim == 3) {
        v = 0.125f * (xc[node(gc, x0, y0, z0)] + xc[node(gc, x1, y0, z0)] + xc[node(gc, x0, y1, z0)] +
                      xc[node(gc, x1, y1, z0)] + xc[node(gc, x0, y0, z1)] + xc[node(gc, x1, y0, z1)] +
                      xc[node(gc, x0, y1, z1)] + xc[node(gc, x1, y1, z1)]);
    } else {
        v = 0.25f * (xc[node(gc, x0, y0, 0)] + xc[node(gc, x1, y0, 0)] + xc[node(gc, x0, y1, 0)] +
                     xc[node(gc, x1, y1, 0)]);
    }
    xf[i] += v;
}

__global__ void k_coarsen_mask(Geom gf, const unsigned char* __restrict__ mf, Geom gc, unsigned char* __restrict__ mc) {
    const long long J = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (J >= gc.np) return;
    int jx, jy, jz;
    coords(gc, J, jx, jy, jz);
    mc[J] = mf[node(gf, 2 * jx, 2 * jy, 2 * jz)];
}

// Coarsest level: damped Jacobi sweeps in shared memory inside one block.
__global__ void __launch_bounds__(1024) k_coarse(Geom g, const unsigned char* __restrict__ mask, float* __restrict__ xg,
                                                 const float* __restrict__ b, int sweeps, float omega) {
    extern __shared__ float sm[];
    float* x = sm;
    float* xn = sm + g.np;
    const float h2 = (float)(g.h * g.h);
    const float twod = (float)(2 * g.dim);
    for (long long j = threadIdx.x; j < g.np; j += blockDim.x) x[j] = 0.f;
    __syncthreads();
    for (int s = 0; s < sweeps; ++s) {
        for (long long j = threadIdx.x; j < g.np; j += blockDim.x) {
            if (mask && mask[j]) {
                xn[j] = 0.f;
                continue;
            }
            int ix, iy, iz;
            coords(g, j, ix, iy, iz);
            const float W = (float)weight(g, ix, iy, iz);
            LdM<float> f{x, mask};
            const float L = lap_t<2, float>(g, f, j, ix, iy, iz);
            xn[j] = x[j] + omega * (h2 * b[j] / W - L) / twod;
        }
        __syncthreads();
        for (long long j = threadIdx.x; j < g.np; j += blockDim.x) x[j] = xn[j];
        __syncthreads();
    }
    for (long long j = threadIdx.x; j < g.np; j += blockDim.x) xg[j] = x[j];
}

// ---- FP64 PCG pieces ----------------------------------------------------------------------
// y = K x (masked); optional dot(dotwith, y) into sc[slot].
template <int ORDER>
__global__ void __launch_bounds__(kT) k_applyK(Geom g, const unsigned char* __restrict__ mask,
                                               const double* __restrict__ x, double* __restrict__ y,
                                               const double* __restrict__ dotwith, Red red, int slot) {
    double acc[1] = {0.0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    const double ih2 = 1.0 / (g.h * g.h);
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < g.np; j += stride) {
        if (mask && mask[j]) {
            y[j] = 0.0;
            continue;
        }
        int ix, iy, iz;
        coords(g, j, ix, iy, iz);
        LdM<double> f{x, mask};
        const double v = weight(g, ix, iy, iz) * ih2 * lap_t<ORDER, double>(g, f, j, ix, iy, iz);
        y[j] = v;
        if (dotwith) acc[0] += dotwith[j] * v;
    }
    if (dotwith) {
        if (grid_sum<1>(acc, red.partials, red.ticket) && threadIdx.x == 0) red.sc[slot] = acc[0];
    }
}

__global__ void k_to_float(long long n, const double* __restrict__ in, float* __restrict__ out) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) out[j] = (float)in[j];
}

__global__ void __launch_bounds__(kT) k_reduce_sum(long long n, const double* __restrict__ x, Red red, int slot) {
    double acc[1] = {0.0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) acc[0] += x[j];
    if (grid_sum<1>(acc, red.partials, red.ticket) && threadIdx.x == 0) red.sc[slot] = acc[0];
}

// b = rhs - (sum rhs / volume) W (range projection when K is singular), masked; ||b||^2.
__global__ void __launch_bounds__(kT) k_project(Geom g, const double* __restrict__ in, double* __restrict__ out,
                                                const unsigned char* __restrict__ mask, double inv_volume,
                                                int project, Red red) {
    const double mu = project ? red.sc[SC_P_BSUM] * inv_volume : 0.0;
    double acc[1] = {0.0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < g.np; j += stride) {
        double v = 0.0;
        if (!(mask && mask[j])) {
            v = in[j];
            if (project) {
                int ix, iy, iz;
                coords(g, j, ix, iy, iz);
                v -= mu * weight(g, ix, iy, iz);
            }
        }
        out[j] = v;
        acc[0] += v * v;
    }
    if (grid_sum<1>(acc, red.partials, red.ticket) && threadIdx.x == 0) red.sc[SC_P_BB] = acc[0];
}

// After the preconditioner: zd = z (FP64), rz = r.z, zAp = z.Ap; flexible (Polak-Ribiere)
// beta = (z_new . (r_new - r_old)) / rz_old = -alpha zAp / rz_old.
__global__ void __launch_bounds__(kT) k_dots_after_precond(long long n, const double* __restrict__ r,
                                                           const float* __restrict__ z, const double* __restrict__ Ap,
                                                           double* __restrict__ zd, Red red, int first) {
    double acc[2] = {0.0, 0.0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        const double zz = (double)z[j];
        zd[j] = zz;
        acc[0] += r[j] * zz;
        if (!first) acc[1] += zz * Ap[j];
    }
    if (grid_sum<2>(acc, red.partials, red.ticket) && threadIdx.x == 0) {
        const double rz_old = red.sc[SC_P_RZ];
        // a zero residual (zero right-hand side) gives rz = 0: no direction update
        red.sc[SC_P_BETA] = (first || rz_old == 0.0) ? 0.0 : -red.sc[SC_P_ALPHA] * acc[1] / rz_old;
        red.sc[SC_P_RZ] = acc[0];
    }
}

__global__ void k_p_update(long long n, double* __restrict__ p, const double* __restrict__ zd,
                           const double* __restrict__ sc, int first) {
    const double beta = first ? 0.0 : sc[SC_P_BETA];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride)
        p[j] = first ? zd[j] : zd[j] + beta * p[j];
}

// alpha = rz / pAp; x += alpha p; r -= alpha Ap; rr = r.r.
__global__ void __launch_bounds__(kT) k_xr_update(long long n, double* __restrict__ x, double* __restrict__ r,
                                                  const double* __restrict__ p, const double* __restrict__ Ap, Red red) {
    const double pap = red.sc[SC_P_PAP];
    const double alpha = pap != 0.0 ? red.sc[SC_P_RZ] / pap : 0.0;  // p = 0 only for a zero residual
    double acc[1] = {0.0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        x[j] += alpha * p[j];
        const double rv = r[j] - alpha * Ap[j];
        r[j] = rv;
        acc[0] += rv * rv;
    }
    if (grid_sum<1>(acc, red.partials, red.ticket) && threadIdx.x == 0) {
        red.sc[SC_P_ALPHA] = alpha;
        red.sc[SC_P_RR] = acc[0];
    }
}

// x -= (sum W x / volume): W-weighted mean zero.
__global__ void __launch_bounds__(kT) k_wsum(Geom g, const double* __restrict__ x, Red red) {
    double acc[1] = {0.0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < g.np; j += stride) {
        int ix, iy, iz;
        coords(g, j, ix, iy, iz);
        acc[0] += weight(g, ix, iy, iz) * x[j];
    }
    if (grid_sum<1>(acc, red.partials, red.ticket) && threadIdx.x == 0) red.sc[SC_P_XW] = acc[0];
}

__global__ void k_sub_const(long long n, double* __restrict__ x, const double* __restrict__ sc, double inv_volume) {
    const double mu = sc[SC_P_XW] * inv_volume;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) x[j] -= mu;
}

}  // namespace

void launch_mg_coarsen_mask(const MGLevel& fine, const MGLevel& coarse, cudaStream_t st) {
    note_launch((fine.mask && coarse.mask) ? 1 : 0);
    if (!fine.mask || !coarse.mask) return;
    k_coarsen_mask<<<node_blocks(coarse.g.np), kT, 0, st>>>(fine.g, fine.mask, coarse.g, coarse.mask);
}

void launch_mg_jacobi(const MGLevel& L, const float* xin, float* xout, const float* b, float omega, bool zero_init,
                      cudaStream_t st) {
    note_launch(1);
    k_jacobi<<<node_blocks(L.g.np), kT, 0, st>>>(L.g, L.mask, xin, xout, b, omega, zero_init ? 1 : 0);
}

void launch_mg_residual(const MGLevel& L, const float* x, const float* b, float* r, cudaStream_t st) {
    note_launch(1);
    k_residual<<<node_blocks(L.g.np), kT, 0, st>>>(L.g, L.mask, x, b, r);
}

void launch_mg_restrict(const MGLevel& fine, const float* rf, const MGLevel& coarse, float* bc, cudaStream_t st) {
    note_launch(1);
    k_restrict<<<node_blocks(coarse.g.np), kT, 0, st>>>(fine.g, rf, coarse.g, coarse.mask, bc);
}

void launch_mg_prolong_add(const MGLevel& coarse, const float* xc, const MGLevel& fine, float* xf, cudaStream_t st) {
    note_launch(1);
    k_prolong_add<<<node_blocks(fine.g.np), kT, 0, st>>>(coarse.g, xc, fine.g, fine.mask, xf);
}

int mg_coarse_max_nodes() { return kCoarseMax; }

void launch_mg_coarse_solve(const MGLevel& L, float* x, const float* b, int sweeps, float omega, cudaStream_t st) {
    note_launch(1);
    const size_t smem = 2 * (size_t)L.g.np * sizeof(float);
    k_coarse<<<1, 1024, smem, st>>>(L.g, L.mask, x, b, sweeps, omega);
}

void launch_applyK(const Geom& g, int order, const unsigned char* mask, const double* x, double* y,
                   const double* dotwith, Red red, int slot, cudaStream_t st) {
    note_launch(1);
    if (order == 2)
        k_applyK<2><<<vec_blocks(g.np), kT, 0, st>>>(g, mask, x, y, dotwith, red, slot);
    else
        k_applyK<4><<<vec_blocks(g.np), kT, 0, st>>>(g, mask, x, y, dotwith, red, slot);
}

void launch_to_float(long long n, const double* in, float* out, cudaStream_t st) {
    note_launch(1);
    k_to_float<<<vec_blocks(n), kT, 0, st>>>(n, in, out);
}

void launch_reduce_sum(long long n, const double* x, Red red, int slot, cudaStream_t st) {
    note_launch(1);
    k_reduce_sum<<<vec_blocks(n), kT, 0, st>>>(n, x, red, slot);
}

void launch_pcg_project(const Geom& g, const double* in, double* out, const unsigned char* mask, double volume,
                        Red red, bool project, cudaStream_t st) {
    note_launch(1);  // plus launch_reduce_sum's own count
    if (project) launch_reduce_sum(g.np, in, red, SC_P_BSUM, st);
    k_project<<<vec_blocks(g.np), kT, 0, st>>>(g, in, out, mask, 1.0 / volume, project ? 1 : 0, red);
}

void launch_pcg_dots_after_precond(long long n, const double* r, const float* z, const double* Ap, double* zd,
                                   Red red, cudaStream_t st) {
    note_launch(1);
    // "first" is encoded by Ap == nullptr
    k_dots_after_precond<<<vec_blocks(n), kT, 0, st>>>(n, r, z, Ap, zd, red, Ap == nullptr ? 1 : 0);
}

void launch_pcg_xr_update(long long n, double* x, double* r, const double* p, const double* Ap, Red red,
                          cudaStream_t st) {
    note_launch(1);
    k_xr_update<<<vec_blocks(n), kT, 0, st>>>(n, x, r, p, Ap, red);
}

void launch_pcg_p_update(long long n, double* p, const double* zd, Red red, bool first, cudaStream_t st) {
    note_launch(1);
    k_p_update<<<vec_blocks(n), kT, 0, st>>>(n, p, zd, red.sc, first ? 1 : 0);
}

void launch_mean_remove(const Geom& g, double* x, double volume, Red red, cudaStream_t st) {
    note_launch(2);
    k_wsum<<<vec_blocks(g.np), kT, 0, st>>>(g, x, red);
    k_sub_const<<<vec_blocks(g.np), kT, 0, st>>>(g.np, x, red.sc, 1.0 / volume);
}

}  // namespace cmcg
