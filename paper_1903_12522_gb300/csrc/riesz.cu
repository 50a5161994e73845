// Riesz map of Eq. CMCG_PRECONDITIONIER: K s = rhs with K = W (-Lap_h) (the discrete
// (grad s, grad phi)), solved matrix-free on the GPU.  The paper solves this SPD,
// omega-independent problem with a two-level Schwarz method (Sec. 4.3); here it is FP64
// flexible PCG whose preconditioner is one geometric multigrid V-cycle in FP32:
//   - vertex-centred coarsening n -> ceil(n/2) per axis (nested 2:1 for even n, general
//     linear interpolation for odd n), rediscretised K on each level, Dirichlet mask taken
//     from the nearest fine node;
//   - damped Jacobi smoothing, residual restriction by the transpose of (bi/tri)linear
//     interpolation, prolongation by that interpolation;
//   - the levels below kBlockMaxNodes nodes run as one V-cycle inside one thread block in
//     shared memory; its coarsest level is solved by Jacobi sweeps.
#include <math.h>

#include "common.cuh"
#include "kernels.h"

namespace cmcg {

namespace {

constexpr int kT = 256;

inline unsigned vec_blocks(long long n) {
    long long b = (n + kT - 1) / kT;
    if (b > kMaxBlocksReduce) b = kMaxBlocksReduce;
    if (b < 1) b = 1;
    return (unsigned)b;
}

inline unsigned node_blocks(long long n) { return (unsigned)((n + kT - 1) / kT); }

inline dim3 mg_grid(const Geom& g, int zc) {
    const long long plane = (long long)g.sx * g.sy;
    return dim3((unsigned)((plane + kT - 1) / kT), (unsigned)((g.sz + zc - 1) / zc), 1);
}

template <typename R>
struct Ld {
    const R* __restrict__ p;
    __device__ __forceinline__ R operator()(long long i) const { return p[i]; }
};

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
// K-form on every level: K = (h^d / h^2) s Lt with s = prod_a w(j_a) in {1, 1/2, 1/4, 1/8};
// diag K = (h^d / h^2) s 2d.  Damped Jacobi: x += omega (b - K x) / diag K.
// Iterates are kept exactly 0 on Dirichlet nodes, so neighbour loads need no mask.
__device__ __forceinline__ int axis_ends(const Geom& g, int ix, int iy, int iz) {
    int e = (ix == 0 || ix == g.nx) + (iy == 0 || iy == g.ny);
    if (g.dim == 3) e += (iz == 0 || iz == g.nz);
    return e;
}

struct MGConst {
    float cK;     // h^d / h^2
    float cB;     // h^2 / (2d h^d)
    float inv2d;  // 1 / (2d)
};

__device__ __forceinline__ MGConst mg_const(const Geom& g) {
    MGConst c;
    const float h = (float)g.h;
    const float hd = g.dim == 3 ? h * h * h : h * h;
    c.cK = hd / (h * h);
    c.inv2d = 1.f / (float)(2 * g.dim);
    c.cB = (h * h) / (hd * (float)(2 * g.dim));
    return c;
}

// One damped Jacobi update at node j (xin == nullptr: from x = 0).
__device__ __forceinline__ float jacobi_node(const Geom& g, const MGConst& c, const float* xin, float bj, float omega,
                                             long long j, int ix, int iy, int iz) {
    const float inv_s = (float)(1 << axis_ends(g, ix, iy, iz));
    if (!xin) return omega * c.cB * inv_s * bj;
    Ld<float> f{xin};
    const float L = lap_t<2, float>(g, f, j, ix, iy, iz);
    return xin[j] + omega * (c.cB * inv_s * bj - c.inv2d * L);
}

__device__ __forceinline__ float residual_node(const Geom& g, const MGConst& c, const float* x, float bj, long long j,
                                               int ix, int iy, int iz) {
    const float s = 1.f / (float)(1 << axis_ends(g, ix, iy, iz));
    Ld<float> f{x};
    return bj - c.cK * s * lap_t<2, float>(g, f, j, ix, iy, iz);
}

// Coarsening n_f -> n_c = ceil(n_f / 2) per axis: fine node i sits at coarse coordinate
// xi = i n_c / n_f; it interpolates from coarse nodes J0 = floor(xi) (weight 1 - t) and
// J0 + 1 (weight t), t = xi - J0.  For even n_f this is the nested 2:1 scheme (t in {0, 1/2}).
// Restriction is the exact transpose of this interpolation.
struct Interp1 {
    int j0;
    float t;
};

__device__ __forceinline__ Interp1 interp1(int i, int nf, int nc) {
    const long long num = (long long)i * nc;
    Interp1 r;
    r.j0 = (int)(num / nf);
    r.t = (float)(num - (long long)r.j0 * nf) / (float)nf;
    if (r.j0 >= nc) {
        r.j0 = nc;
        r.t = 0.f;
    }
    return r;
}

// weight with which fine node i contributes to coarse node J along one axis
__device__ __forceinline__ float interp_weight(int i, int J, int nf, int nc) {
    const Interp1 p = interp1(i, nf, nc);
    if (p.j0 == J) return 1.f - p.t;
    if (p.j0 + 1 == J) return p.t;
    return 0.f;
}

__device__ __forceinline__ void fine_range(int J, int nf, int nc, int& lo, int& hi) {
    // fine nodes whose interpolation stencil can include coarse node J
    lo = (int)(((long long)(J - 1) * nf) / nc);
    hi = (int)(((long long)(J + 1) * nf + nc - 1) / nc);
    lo = lo < 0 ? 0 : lo;
    hi = hi > nf ? nf : hi;
}

__device__ __forceinline__ bool nested(const Geom& gf, const Geom& gc) {
    return gf.nx == 2 * gc.nx && gf.ny == 2 * gc.ny && (gf.dim == 2 || gf.nz == 2 * gc.nz);
}

// nested 2:1 case: weights 1 at 2J and 1/2 at 2J +- 1 per axis
__device__ __forceinline__ float restrict_nested(const Geom& gf, const float* rf, int jx, int jy, int jz) {
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
            const float* row = rf + node(gf, 0, fy, fz);
            float racc = row[cx];
            if (cx > 0) racc += 0.5f * row[cx - 1];
            if (cx < gf.nx) racc += 0.5f * row[cx + 1];
            acc += wy * wz * racc;
        }
    }
    return acc;
}

__device__ __forceinline__ float restrict_node(const Geom& gf, const Geom& gc, const float* rf, int jx, int jy,
                                               int jz) {
    if (nested(gf, gc)) return restrict_nested(gf, rf, jx, jy, jz);
    int xlo, xhi, ylo, yhi, zlo = 0, zhi = 0;
    fine_range(jx, gf.nx, gc.nx, xlo, xhi);
    fine_range(jy, gf.ny, gc.ny, ylo, yhi);
    if (gf.dim == 3) fine_range(jz, gf.nz, gc.nz, zlo, zhi);
    float acc = 0.f;
    for (int fz = zlo; fz <= zhi; ++fz) {
        const float wz = gf.dim == 3 ? interp_weight(fz, jz, gf.nz, gc.nz) : 1.f;
        if (wz == 0.f) continue;
        for (int fy = ylo; fy <= yhi; ++fy) {
            const float wy = interp_weight(fy, jy, gf.ny, gc.ny);
            if (wy == 0.f) continue;
            for (int fx = xlo; fx <= xhi; ++fx) {
                const float wx = interp_weight(fx, jx, gf.nx, gc.nx);
                if (wx == 0.f) continue;
                acc += wx * wy * wz * rf[node(gf, fx, fy, fz)];
            }
        }
    }
    return acc;
}

__device__ __forceinline__ Interp1 interp1_fast(int i, int nf, int nc) {
    if (nf == 2 * nc) {
        Interp1 r;
        r.j0 = i >> 1;
        r.t = (i & 1) ? 0.5f : 0.f;
        return r;
    }
    return interp1(i, nf, nc);
}

__device__ __forceinline__ float prolong_node(const Geom& gc, const float* xc, const Geom& gf, int ix, int iy, int iz) {
    const Interp1 px = interp1_fast(ix, gf.nx, gc.nx), py = interp1_fast(iy, gf.ny, gc.ny);
    const int x1 = px.t > 0.f ? px.j0 + 1 : px.j0, y1 = py.t > 0.f ? py.j0 + 1 : py.j0;
    const float ax = 1.f - px.t, ay = 1.f - py.t;
    float v = ay * (ax * xc[node(gc, px.j0, py.j0, 0)] + px.t * xc[node(gc, x1, py.j0, 0)]) +
              py.t * (ax * xc[node(gc, px.j0, y1, 0)] + px.t * xc[node(gc, x1, y1, 0)]);
    if (gf.dim == 3) {
        const Interp1 pz = interp1_fast(iz, gf.nz, gc.nz);
        const int z1 = pz.t > 0.f ? pz.j0 + 1 : pz.j0;
        const long long offz0 = (long long)pz.j0 * gc.sx * gc.sy, offz1 = (long long)z1 * gc.sx * gc.sy;
        const float* c0 = xc + offz0;
        const float* c1 = xc + offz1;
        const float v0 = ay * (ax * c0[node(gc, px.j0, py.j0, 0)] + px.t * c0[node(gc, x1, py.j0, 0)]) +
                         py.t * (ax * c0[node(gc, px.j0, y1, 0)] + px.t * c0[node(gc, x1, y1, 0)]);
        const float v1 = ay * (ax * c1[node(gc, px.j0, py.j0, 0)] + px.t * c1[node(gc, x1, py.j0, 0)]) +
                         py.t * (ax * c1[node(gc, px.j0, y1, 0)] + px.t * c1[node(gc, x1, y1, 0)]);
        v = (1.f - pz.t) * v0 + pz.t * v1;
    }
    return v;
}

struct PlaneIt {
    int ix, iy, z0, z1;
    bool valid;
};

__device__ __forceinline__ PlaneIt plane_it(const Geom& g, int zc) {
    PlaneIt m;
    const unsigned plane = (unsigned)g.sx * (unsigned)g.sy;
    const unsigned p = blockIdx.x * blockDim.x + threadIdx.x;
    m.valid = p < plane;
    const unsigned pp = m.valid ? p : 0u;
    m.iy = (int)(pp / (unsigned)g.sx);
    m.ix = (int)(pp - (unsigned)m.iy * (unsigned)g.sx);
    m.z0 = blockIdx.y * zc;
    m.z1 = min(m.z0 + zc, g.sz);
    if (m.valid && !column_in_range(g, m.ix, m.iy, m.z0, m.z1, 1, kSiteMultigrid)) m.valid = false;
    return m;
}

__global__ void __launch_bounds__(kT) k_jacobi(Geom g, const unsigned char* __restrict__ mask,
                                               const float* __restrict__ xin, float* __restrict__ xout,
                                               const float* __restrict__ b, float omega, int zc) {
    const PlaneIt m = plane_it(g, zc);
    if (!m.valid) return;
    const MGConst c = mg_const(g);
    for (int iz = m.z0; iz < m.z1; ++iz) {
        const long long j = node(g, m.ix, m.iy, iz);
        // the mask, b and the stencil are loaded together and the mask selects at the end: a
        // branch on the mask byte would put its load's latency before every other load
        const bool dir = mask && mask[j];
        const float v = jacobi_node(g, c, xin, b[j], omega, j, m.ix, m.iy, iz);
        xout[j] = dir ? 0.f : v;
    }
}

__global__ void __launch_bounds__(kT) k_residual(Geom g, const unsigned char* __restrict__ mask,
                                                 const float* __restrict__ x, const float* __restrict__ b,
                                                 float* __restrict__ r, int zc) {
    const PlaneIt m = plane_it(g, zc);
    if (!m.valid) return;
    const MGConst c = mg_const(g);
    for (int iz = m.z0; iz < m.z1; ++iz) {
        const long long j = node(g, m.ix, m.iy, iz);
        const bool dir = mask && mask[j];  // selected at the end (see k_jacobi)
        const float v = residual_node(g, c, x, b[j], j, m.ix, m.iy, iz);
        r[j] = dir ? 0.f : v;
    }
}

// 3D Jacobi sweep (from a given x) and residual, two z-planes per loop trip: both planes' loads
// (x with its x/y neighbours, b, the mask byte) are issued before either update, and the
// z-neighbours come from registers.  The expressions are those of jacobi_node / residual_node
// with the 7-point Laplacian summed in lap_t's order, so the results are bitwise equal to
// k_jacobi / k_residual.
struct Col3 {
    long long sZ, oxm, oxp, oym, oyp;
    int exy;  // axis ends of the column in x and y
};

__device__ __forceinline__ Col3 col3(const Geom& g, int ix, int iy) {
    Col3 c;
    c.sZ = (long long)g.sx * g.sy;
    c.oxm = off_m1(ix, 1);
    c.oxp = off_p1(ix, g.nx, 1);
    c.oym = off_m1(iy, g.sx);
    c.oyp = off_p1(iy, g.ny, g.sx);
    c.exy = (ix == 0 || ix == g.nx) + (iy == 0 || iy == g.ny);
    return c;
}

// MODE 0: Jacobi x_out = x + omega (cB s^-1 b - L / 6); MODE 1: residual r = b - cK s L.
template <int MODE>
__global__ void __launch_bounds__(kT) k_mg3_z2(Geom g, const unsigned char* __restrict__ mask,
                                               const float* __restrict__ x, const float* __restrict__ b,
                                               float* __restrict__ out, float omega, int zc) {
    const PlaneIt m = plane_it(g, zc);
    if (!m.valid || m.z0 >= m.z1) return;
    const MGConst c = mg_const(g);
    const Col3 o = col3(g, m.ix, m.iy);
    const long long sZ = o.sZ;
    auto update = [&](float xc, float xm, float xp, float sx, float sy, long long jj, int iz, float bj, bool dir) {
        float acc = sx;
        acc += sy;
        acc += xm + xp;
        const float L = 6.f * xc - acc;
        const int e = o.exy + (iz == 0 || iz == g.nz);
        float v;
        if (MODE == 0) {
            const float inv_s = (float)(1 << e);
            v = xc + omega * (c.cB * inv_s * bj - c.inv2d * L);
        } else {
            const float s = 1.f / (float)(1 << e);
            v = bj - c.cK * s * L;
        }
        out[jj] = dir ? 0.f : v;
    };
    long long j = node(g, m.ix, m.iy, m.z0);
    float xm = x[j + (m.z0 > 0 ? -sZ : sZ)];
    float xc = x[j];
    int iz = m.z0;
    for (; iz + 1 < m.z1; iz += 2) {
        const long long j1 = j + sZ;
        const float x1 = x[j1];                               // plane iz+1 (exists: iz+1 < z1 <= sz)
        const float x2 = x[j1 + (iz + 1 < g.nz ? sZ : -sZ)];  // plane iz+2 (mirrored at the top)
        const float sx0 = x[j + o.oxm] + x[j + o.oxp], sy0 = x[j + o.oym] + x[j + o.oyp];
        const float sx1 = x[j1 + o.oxm] + x[j1 + o.oxp], sy1 = x[j1 + o.oym] + x[j1 + o.oyp];
        const float b0 = b[j], b1 = b[j1];
        const bool d0 = mask && mask[j], d1 = mask && mask[j1];
        update(xc, xm, x1, sx0, sy0, j, iz, b0, d0);
        update(x1, xc, x2, sx1, sy1, j1, iz + 1, b1, d1);
        xm = x1;
        xc = x2;
        j += 2 * sZ;
    }
    if (iz < m.z1) {
        const float xp = x[j + (iz < g.nz ? sZ : -sZ)];
        const float sx0 = x[j + o.oxm] + x[j + o.oxp], sy0 = x[j + o.oym] + x[j + o.oyp];
        update(xc, xm, xp, sx0, sy0, j, iz, b[j], mask && mask[j]);
    }
}

// 3D prolongation x_f += P x_c along a thread's fine z-column.  Every fine plane blends the
// xy-interpolated values of at most two coarse planes; those are kept in registers and
// reused by the next fine plane (for 2:1 coarsening, one new coarse plane per two fine
// planes).  Same expressions as prolong_node: bitwise equal to k_prolong_add.
__global__ void __launch_bounds__(kT) k_prolong_add3(Geom gc, const float* __restrict__ xc, Geom gf,
                                                     const unsigned char* __restrict__ maskf, float* __restrict__ xf,
                                                     int zc) {
    const PlaneIt m = plane_it(gf, zc);
    if (!m.valid || m.z0 >= m.z1) return;
    const Interp1 px = interp1_fast(m.ix, gf.nx, gc.nx), py = interp1_fast(m.iy, gf.ny, gc.ny);
    const int x1 = px.t > 0.f ? px.j0 + 1 : px.j0, y1 = py.t > 0.f ? py.j0 + 1 : py.j0;
    const float ax = 1.f - px.t, ay = 1.f - py.t;
    const long long o00 = node(gc, px.j0, py.j0, 0), o10 = node(gc, x1, py.j0, 0);
    const long long o01 = node(gc, px.j0, y1, 0), o11 = node(gc, x1, y1, 0);
    const long long planeC = (long long)gc.sx * gc.sy;
    auto pxy = [&](int J) {
        const float* cp = xc + (long long)J * planeC;
        return ay * (ax * cp[o00] + px.t * cp[o10]) + py.t * (ax * cp[o01] + px.t * cp[o11]);
    };
    int ja = -1, jb = -1;  // coarse planes held in va, vb
    float va = 0.f, vb = 0.f;
    for (int iz = m.z0; iz < m.z1; ++iz) {
        const long long i = node(gf, m.ix, m.iy, iz);
        const bool dir = maskf && maskf[i];  // tested at the store (see k_jacobi)
        const float x0 = xf[i];
        const Interp1 pz = interp1_fast(iz, gf.nz, gc.nz);  // the same for every thread of the block
        const int z1 = pz.t > 0.f ? pz.j0 + 1 : pz.j0;
        const float v0 = pz.j0 == jb ? vb : (pz.j0 == ja ? va : pxy(pz.j0));
        const float v1 = z1 == pz.j0 ? v0 : (z1 == jb ? vb : pxy(z1));
        ja = pz.j0;
        va = v0;
        jb = z1;
        vb = v1;
        const float v = (1.f - pz.t) * v0 + pz.t * v1;
        if (!dir) xf[i] = x0 + v;
    }
}

// 3D restriction for 2:1 coarsening along a thread's coarse z-column.  Coarse plane J gathers
// fine planes 2J-1, 2J, 2J+1; the x-weighted row sums of plane 2J+1 are kept in registers
// for plane J+1, so each coarse plane loads two fine planes.  Rows outside the grid are read
// at a clamped address and left out of the sum, so every load is issued before the sums.  The
// terms and their order are those of restrict_nested: bitwise equal to k_restrict.
__global__ void __launch_bounds__(kT) k_restrict3_nested(Geom gf, const float* __restrict__ rf, Geom gc,
                                                         const unsigned char* __restrict__ maskc,
                                                         float* __restrict__ bc, int zc) {
    const PlaneIt m = plane_it(gc, zc);
    if (!m.valid || m.z0 >= m.z1) return;
    const int cx = 2 * m.ix, cy = 2 * m.iy;
    const bool xm = cx > 0, xp = cx < gf.nx;
    const int xl = xm ? cx - 1 : cx, xr = xp ? cx + 1 : cx;
    bool yok[3];
    long long yoff[3];
    for (int d = 0; d < 3; ++d) {
        const int fy = cy + d - 1;
        yok[d] = fy >= 0 && fy <= gf.ny;
        yoff[d] = (long long)(yok[d] ? fy : cy) * gf.sx;
    }
    const long long sZ = (long long)gf.sx * gf.sy;
    auto rows = [&](int fz, float* r) {  // row sums of fine plane fz (0 <= fz <= nz)
        const float* pl = rf + (long long)fz * sZ;
        float a[3], l[3], q[3];
        for (int d = 0; d < 3; ++d) {
            a[d] = pl[yoff[d] + cx];
            l[d] = pl[yoff[d] + xl];
            q[d] = pl[yoff[d] + xr];
        }
        for (int d = 0; d < 3; ++d) {
            float racc = a[d];
            if (xm) racc += 0.5f * l[d];
            if (xp) racc += 0.5f * q[d];
            r[d] = racc;
        }
    };
    float lo[3] = {0.f, 0.f, 0.f};  // row sums of fine plane 2J - 1
    bool have_lo = false;
    for (int jz = m.z0; jz < m.z1; ++jz) {
        const long long J = node(gc, m.ix, m.iy, jz);
        const bool dir = maskc && maskc[J];
        const int cz = 2 * jz;
        const bool zlo = cz - 1 >= 0, zhi = cz + 1 <= gf.nz;
        if (zlo && !have_lo) rows(cz - 1, lo);
        float mid[3], hi[3] = {0.f, 0.f, 0.f};
        rows(cz, mid);
        if (zhi) rows(cz + 1, hi);
        float acc = 0.f;
        if (zlo)
            for (int d = 0; d < 3; ++d)
                if (yok[d]) acc += (d == 1 ? 1.f : 0.5f) * 0.5f * lo[d];
        for (int d = 0; d < 3; ++d)
            if (yok[d]) acc += (d == 1 ? 1.f : 0.5f) * 1.f * mid[d];
        if (zhi)
            for (int d = 0; d < 3; ++d)
                if (yok[d]) acc += (d == 1 ? 1.f : 0.5f) * 0.5f * hi[d];
        bc[J] = dir ? 0.f : acc;
        for (int d = 0; d < 3; ++d) lo[d] = hi[d];
        have_lo = zhi;
    }
}

// b_c[J] = sum over fine nodes i with |i - 2J|_inf <= 1 of prod_a (1 or 1/2) r_f[i].
__global__ void __launch_bounds__(kT) k_restrict(Geom gf, const float* __restrict__ rf, Geom gc,
                                                 const unsigned char* __restrict__ maskc, float* __restrict__ bc,
                                                 int zc) {
    const PlaneIt m = plane_it(gc, zc);
    if (!m.valid) return;
    for (int iz = m.z0; iz < m.z1; ++iz) {
        const long long J = node(gc, m.ix, m.iy, iz);
        const bool dir = maskc && maskc[J];  // selected at the end (see k_jacobi)
        const float v = restrict_node(gf, gc, rf, m.ix, m.iy, iz);
        bc[J] = dir ? 0.f : v;
    }
}

// x_f[i] += interpolated x_c.
__global__ void __launch_bounds__(kT) k_prolong_add(Geom gc, const float* __restrict__ xc, Geom gf,
                                                    const unsigned char* __restrict__ maskf, float* __restrict__ xf,
                                                    int zc) {
    const PlaneIt m = plane_it(gf, zc);
    if (!m.valid) return;
    for (int iz = m.z0; iz < m.z1; ++iz) {
        const long long i = node(gf, m.ix, m.iy, iz);
        const bool dir = maskf && maskf[i];  // tested at the store (see k_jacobi)
        const float v = prolong_node(gc, xc, gf, m.ix, m.iy, iz);
        const float x0 = xf[i];
        if (!dir) xf[i] = x0 + v;
    }
}

__global__ void k_coarsen_mask(Geom gf, const unsigned char* __restrict__ mf, Geom gc, unsigned char* __restrict__ mc) {
    const long long J = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (J >= gc.np) return;
    int jx, jy, jz;
    coords(gc, J, jx, jy, jz);
    // the fine node nearest to the coarse node's position
    const int fx = (int)(((long long)jx * gf.nx * 2 + gc.nx) / (2 * gc.nx));
    const int fy = (int)(((long long)jy * gf.ny * 2 + gc.ny) / (2 * gc.ny));
    const int fz = gf.dim == 3 ? (int)(((long long)jz * gf.nz * 2 + gc.nz) / (2 * gc.nz)) : 0;
    mc[J] = mf[node(gf, fx, fy, fz)];
}

// The coarse end of the V-cycle inside one thread block: levels 0..n-1 of BlockLevels live
// in shared memory (x, x2, b, r per level); b of the first level comes from global memory and
// its x goes back.  Same smoother, restriction and prolongation as the grid-wide kernels.
__device__ void blk_jacobi(const Geom& g, const unsigned char* mask, const float* xin, float* xout, const float* b,
                           float omega) {
    const MGConst c = mg_const(g);
    for (int j = threadIdx.x; j < (int)g.np; j += blockDim.x) {
        if (mask && mask[j]) {
            xout[j] = 0.f;
            continue;
        }
        int ix, iy, iz;
        coords(g, j, ix, iy, iz);
        xout[j] = jacobi_node(g, c, xin, b[j], omega, j, ix, iy, iz);
    }
    __syncthreads();
}

__global__ void __launch_bounds__(1024) k_block_vcycle(BlockLevels lv, const float* __restrict__ bglob,
                                                       float* __restrict__ xglob, float omega, int nu,
                                                       int coarse_sweeps) {
    extern __shared__ float sm[];
    float *x[kBlockLevelsMax], *x2[kBlockLevelsMax], *b[kBlockLevelsMax], *r[kBlockLevelsMax];
    {
        float* p = sm;
        for (int l = 0; l < lv.n; ++l) {
            const int np = (int)lv.g[l].np;
            x[l] = p;
            x2[l] = p + np;
            b[l] = p + 2 * np;
            r[l] = p + 3 * np;
            p += 4 * np;
        }
    }
    for (int j = threadIdx.x; j < (int)lv.g[0].np; j += blockDim.x) b[0][j] = bglob[j];
    __syncthreads();
    // descend
    for (int l = 0; l + 1 < lv.n; ++l) {
        const Geom& g = lv.g[l];
        blk_jacobi(g, lv.mask[l], nullptr, x[l], b[l], omega);
        for (int s = 1; s < nu; ++s) {
            blk_jacobi(g, lv.mask[l], x[l], x2[l], b[l], omega);
            float* t = x[l]; x[l] = x2[l]; x2[l] = t;
        }
        const MGConst c = mg_const(g);
        for (int j = threadIdx.x; j < (int)g.np; j += blockDim.x) {
            int ix, iy, iz;
            coords(g, j, ix, iy, iz);
            r[l][j] = (lv.mask[l] && lv.mask[l][j]) ? 0.f : residual_node(g, c, x[l], b[l][j], j, ix, iy, iz);
        }
        __syncthreads();
        const Geom& gc = lv.g[l + 1];
        for (int J = threadIdx.x; J < (int)gc.np; J += blockDim.x) {
            int jx, jy, jz;
            coords(gc, J, jx, jy, jz);
            b[l + 1][J] = (lv.mask[l + 1] && lv.mask[l + 1][J]) ? 0.f : restrict_node(g, gc, r[l], jx, jy, jz);
        }
        __syncthreads();
    }
    // coarsest
    {
        const int l = lv.n - 1;
        blk_jacobi(lv.g[l], lv.mask[l], nullptr, x[l], b[l], omega);
        for (int s = 1; s < coarse_sweeps; ++s) {
            blk_jacobi(lv.g[l], lv.mask[l], x[l], x2[l], b[l], omega);
            float* t = x[l]; x[l] = x2[l]; x2[l] = t;
        }
    }
    // ascend
    for (int l = lv.n - 2; l >= 0; --l) {
        const Geom& g = lv.g[l];
        const Geom& gc = lv.g[l + 1];
        for (int j = threadIdx.x; j < (int)g.np; j += blockDim.x) {
            if (lv.mask[l] && lv.mask[l][j]) continue;
            int ix, iy, iz;
            coords(g, j, ix, iy, iz);
            x[l][j] += prolong_node(gc, x[l + 1], g, ix, iy, iz);
        }
        __syncthreads();
        for (int s = 0; s < nu; ++s) {
            blk_jacobi(g, lv.mask[l], x[l], x2[l], b[l], omega);
            float* t = x[l]; x[l] = x2[l]; x2[l] = t;
        }
    }
    for (int j = threadIdx.x; j < (int)lv.g[0].np; j += blockDim.x) xglob[j] = x[0][j];
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
        Ld<double> f{x};  // PCG vectors are zero on Dirichlet nodes
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
    const int zc = L.g.dim == 3 ? 8 : 1;
    if (L.g.dim == 3 && !zero_init)
        k_mg3_z2<0><<<mg_grid(L.g, zc), kT, 0, st>>>(L.g, L.mask, xin, b, xout, omega, zc);
    else
        k_jacobi<<<mg_grid(L.g, zc), kT, 0, st>>>(L.g, L.mask, zero_init ? nullptr : xin, xout, b, omega, zc);
}

void launch_mg_residual(const MGLevel& L, const float* x, const float* b, float* r, cudaStream_t st) {
    note_launch(1);
    const int zc = L.g.dim == 3 ? 8 : 1;
    if (L.g.dim == 3)
        k_mg3_z2<1><<<mg_grid(L.g, zc), kT, 0, st>>>(L.g, L.mask, x, b, r, 0.f, zc);
    else
        k_residual<<<mg_grid(L.g, zc), kT, 0, st>>>(L.g, L.mask, x, b, r, zc);
}

void launch_mg_restrict(const MGLevel& fine, const float* rf, const MGLevel& coarse, float* bc, cudaStream_t st) {
    note_launch(1);
    const int zc = coarse.g.dim == 3 ? 4 : 1;
    const Geom& gf = fine.g;
    const Geom& gc = coarse.g;
    if (gf.dim == 3 && gf.nx == 2 * gc.nx && gf.ny == 2 * gc.ny && gf.nz == 2 * gc.nz)
        k_restrict3_nested<<<mg_grid(gc, zc), kT, 0, st>>>(gf, rf, gc, coarse.mask, bc, zc);
    else
        k_restrict<<<mg_grid(gc, zc), kT, 0, st>>>(gf, rf, gc, coarse.mask, bc, zc);
}

void launch_mg_prolong_add(const MGLevel& coarse, const float* xc, const MGLevel& fine, float* xf, cudaStream_t st) {
    note_launch(1);
    const int zc = fine.g.dim == 3 ? 8 : 1;
    if (fine.g.dim == 3)
        k_prolong_add3<<<mg_grid(fine.g, zc), kT, 0, st>>>(coarse.g, xc, fine.g, fine.mask, xf, zc);
    else
        k_prolong_add<<<mg_grid(fine.g, zc), kT, 0, st>>>(coarse.g, xc, fine.g, fine.mask, xf, zc);
}

int mg_block_max_nodes() { return kBlockMaxNodes; }

size_t mg_block_smem_bytes(const BlockLevels& lv) {
    size_t n = 0;
    for (int l = 0; l < lv.n; ++l) n += 4 * (size_t)lv.g[l].np;
    return n * sizeof(float);
}

void launch_mg_block_vcycle(const BlockLevels& lv, const float* b, float* x, float omega, int nu, int coarse_sweeps,
                            cudaStream_t st) {
    note_launch(1);
    const size_t smem = mg_block_smem_bytes(lv);
    cudaFuncSetAttribute(k_block_vcycle, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_block_vcycle<<<1, 1024, smem, st>>>(lv, b, x, omega, nu, coarse_sweeps);
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

namespace cmcg {
CMCG_CHECK_TU(riesz)
}  // namespace cmcg
