// Leapfrog period kernels: forward period (Eq. WE) and its exact transpose (the discrete
// adjoint wave equation, Eq. AWE), with the absorbing-boundary terms, the time-harmonic
// source and the period-end energy functional (Eq. cost_functional_J) fused in.
//
// Notation (all pointwise except Lt): kappa = c^2 dt^2 / h^2, beta = (dt/2) M^-1 B =
// nb sqrt(kappa) with nb the number of absorbing faces through the node, S = dt^2 M^-1 F^
// (complex), so dt^2 M^-1 F^n = Re(S exp(-i omega t_n)).  Dirichlet nodes have kappa = 0 and
// hold 0 in every field.
//
//   start : y1 = y0 + dt (1 - beta) v0 + (S_re - kappa Lt y0) / 2
//   step  : y^{n+1} = [2 y^n - (1 - beta) y^{n-1} - kappa Lt y^n + Re(S e^{-i w t_n})] / (1 + beta)
//   end   : vN = [(yN - yN-1)/dt + (Re(S e^{-i w T}) - kappa Lt yN) / (2 dt)] / (1 + beta)
//           e = (yN - w0, vN - w1),  z = E e = (W Lt e0 / h^2, M e1),  J = e.z / 2
// The adjoint runs the SAME step kernel backwards in time on primal-scaled cotangents
// u_n = D^-1 ybar_{n+1}:  D u_{n-1} = (2M - dt^2 K) u_n - C u_{n+1}, with two variants:
// PREV_SCALED (the first step's "previous" term is already C u / M) and NO_DIV (the last
// step returns s = (1 + beta) u_0 = M^-1 ybar_1, which the final kernel needs).
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace cmcg {

namespace {

constexpr int kThreads = 256;

struct PlaneMap {
    int ix, iy, z0, z1;
    bool valid;
};

// radius: the stencil's reach along each axis (the checked build tests the column's index
// range against the grid and drops a column that would leave it)
__device__ __forceinline__ PlaneMap plane_map(const Geom& g, int zc, int radius = 1) {
    PlaneMap m;
    const long long plane = (long long)g.sx * g.sy;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    m.valid = p < plane;
    const long long pp = m.valid ? p : 0;
    m.iy = (int)(pp / g.sx);
    m.ix = (int)(pp - (long long)m.iy * g.sx);
    m.z0 = blockIdx.y * zc;
    m.z1 = min(m.z0 + zc, g.sz);
    if (m.valid && !column_in_range(g, m.ix, m.iy, m.z0, m.z1, radius, kSiteColumn)) m.valid = false;
    return m;
}

template <typename T>
struct Ld {
    const T* __restrict__ p;
    __device__ __forceinline__ T operator()(long long i) const { return p[i]; }
};

template <typename T>
struct LdD {  // loads T, returns double
    const T* __restrict__ p;
    __device__ __forceinline__ double operator()(long long i) const { return (double)p[i]; }
};

template <typename T>
struct DiffT {  // a[i] - b[i] in T
    const T* __restrict__ a;
    const T* __restrict__ b;
    __device__ __forceinline__ T operator()(long long i) const { return a[i] - b[i]; }
};


// ---------------------------------------------------------------------------------------
// Leapfrog step, generic (any dim / order): one thread per (x, y) column, marching z.
template <typename T, int ORDER, int FLAGS>
__global__ void __launch_bounds__(kThreads) k_step(const T* __restrict__ cur, T* __restrict__ prev_out,
                                                   const T* __restrict__ kap, const T* __restrict__ S,
                                                   double cs, double sn, Geom g, int zc) {
    const PlaneMap m = plane_map(g, zc, ORDER / 2);
    if (!m.valid) return;
    Ld<T> f{cur};
    for (int iz = m.z0; iz < m.z1; ++iz) {
        const long long j = node(g, m.ix, m.iy, iz);
        const T L = lap_t<ORDER, T>(g, f, j, m.ix, m.iy, iz);
        const T k = kap[j];
        const T yp = prev_out[j];
        T rhs = T(2) * cur[j] - k * L;
        if (FLAGS & kStepSrc) rhs += S[2 * j] * (T)cs + S[2 * j + 1] * (T)sn;
        const int nb = num_abc(g, m.ix, m.iy, iz);
        T out;
        if (nb == 0) {
            out = rhs - yp;
        } else {
            const T beta = (T)nb * sqrt(k);
            const T v = rhs - ((FLAGS & kStepPrevScaled) ? yp : (T(1) - beta) * yp);
            out = (FLAGS & kStepNoDiv) ? v : v / (T(1) + beta);
        }
        prev_out[j] = out;
    }
}

// Fundamental-frequency filter of Sec. 2.2, fused into a forced forward period:
//   U = (1/N) sum_{n=0}^{N-1} (y^n + (i/wh) v^n) e^{i w t_n},  v^n = (y^{n+1} - y^{n-1}) / (2 dt)
// (rectangle rule; exact for the discrete time-harmonic solution, and the constant shift of
// Theorem 1 and the other harmonics drop out).  The step below is the forced leapfrog step
// that also adds its term n to the complex accumulator acc (interleaved re, im).
template <int ORDER>
__global__ void __launch_bounds__(kThreads) k_step_filter(const double* __restrict__ cur, double* __restrict__ prev_out,
                                                          const double* __restrict__ kap, const double* __restrict__ S,
                                                          double cs, double sn, double* __restrict__ acc, double fc,
                                                          double fs, double cv, Geom g, int zc) {
    const PlaneMap m = plane_map(g, zc, ORDER / 2);
    if (!m.valid) return;
    Ld<double> f{cur};
    for (int iz = m.z0; iz < m.z1; ++iz) {
        const long long j = node(g, m.ix, m.iy, iz);
        const double L = lap_t<ORDER, double>(g, f, j, m.ix, m.iy, iz);
        const double k = kap[j];
        const double yp = prev_out[j];
        const double yc = cur[j];
        const double rhs = 2.0 * yc - k * L + (S[2 * j] * cs + S[2 * j + 1] * sn);
        const int nb = num_abc(g, m.ix, m.iy, iz);
        double out;
        if (nb == 0) {
            out = rhs - yp;
        } else {
            const double beta = nb * sqrt(k);
            out = (rhs - (1.0 - beta) * yp) / (1.0 + beta);
        }
        prev_out[j] = out;
        const double a = yc, b = cv * (out - yp);  // y^n and v^n / wh
        acc[2 * j] += a * fc - b * fs;
        acc[2 * j + 1] += a * fs + b * fc;
    }
}

// Source columns: scol[x + sx y] = 1 if S != 0 at some node (x, y, z) with 0 < z < nz.  A
// boundary datum on the six faces of a box leaves only the x- and y-face columns flagged.
__global__ void k_source_columns(Geom g, const double* __restrict__ S, unsigned char* __restrict__ scol) {
    const long long plane = (long long)g.sx * g.sy;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < plane; c += stride) {
        bool any = false;
        for (int z = 1; z < g.nz && !any; ++z) {
            const long long j = c + plane * z;
            any = S[2 * j] != 0.0 || S[2 * j + 1] != 0.0;
        }
        scol[c] = any ? 1 : 0;
    }
}

// acc = w0 + i w1 / wh (the n = 0 term; zero on Dirichlet nodes).
__global__ void k_filter_init(long long n, const double* __restrict__ w0, const double* __restrict__ w1,
                              const double* __restrict__ kap64, double inv_wh, double* __restrict__ acc) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        const bool act = kap64[j] != 0.0;
        acc[2 * j] = act ? w0[j] : 0.0;
        acc[2 * j + 1] = act ? w1[j] * inv_wh : 0.0;
    }
}

__global__ void k_scale_complex(long long n, double* __restrict__ u, double s) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < 2 * n; j += stride) u[j] *= s;
}

// Leapfrog step, 3D 2nd order: z-neighbours carried in registers along the march.
template <typename T, int FLAGS>
__global__ void __launch_bounds__(kThreads) k_step3d7(const T* __restrict__ cur, T* __restrict__ prev_out,
                                                      const T* __restrict__ kap, const T* __restrict__ S,
                                                      double cs, double sn, Geom g, int zc,
                                                      const unsigned char* __restrict__ scol) {
    const PlaneMap m = plane_map(g, zc);
    if (!m.valid || m.z0 >= m.z1) return;
    const long long sZ = (long long)g.sx * g.sy;
    long long j = node(g, m.ix, m.iy, m.z0);
    const long long oxm = off_m1(m.ix, 1), oxp = off_p1(m.ix, g.nx, 1);
    const long long oym = off_m1(m.iy, g.sx), oyp = off_p1(m.iy, g.ny, g.sx);
    int nbxy = 0;
    nbxy += (m.ix == 0) & (int)(g.abc & 1u);
    nbxy += (m.ix == g.nx) & (int)((g.abc >> 1) & 1u);
    nbxy += (m.iy == 0) & (int)((g.abc >> 2) & 1u);
    nbxy += (m.iy == g.ny) & (int)((g.abc >> 3) & 1u);
    // a column without source inside the grid (0 < z < nz) reads S only on its two z-faces
    const bool col_src = !(FLAGS & kStepSrc) || !scol || scol[m.ix + (long long)g.sx * m.iy];
    T ym = cur[j + (m.z0 > 0 ? -sZ : sZ)];
    T yc = cur[j];
    for (int iz = m.z0; iz < m.z1; ++iz) {
        const T yz = cur[j + (iz < g.nz ? sZ : -sZ)];
        const T L = T(6) * yc - ((cur[j + oxm] + cur[j + oxp]) + (cur[j + oym] + cur[j + oyp]) + (ym + yz));
        const T k = __ldcs(kap + j);  // streamed: keep L2 for the two wave fields reused next step
        const T yp = prev_out[j];
        T rhs = T(2) * yc - k * L;
        if ((FLAGS & kStepSrc) && (col_src || iz == 0 || iz == g.nz)) rhs += S[2 * j] * (T)cs + S[2 * j + 1] * (T)sn;
        const int nb = nbxy + ((iz == 0) & (int)((g.abc >> 4) & 1u)) + ((iz == g.nz) & (int)((g.abc >> 5) & 1u));
        T out;
        if (nb == 0) {
            out = rhs - yp;
        } else {
            const T beta = (T)nb * sqrt(k);
            const T v = rhs - ((FLAGS & kStepPrevScaled) ? yp : (T(1) - beta) * yp);
            out = (FLAGS & kStepNoDiv) ? v : v / (T(1) + beta);
        }
        prev_out[j] = out;
        ym = yc;
        yc = yz;
        j += sZ;
    }
}

// Leapfrog step, 3D 2nd order, two z-planes per loop iteration: both planes' loads are
// issued before either update (more loads in flight per thread).
template <typename T, int FLAGS>
__global__ void __launch_bounds__(kThreads) k_step3d7_z2(const T* __restrict__ cur, T* __restrict__ prev_out,
                                                         const T* __restrict__ kap, const T* __restrict__ S,
                                                         double cs, double sn, Geom g, int zc,
                                                         const unsigned char* __restrict__ scol) {
    const PlaneMap m = plane_map(g, zc);
    if (!m.valid || m.z0 >= m.z1) return;
    const long long sZ = (long long)g.sx * g.sy;
    long long j = node(g, m.ix, m.iy, m.z0);
    const long long oxm = off_m1(m.ix, 1), oxp = off_p1(m.ix, g.nx, 1);
    const long long oym = off_m1(m.iy, g.sx), oyp = off_p1(m.iy, g.ny, g.sx);
    int nbxy = 0;
    nbxy += (m.ix == 0) & (int)(g.abc & 1u);
    nbxy += (m.ix == g.nx) & (int)((g.abc >> 1) & 1u);
    nbxy += (m.iy == 0) & (int)((g.abc >> 2) & 1u);
    nbxy += (m.iy == g.ny) & (int)((g.abc >> 3) & 1u);
    // a column without source inside the grid (0 < z < nz) reads S only on its two z-faces
    const bool col_src = !(FLAGS & kStepSrc) || !scol || scol[m.ix + (long long)g.sx * m.iy];
    auto update = [&](T yc, T ym, T yz, long long jj, int iz, T sxy, T k, T yp) {
        const T L = T(6) * yc - (sxy + (ym + yz));
        T rhs = T(2) * yc - k * L;
        if ((FLAGS & kStepSrc) && (col_src || iz == 0 || iz == g.nz))
            rhs += S[2 * jj] * (T)cs + S[2 * jj + 1] * (T)sn;
        const int nb = nbxy + ((iz == 0) & (int)((g.abc >> 4) & 1u)) + ((iz == g.nz) & (int)((g.abc >> 5) & 1u));
        T out;
        if (nb == 0) {
            out = rhs - yp;
        } else {
            const T beta = (T)nb * sqrt(k);
            const T v = rhs - ((FLAGS & kStepPrevScaled) ? yp : (T(1) - beta) * yp);
            out = (FLAGS & kStepNoDiv) ? v : v / (T(1) + beta);
        }
        prev_out[jj] = out;
    };
    T ym = cur[j + (m.z0 > 0 ? -sZ : sZ)];
    T yc = cur[j];
    int iz = m.z0;
    for (; iz + 1 < m.z1; iz += 2) {
        const long long j1 = j + sZ;
        const T y1 = cur[j1];                                    // plane iz+1 (exists: iz+1 < z1 <= sz)
        const T y2 = cur[j1 + (iz + 1 < g.nz ? sZ : -sZ)];       // plane iz+2 (mirrored at the top)
        const T s0 = (cur[j + oxm] + cur[j + oxp]) + (cur[j + oym] + cur[j + oyp]);
        const T s1 = (cur[j1 + oxm] + cur[j1 + oxp]) + (cur[j1 + oym] + cur[j1 + oyp]);
        const T k0 = __ldcs(kap + j), k1 = __ldcs(kap + j1);
        const T p0 = prev_out[j], p1 = prev_out[j1];
        update(yc, ym, y1, j, iz, s0, k0, p0);
        update(y1, yc, y2, j1, iz + 1, s1, k1, p1);
        ym = y1;
        yc = y2;
        j += 2 * sZ;
    }
    if (iz < m.z1) {
        const T yz = cur[j + (iz < g.nz ? sZ : -sZ)];
        const T s0 = (cur[j + oxm] + cur[j + oxp]) + (cur[j + oym] + cur[j + oyp]);
        update(yc, ym, yz, j, iz, s0, __ldcs(kap + j), prev_out[j]);
    }
}

// Leapfrog step, 2D 5-point or 3D 7-point, FP32, vector form.  Each thread owns one aligned float4 chunk of
// the flat node index, nodes 4c .. 4c+3 (which may straddle a row or a plane), and reads y^n,
// y^{n-1} and kappa and writes y^{n+1} with 16-byte accesses.  The neighbours at a flat offset
// d = 4a + r (0 <= r < 4) of the four nodes are positions r .. r+3 of chunks c+a and c+a+1;
// the x-neighbours of the chunk's two end nodes are single loads.  Every load is issued before
// any arithmetic.  At a face the neighbour outside is replaced by the mirror value afterwards
// (ghost-point Neumann, as in the other step kernels), so a chunk index is clamped into range
// only where all of its values are discarded.  Same expression, in the same order, as
// k_step / k_step3d7.  The last chunk may extend past the last node: its loads read the slack behind
// every FP32 field (at least 16 bytes), and only its real nodes are stored.
struct Win4 {
    float v[4];
};

__device__ __forceinline__ float4 ld4g(const float* __restrict__ f, long long ch) {
    return __ldg(reinterpret_cast<const float4*>(f) + ch);
}

__device__ __forceinline__ long long clamp_ch(long long ch, long long nch) {
    return ch < 0 ? 0 : (ch >= nch ? nch - 1 : ch);
}

// w.v[e] = f[4 ca + r + e] (e = 0..3), r the same for every thread of the grid.
__device__ __forceinline__ Win4 window4(const float* __restrict__ f, long long ca, int r, long long nch) {
    const long long c0 = clamp_ch(ca, nch), c1 = clamp_ch(ca + 1, nch);
    Win4 w;
    if (r == 0) {
        const float4 a = ld4g(f, c0);
        w.v[0] = a.x, w.v[1] = a.y, w.v[2] = a.z, w.v[3] = a.w;
    } else if (r == 1) {
        const float4 a = ld4g(f, c0);
        const float b = __ldg(f + 4 * c1);
        w.v[0] = a.y, w.v[1] = a.z, w.v[2] = a.w, w.v[3] = b;
    } else if (r == 2) {
        const float2 a = __ldg(reinterpret_cast<const float2*>(f + 4 * c0 + 2));
        const float2 b = __ldg(reinterpret_cast<const float2*>(f + 4 * c1));
        w.v[0] = a.x, w.v[1] = a.y, w.v[2] = b.x, w.v[3] = b.y;
    } else {
        const float a = __ldg(f + 4 * c0 + 3);
        const float4 b = ld4g(f, c1);
        w.v[0] = a, w.v[1] = b.x, w.v[2] = b.y, w.v[3] = b.z;
    }
    return w;
}

template <int DIM, int FLAGS>
__device__ __forceinline__ void step_v4_chunk(const float* __restrict__ cur, float* __restrict__ prev_out,
                                              const float* __restrict__ kap, const float* __restrict__ S, double cs,
                                              double sn, const Geom& g, long long c) {
    const long long nch = (g.np + 3) >> 2;
    if (c >= nch) return;
    // chunks read: c and the windows at flat offsets +-sx (+-sx sy), clamped into [0, nch)
    if (!CMCG_RANGE_OK(4 * c, 4 * c + 3, 4 * nch, kSiteVector)) return;
    const long long sY = g.sx, sZ = (long long)g.sx * g.sy;
    const long long i0 = 4 * c;
    const float4 yc4 = ld4g(cur, c);
    const float xl = __ldg(cur + (i0 > 0 ? i0 - 1 : 0));
    const float xr = __ldg(cur + (i0 + 4 < g.np ? i0 + 4 : g.np - 1));
    const Win4 yP = window4(cur, c + (sY >> 2), (int)(sY & 3), nch);
    const Win4 yM = window4(cur, c + ((-sY) >> 2), (int)((-sY) & 3), nch);
    Win4 zP{}, zM{};
    if (DIM == 3) {
        zP = window4(cur, c + (sZ >> 2), (int)(sZ & 3), nch);
        zM = window4(cur, c + ((-sZ) >> 2), (int)((-sZ) & 3), nch);
    }
    const float4 k4 = __ldcs(reinterpret_cast<const float4*>(kap) + c);  // streamed, as in k_step3d7
    const float4 p4 = reinterpret_cast<const float4*>(prev_out)[c];
    float2 s2[4];
    if (FLAGS & kStepSrc) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const long long j = i0 + e < g.np ? i0 + e : g.np - 1;
            s2[e] = __ldg(reinterpret_cast<const float2*>(S) + j);
        }
    }
    // coordinates of node i0 (the flat index is below 2^31 for this kernel)
    const unsigned u0 = (unsigned)i0;
    int iz = (int)(u0 / (unsigned)sZ);
    const unsigned rem = u0 - (unsigned)iz * (unsigned)sZ;
    int iy = (int)(rem / (unsigned)g.sx);
    int ix = (int)(rem - (unsigned)iy * (unsigned)g.sx);
    const float yc[4] = {yc4.x, yc4.y, yc4.z, yc4.w};
    const float kk[4] = {k4.x, k4.y, k4.z, k4.w};
    const float pp[4] = {p4.x, p4.y, p4.z, p4.w};
    float out[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        float xm = e == 0 ? xl : yc[e - 1];
        float xp = e == 3 ? xr : yc[e + 1];
        if (ix == 0) xm = xp;
        if (ix == g.nx) xp = xm;
        float ym = yM.v[e], yp = yP.v[e];
        if (iy == 0) ym = yp;
        if (iy == g.ny) yp = ym;
        float L;
        if (DIM == 3) {
            float zm = zM.v[e], zp = zP.v[e];
            if (iz == 0) zm = zp;
            if (iz == g.nz) zp = zm;
            L = 6.f * yc[e] - (((xm + xp) + (ym + yp)) + (zm + zp));
        } else {
            L = 4.f * yc[e] - ((xm + xp) + (ym + yp));
        }
        const float k = kk[e];
        float rhs = 2.f * yc[e] - k * L;
        if (FLAGS & kStepSrc) rhs += s2[e].x * (float)cs + s2[e].y * (float)sn;
        int nb = 0;
        nb += (ix == 0) & (int)(g.abc & 1u);
        nb += (ix == g.nx) & (int)((g.abc >> 1) & 1u);
        nb += (iy == 0) & (int)((g.abc >> 2) & 1u);
        nb += (iy == g.ny) & (int)((g.abc >> 3) & 1u);
        if (DIM == 3) {
            nb += (iz == 0) & (int)((g.abc >> 4) & 1u);
            nb += (iz == g.nz) & (int)((g.abc >> 5) & 1u);
        }
        const float yq = pp[e];
        if (nb == 0) {
            out[e] = rhs - yq;
        } else {
            const float beta = (float)nb * sqrtf(k);
            const float v = rhs - ((FLAGS & kStepPrevScaled) ? yq : (1.f - beta) * yq);
            out[e] = (FLAGS & kStepNoDiv) ? v : v / (1.f + beta);
        }
        if (++ix == g.sx) {
            ix = 0;
            if (++iy == g.sy) {
                iy = 0;
                ++iz;
            }
        }
    }
    if (i0 + 3 < g.np) {
        reinterpret_cast<float4*>(prev_out)[c] = make_float4(out[0], out[1], out[2], out[3]);
    } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (i0 + e < g.np) prev_out[i0 + e] = out[e];
    }
}

template <int DIM, int FLAGS>
__global__ void __launch_bounds__(kThreads) k_step_v4(const float* __restrict__ cur, float* __restrict__ prev_out,
                                                      const float* __restrict__ kap, const float* __restrict__ S,
                                                      double cs, double sn, Geom g) {
    step_v4_chunk<DIM, FLAGS>(cur, prev_out, kap, S, cs, sn, g, (long long)blockIdx.x * kThreads + threadIdx.x);
}

// Can the vector-form step run on these fields?  16-byte aligned fields (each carries at
// least 16 bytes of slack behind its last node) and a flat index below 2^31.
inline bool step_v4_ok(const Geom& g, const void* cur, const void* prev, const void* kap) {
    const uintptr_t a = (uintptr_t)cur | (uintptr_t)prev | (uintptr_t)kap;
    return (a & 15u) == 0 && g.np + 4 < (1ll << 31);
}

// Leapfrog step, 3D 2nd order, K z-planes per loop iteration (K >= 2): all K planes' loads are
// issued before any update.  Same expression, in the same order, as k_step3d7.
template <typename T, int FLAGS, int K>
__global__ void __launch_bounds__(kThreads) k_step3d7_zk(const T* __restrict__ cur, T* __restrict__ prev_out,
                                                         const T* __restrict__ kap, const T* __restrict__ S,
                                                         double cs, double sn, Geom g, int zc,
                                                         const unsigned char* __restrict__ scol) {
    const PlaneMap m = plane_map(g, zc);
    if (!m.valid || m.z0 >= m.z1) return;
    const long long sZ = (long long)g.sx * g.sy;
    long long j = node(g, m.ix, m.iy, m.z0);
    const long long oxm = off_m1(m.ix, 1), oxp = off_p1(m.ix, g.nx, 1);
    const long long oym = off_m1(m.iy, g.sx), oyp = off_p1(m.iy, g.ny, g.sx);
    int nbxy = 0;
    nbxy += (m.ix == 0) & (int)(g.abc & 1u);
    nbxy += (m.ix == g.nx) & (int)((g.abc >> 1) & 1u);
    nbxy += (m.iy == 0) & (int)((g.abc >> 2) & 1u);
    nbxy += (m.iy == g.ny) & (int)((g.abc >> 3) & 1u);
    // a column without source inside the grid (0 < z < nz) reads S only on its two z-faces
    const bool col_src = !(FLAGS & kStepSrc) || !scol || scol[m.ix + (long long)g.sx * m.iy];
    auto update = [&](T yc, T ym, T yz, long long jj, int iz, T sxy, T k, T yp) {
        const T L = T(6) * yc - (sxy + (ym + yz));
        T rhs = T(2) * yc - k * L;
        if ((FLAGS & kStepSrc) && (col_src || iz == 0 || iz == g.nz))
            rhs += S[2 * jj] * (T)cs + S[2 * jj + 1] * (T)sn;
        const int nb = nbxy + ((iz == 0) & (int)((g.abc >> 4) & 1u)) + ((iz == g.nz) & (int)((g.abc >> 5) & 1u));
        T out;
        if (nb == 0) {
            out = rhs - yp;
        } else {
            const T beta = (T)nb * sqrt(k);
            const T v = rhs - ((FLAGS & kStepPrevScaled) ? yp : (T(1) - beta) * yp);
            out = (FLAGS & kStepNoDiv) ? v : v / (T(1) + beta);
        }
        prev_out[jj] = out;
    };
    T ym = cur[j + (m.z0 > 0 ? -sZ : sZ)];
    T yc = cur[j];
    int iz = m.z0;
    for (; iz + K - 1 < m.z1; iz += K) {
        T y[K + 1], sxy[K], kk[K], pp[K];
        // planes iz+1 .. iz+K (the top one mirrored to nz-1 past the last plane)
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int q = iz + k + 1;
            y[k + 1] = cur[j + (long long)(q <= g.nz ? k + 1 : k - 1) * sZ];
        }
        y[0] = yc;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const long long jk = j + (long long)k * sZ;
            sxy[k] = (cur[jk + oxm] + cur[jk + oxp]) + (cur[jk + oym] + cur[jk + oyp]);
            kk[k] = __ldcs(kap + jk);
            pp[k] = prev_out[jk];
        }
        T below = ym;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            update(y[k], below, y[k + 1], j + (long long)k * sZ, iz + k, sxy[k], kk[k], pp[k]);
            below = y[k];
        }
        ym = y[K - 1];
        yc = y[K];
        j += (long long)K * sZ;
    }
    for (; iz < m.z1; ++iz) {
        const T yz = cur[j + (iz < g.nz ? sZ : -sZ)];
        const T s0 = (cur[j + oxm] + cur[j + oxp]) + (cur[j + oym] + cur[j + oyp]);
        update(yc, ym, yz, j, iz, s0, __ldcs(kap + j), prev_out[j]);
        ym = yc;
        yc = yz;
        j += sZ;
    }
}

// Leapfrog step, 3D 4th order (13-point): the five z-planes z-2..z+2 carried in registers
// (even reflection at the faces), x/y neighbours at distance 1 and 2 loaded.
__device__ __forceinline__ int refl(int i, int n) { return i < 0 ? -i : (i > n ? 2 * n - i : i); }

template <typename T, int FLAGS>
__global__ void __launch_bounds__(kThreads) k_step3d13(const T* __restrict__ cur, T* __restrict__ prev_out,
                                                       const T* __restrict__ kap, const T* __restrict__ S,
                                                       double cs, double sn, Geom g, int zc) {
    const PlaneMap m = plane_map(g, zc, 2);
    if (!m.valid || m.z0 >= m.z1) return;
    const long long sZ = (long long)g.sx * g.sy;
    const long long col = (long long)m.ix + (long long)g.sx * m.iy;
    const long long ox1m = off_m1(m.ix, 1), ox1p = off_p1(m.ix, g.nx, 1);
    const long long ox2m = off_m2(m.ix, 1), ox2p = off_p2(m.ix, g.nx, 1);
    const long long oy1m = off_m1(m.iy, g.sx), oy1p = off_p1(m.iy, g.ny, g.sx);
    const long long oy2m = off_m2(m.iy, g.sx), oy2p = off_p2(m.iy, g.ny, g.sx);
    int nbxy = 0;
    nbxy += (m.ix == 0) & (int)(g.abc & 1u);
    nbxy += (m.ix == g.nx) & (int)((g.abc >> 1) & 1u);
    nbxy += (m.iy == 0) & (int)((g.abc >> 2) & 1u);
    nbxy += (m.iy == g.ny) & (int)((g.abc >> 3) & 1u);
    T zm2 = cur[col + refl(m.z0 - 2, g.nz) * sZ];
    T zm1 = cur[col + refl(m.z0 - 1, g.nz) * sZ];
    T zc0 = cur[col + (long long)m.z0 * sZ];
    T zp1 = cur[col + refl(m.z0 + 1, g.nz) * sZ];
    const T c1 = T(4) / T(3), c2 = T(1) / T(12);
    for (int iz = m.z0; iz < m.z1; ++iz) {
        const long long j = col + (long long)iz * sZ;
        const T zp2 = cur[col + refl(iz + 2, g.nz) * sZ];
        const T a1 = (cur[j + ox1m] + cur[j + ox1p]) + (cur[j + oy1m] + cur[j + oy1p]) + (zm1 + zp1);
        const T a2 = (cur[j + ox2m] + cur[j + ox2p]) + (cur[j + oy2m] + cur[j + oy2p]) + (zm2 + zp2);
        const T L = T(7.5) * zc0 - c1 * a1 + c2 * a2;
        const T k = kap[j];
        const T yp = prev_out[j];
        T rhs = T(2) * zc0 - k * L;
        if (FLAGS & kStepSrc) rhs += S[2 * j] * (T)cs + S[2 * j + 1] * (T)sn;
        const int nb = nbxy + ((iz == 0) & (int)((g.abc >> 4) & 1u)) + ((iz == g.nz) & (int)((g.abc >> 5) & 1u));
        T out;
        if (nb == 0) {
            out = rhs - yp;
        } else {
            const T beta = (T)nb * sqrt(k);
            const T v = rhs - ((FLAGS & kStepPrevScaled) ? yp : (T(1) - beta) * yp);
            out = (FLAGS & kStepNoDiv) ? v : v / (T(1) + beta);
        }
        prev_out[j] = out;
        zm2 = zm1;
        zm1 = zc0;
        zc0 = zp1;
        zp1 = zp2;
    }
}

// The 13-point step with two z-planes per loop trip: both planes' loads are issued before
// either update (more loads in flight per thread), the same expression in the same order as
// k_step3d13.  With a source, a column without source inside the grid (0 < z < nz) reads S
// only on its two z-faces.
template <typename T, int FLAGS>
__global__ void __launch_bounds__(kThreads) k_step3d13_z2(const T* __restrict__ cur, T* __restrict__ prev_out,
                                                          const T* __restrict__ kap, const T* __restrict__ S,
                                                          double cs, double sn, Geom g, int zc,
                                                          const unsigned char* __restrict__ scol) {
    const PlaneMap m = plane_map(g, zc, 2);
    if (!m.valid || m.z0 >= m.z1) return;
    const long long sZ = (long long)g.sx * g.sy;
    const long long col = (long long)m.ix + (long long)g.sx * m.iy;
    const long long ox1m = off_m1(m.ix, 1), ox1p = off_p1(m.ix, g.nx, 1);
    const long long ox2m = off_m2(m.ix, 1), ox2p = off_p2(m.ix, g.nx, 1);
    const long long oy1m = off_m1(m.iy, g.sx), oy1p = off_p1(m.iy, g.ny, g.sx);
    const long long oy2m = off_m2(m.iy, g.sx), oy2p = off_p2(m.iy, g.ny, g.sx);
    int nbxy = 0;
    nbxy += (m.ix == 0) & (int)(g.abc & 1u);
    nbxy += (m.ix == g.nx) & (int)((g.abc >> 1) & 1u);
    nbxy += (m.iy == 0) & (int)((g.abc >> 2) & 1u);
    nbxy += (m.iy == g.ny) & (int)((g.abc >> 3) & 1u);
    const bool col_src = !(FLAGS & kStepSrc) || !scol || scol[col];
    const T c1 = T(4) / T(3), c2 = T(1) / T(12);
    auto update = [&](long long j, int iz, T zc0, T zm1, T zp1, T zm2, T zp2, T a1xy, T a2xy, T k, T yp) {
        const T a1 = a1xy + (zm1 + zp1);
        const T a2 = a2xy + (zm2 + zp2);
        const T L = T(7.5) * zc0 - c1 * a1 + c2 * a2;
        T rhs = T(2) * zc0 - k * L;
        if ((FLAGS & kStepSrc) && (col_src || iz == 0 || iz == g.nz)) rhs += S[2 * j] * (T)cs + S[2 * j + 1] * (T)sn;
        const int nb = nbxy + ((iz == 0) & (int)((g.abc >> 4) & 1u)) + ((iz == g.nz) & (int)((g.abc >> 5) & 1u));
        T out;
        if (nb == 0) {
            out = rhs - yp;
        } else {
            const T beta = (T)nb * sqrt(k);
            const T v = rhs - ((FLAGS & kStepPrevScaled) ? yp : (T(1) - beta) * yp);
            out = (FLAGS & kStepNoDiv) ? v : v / (T(1) + beta);
        }
        prev_out[j] = out;
    };
    T zm2 = cur[col + refl(m.z0 - 2, g.nz) * sZ];
    T zm1 = cur[col + refl(m.z0 - 1, g.nz) * sZ];
    T zc0 = cur[col + (long long)m.z0 * sZ];
    T zp1 = cur[col + refl(m.z0 + 1, g.nz) * sZ];
    int iz = m.z0;
    for (; iz + 1 < m.z1; iz += 2) {
        const long long j = col + (long long)iz * sZ, j1 = j + sZ;
        const T zp2 = cur[col + refl(iz + 2, g.nz) * sZ];
        const T zp3 = cur[col + refl(iz + 3, g.nz) * sZ];
        const T a1a = (cur[j + ox1m] + cur[j + ox1p]) + (cur[j + oy1m] + cur[j + oy1p]);
        const T a2a = (cur[j + ox2m] + cur[j + ox2p]) + (cur[j + oy2m] + cur[j + oy2p]);
        const T a1b = (cur[j1 + ox1m] + cur[j1 + ox1p]) + (cur[j1 + oy1m] + cur[j1 + oy1p]);
        const T a2b = (cur[j1 + ox2m] + cur[j1 + ox2p]) + (cur[j1 + oy2m] + cur[j1 + oy2p]);
        const T k0 = kap[j], k1 = kap[j1];
        const T p0 = prev_out[j], p1 = prev_out[j1];
        update(j, iz, zc0, zm1, zp1, zm2, zp2, a1a, a2a, k0, p0);
        update(j1, iz + 1, zp1, zc0, zp2, zm1, zp3, a1b, a2b, k1, p1);
        zm2 = zc0;
        zm1 = zp1;
        zc0 = zp2;
        zp1 = zp3;
    }
    if (iz < m.z1) {
        const long long j = col + (long long)iz * sZ;
        const T zp2 = cur[col + refl(iz + 2, g.nz) * sZ];
        const T a1a = (cur[j + ox1m] + cur[j + ox1p]) + (cur[j + oy1m] + cur[j + oy1p]);
        const T a2a = (cur[j + ox2m] + cur[j + ox2p]) + (cur[j + oy2m] + cur[j + oy2p]);
        update(j, iz, zc0, zm1, zp1, zm2, zp2, a1a, a2a, kap[j], prev_out[j]);
    }
}

// ---------------------------------------------------------------------------------------
// The endpoint kernels compute in the stepping precision T: the FP32 path does its stencils
// and pointwise algebra in FP32 and only its FP64-facing outputs (z, ghat, g~1) and the
// reductions in FP64.  w0t is the T-precision copy of the initial displacement w0.
template <typename R>
__device__ __forceinline__ R weight_t(const Geom& g, int ix, int iy, int iz) {
    const R h = (R)g.h;
    R w = (g.dim == 3) ? h * h * h : h * h;
    if (ix == 0 || ix == g.nx) w *= R(0.5);
    if (iy == 0 || iy == g.ny) w *= R(0.5);
    if (g.dim == 3 && (iz == 0 || iz == g.nz)) w *= R(0.5);
    return w;
}

// Period start: y0 = w0, y1 = w0 + dt (1 - beta) w1 + (S_re - kappa Lt w0) / 2.
template <typename T, int ORDER, bool SRC, typename V = double>
__global__ void __launch_bounds__(kThreads) k_start(const T* __restrict__ w0t, const V* __restrict__ w1,
                                                    T* __restrict__ y0, T* __restrict__ y1,
                                                    const T* __restrict__ kap, const double* __restrict__ S,
                                                    Geom g, double dt, int zc) {
    const PlaneMap m = plane_map(g, zc, ORDER / 2);
    if (!m.valid || m.z0 >= m.z1) return;
    Ld<T> f{w0t};
    const T dtT = (T)dt;
    const bool col = ORDER == 2 && g.dim == 3;
    auto cl = column_lap<T>(g, f, m.ix, m.iy);
    if (col) cl.start(node(g, m.ix, m.iy, m.z0), m.z0);
    for (int iz = m.z0; iz < m.z1; ++iz) {
        const long long j = node(g, m.ix, m.iy, iz);
        // every load is issued before the Dirichlet test (kappa = 0), which only selects the
        // stores: a branch on kappa would put its load's latency before all the others
        const T k = kap[j];
        const T L = col ? cl.lap(j) : lap_t<ORDER, T>(g, f, j, m.ix, m.iy, iz);
        const int nbf = num_abc(g, m.ix, m.iy, iz);
        const T beta = nbf ? (T)nbf * sqrt(k) : T(0);
        const T w0j = w0t[j];
        T v = w0j + dtT * (T(1) - beta) * (T)w1[j] - T(0.5) * k * L;
        if (SRC) v += (T)(0.5 * S[2 * j]);
        const bool dir = k == T(0);
        y0[j] = dir ? T(0) : w0j;
        y1[j] = dir ? T(0) : v;
        if (col && iz + 1 < m.z1) cl.advance(j, iz);
    }
}

// Period end: vN, mismatch, energy operator and J (MODE 0), or (uT, vT) (MODE 1).  MODE 2
// (FP32 periods inside a gradient) is MODE 0 with an FP32 hand-off to the adjoint period: out0
// holds z0 and out1 holds t = e1 / (1 + beta) = D^-1 z1 (D = M (1 + beta)), both as floats,
// which is what the adjoint start needs, so it has no separate D^-1 pass.
// The FP32 instantiations of k_end and k_adj_final are held to five resident blocks per SM
// (48 registers) for occupancy; the FP64 ones would spill.  k_end: 384 -> 323 us per launch
// at 257^3; k_adj_final with the hand-off would otherwise take 53 registers.
template <typename T>
constexpr int kEndMinBlocks = std::is_same<T, float>::value ? 5 : 1;

template <typename T, int ORDER, bool SRC, int MODE, typename V = double>
__global__ void __launch_bounds__(kThreads, kEndMinBlocks<T>) k_end(const T* __restrict__ yN, const T* __restrict__ yNm1,
                                                  const T* __restrict__ w0t, const V* __restrict__ w1,
                                                  const T* __restrict__ kap, const T* __restrict__ mass,
                                                  const double* __restrict__ S, double cs, double sn,
                                                  double* __restrict__ out0, double* __restrict__ out1,
                                                  Red red, Geom g, double dt, int zc) {
    const PlaneMap m = plane_map(g, zc, ORDER / 2);
    double acc[1] = {0.0};
    KahanF accf;  // FP32 periods: the thread's part of J without FP64 arithmetic
    if (m.valid) {
        Ld<T> fy{yN};
        DiffT<T> fe{yN, w0t};
        const T ih2 = T(1) / (T)(g.h * g.h);
        const T dtT = (T)dt;
        for (int iz = m.z0; iz < m.z1; ++iz) {
            const long long j = node(g, m.ix, m.iy, iz);
            const T k = kap[j];  // Dirichlet (kappa = 0) only selects the stores (see k_start)
            const bool dir = k == T(0);
            const T L = lap_t<ORDER, T>(g, fy, j, m.ix, m.iy, iz);
            const int nbf = num_abc(g, m.ix, m.iy, iz);
        const T beta = nbf ? (T)nbf * sqrt(k) : T(0);
            T src = T(0);
            if (SRC) src = (T)(S[2 * j] * cs + S[2 * j + 1] * sn);
            const T yn = yN[j];
            const T vN = ((yn - yNm1[j]) / dtT + (src - k * L) / (T(2) * dtT)) / (T(1) + beta);
            if (MODE == 1) {
                out0[j] = dir ? 0.0 : (double)yn;
                out1[j] = dir ? 0.0 : (double)vN;
            } else {
                const T e0 = yn - w0t[j];
                const T e1 = vN - (T)w1[j];
                const T W = weight_t<T>(g, m.ix, m.iy, iz);
                const T z0 = W * ih2 * lap_t<ORDER, T>(g, fe, j, m.ix, m.iy, iz);
                const T z1 = (T)mass[j] * e1;
                if (MODE == 2) {
                    ((float*)out0)[j] = dir ? 0.f : (float)z0;
                    ((float*)out1)[j] = dir ? 0.f : (float)(e1 / (T(1) + beta));
                } else {
                    out0[j] = dir ? 0.0 : (double)z0;
                    out1[j] = dir ? 0.0 : (double)z1;
                }
                if (std::is_same<T, float>::value)
                    accf.add(dir ? 0.0f : (float)(e0 * z0 + e1 * z1));
                else
                    acc[0] += dir ? 0.0 : 0.5 * (double)(e0 * z0 + e1 * z1);
            }
        }
    }
    if (MODE != 1) {
        if (std::is_same<T, float>::value) acc[0] = 0.5 * accf.value();
        if (grid_sum<1>(acc, red.partials, red.ticket) && threadIdx.x == 0) red.sc[SC_J] = acc[0];
    }
}

// Adjoint start, part 1: t = D^-1 b = b / (M (1 + beta)).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_adj_prep(const double* __restrict__ b, const T* __restrict__ mass,
                                                       const T* __restrict__ kap, T* __restrict__ t, Geom g, int zc) {
    const PlaneMap m = plane_map(g, zc);
    if (!m.valid) return;
    for (int iz = m.z0; iz < m.z1; ++iz) {
        const long long j = node(g, m.ix, m.iy, iz);
        const T k = kap[j];  // Dirichlet (kappa = 0) only selects the store (see k_start)
        const int nbf = num_abc(g, m.ix, m.iy, iz);
        const T beta = nbf ? (T)nbf * sqrt(k) : T(0);
        const T v = (T)b[j] / ((T)mass[j] * (T(1) + beta));  // 0/0 on Dirichlet nodes: not stored
        t[j] = k == T(0) ? T(0) : v;
    }
}

// Adjoint start, part 2 (transposed end velocity):
//   ybar_N = a + M t / dt - (dt/2) K t,  u_{N-1} = D^-1 ybar_N,  prev = C u_N / M = t / dt.
template <typename T, int ORDER, typename A>
__global__ void __launch_bounds__(kThreads) k_adj_start(const A* __restrict__ a, const T* __restrict__ t,
                                                        const T* __restrict__ mass, const T* __restrict__ kap,
                                                        T* __restrict__ cur, T* __restrict__ prev, Geom g, double dt,
                                                        int zc) {
    const PlaneMap m = plane_map(g, zc, ORDER / 2);
    if (!m.valid) return;
    Ld<T> f{t};
    const T dtT = (T)dt;
    for (int iz = m.z0; iz < m.z1; ++iz) {
        const long long j = node(g, m.ix, m.iy, iz);
        const T k = kap[j];  // Dirichlet (kappa = 0) only selects the stores (see k_start)
        const T L = lap_t<ORDER, T>(g, f, j, m.ix, m.iy, iz);
        const int nbf = num_abc(g, m.ix, m.iy, iz);
        const T beta = nbf ? (T)nbf * sqrt(k) : T(0);
        const T tj = t[j];
        const T u = ((T)a[j] / (T)mass[j] + tj / dtT - k * L / (T(2) * dtT)) / (T(1) + beta);  // 0/0 at Dirichlet
        const bool dir = k == T(0);
        cur[j] = dir ? T(0) : u;
        prev[j] = dir ? T(0) : tj / dtT;
    }
}

// Adjoint final (transposed start half-kick), from s = M^-1 ybar_1 and u_1:
//   q0 = M (s - (1 - beta) u_1) - (dt^2/2) K s,   q1 = dt M (1 - beta) s.
// MODE 1 writes q.  MODE 0 forms the CG gradient ghat = q - z, g~1 = ghat1 / M (only when gt1
// is given: the exact Riesz map needs it, the V-cycle does not), and reduces
// (ghat . d, sum ghat0).  MODE 2 (FP32) is MODE 0 on the FP32 hand-off of k_end: z0 in z0, and
// z1 = M (1 + beta) t from t in z1.
template <typename T, int ORDER, int MODE, typename V = double>
__global__ void __launch_bounds__(kThreads, kEndMinBlocks<T>) k_adj_final(const T* __restrict__ s, const T* __restrict__ u1,
                                                        const T* __restrict__ mass, const T* __restrict__ kap,
                                                        const double* __restrict__ minv,
                                                        const double* __restrict__ z0, const double* __restrict__ z1,
                                                        const V* __restrict__ d0, const V* __restrict__ d1,
                                                        V* __restrict__ o0, V* __restrict__ o1,
                                                        double* __restrict__ gt1, Red red, Geom g, double dt, int zc) {
    const PlaneMap m = plane_map(g, zc, ORDER / 2);
    double acc[2] = {0.0, 0.0};
    KahanF accf0, accf1;
    if (m.valid && m.z0 < m.z1) {
        Ld<T> f{s};
        const T ih2 = T(1) / (T)(g.h * g.h);
        const T dtT = (T)dt;
        const bool col = ORDER == 2 && g.dim == 3;
        auto cl = column_lap<T>(g, f, m.ix, m.iy);
        if (col) cl.start(node(g, m.ix, m.iy, m.z0), m.z0);
        for (int iz = m.z0; iz < m.z1; ++iz) {
            const long long j = node(g, m.ix, m.iy, iz);
            const T k = kap[j];  // Dirichlet (kappa = 0) only selects the stores (see k_start)
            const bool dir = k == T(0);
            const T L = col ? cl.lap(j) : lap_t<ORDER, T>(g, f, j, m.ix, m.iy, iz);
            const int nbf = num_abc(g, m.ix, m.iy, iz);
        const T beta = nbf ? (T)nbf * sqrt(k) : T(0);
            const T W = weight_t<T>(g, m.ix, m.iy, iz);
            const T M = (T)mass[j];
            const T sj = s[j];
            const T q0 = M * (sj - (T(1) - beta) * u1[j]) - T(0.5) * dtT * dtT * W * ih2 * L;
            const T q1 = dtT * M * (T(1) - beta) * sj;
            if (MODE == 1) {
                o0[j] = dir ? V(0) : (V)q0;
                o1[j] = dir ? V(0) : (V)q1;
            } else if (std::is_same<T, float>::value) {
                // FP32 periods: z came from FP32 values, so the differences and products stay in
                // FP32 (FP64 only holds the stored vectors)
                float zz0, zz1;
                if (MODE == 2) {
                    zz0 = ((const float*)z0)[j];
                    zz1 = (float)M * ((float)(T(1) + beta) * ((const float*)z1)[j]);
                } else {
                    zz0 = (float)z0[j];
                    zz1 = (float)z1[j];
                }
                const float g0 = (float)q0 - zz0;
                const float g1 = (float)q1 - zz1;
                const float pd = g0 * (float)d0[j] + g1 * (float)d1[j];
                o0[j] = dir ? V(0) : (V)g0;
                o1[j] = dir ? V(0) : (V)g1;
                if (gt1) gt1[j] = dir ? 0.0 : (double)(g1 * (float)minv[j]);
                accf0.add(dir ? 0.0f : pd);
                accf1.add(dir ? 0.0f : g0);
            } else {
                const double g0 = (double)q0 - z0[j];
                const double g1 = (double)q1 - z1[j];
                const double pd = g0 * (double)d0[j] + g1 * (double)d1[j];
                o0[j] = dir ? V(0) : (V)g0;
                o1[j] = dir ? V(0) : (V)g1;
                if (gt1) gt1[j] = dir ? 0.0 : g1 * minv[j];
                acc[0] += dir ? 0.0 : pd;
                acc[1] += dir ? 0.0 : g0;
            }
            if (col && iz + 1 < m.z1) cl.advance(j, iz);
        }
    }
    if (MODE != 1) {
        if (std::is_same<T, float>::value) {
            acc[0] = accf0.value();
            acc[1] = accf1.value();
        }
        if (grid_sum<2>(acc, red.partials, red.ticket) && threadIdx.x == 0) {
            red.sc[SC_GD] = acc[0];
            red.sc[SC_GSUM] = acc[1];
        }
    }
}

// S = dt^2 M^-1 (W f + A g) = kappa h^2 (f + (2 nb / h) g), zero on Dirichlet nodes
// (or added to S when accumulating).
__global__ void __launch_bounds__(kThreads) k_make_source(const double* __restrict__ f, const double* __restrict__ gb,
                                                          const double* __restrict__ kap64, double* __restrict__ S,
                                                          Geom g, int zc, int accumulate) {
    const PlaneMap m = plane_map(g, zc);
    if (!m.valid) return;
    for (int iz = m.z0; iz < m.z1; ++iz) {
        const long long j = node(g, m.ix, m.iy, iz);
        const double k = kap64[j];
        const double sc = k * g.h * g.h;
        double re = 0.0, im = 0.0;
        if (f) {
            re += f[2 * j];
            im += f[2 * j + 1];
        }
        if (gb) {
            const double a = 2.0 * num_abc(g, m.ix, m.iy, iz) / g.h;
            re += a * gb[2 * j];
            im += a * gb[2 * j + 1];
        }
        if (accumulate) {
            S[2 * j] += sc * re;
            S[2 * j + 1] += sc * im;
        } else {
            S[2 * j] = sc * re;
            S[2 * j + 1] = sc * im;
        }
    }
}

// ---------------------------------------------------------------------------------------
// Batched persistent step loop: one cooperative launch advances the step loops of many solves
// (uneven grids and step counts) together.  Per step, the blocks stride over the work items of
// every solve that still has steps left (a work item is one block of the solve's own launch
// grid: 256 plane nodes x zc planes), then meet at a grid barrier.  Solve i uses buf0 as y^n
// at its step 0 and the two buffers alternate; adjoint loops use the PREV_SCALED / NO_DIV
// variants on their first / last step.  Every barrier wait is bounded: on time-out the kernel
// sets *err and all blocks return.
constexpr long long kBarrierSpinLimit = 1ll << 24;

__device__ bool grid_barrier(unsigned* bar, int* err, unsigned nblocks, long long spin_limit) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* vgen = bar + 1;
        const unsigned gen = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(bar, 1u);
        ok = 1;
        if (arrived == nblocks - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            long long spins = 0;
            while (*vgen == gen) {
                if (++spins > spin_limit || *(volatile int*)err) {
                    atomicExch(err, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// The 3D 7-point step of one work item's column: two z-planes per loop trip with every load
// issued first and the z-neighbours in registers, as in k_step3d7_z2 (the same expression in
// the same order as the generic work-item step below).
template <int FLAGS>
__device__ __forceinline__ void step_item3d7(const float* __restrict__ cur, float* __restrict__ prev,
                                             const float* __restrict__ kap, const Geom& g, int ix, int iy, int z0,
                                             int z1, const float* __restrict__ S, float csf, float snf,
                                             bool col_src) {
    const long long sZ = (long long)g.sx * g.sy;
    long long j = node(g, ix, iy, z0);
    const long long oxm = off_m1(ix, 1), oxp = off_p1(ix, g.nx, 1);
    const long long oym = off_m1(iy, g.sx), oyp = off_p1(iy, g.ny, g.sx);
    int nbxy = 0;
    nbxy += (ix == 0) & (int)(g.abc & 1u);
    nbxy += (ix == g.nx) & (int)((g.abc >> 1) & 1u);
    nbxy += (iy == 0) & (int)((g.abc >> 2) & 1u);
    nbxy += (iy == g.ny) & (int)((g.abc >> 3) & 1u);
    auto update = [&](float yc, float ym, float yz, long long jj, int iz, float sxy, float k, float yp) {
        const float L = 6.f * yc - (sxy + (ym + yz));
        float rhs = 2.f * yc - k * L;
        if ((FLAGS & kStepSrc) && (col_src || iz == 0 || iz == g.nz)) rhs += S[2 * jj] * csf + S[2 * jj + 1] * snf;
        const int nb = nbxy + ((iz == 0) & (int)((g.abc >> 4) & 1u)) + ((iz == g.nz) & (int)((g.abc >> 5) & 1u));
        float out;
        if (nb == 0) {
            out = rhs - yp;
        } else {
            const float beta = (float)nb * sqrtf(k);
            const float v = rhs - ((FLAGS & kStepPrevScaled) ? yp : (1.f - beta) * yp);
            out = (FLAGS & kStepNoDiv) ? v : v / (1.f + beta);
        }
        prev[jj] = out;
    };
    float ym = cur[j + (z0 > 0 ? -sZ : sZ)];
    float yc = cur[j];
    int iz = z0;
    for (; iz + 1 < z1; iz += 2) {
        const long long j1 = j + sZ;
        const float y1 = cur[j1];
        const float y2 = cur[j1 + (iz + 1 < g.nz ? sZ : -sZ)];
        const float s0 = (cur[j + oxm] + cur[j + oxp]) + (cur[j + oym] + cur[j + oyp]);
        const float s1 = (cur[j1 + oxm] + cur[j1 + oxp]) + (cur[j1 + oym] + cur[j1 + oyp]);
        const float k0 = kap[j], k1 = kap[j1];
        const float p0 = prev[j], p1 = prev[j1];
        update(yc, ym, y1, j, iz, s0, k0, p0);
        update(y1, yc, y2, j1, iz + 1, s1, k1, p1);
        ym = y1;
        yc = y2;
        j += 2 * sZ;
    }
    if (iz < z1) {
        const float yz = cur[j + (iz < g.nz ? sZ : -sZ)];
        const float s0 = (cur[j + oxm] + cur[j + oxp]) + (cur[j + oym] + cur[j + oyp]);
        update(yc, ym, yz, j, iz, s0, kap[j], prev[j]);
    }
}

// The step of one work item (block-sized piece of one solve's grid).
// With kStepSrc (the forced steps of a run-up), S is the FP32 source and (cs, sn) the step's
// source factors, as in the one-solve step kernels.
template <int ORDER, int FLAGS>
__device__ __forceinline__ void step_item(const float* __restrict__ cur, float* __restrict__ prev,
                                          const float* __restrict__ kap, const Geom& g, int zc, int bx, int bz,
                                          int vec4, const float* __restrict__ S, double cs, double sn,
                                          const unsigned char* __restrict__ scol) {
    if (ORDER == 2 && g.dim == 2 && vec4) {  // 2D: one aligned float4 chunk of the flat index per thread
        step_v4_chunk<2, FLAGS>(cur, prev, kap, S, cs, sn, g, (long long)bx * kThreads + threadIdx.x);
        return;
    }
    const long long plane = (long long)g.sx * g.sy;
    const long long p = (long long)bx * kThreads + threadIdx.x;
    if (p >= plane) return;
    const int iy = (int)(p / g.sx);
    const int ix = (int)(p - (long long)iy * g.sx);
    const int z0 = bz * zc, z1 = min(z0 + zc, g.sz);
    if (!column_in_range(g, ix, iy, z0, z1, ORDER / 2, kSiteBatch)) return;
    if (ORDER == 2 && g.dim == 3) {
        const bool col_src = !(FLAGS & kStepSrc) || !scol || scol[ix + (long long)g.sx * iy];
        step_item3d7<FLAGS>(cur, prev, kap, g, ix, iy, z0, z1, S, (float)cs, (float)sn, col_src);
        return;
    }
    Ld<float> f{cur};
    for (int iz = z0; iz < z1; ++iz) {
        const long long j = node(g, ix, iy, iz);
        const float L = lap_t<ORDER, float>(g, f, j, ix, iy, iz);
        const float k = kap[j];
        const float yp = prev[j];
        float rhs = 2.f * cur[j] - k * L;
        if (FLAGS & kStepSrc) rhs += S[2 * j] * (float)cs + S[2 * j + 1] * (float)sn;
        const int nb = num_abc(g, ix, iy, iz);
        float out;
        if (nb == 0) {
            out = rhs - yp;
        } else {
            const float beta = (float)nb * sqrtf(k);
            const float v = rhs - ((FLAGS & kStepPrevScaled) ? yp : (1.f - beta) * yp);
            out = (FLAGS & kStepNoDiv) ? v : v / (1.f + beta);
        }
        prev[j] = out;
    }
}

template <int ORDER>
__device__ __forceinline__ void step_item_flags(const float* cur, float* prev, const float* kap, const Geom& g, int zc,
                                                int bx, int bz, int flags, int vec4) {
    switch (flags) {
        case 0: step_item<ORDER, 0>(cur, prev, kap, g, zc, bx, bz, vec4, nullptr, 0.0, 0.0, nullptr); break;
        case kStepPrevScaled:
            step_item<ORDER, kStepPrevScaled>(cur, prev, kap, g, zc, bx, bz, vec4, nullptr, 0.0, 0.0, nullptr);
            break;
        case kStepNoDiv:
            step_item<ORDER, kStepNoDiv>(cur, prev, kap, g, zc, bx, bz, vec4, nullptr, 0.0, 0.0, nullptr);
            break;
        default:
            step_item<ORDER, kStepPrevScaled | kStepNoDiv>(cur, prev, kap, g, zc, bx, bz, vec4, nullptr, 0.0, 0.0,
                                                           nullptr);
            break;
    }
}

// Source factors (theta_tr(t_n) cos(omega t_n), theta_tr(t_n) sin(omega t_n)) of run-up step n
// (Eq. transientfunction): since omega dt = 2 pi / N, the phase is 2 pi (n mod N) / N, which
// the FP32 sin(pi x) / cos(pi x) evaluate without the large-argument reduction; the ramp
// argument pi t_n / (2 t_tr) is pi n / (2 l N) with t_tr = l T.  The steps take these factors
// in FP32, as they take the host's FP64 ones.
__device__ __forceinline__ void runup_factors(int n, int N, int total, double* cs, double* sn) {
    const int k = n % N;
    float sw, cw;
    sincospif(2.0f * (float)k / (float)N, &sw, &cw);
    float th = 1.0f;
    if (n < total) {
        const float r = sinpif(0.5f * (float)n / (float)total);
        th = (2.0f - r) * r;
    }
    *cs = (double)(th * cw);
    *sn = (double)(th * sw);
}

// FORCED: the run-ups of several solves stepping together (steps n = s + 1 of the ramped
// forced leapfrog from rest); otherwise homogeneous period step loops.
template <bool FORCED>
__global__ void __launch_bounds__(kThreads) k_batch_steps(const BatchItem* __restrict__ items, int nitems,
                                                          int total_blocks, int max_steps, unsigned* bar, int* err,
                                                          long long spin_limit) {
    for (int s = 0; s < max_steps; ++s) {
        for (int w = blockIdx.x; w < total_blocks; w += gridDim.x) {
            int lo = 0, hi = nitems - 1;  // last item with offset <= w
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (items[mid].offset <= w) lo = mid;
                else hi = mid - 1;
            }
            const BatchItem& it = items[lo];
            if (s >= it.nsteps) continue;
            const int lb = w - it.offset;
            const int bz = lb / it.blocks_xy, bx = lb - bz * it.blocks_xy;
            const float* cur = (s & 1) ? it.buf1 : it.buf0;
            float* prev = (s & 1) ? it.buf0 : it.buf1;
            if (FORCED) {
                double cs, sn;
                runup_factors(s + 1, it.steps_per_period, it.runup_steps, &cs, &sn);
                if (it.order == 2)
                    step_item<2, kStepSrc>(cur, prev, it.kap, it.g, it.zc, bx, bz, it.vec4, it.S, cs, sn, it.scol);
                else
                    step_item<4, kStepSrc>(cur, prev, it.kap, it.g, it.zc, bx, bz, 0, it.S, cs, sn, it.scol);
                continue;
            }
            int flags = 0;
            if (it.adjoint) {
                if (s == 0) flags |= kStepPrevScaled;
                if (s == it.nsteps - 1) flags |= kStepNoDiv;
            }
            if (it.order == 2) step_item_flags<2>(cur, prev, it.kap, it.g, it.zc, bx, bz, flags, it.vec4);
            else step_item_flags<4>(cur, prev, it.kap, it.g, it.zc, bx, bz, flags, 0);
        }
        if (s + 1 < max_steps && !grid_barrier(bar, err, gridDim.x, spin_limit)) return;
    }
}

// A barrier that can never complete (one more arrival expected than blocks exist): used only
// by the self-test of the time-out path.
__global__ void k_barrier_selftest(unsigned* bar, int* err, long long spin_limit) {
    grid_barrier(bar, err, gridDim.x + 1, spin_limit);
}

inline dim3 plane_grid(const Geom& g, int zc) {
    const long long plane = (long long)g.sx * g.sy;
    return dim3((unsigned)((plane + kThreads - 1) / kThreads), (unsigned)((g.sz + zc - 1) / zc), 1);
}

template <typename T, int ORDER, int FLAGS>
void step_dispatch(const Geom& g, const T* cur, T* prev, const T* kap, const T* S, double cs, double sn,
                   int zc, const unsigned char* scol, cudaStream_t st) {
    // zc < 0 selects the variants of the 3D 7-point kernel with several z-planes per loop
    // iteration: -zc = planes per thread, plus kZk4 for four planes per iteration (else two);
    // kZcFlat the FP32 vector form (other types and stencils: their default kernel)
    if (zc == kZcFlat) {
        if constexpr (std::is_same<T, float>::value) {
            if (ORDER == 2 && step_v4_ok(g, cur, prev, kap)) {
                const long long nch = (g.np + 3) >> 2;
                const unsigned blocks = (unsigned)((nch + kThreads - 1) / kThreads);
                if (g.dim == 3)
                    k_step_v4<3, FLAGS><<<blocks, kThreads, 0, st>>>(cur, prev, kap, S, cs, sn, g);
                else
                    k_step_v4<2, FLAGS><<<blocks, kThreads, 0, st>>>(cur, prev, kap, S, cs, sn, g);
                return;
            }
        }
        zc = g.dim == 3 ? 16 : 1;
    }
    if (ORDER == 2 && g.dim == 3 && zc < 0 && (-zc) >= kZk4) {
        const int z = -zc - kZk4;
        k_step3d7_zk<T, FLAGS, 4><<<plane_grid(g, z), kThreads, 0, st>>>(cur, prev, kap, S, cs, sn, g, z, scol);
    } else if (ORDER == 2 && g.dim == 3 && zc < 0) {
        k_step3d7_z2<T, FLAGS><<<plane_grid(g, -zc), kThreads, 0, st>>>(cur, prev, kap, S, cs, sn, g, -zc, scol);
    } else if (ORDER == 2 && g.dim == 3) {
        k_step3d7<T, FLAGS><<<plane_grid(g, zc), kThreads, 0, st>>>(cur, prev, kap, S, cs, sn, g, zc, scol);
    } else if (ORDER == 4 && g.dim == 3 && zc < 0) {
        k_step3d13_z2<T, FLAGS><<<plane_grid(g, -zc), kThreads, 0, st>>>(cur, prev, kap, S, cs, sn, g, -zc, scol);
    } else if (ORDER == 4 && g.dim == 3) {
        k_step3d13<T, FLAGS><<<plane_grid(g, zc), kThreads, 0, st>>>(cur, prev, kap, S, cs, sn, g, zc);
    } else {
        k_step<T, ORDER, FLAGS><<<plane_grid(g, zc), kThreads, 0, st>>>(cur, prev, kap, S, cs, sn, g, zc);
    }
}

template <typename T, int ORDER>
void step_flags(const Geom& g, const T* cur, T* prev, const T* kap, const T* S, double cs, double sn,
                int flags, int zc, const unsigned char* scol, cudaStream_t st) {
    switch (flags) {
        case 0: step_dispatch<T, ORDER, 0>(g, cur, prev, kap, S, cs, sn, zc, scol, st); break;
        case kStepSrc: step_dispatch<T, ORDER, kStepSrc>(g, cur, prev, kap, S, cs, sn, zc, scol, st); break;
        case kStepPrevScaled: step_dispatch<T, ORDER, kStepPrevScaled>(g, cur, prev, kap, S, cs, sn, zc, scol, st); break;
        case kStepNoDiv: step_dispatch<T, ORDER, kStepNoDiv>(g, cur, prev, kap, S, cs, sn, zc, scol, st); break;
        case kStepPrevScaled | kStepNoDiv:
            step_dispatch<T, ORDER, kStepPrevScaled | kStepNoDiv>(g, cur, prev, kap, S, cs, sn, zc, scol, st);
            break;
        default: break;
    }
}

}  // namespace

// ---- launchers ------------------------------------------------------------------------
template <typename T>
void launch_step(const Geom& g, int order, const T* cur, T* prev, const T* kap, const T* S, double cs,
                 double sn, int flags, int zc, cudaStream_t st, const unsigned char* scol) {
    note_launch(1);
    if (order == 2)
        step_flags<T, 2>(g, cur, prev, kap, S, cs, sn, flags, zc, scol, st);
    else
        step_flags<T, 4>(g, cur, prev, kap, S, cs, sn, flags, zc, scol, st);
}

void launch_source_columns(const Geom& g, const double* S, unsigned char* scol, cudaStream_t st) {
    note_launch(1);
    const long long plane = (long long)g.sx * g.sy;
    const unsigned blocks = (unsigned)std::min<long long>((plane + kThreads - 1) / kThreads, 4096);
    k_source_columns<<<blocks, kThreads, 0, st>>>(g, S, scol);
}

template <typename T>
void launch_start(const Geom& g, int order, const T* w0t, const double* w1, T* y0, T* y1, const T* kap,
                  const double* S, double dt, int zc, cudaStream_t st, bool w1_float) {
    note_launch(1);
    const dim3 grid = plane_grid(g, zc);
    if constexpr (std::is_same<T, float>::value) {
        if (w1_float) {  // FP32 CG vectors: w1 holds floats
            const float* w1f = (const float*)w1;
            if (order == 2) {
                if (S) k_start<T, 2, true, float><<<grid, kThreads, 0, st>>>(w0t, w1f, y0, y1, kap, S, g, dt, zc);
                else k_start<T, 2, false, float><<<grid, kThreads, 0, st>>>(w0t, w1f, y0, y1, kap, S, g, dt, zc);
            } else {
                if (S) k_start<T, 4, true, float><<<grid, kThreads, 0, st>>>(w0t, w1f, y0, y1, kap, S, g, dt, zc);
                else k_start<T, 4, false, float><<<grid, kThreads, 0, st>>>(w0t, w1f, y0, y1, kap, S, g, dt, zc);
            }
            return;
        }
    }
    if (order == 2) {
        if (S) k_start<T, 2, true><<<grid, kThreads, 0, st>>>(w0t, w1, y0, y1, kap, S, g, dt, zc);
        else k_start<T, 2, false><<<grid, kThreads, 0, st>>>(w0t, w1, y0, y1, kap, S, g, dt, zc);
    } else {
        if (S) k_start<T, 4, true><<<grid, kThreads, 0, st>>>(w0t, w1, y0, y1, kap, S, g, dt, zc);
        else k_start<T, 4, false><<<grid, kThreads, 0, st>>>(w0t, w1, y0, y1, kap, S, g, dt, zc);
    }
}

template <typename T>
void launch_end(const Geom& g, int order, int mode, const T* yN, const T* yNm1, const T* w0t, const double* w1,
                const T* kap, const T* mass, const double* S, double cs, double sn, double* out0, double* out1,
                Red red, double dt, int zc, cudaStream_t st) {
    note_launch(1);
    const dim3 grid = plane_grid(g, zc);
#define CMCG_END(O, SRC, MODE)                                                                                \
    k_end<T, O, SRC, MODE><<<grid, kThreads, 0, st>>>(yN, yNm1, w0t, w1, kap, mass, S, cs, sn, out0, out1, red, \
                                                      g, dt, zc)
    const bool src = S != nullptr;
    if constexpr (std::is_same<T, float>::value) {
        if (mode == 2) {
            if (order == 2) { if (src) CMCG_END(2, true, 2); else CMCG_END(2, false, 2); }
            else { if (src) CMCG_END(4, true, 2); else CMCG_END(4, false, 2); }
            return;
        }
        if (mode == 3) {  // mode 2 with FP32 CG vectors: w1 holds floats
            const float* w1f = (const float*)w1;
#define CMCG_END3(O, SRC)                                                                                      \
    k_end<T, O, SRC, 2, float><<<grid, kThreads, 0, st>>>(yN, yNm1, w0t, w1f, kap, mass, S, cs, sn, out0, out1, \
                                                          red, g, dt, zc)
            if (order == 2) { if (src) CMCG_END3(2, true); else CMCG_END3(2, false); }
            else { if (src) CMCG_END3(4, true); else CMCG_END3(4, false); }
#undef CMCG_END3
            return;
        }
    }
    if (order == 2) {
        if (mode == 0) { if (src) CMCG_END(2, true, 0); else CMCG_END(2, false, 0); }
        else { if (src) CMCG_END(2, true, 1); else CMCG_END(2, false, 1); }
    } else {
        if (mode == 0) { if (src) CMCG_END(4, true, 0); else CMCG_END(4, false, 0); }
        else { if (src) CMCG_END(4, true, 1); else CMCG_END(4, false, 1); }
    }
#undef CMCG_END
}

template <typename T>
void launch_adj_prep(const Geom& g, const double* b, const T* mass, const T* kap, T* t, int zc,
                     cudaStream_t st) {
    note_launch(1);
    k_adj_prep<T><<<plane_grid(g, zc), kThreads, 0, st>>>(b, mass, kap, t, g, zc);
}

template <typename T, typename A>
void launch_adj_start(const Geom& g, int order, const A* a, const T* t, const T* mass, const T* kap,
                      T* cur, T* prev, double dt, int zc, cudaStream_t st) {
    note_launch(1);
    if (order == 2)
        k_adj_start<T, 2, A><<<plane_grid(g, zc), kThreads, 0, st>>>(a, t, mass, kap, cur, prev, g, dt, zc);
    else
        k_adj_start<T, 4, A><<<plane_grid(g, zc), kThreads, 0, st>>>(a, t, mass, kap, cur, prev, g, dt, zc);
}

template <typename T>
void launch_adj_final(const Geom& g, int order, int mode, const T* s, const T* u1, const T* mass, const T* kap,
                      const double* minv, const double* z0, const double* z1, const double* d0, const double* d1,
                      double* o0, double* o1, double* gt1, Red red, double dt, int zc, cudaStream_t st) {
    note_launch(1);
    const dim3 grid = plane_grid(g, zc);
#define CMCG_FIN(O, MODE)                                                                                        \
    k_adj_final<T, O, MODE><<<grid, kThreads, 0, st>>>(s, u1, mass, kap, minv, z0, z1, d0, d1, o0, o1, gt1, red, g, \
                                                       dt, zc)
    if constexpr (std::is_same<T, float>::value) {
        if (mode == 2) {
            if (order == 2) CMCG_FIN(2, 2); else CMCG_FIN(4, 2);
            return;
        }
        if (mode == 3) {  // mode 2 with FP32 CG vectors: d and the gradient are floats
            const float *d0f = (const float*)d0, *d1f = (const float*)d1;
            float *o0f = (float*)o0, *o1f = (float*)o1;
#define CMCG_FIN3(O)                                                                                               \
    k_adj_final<T, O, 2, float><<<grid, kThreads, 0, st>>>(s, u1, mass, kap, minv, z0, z1, d0f, d1f, o0f, o1f, gt1, \
                                                           red, g, dt, zc)
            if (order == 2) CMCG_FIN3(2); else CMCG_FIN3(4);
#undef CMCG_FIN3
            return;
        }
    }
    if (order == 2) {
        if (mode == 0) CMCG_FIN(2, 0); else CMCG_FIN(2, 1);
    } else {
        if (mode == 0) CMCG_FIN(4, 0); else CMCG_FIN(4, 1);
    }
#undef CMCG_FIN
}

void launch_make_source(const Geom& g, const double* f, const double* gb, const double* kap64, double* S, int zc,
                        bool accumulate, cudaStream_t st) {
    note_launch(1);
    k_make_source<<<plane_grid(g, zc), kThreads, 0, st>>>(f, gb, kap64, S, g, zc, accumulate ? 1 : 0);
}

long long plane_blocks(const Geom& g, int zc) {
    const dim3 d = plane_grid(g, zc);
    return (long long)d.x * d.y;
}

#define CMCG_INST(T)                                                                                           \
    template void launch_step<T>(const Geom&, int, const T*, T*, const T*, const T*, double, double, int,        \
                                 int, cudaStream_t, const unsigned char*);                                     \
    template void launch_start<T>(const Geom&, int, const T*, const double*, T*, T*, const T*, const double*,   \
                                  double, int, cudaStream_t, bool);                                            \
    template void launch_end<T>(const Geom&, int, int, const T*, const T*, const T*, const double*, const T*,   \
                                const T*, const double*, double, double, double*, double*, Red, double,         \
                                int, cudaStream_t);                                                            \
    template void launch_adj_prep<T>(const Geom&, const double*, const T*, const T*, T*, int, cudaStream_t);    \
    template void launch_adj_start<T, double>(const Geom&, int, const double*, const T*, const T*, const T*,    \
                                              T*, T*, double, int, cudaStream_t);                               \
    template void launch_adj_final<T>(const Geom&, int, int, const T*, const T*, const T*, const T*,           \
                                      const double*, const double*, const double*, const double*, const double*, \
                                      double*, double*, double*, Red, double, int, cudaStream_t);
CMCG_INST(float)
CMCG_INST(double)
#undef CMCG_INST
template void launch_adj_start<float, float>(const Geom&, int, const float*, const float*, const float*,
                                             const float*, float*, float*, double, int, cudaStream_t);

}  // namespace cmcg

namespace cmcg {

int batch_steps_max_blocks(bool forced) {
    int per_sm = 0, sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (forced) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_steps<true>, kThreads, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_steps<false>, kThreads, 0);
    return per_sm * sms;
}

bool step_vec4_ok(const Geom& g, const void* cur, const void* prev, const void* kap) {
    return step_v4_ok(g, cur, prev, kap);
}

cudaError_t launch_batch_steps(const BatchItem* items, int nitems, int total_blocks, int max_steps, unsigned* bar,
                               int* err, int grid, cudaStream_t st, bool forced) {
    note_launch(1);
    long long spin = kBarrierSpinLimit;
    void* args[] = {(void*)&items, (void*)&nitems, (void*)&total_blocks, (void*)&max_steps, (void*)&bar, (void*)&err,
                    (void*)&spin};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kThreads);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, forced ? (const void*)k_batch_steps<true> : (const void*)k_batch_steps<false>, args);
}

cudaError_t launch_barrier_selftest(unsigned* bar, int* err, long long spin_limit, cudaStream_t st) {
    note_launch(1);
    k_barrier_selftest<<<1, kThreads, 0, st>>>(bar, err, spin_limit);
    return cudaGetLastError();
}

}  // namespace cmcg

namespace cmcg {

void launch_filter_init(long long n, const double* w0, const double* w1, const double* kap64, double inv_wh,
                        double* acc, cudaStream_t st) {
    note_launch(1);
    const unsigned blocks = (unsigned)std::min<long long>((n + kThreads - 1) / kThreads, 152 * 8);
    k_filter_init<<<blocks, kThreads, 0, st>>>(n, w0, w1, kap64, inv_wh, acc);
}

void launch_step_filter(const Geom& g, int order, const double* cur, double* prev, const double* kap,
                        const double* S, double cs, double sn, double* acc, double fc, double fs, double cv, int zc,
                        cudaStream_t st) {
    note_launch(1);
    if (order == 2)
        k_step_filter<2><<<plane_grid(g, zc), kThreads, 0, st>>>(cur, prev, kap, S, cs, sn, acc, fc, fs, cv, g, zc);
    else
        k_step_filter<4><<<plane_grid(g, zc), kThreads, 0, st>>>(cur, prev, kap, S, cs, sn, acc, fc, fs, cv, g, zc);
}

void launch_scale_complex(long long n, double* u, double s, cudaStream_t st) {
    note_launch(1);
    const unsigned blocks = (unsigned)std::min<long long>((2 * n + kThreads - 1) / kThreads, 152 * 8);
    k_scale_complex<<<blocks, kThreads, 0, st>>>(n, u, s);
}

}  // namespace cmcg

namespace cmcg {
CMCG_CHECK_TU(wave)
}  // namespace cmcg
