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

#include "common.cuh"
#include "kernels.h"

namespace cmcg {

namespace {

constexpr int kThreads = 256;

struct PlaneMap {
    int ix, iy, z0, z1;
    bool valid;
};

__device__ __forceinline__ PlaneMap plane_map(const Geom& g, int zc) {
    PlaneMap m;
    const long long plane = (long long)g.sx * g.sy;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    m.valid = p < plane;
    const long long pp = m.valid ? p : 0;
    m.iy = (int)(pp / g.sx);
    m.ix = (int)(pp - (long long)m.iy * g.sx);
    m.z0 = blockIdx.y * zc;
    m.z1 = min(m.z0 + zc, g.sz);
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
                                                   const T* __restrict__ kap, const double* __restrict__ S,
                                                   double cs, double sn, Geom g, int zc) {
    const PlaneMap m = plane_map(g, zc);
    if (!m.valid) return;
    Ld<T> f{cur};
    for (int iz = m.z0; iz < m.z1; ++iz) {
        const long long j = node(g, m.ix, m.iy, iz);
        const T L = lap_t<ORDER, T>(g, f, j, m.ix, m.iy, iz);
        const T k = kap[j];
        const T yp = prev_out[j];
        T rhs = T(2) * cur[j] - k * L;
        if (FLAGS & kStepSrc) rhs += (T)(S[2 * j] * cs + S[2 * j + 1] * sn);
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

// Leapfrog step, 3D 2nd order: z-neighbours carried in registers along the march.
template <typename T, int FLAGS>
__global__ void __launch_bounds__(kThreads) k_step3d7(const T* __restrict__ cur, T* __restrict__ prev_out,
                                                      const T* __restrict__ kap, const double* __restrict__ S,
                                                      double cs, double sn, Geom g, int zc) {
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
    T ym = cur[j + (m.z0 > 0 ? -sZ : sZ)];
    T yc = cur[j];
    for (int iz = m.z0; iz < m.z1; ++iz) {
        const T yz = cur[j + (iz < g.nz ? sZ : -sZ)];
        const T L = T(6) * yc - ((cur[j + oxm] + cur[j + oxp]) + (cur[j + oym] + cur[j + oyp]) + (ym + yz));
        const T k = kap[j];
        const T yp = prev_out[j];
        T rhs = T(2) * yc - k * L;
        if (FLAGS & kStepSrc) rhs += (T)(S[2 * j] * cs + S[2 * j + 1] * sn);
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
template <typename T, int ORDER, bool SRC>
__global__ void __launch_bounds__(kThreads) k_start(const T* __restrict__ w0t, const double* __restrict__ w1,
                                                    T* __restrict__ y0, T* __restrict__ y1,
                                                    const T* __restrict__ kap, const double* __restrict__ S,
                                                    Geom g, double dt, int zc) {
    const PlaneMap m = plane_map(g, zc);
    if (!m.valid) return;
    Ld<T> f{w0t};
    const T dtT = (T)dt;
    for (int iz = m.z0; iz < m.z1; ++iz) {
        const long long j = node(g, m.ix, m.iy, iz);
        const T k = kap[j];
        if (k == T(0)) {
            y0[j] = T(0);
            y1[j] = T(0);
            continue;
        }
        const T L = lap_t<ORDER, T>(g, f, j, m.ix, m.iy, iz);
        const T beta = (T)num_abc(g, m.ix, m.iy, iz) * sqrt(k);
        const T w0j = w0t[j];
        T v = w0j + dtT * (T(1) - beta) * (T)w1[j] - T(0.5) * k * L;
        if (SRC) v += (T)(0.5 * S[2 * j]);
        y0[j] = w0j;
        y1[j] = v;
    }
}

// Period end: vN, mismatch, energy operator and J (MODE 0), or (uT, vT) (MODE 1).
template <typename T, int ORDER, bool SRC, int MODE>
__global__ void __launch_bounds__(kThreads) k_end(const T* __restrict__ yN, const T* __restrict__ yNm1,
                                                  const T* __restrict__ w0t, const double* __restrict__ w1,
                                                  const T* __restrict__ kap, const double* __restrict__ mass,
                                                  const double* __restrict__ S, double cs, double sn,
                                                  double* __restrict__ out0, double* __restrict__ out1,
                                                  Red red, Geom g, double dt, int zc) {
    const PlaneMap m = plane_map(g, zc);
    double acc[1] = {0.0};
    if (m.valid) {
        Ld<T> fy{yN};
        DiffT<T> fe{yN, w0t};
        const T ih2 = T(1) / (T)(g.h * g.h);
        const T dtT = (T)dt;
        for (int iz = m.z0; iz < m.z1; ++iz) {
            const long long j = node(g, m.ix, m.iy, iz);
            const T k = kap[j];
            if (k == T(0)) {
                out0[j] = 0.0;
                out1[j] = 0.0;
                continue;
            }
            const T L = lap_t<ORDER, T>(g, fy, j, m.ix, m.iy, iz);
            const T beta = (T)num_abc(g, m.ix, m.iy, iz) * sqrt(k);
            T src = T(0);
            if (SRC) src = (T)(S[2 * j] * cs + S[2 * j + 1] * sn);
            const T yn = yN[j];
            const T vN = ((yn - yNm1[j]) / dtT + (src - k * L) / (T(2) * dtT)) / (T(1) + beta);
            if (MODE == 1) {
                out0[j] = (double)yn;
                out1[j] = (double)vN;
            } else {
                const T e0 = yn - w0t[j];
                const T e1 = vN - (T)w1[j];
                const T W = weight_t<T>(g, m.ix, m.iy, iz);
                const T z0 = W * ih2 * lap_t<ORDER, T>(g, fe, j, m.ix, m.iy, iz);
                const T z1 = (T)mass[j] * e1;
                out0[j] = (double)z0;
                out1[j] = (double)z1;
                acc[0] += 0.5 * (double)(e0 * z0 + e1 * z1);
            }
        }
    }
    if (MODE == 0) {
        if (grid_sum<1>(acc, red.partials, red.ticket) && threadIdx.x == 0) red.sc[SC_J] = acc[0];
    }
}

// Adjoint start, part 1: t = D^-1 b = b / (M (1 + beta)).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_adj_prep(const double* __restrict__ b, const double* __restrict__ mass,
                                                       const T* __restrict__ kap, T* __restrict__ t, Geom g, int zc) {
    const PlaneMap m = plane_map(g, zc);
    if (!m.valid) return;
    for (int iz = m.z0; iz < m.z1; ++iz) {
        const long long j = node(g, m.ix, m.iy, iz);
        const T k = kap[j];
        if (k == T(0)) {
            t[j] = T(0);
            continue;
        }
        const T beta = (T)num_abc(g, m.ix, m.iy, iz) * sqrt(k);
        t[j] = (T)b[j] / ((T)mass[j] * (T(1) + beta));
    }
}

// Adjoint start, part 2 (transposed end velocity):
//   ybar_N = a + M t / dt - (dt/2) K t,  u_{N-1} = D^-1 ybar_N,  prev = C u_N / M = t / dt.
template <typename T, int ORDER>
__global__ void __launch_bounds__(kThreads) k_adj_start(const double* __restrict__ a, const T* __restrict__ t,
                                                        const double* __restrict__ mass, const T* __restrict__ kap,
                                                        T* __restrict__ cur, T* __restrict__ prev, Geom g, double dt,
                                                        int zc) {
    const PlaneMap m = plane_map(g, zc);
    if (!m.valid) return;
    Ld<T> f{t};
    const T dtT = (T)dt;
    for (int iz = m.z0; iz < m.z1; ++iz) {
        const long long j = node(g, m.ix, m.iy, iz);
        const T k = kap[j];
        if (k == T(0)) {
            cur[j] = T(0);
            prev[j] = T(0);
            continue;
        }
        const T L = lap_t<ORDER, T>(g, f, j, m.ix, m.iy, iz);
        const T beta = (T)num_abc(g, m.ix, m.iy, iz) * sqrt(k);
        const T tj = t[j];
        const T u = ((T)a[j] / (T)mass[j] + tj / dtT - k * L / (T(2) * dtT)) / (T(1) + beta);
        cur[j] = u;
        prev[j] = tj / dtT;
    }
}

// Adjoint final (transposed start half-kick), from s = M^-1 ybar_1 and u_1:
//   q0 = M (s - (1 - beta) u_1) - (dt^2/2) K s,   q1 = dt M (1 - beta) s.
// MODE 1 writes q.  MODE 0 forms the CG gradient ghat = q - z, g~1 = ghat1 / M, and reduces
// (ghat . d, sum ghat0) in FP64.
template <typename T, int ORDER, int MODE>
__global__ void __launch_bounds__(kThreads) k_adj_final(const T* __restrict__ s, const T* __restrict__ u1,
                                                        const double* __restrict__ mass, const T* __restrict__ kap,
                                                        const double* __restrict__ minv,
                                                        const double* __restrict__ z0, const double* __restrict__ z1,
                                                        const double* __restrict__ d0, const double* __restrict__ d1,
                                                        double* __restrict__ o0, double* __restrict__ o1,
                                                        double* __restrict__ gt1, Red red, Geom g, double dt, int zc) {
    const PlaneMap m = plane_map(g, zc);
    double acc[2] = {0.0, 0.0};
    if (m.valid) {
        Ld<T> f{s};
        const T ih2 = T(1) / (T)(g.h * g.h);
        const T dtT = (T)dt;
        for (int iz = m.z0; iz < m.z1; ++iz) {
            const long long j = node(g, m.ix, m.iy, iz);
            const T k = kap[j];
            if (k == T(0)) {
                o0[j] = 0.0;
                o1[j] = 0.0;
                if (MODE == 0) gt1[j] = 0.0;
                continue;
            }
            const T L = lap_t<ORDER, T>(g, f, j, m.ix, m.iy, iz);
            const T beta = (T)num_abc(g, m.ix, m.iy, iz) * sqrt(k);
            const T W = weight_t<T>(g, m.ix, m.iy, iz);
            const T M = (T)mass[j];
            const T sj = s[j];
            const T q0 = M * (sj - (T(1) - beta) * u1[j]) - T(0.5) * dtT * dtT * W * ih2 * L;
            const T q1 = dtT * M * (T(1) - beta) * sj;
            if (MODE == 1) {
                o0[j] = (double)q0;
                o1[j] = (double)q1;
            } else {
                const double g0 = (double)q0 - z0[j];
                const double g1 = (double)q1 - z1[j];
                o0[j] = g0;
                o1[j] = g1;
                gt1[j] = g1 * minv[j];
                acc[0] += g0 * d0[j] + g1 * d1[j];
                acc[1] += g0;
            }
        }
    }
    if (MODE == 0) {
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

inline dim3 plane_grid(const Geom& g, int zc) {
    const long long plane = (long long)g.sx * g.sy;
    return dim3((unsigned)((plane + kThreads - 1) / kThreads), (unsigned)((g.sz + zc - 1) / zc), 1);
}

template <typename T, int ORDER, int FLAGS>
void step_dispatch(const Geom& g, const T* cur, T* prev, const T* kap, const double* S, double cs, double sn,
                   int zc, cudaStream_t st) {
    if (ORDER == 2 && g.dim == 3) {
        k_step3d7<T, FLAGS><<<plane_grid(g, zc), kThreads, 0, st>>>(cur, prev, kap, S, cs, sn, g, zc);
    } else {
        k_step<T, ORDER, FLAGS><<<plane_grid(g, zc), kThreads, 0, st>>>(cur, prev, kap, S, cs, sn, g, zc);
    }
}

template <typename T, int ORDER>
void step_flags(const Geom& g, const T* cur, T* prev, const T* kap, const double* S, double cs, double sn,
                int flags, int zc, cudaStream_t st) {
    switch (flags) {
        case 0: step_dispatch<T, ORDER, 0>(g, cur, prev, kap, S, cs, sn, zc, st); break;
        case kStepSrc: step_dispatch<T, ORDER, kStepSrc>(g, cur, prev, kap, S, cs, sn, zc, st); break;
        case kStepPrevScaled: step_dispatch<T, ORDER, kStepPrevScaled>(g, cur, prev, kap, S, cs, sn, zc, st); break;
        case kStepNoDiv: step_dispatch<T, ORDER, kStepNoDiv>(g, cur, prev, kap, S, cs, sn, zc, st); break;
        case kStepPrevScaled | kStepNoDiv:
            step_dispatch<T, ORDER, kStepPrevScaled | kStepNoDiv>(g, cur, prev, kap, S, cs, sn, zc, st);
            break;
        default: break;
    }
}

}  // namespace

// ---- launchers ------------------------------------------------------------------------
template <typename T>
void launch_step(const Geom& g, int order, const T* cur, T* prev, const T* kap, const double* S, double cs,
                 double sn, int flags, int zc, cudaStream_t st) {
    note_launch(1);
    if (order == 2)
        step_flags<T, 2>(g, cur, prev, kap, S, cs, sn, flags, zc, st);
    else
        step_flags<T, 4>(g, cur, prev, kap, S, cs, sn, flags, zc, st);
}

template <typename T>
void launch_start(const Geom& g, int order, const T* w0t, const double* w1, T* y0, T* y1, const T* kap,
                  const double* S, double dt, int zc, cudaStream_t st) {
    note_launch(1);
    const dim3 grid = plane_grid(g, zc);
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
                const T* kap, const double* mass, const double* S, double cs, double sn, double* out0, double* out1,
                Red red, double dt, int zc, cudaStream_t st) {
    note_launch(1);
    const dim3 grid = plane_grid(g, zc);
#define CMCG_END(O, SRC, MODE)                                                                                \
    k_end<T, O, SRC, MODE><<<grid, kThreads, 0, st>>>(yN, yNm1, w0t, w1, kap, mass, S, cs, sn, out0, out1, red, \
                                                      g, dt, zc)
    const bool src = S != nullptr;
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
void launch_adj_prep(const Geom& g, const double* b, const double* mass, const T* kap, T* t, int zc,
                     cudaStream_t st) {
    note_launch(1);
    k_adj_prep<T><<<plane_grid(g, zc), kThreads, 0, st>>>(b, mass, kap, t, g, zc);
}

template <typename T>
void launch_adj_start(const Geom& g, int order, const double* a, const T* t, const double* mass, const T* kap,
                      T* cur, T* prev, double dt, int zc, cudaStream_t st) {
    note_launch(1);
    if (order == 2)
        k_adj_start<T, 2><<<plane_grid(g, zc), kThreads, 0, st>>>(a, t, mass, kap, cur, prev, g, dt, zc);
    else
        k_adj_start<T, 4><<<plane_grid(g, zc), kThreads, 0, st>>>(a, t, mass, kap, cur, prev, g, dt, zc);
}

template <typename T>
void launch_adj_final(const Geom& g, int order, int mode, const T* s, const T* u1, const double* mass, const T* kap,
                      const double* minv, const double* z0, const double* z1, const double* d0, const double* d1,
                      double* o0, double* o1, double* gt1, Red red, double dt, int zc, cudaStream_t st) {
    note_launch(1);
    const dim3 grid = plane_grid(g, zc);
#define CMCG_FIN(O, MODE)                                                                                        \
    k_adj_final<T, O, MODE><<<grid, kThreads, 0, st>>>(s, u1, mass, kap, minv, z0, z1, d0, d1, o0, o1, gt1, red, g, \
                                                       dt, zc)
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
    template void launch_step<T>(const Geom&, int, const T*, T*, const T*, const double*, double, double, int,   \
                                 int, cudaStream_t);                                                           \
    template void launch_start<T>(const Geom&, int, const T*, const double*, T*, T*, const T*, const double*,   \
                                  double, int, cudaStream_t);                                                  \
    template void launch_end<T>(const Geom&, int, int, const T*, const T*, const T*, const double*, const T*,   \
                                const double*, const double*, double, double, double*, double*, Red, double,    \
                                int, cudaStream_t);                                                            \
    template void launch_adj_prep<T>(const Geom&, const double*, const double*, const T*, T*, int, cudaStream_t); \
    template void launch_adj_start<T>(const Geom&, int, const double*, const T*, const double*, const T*, T*,   \
                                      T*, double, int, cudaStream_t);                                          \
    template void launch_adj_final<T>(const Geom&, int, int, const T*, const T*, const double*, const T*,       \
                                      const double*, const double*, const double*, const double*, const double*, \
                                      double*, double*, double*, Red, double, int, cudaStream_t);
CMCG_INST(float)
CMCG_INST(double)
#undef CMCG_INST

}  // namespace cmcg
