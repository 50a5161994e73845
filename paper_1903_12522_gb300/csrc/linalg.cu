// Coefficient setup, the CG recurrences of the CMCG Algorithm (Sec. 2.3, Steps (4) and
// 5.3-5.8) with every scalar kept on the device, and the solution recovery of Step (6) with
// the compatibility-condition shift of Sec. 2.1.
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

// ---- setup -------------------------------------------------------------------------------
// kappa = c^2 dt^2 / h^2, M = W / c^2, zero on Dirichlet nodes.  Reduces (sum M, sum B,
// sum W) over active nodes, the number of invalid c and the number of Dirichlet nodes into
// sc[0..5), max c into sc[5] and min c into sc[6] (as bit patterns of positive doubles, which
// order like unsigned integers; sc[6] must start as all ones).
__global__ void __launch_bounds__(kT) k_setup(const double* __restrict__ c, const unsigned char* __restrict__ umask,
                                              unsigned face_dir, double dt, double* __restrict__ kap64,
                                              float* __restrict__ kap32, double* __restrict__ mass,
                                              unsigned char* __restrict__ mask, Red red, Geom g) {
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    unsigned long long cmax_bits = 0ull, cmin_bits = ~0ull;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < g.np; j += stride) {
        const unsigned t = (unsigned)j / (unsigned)g.sx;
        const int ix = (int)((unsigned)j - t * (unsigned)g.sx);
        const int iz = (int)(t / (unsigned)g.sy);
        const int iy = (int)(t - (unsigned)iz * (unsigned)g.sy);
        bool dir = umask ? (umask[j] != 0) : false;
        dir |= (ix == 0) && (face_dir & 1u);
        dir |= (ix == g.nx) && (face_dir & 2u);
        dir |= (iy == 0) && (face_dir & 4u);
        dir |= (iy == g.ny) && (face_dir & 8u);
        if (g.dim == 3) {
            dir |= (iz == 0) && (face_dir & 16u);
            dir |= (iz == g.nz) && (face_dir & 32u);
        }
        const double cj = c[j];
        if (!(cj > 0.0) || !isfinite(cj)) acc[3] += 1.0;
        const double W = weight(g, ix, iy, iz);
        if (dir) {
            kap64[j] = 0.0;
            mass[j] = 0.0;
            if (kap32) kap32[j] = 0.f;
            mask[j] = 1;
            acc[4] += 1.0;
        } else {
            const double k = cj * cj * dt * dt / (g.h * g.h);
            kap64[j] = k;
            mass[j] = W / (cj * cj);
            if (kap32) kap32[j] = (float)k;
            mask[j] = 0;
            acc[0] += W / (cj * cj);
            acc[1] += W * 2.0 * num_abc(g, ix, iy, iz) / g.h / cj;
            acc[2] += W;
        }
        if (cj > 0.0 && isfinite(cj)) {
            const unsigned long long bits = (unsigned long long)__double_as_longlong(cj);
            cmax_bits = bits > cmax_bits ? bits : cmax_bits;
            cmin_bits = bits < cmin_bits ? bits : cmin_bits;
        }
    }
    // max c: order-independent atomic on the bit pattern of positive doubles
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long other = __shfl_down_sync(0xffffffffu, cmax_bits, o);
        cmax_bits = other > cmax_bits ? other : cmax_bits;
        other = __shfl_down_sync(0xffffffffu, cmin_bits, o);
        cmin_bits = other < cmin_bits ? other : cmin_bits;
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax((unsigned long long*)&red.sc[5], cmax_bits);
        atomicMin((unsigned long long*)&red.sc[6], cmin_bits);
    }
    if (grid_sum<5>(acc, red.partials, red.ticket) && threadIdx.x == 0) {
        for (int k = 0; k < 5; ++k) red.sc[k] = acc[k];
    }
}

__global__ void k_mask_copy(const double* __restrict__ in, const double* __restrict__ kap64, double* __restrict__ out,
                            long long n) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride)
        out[j] = kap64[j] == 0.0 ? 0.0 : in[j];
}

__global__ void k_fill(double* p, long long n, double v) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) p[j] = v;
}

// Warm start: the periodic initial state of a time-harmonic field U (interleaved re, im) is
// (v0, v1) = (Re U, omega_hat Im U), the fixed-point relation of step (6) read backwards;
// Dirichlet nodes (kappa = 0) hold 0.
__global__ void k_warm_start(long long n, const double* __restrict__ u, const double* __restrict__ kap64, double wh,
                             double* __restrict__ w0, double* __restrict__ w1) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        const bool act = kap64[j] != 0.0;
        w0[j] = act ? u[2 * j] : 0.0;
        w1[j] = act ? wh * u[2 * j + 1] : 0.0;
    }
}

// ---- CG -----------------------------------------------------------------------------------
// Step (4): r = d = g~, rhat = ghat (= E r), gamma = r . rhat = ||r||_E^2.
__global__ void __launch_bounds__(kT) k_cg_init(long long n, const double* __restrict__ gt0,
                                                const double* __restrict__ gt1, const double* __restrict__ gh0,
                                                const double* __restrict__ gh1, double* __restrict__ r0,
                                                double* __restrict__ r1, double* __restrict__ rh0,
                                                double* __restrict__ rh1, double* __restrict__ d0,
                                                double* __restrict__ d1, Red red) {
    double acc[1] = {0.0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        const double a0 = gt0[j], a1 = gt1[j], b0 = gh0[j], b1 = gh1[j];
        r0[j] = a0;
        r1[j] = a1;
        d0[j] = a0;
        d1[j] = a1;
        rh0[j] = b0;
        rh1[j] = b1;
        acc[0] += a0 * b0 + a1 * b1;
    }
    if (grid_sum<1>(acc, red.partials, red.ticket) && threadIdx.x == 0) {
        red.sc[SC_GAMMA] = acc[0];
        red.sc[SC_GAMMA0] = acc[0];
        red.sc[SC_REL] = acc[0] > 0.0 ? 1.0 : 0.0;
        red.sc[SC_STATUS] = (isfinite(acc[0]) && acc[0] >= 0.0) ? 0.0 : 1.0;
    }
}

// Steps 5.3-5.6: alpha = gamma / (ghat . d); v -= alpha d; r -= alpha g~; rhat -= alpha ghat;
// gamma' = r . rhat; beta = gamma'/gamma (stored for Step 5.7); rel = sqrt(gamma'/gamma0).
__global__ void __launch_bounds__(kT) k_cg_update(long long n, double* __restrict__ w0, double* __restrict__ w1,
                                                  double* __restrict__ r0, double* __restrict__ r1,
                                                  double* __restrict__ rh0, double* __restrict__ rh1,
                                                  const double* __restrict__ d0, const double* __restrict__ d1,
                                                  const double* __restrict__ gt0, const double* __restrict__ gt1,
                                                  const double* __restrict__ gh0, const double* __restrict__ gh1,
                                                  double sign, Red red) {
    const double gamma = red.sc[SC_GAMMA];
    const double gd = red.sc[SC_GD];
    const double alpha = gamma / gd;
    double acc[1] = {0.0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        const double a0 = d0[j], a1 = d1[j];
        w0[j] += sign * alpha * a0;
        w1[j] += sign * alpha * a1;
        const double x0 = r0[j] - alpha * gt0[j];
        const double x1 = r1[j] - alpha * gt1[j];
        const double y0 = rh0[j] - alpha * gh0[j];
        const double y1 = rh1[j] - alpha * gh1[j];
        r0[j] = x0;
        r1[j] = x1;
        rh0[j] = y0;
        rh1[j] = y1;
        acc[0] += x0 * y0 + x1 * y1;
    }
    if (grid_sum<1>(acc, red.partials, red.ticket) && threadIdx.x == 0) {
        const double gnew = acc[0];
        red.sc[SC_ALPHA] = alpha;
        red.sc[SC_GAMMA_NEW] = gnew;
        red.sc[SC_BETA] = gnew / gamma;
        red.sc[SC_GAMMA] = gnew;
        const double g0 = red.sc[SC_GAMMA0];
        red.sc[SC_REL] = sqrt(fmax(gnew, 0.0) / g0);
        const bool bad = !isfinite(alpha) || !(gd > 0.0) || !isfinite(gnew);
        if (bad) red.sc[SC_STATUS] = 1.0;
    }
}

// Step 5.7: d = r + beta d; with d0f, also float(d0) (what FP32 periods read).  V: the CG
// vectors' type (float: the inner solve of mixed precision, whose periods read d0 directly).
template <typename V>
__global__ void __launch_bounds__(kT) k_cg_direction(long long n, const V* __restrict__ r0,
                                                     const V* __restrict__ r1, V* __restrict__ d0,
                                                     V* __restrict__ d1, float* __restrict__ d0f,
                                                     const double* __restrict__ sc) {
    const V beta = (V)sc[SC_BETA];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        const V v = r0[j] + beta * d0[j];
        d0[j] = v;
        d1[j] = r1[j] + beta * d1[j];
        if (d0f) d0f[j] = (float)v;
    }
}

// r . rhat into sc[slot] (used by the defect-correction outer residual).
__global__ void __launch_bounds__(kT) k_dot2(long long n, const double* __restrict__ a0, const double* __restrict__ a1,
                                             const double* __restrict__ b0, const double* __restrict__ b1, Red red,
                                             int slot) {
    double acc[1] = {0.0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride)
        acc[0] += a0[j] * b0[j] + a1[j] * b1[j];
    if (grid_sum<1>(acc, red.partials, red.ticket) && threadIdx.x == 0) red.sc[slot] = acc[0];
}

// Step (6): u = v0 + i v1 / omega_hat (interleaved complex) and the sums entering the
// compatibility condition: 1.F^, 1.(M u), 1.(B u), with F^ = W S / (kappa h^2) recovered
// from the stored source S = dt^2 M^-1 F^ (S may be null: no source).
__global__ void __launch_bounds__(kT) k_recover(Geom g, const double* __restrict__ w0, const double* __restrict__ w1,
                                                double inv_wh, const double* __restrict__ S,
                                                const double* __restrict__ kap64, const double* __restrict__ mass,
                                                double* __restrict__ u, Red red) {
    double acc[6] = {0, 0, 0, 0, 0, 0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < g.np; j += stride) {
        const double k = kap64[j];
        if (k == 0.0) {
            u[2 * j] = 0.0;
            u[2 * j + 1] = 0.0;
            continue;
        }
        const unsigned t = (unsigned)j / (unsigned)g.sx;
        const int ix = (int)((unsigned)j - t * (unsigned)g.sx);
        const int iz = (int)(t / (unsigned)g.sy);
        const int iy = (int)(t - (unsigned)iz * (unsigned)g.sy);
        const double re = w0[j], im = w1[j] * inv_wh;
        u[2 * j] = re;
        u[2 * j + 1] = im;
        const double W = weight(g, ix, iy, iz);
        const double M = mass[j];
        const double a = 2.0 * num_abc(g, ix, iy, iz) / g.h;   // A / W
        const double B = a * sqrt(W * M);                       // A / c
        if (S) {
            const double sc = W / (k * g.h * g.h);
            acc[0] += sc * S[2 * j];
            acc[1] += sc * S[2 * j + 1];
        }
        acc[2] += M * re;
        acc[3] += M * im;
        acc[4] += B * re;
        acc[5] += B * im;
    }
    if (grid_sum<6>(acc, red.partials, red.ticket) && threadIdx.x == 0) {
        for (int k = 0; k < 6; ++k) red.sc[SC_R0 + k] = acc[k];
    }
}

// The sums of the discrete compatibility condition for a complex field u (interleaved):
// 1.F^ (re, im), 1.M u (re, im), 1.B u (re, im) into sc[SC_R0 .. SC_R0 + 5].
__global__ void __launch_bounds__(kT) k_compat_sums(Geom g, const double* __restrict__ u, const double* __restrict__ S,
                                                    const double* __restrict__ kap64,
                                                    const double* __restrict__ mass, Red red) {
    double acc[6] = {0, 0, 0, 0, 0, 0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < g.np; j += stride) {
        const double k = kap64[j];
        if (k == 0.0) continue;
        const unsigned t = (unsigned)j / (unsigned)g.sx;
        const int ix = (int)((unsigned)j - t * (unsigned)g.sx);
        const int iz = (int)(t / (unsigned)g.sy);
        const int iy = (int)(t - (unsigned)iz * (unsigned)g.sy);
        const double re = u[2 * j], im = u[2 * j + 1];
        const double W = weight(g, ix, iy, iz);
        const double M = mass[j];
        const double B = 2.0 * num_abc(g, ix, iy, iz) / g.h * sqrt(W * M);
        if (S) {
            const double sc = W / (k * g.h * g.h);
            acc[0] += sc * S[2 * j];
            acc[1] += sc * S[2 * j + 1];
        }
        acc[2] += M * re;
        acc[3] += M * im;
        acc[4] += B * re;
        acc[5] += B * im;
    }
    if (grid_sum<6>(acc, red.partials, red.ticket) && threadIdx.x == 0) {
        for (int k = 0; k < 6; ++k) red.sc[SC_R0 + k] = acc[k];
    }
}

__global__ void k_axpy(long long n, double a, const double* __restrict__ x, double* __restrict__ y) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) y[j] += a * x[j];
}

__global__ void k_shift(long long n, double* __restrict__ u, const double* __restrict__ kap64, double lre,
                        double lim) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        if (kap64[j] != 0.0) {
            u[2 * j] -= lre;
            u[2 * j + 1] -= lim;
        }
    }
}

// 1/M on active nodes (0 on Dirichlet nodes).
__global__ void k_reciprocal(long long n, const double* __restrict__ m, double* __restrict__ out) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride)
        out[j] = m[j] != 0.0 ? 1.0 / m[j] : 0.0;
}

// ---- flexible CG with an approximate Riesz map B ~ E^-1 --------------------------------
// Step 5.3-5.5 with the dual residual: alpha = gamma / (ghat_d . d); v -= alpha d;
// rhat -= alpha ghat_d.  The primal residual z = B rhat is formed afterwards (k_fcg_dots); with
// bf, float(rhat0) is written for its V-cycle.
template <typename V>
__global__ void __launch_bounds__(kT) k_fcg_update(long long n, V* __restrict__ w0, V* __restrict__ w1,
                                                   V* __restrict__ rh0, V* __restrict__ rh1,
                                                   const V* __restrict__ d0, const V* __restrict__ d1,
                                                   const V* __restrict__ gh0, const V* __restrict__ gh1,
                                                   float* __restrict__ bf, double* __restrict__ sc) {
    const V alpha = (V)(sc[SC_GAMMA] / sc[SC_GD]);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        w0[j] -= alpha * d0[j];
        w1[j] -= alpha * d1[j];
        const V r = rh0[j] - alpha * gh0[j];
        rh0[j] = r;
        rh1[j] -= alpha * gh1[j];
        if (bf) bf[j] = (float)r;
    }
}

// FP32 CG vectors, four nodes per thread and loop trip (float4 loads and stores; the vectors
// start 256-byte aligned); the last n % 4 nodes take the scalar loop.  Same arithmetic per
// node as the scalar kernels.
__global__ void __launch_bounds__(kT) k_fcg_update_f4(long long n, float* __restrict__ w0, float* __restrict__ w1,
                                                      float* __restrict__ rh0, float* __restrict__ rh1,
                                                      const float* __restrict__ d0, const float* __restrict__ d1,
                                                      const float* __restrict__ gh0, const float* __restrict__ gh1,
                                                      float* __restrict__ bf, double* __restrict__ sc) {
    const float alpha = (float)(sc[SC_GAMMA] / sc[SC_GD]);
    const long long n4 = n >> 2;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (long long q = t0; q < n4; q += stride) {
        float4 a = reinterpret_cast<float4*>(w0)[q], b = reinterpret_cast<float4*>(w1)[q];
        const float4 e = reinterpret_cast<const float4*>(d0)[q], f = reinterpret_cast<const float4*>(d1)[q];
        float4 r = reinterpret_cast<float4*>(rh0)[q], u = reinterpret_cast<float4*>(rh1)[q];
        const float4 g = reinterpret_cast<const float4*>(gh0)[q], h = reinterpret_cast<const float4*>(gh1)[q];
        a.x -= alpha * e.x, a.y -= alpha * e.y, a.z -= alpha * e.z, a.w -= alpha * e.w;
        b.x -= alpha * f.x, b.y -= alpha * f.y, b.z -= alpha * f.z, b.w -= alpha * f.w;
        r.x = r.x - alpha * g.x, r.y = r.y - alpha * g.y, r.z = r.z - alpha * g.z, r.w = r.w - alpha * g.w;
        u.x -= alpha * h.x, u.y -= alpha * h.y, u.z -= alpha * h.z, u.w -= alpha * h.w;
        reinterpret_cast<float4*>(w0)[q] = a;
        reinterpret_cast<float4*>(w1)[q] = b;
        reinterpret_cast<float4*>(rh0)[q] = r;
        reinterpret_cast<float4*>(rh1)[q] = u;
        if (bf) reinterpret_cast<float4*>(bf)[q] = r;
    }
    for (long long j = 4 * n4 + t0; j < n; j += stride) {
        w0[j] -= alpha * d0[j];
        w1[j] -= alpha * d1[j];
        const float r = rh0[j] - alpha * gh0[j];
        rh0[j] = r;
        rh1[j] -= alpha * gh1[j];
        if (bf) bf[j] = r;
    }
}

__global__ void __launch_bounds__(kT) k_cg_direction_f4(long long n, const float* __restrict__ r0,
                                                        const float* __restrict__ r1, float* __restrict__ d0,
                                                        float* __restrict__ d1, const double* __restrict__ sc) {
    const float beta = (float)sc[SC_BETA];
    const long long n4 = n >> 2;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (long long q = t0; q < n4; q += stride) {
        const float4 a = reinterpret_cast<const float4*>(r0)[q], b = reinterpret_cast<const float4*>(r1)[q];
        float4 c = reinterpret_cast<float4*>(d0)[q], d = reinterpret_cast<float4*>(d1)[q];
        c.x = a.x + beta * c.x, c.y = a.y + beta * c.y, c.z = a.z + beta * c.z, c.w = a.w + beta * c.w;
        d.x = b.x + beta * d.x, d.y = b.y + beta * d.y, d.z = b.z + beta * d.z, d.w = b.w + beta * d.w;
        reinterpret_cast<float4*>(d0)[q] = c;
        reinterpret_cast<float4*>(d1)[q] = d;
    }
    for (long long j = 4 * n4 + t0; j < n; j += stride) {
        d0[j] = r0[j] + beta * d0[j];
        d1[j] = r1[j] + beta * d1[j];
    }
}

// y += x with x in FP32 (the inner correction of mixed precision added to the FP64 iterate).
__global__ void k_add_float(long long n, const float* __restrict__ x, double* __restrict__ y) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) y[j] += (double)x[j];
}

// z0 from the FP32 V-cycle output with the W-weighted mean removed when K is singular,
// z1 = M^-1 rhat1; gamma' = z . rhat; for the Polak-Ribiere update also z . ghat_d:
// beta = -alpha (z . ghat_d) / gamma (= gamma'/gamma when B is exactly E^-1).  first != 0:
// Step (4), gamma0 = gamma', no beta.
template <typename V>
__global__ void __launch_bounds__(kT) k_fcg_dots(Geom g, const float* __restrict__ zf, double inv_volume,
                                                 int remove_mean, const V* __restrict__ rh0,
                                                 const V* __restrict__ rh1, const V* __restrict__ minv,
                                                 const V* __restrict__ gh0, const V* __restrict__ gh1,
                                                 V* __restrict__ z0, V* __restrict__ z1, Red red,
                                                 int first, int lowp) {
    const double mu = remove_mean ? red.sc[SC_P_XW] * inv_volume : 0.0;
    double acc[2] = {0.0, 0.0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    if (lowp) {
        // inside an FP32-period solve: the same quantities with FP32 arithmetic and
        // compensated FP32 partial sums (no FP64 arithmetic per node)
        KahanF s0, s1;
        const float muf = (float)mu;
        for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < g.np; j += stride) {
            const float m = (float)minv[j];
            const float a0 = m != 0.0f ? zf[j] - muf : 0.0f;
            const float r1 = (float)rh1[j];
            const float a1 = r1 * m;
            z0[j] = (V)a0;
            z1[j] = (V)a1;
            s0.add(a0 * (float)rh0[j] + a1 * r1);
            if (!first) s1.add(a0 * (float)gh0[j] + a1 * (float)gh1[j]);
        }
        acc[0] = s0.value();
        acc[1] = s1.value();
    } else {
        for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < g.np; j += stride) {
            const double m = minv[j];
            const double a0 = m != 0.0 ? (double)zf[j] - mu : 0.0;
            const double a1 = (double)rh1[j] * m;
            z0[j] = (V)a0;
            z1[j] = (V)a1;
            acc[0] += a0 * (double)rh0[j] + a1 * (double)rh1[j];
            if (!first) acc[1] += a0 * (double)gh0[j] + a1 * (double)gh1[j];
        }
    }
    if (grid_sum<2>(acc, red.partials, red.ticket) && threadIdx.x == 0) {
        const double gnew = acc[0];
        if (first) {
            red.sc[SC_GAMMA0] = gnew;
            red.sc[SC_REL] = gnew > 0.0 ? 1.0 : 0.0;
            red.sc[SC_STATUS] = (isfinite(gnew) && gnew >= 0.0) ? 0.0 : 1.0;
        } else {
            const double gamma = red.sc[SC_GAMMA];
            const double alpha = gamma / red.sc[SC_GD];
            red.sc[SC_ALPHA] = alpha;
            red.sc[SC_BETA] = -alpha * acc[1] / gamma;
            red.sc[SC_REL] = sqrt(fmax(gnew, 0.0) / red.sc[SC_GAMMA0]);
            if (!isfinite(alpha) || !(red.sc[SC_GD] > 0.0) || !isfinite(gnew)) red.sc[SC_STATUS] = 1.0;
        }
        red.sc[SC_GAMMA_NEW] = gnew;
        red.sc[SC_GAMMA] = gnew;
    }
}

// sum_j W_j x_j of an FP32 field into sc[SC_P_XW].
__global__ void __launch_bounds__(kT) k_wsum_float(Geom g, const float* __restrict__ x, Red red) {
    double acc[1] = {0.0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < g.np; j += stride) {
        const unsigned t = (unsigned)j / (unsigned)g.sx;
        const int ix = (int)((unsigned)j - t * (unsigned)g.sx);
        const int iz = (int)(t / (unsigned)g.sy);
        const int iy = (int)(t - (unsigned)iz * (unsigned)g.sy);
        int e = (ix == 0 || ix == g.nx) + (iy == 0 || iy == g.ny);
        if (g.dim == 3) e += (iz == 0 || iz == g.nz);
        acc[0] += (double)(x[j] / (float)(1 << e));
    }
    if (grid_sum<1>(acc, red.partials, red.ticket) && threadIdx.x == 0) {
        const double hd = g.dim == 3 ? g.h * g.h * g.h : g.h * g.h;
        red.sc[SC_P_XW] = hd * acc[0];
    }
}

}  // namespace

void launch_setup_coeffs(const Geom& g, const double* c, const unsigned char* user_mask, unsigned face_dir,
                         double dt, double* kap64, float* kap32, double* mass, unsigned char* mask, Red red,
                         cudaStream_t st) {
    note_launch(1);
    k_setup<<<vec_blocks(g.np), kT, 0, st>>>(c, user_mask, face_dir, dt, kap64, kap32, mass, mask, red, g);
}

void launch_mask_copy(const Geom& g, const double* in, const double* kap64, double* out, cudaStream_t st) {
    note_launch(1);
    k_mask_copy<<<vec_blocks(g.np), kT, 0, st>>>(in, kap64, out, g.np);
}

void launch_fill(double* p, long long n, double v, cudaStream_t st) {
    note_launch(1);
    k_fill<<<vec_blocks(n), kT, 0, st>>>(p, n, v);
}

void launch_warm_start(long long n, const double* u, const double* kap64, double wh, double* w0, double* w1,
                       cudaStream_t st) {
    note_launch(1);
    k_warm_start<<<vec_blocks(n), kT, 0, st>>>(n, u, kap64, wh, w0, w1);
}

void launch_cg_init(long long n, const double* gt0, const double* gt1, const double* gh0, const double* gh1,
                    double* r0, double* r1, double* rh0, double* rh1, double* d0, double* d1, Red red,
                    cudaStream_t st) {
    note_launch(1);
    k_cg_init<<<vec_blocks(n), kT, 0, st>>>(n, gt0, gt1, gh0, gh1, r0, r1, rh0, rh1, d0, d1, red);
}

void launch_cg_update(long long n, double* w0, double* w1, double* r0, double* r1, double* rh0, double* rh1,
                      const double* d0, const double* d1, const double* gt0, const double* gt1, const double* gh0,
                      const double* gh1, double sign, Red red, cudaStream_t st) {
    note_launch(1);
    k_cg_update<<<vec_blocks(n), kT, 0, st>>>(n, w0, w1, r0, r1, rh0, rh1, d0, d1, gt0, gt1, gh0, gh1, sign, red);
}

void launch_cg_direction(long long n, const double* r0, const double* r1, double* d0, double* d1, Red red,
                         cudaStream_t st, float* d0f, bool f32vec) {
    note_launch(1);
    if (f32vec && !d0f)
        k_cg_direction_f4<<<vec_blocks((n + 3) / 4), kT, 0, st>>>(n, (const float*)r0, (const float*)r1, (float*)d0,
                                                                  (float*)d1, red.sc);
    else if (f32vec)
        k_cg_direction<float><<<vec_blocks(n), kT, 0, st>>>(n, (const float*)r0, (const float*)r1, (float*)d0,
                                                            (float*)d1, d0f, red.sc);
    else
        k_cg_direction<double><<<vec_blocks(n), kT, 0, st>>>(n, r0, r1, d0, d1, d0f, red.sc);
}

void launch_scalar_residual(long long n, const double* r0, const double* r1, const double* rh0,
                            const double* rh1, Red red, int slot, cudaStream_t st) {
    note_launch(1);
    k_dot2<<<vec_blocks(n), kT, 0, st>>>(n, r0, r1, rh0, rh1, red, slot);
}

void launch_recover(const Geom& g, const double* w0, const double* w1, double omega_hat, const double* S,
                    const double* kap64, const double* mass, double* u, Red red, cudaStream_t st) {
    note_launch(1);
    k_recover<<<vec_blocks(g.np), kT, 0, st>>>(g, w0, w1, 1.0 / omega_hat, S, kap64, mass, u, red);
}

void launch_compat_sums(const Geom& g, const double* u, const double* S, const double* kap64, const double* mass,
                        Red red, cudaStream_t st) {
    note_launch(1);
    k_compat_sums<<<vec_blocks(g.np), kT, 0, st>>>(g, u, S, kap64, mass, red);
}

void launch_axpy(long long n, double a, const double* x, double* y, cudaStream_t st) {
    note_launch(1);
    k_axpy<<<vec_blocks(n), kT, 0, st>>>(n, a, x, y);
}

void launch_shift(long long n, double* u, const double* kap64, double lre, double lim, cudaStream_t st) {
    note_launch(1);
    k_shift<<<vec_blocks(n), kT, 0, st>>>(n, u, kap64, lre, lim);
}

}  // namespace cmcg

namespace cmcg {

void launch_reciprocal(long long n, const double* m, double* out, cudaStream_t st) {
    note_launch(1);
    k_reciprocal<<<vec_blocks(n), kT, 0, st>>>(n, m, out);
}

void launch_fcg_update(long long n, double* w0, double* w1, double* rh0, double* rh1, const double* d0,
                       const double* d1, const double* gh0, const double* gh1, Red red, cudaStream_t st, float* bf,
                       bool f32vec) {
    note_launch(1);
    if (f32vec)
        k_fcg_update_f4<<<vec_blocks((n + 3) / 4), kT, 0, st>>>(n, (float*)w0, (float*)w1, (float*)rh0, (float*)rh1,
                                                                (const float*)d0, (const float*)d1, (const float*)gh0,
                                                                (const float*)gh1, bf, red.sc);
    else
        k_fcg_update<double><<<vec_blocks(n), kT, 0, st>>>(n, w0, w1, rh0, rh1, d0, d1, gh0, gh1, bf, red.sc);
}

void launch_add_float(long long n, const float* x, double* y, cudaStream_t st) {
    note_launch(1);
    k_add_float<<<vec_blocks(n), kT, 0, st>>>(n, x, y);
}

// k_fcg_dots needs more than 32 registers, so fewer than the 8 blocks per SM that
// kMaxBlocksReduce assumes are resident: its grid-stride grid is one full wave of what this
// GPU holds at once (cached per device; deterministic for a given GPU and build).
template <typename V>
static unsigned fcg_dots_blocks(long long n) {
    static int cached[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    int& c = cached[dev & 63];
    if (c == 0) {
        int per_sm = 0, sms = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fcg_dots<V>, kT, 0) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || per_sm < 1 ||
            sms < 1) {
            cudaGetLastError();
            return vec_blocks(n);
        }
        c = per_sm * sms < kMaxBlocksReduce ? per_sm * sms : kMaxBlocksReduce;
    }
    const unsigned b = vec_blocks(n);
    return b < (unsigned)c ? b : (unsigned)c;
}

void launch_fcg_dots(const Geom& g, const float* zf, double volume, bool remove_mean, bool lowp, const double* rh0,
                     const double* rh1, const double* minv, const double* gh0, const double* gh1, double* z0,
                     double* z1, Red red, bool first, cudaStream_t st, bool f32vec) {
    note_launch(1);
    if (f32vec)
        k_fcg_dots<float><<<fcg_dots_blocks<float>(g.np), kT, 0, st>>>(
            g, zf, 1.0 / volume, remove_mean ? 1 : 0, (const float*)rh0, (const float*)rh1, (const float*)minv,
            (const float*)gh0,
            (const float*)gh1, (float*)z0, (float*)z1, red, first ? 1 : 0, 1);
    else
        k_fcg_dots<double><<<fcg_dots_blocks<double>(g.np), kT, 0, st>>>(
            g, zf, 1.0 / volume, remove_mean ? 1 : 0, rh0, rh1, minv, gh0, gh1, z0, z1, red, first ? 1 : 0,
            lowp ? 1 : 0);
}

void launch_wsum_float(const Geom& g, const float* x, Red red, cudaStream_t st) {
    note_launch(1);
    k_wsum_float<<<vec_blocks(g.np), kT, 0, st>>>(g, x, red);
}

}  // namespace cmcg
