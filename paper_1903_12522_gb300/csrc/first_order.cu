// First-order (mixed) formulation of Sec. 3 on a staggered grid: v = y_t on the nodes,
// p = grad y on the grid links, stepped with the staggered leapfrog
//
//   p_a^{n+1/2} = p_a^{n-1/2} + tau (v_{j+e_a} - v_j)                      tau = dt / h
//   v^{n+1}     = [(1 - beta) v^n - sigma sum_a (p_a(j - e_a) - p_a(j)) / w_a(j_a)
//                  + Re(S e^{-i w t_{n+1/2}}) / dt] / (1 + beta)             sigma = kappa h / dt
//
// which is the semi-discrete Eq. mixWE  M v' + B v = -G^T W_e p + F,  p' = G v  with the lumped
// link mass W_e = h^d prod_{b != a} w(j_b) (so G^T W_e G = K of the second-order scheme),
// beta = (dt/2) M^-1 B = nb sqrt(kappa), S = dt^2 M^-1 F^ (the handle's source array) and
// w_a = 1/2 on the two end nodes of axis a.  Missing links (j_a = n_a) hold 0; Dirichlet nodes
// (kappa = 0) hold v = 0.
//
// State layout: p_x | p_y | (p_z) | v, each N_p long; p_a[j] is the link (j, j + e_a).
//
// Adjoint.  With E = diag(W_e, M) the E-adjoint of the homogeneous step, run on the
// variables (q, u) = (E^-1 pbar, (1 + beta)^-1 E^-1 vbar), is the same update with tau and
// sigma negated; so one kernel runs both the forward period and the backward period of
// Eq. mixJ_deriative_2, and the gradient's E-representer P* e - e needs no elliptic solve.
#include <math.h>

#include <algorithm>

#include "solver.h"

namespace cmcg {

namespace {

constexpr int kFT = 256;

inline dim3 fo_grid(const Geom& g, int zc) {
    const long long plane = (long long)g.sx * g.sy;
    return dim3((unsigned)((plane + kFT - 1) / kFT), (unsigned)((g.sz + zc - 1) / zc));
}

inline unsigned fo_vec_blocks(long long n) {
    long long b = (n + kFT - 1) / kFT;
    return (unsigned)std::max<long long>(1, std::min<long long>(b, kMaxBlocksReduce));
}

__device__ __forceinline__ double inv_w(int i, int n) { return (i == 0 || i == n) ? 2.0 : 1.0; }

// Link mass W_e of link (j, j + e_a), 0 where the link does not exist.
__device__ __forceinline__ double link_mass(const Geom& g, int a, int ix, int iy, int iz) {
    const int i[3] = {ix, iy, iz};
    const int n[3] = {g.nx, g.ny, g.nz};
    if (i[a] >= n[a]) return 0.0;
    double w = g.dim == 3 ? g.h * g.h * g.h : g.h * g.h;
    for (int b = 0; b < g.dim; ++b)
        if (b != a && (i[b] == 0 || i[b] == n[b])) w *= 0.5;
    return w;
}

// Component c of element e of a (dim + 1) N_p state, and the node's coordinates.
struct Elem {
    int comp, ix, iy, iz;
    long long j;
};

__device__ __forceinline__ Elem elem(const Geom& g, long long e) {
    Elem r;
    r.comp = (int)(e / g.np);
    r.j = e - (long long)r.comp * g.np;
    const long long t = r.j / g.sx;
    r.ix = (int)(r.j - t * g.sx);
    r.iz = (int)(t / g.sy);
    r.iy = (int)(t - (long long)r.iz * g.sy);
    return r;
}

// Energy weight of element e: W_e for a link component, M for the velocity.
__device__ __forceinline__ double e_weight(const Geom& g, const double* mass, const Elem& r) {
    return r.comp < g.dim ? link_mass(g, r.comp, r.ix, r.iy, r.iz) : mass[r.j];
}

// One staggered leapfrog step for a column of z-planes (3D) or one node (2D).  SRC adds the
// source at t_{n+1/2} (cs, sn already divided by dt); ACC accumulates v^n e^{i w t_n} into acc.
// Consecutive lanes hold consecutive nodes of a row, so v_{j-1}, v_{j+1} and the old value of
// the link (j - 1, j) come from the neighbouring lanes (lane 0 and lane 31 load them); lanes
// past the last column take part in the shuffles but touch no memory.
template <typename T, int DIM, bool SRC, bool ACC>
__global__ void __launch_bounds__(kFT) k_fo_step(const T* __restrict__ sin_, T* __restrict__ sout,
                                                 const T* __restrict__ kap, const double* __restrict__ S, double cs,
                                                 double sn, T tau, T sig, Geom g, int zc, double* __restrict__ acc,
                                                 double ca, double sa) {
    const long long plane = (long long)g.sx * g.sy;
    const long long pidx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = pidx < plane;
    const long long pc = valid ? pidx : plane - 1;  // in-range stand-in for idle lanes
    const int iy = (int)(pc / g.sx);
    const int ix = (int)(pc - (long long)iy * g.sx);
    const int lane = threadIdx.x & 31;
    const int z0 = DIM == 3 ? (int)blockIdx.y * zc : 0;
    const int z1 = DIM == 3 ? min(z0 + zc, g.sz) : 1;
    if (z0 >= z1) return;  // uniform over the block
    const long long np = g.np;
    const long long sZ = plane;
    const T* px = sin_;
    const T* py = sin_ + np;
    const T* pz = sin_ + 2 * np;
    const T* v = sin_ + (long long)DIM * np;
    T* qx = sout;
    T* qy = sout + np;
    T* qz = sout + 2 * np;
    T* w = sout + (long long)DIM * np;
    const T rx = (T)inv_w(ix, g.nx), ry = (T)inv_w(iy, g.ny);
    const bool hx0 = ix > 0, hx1 = ix < g.nx, hy0 = iy > 0, hy1 = iy < g.ny;
    int nbxy = 0;
    nbxy += (ix == 0) & (int)(g.abc & 1u);
    nbxy += (ix == g.nx) & (int)((g.abc >> 1) & 1u);
    nbxy += (iy == 0) & (int)((g.abc >> 2) & 1u);
    nbxy += (iy == g.ny) & (int)((g.abc >> 3) & 1u);
    constexpr unsigned kAll = 0xffffffffu;
    long long j = pc + sZ * z0;
    T vc = v[j];
    T pzl = T(0);  // new value of the z-link below (j - sZ, j)
    if (DIM == 3 && z0 > 0) pzl = pz[j - sZ] + tau * (vc - v[j - sZ]);
    for (int iz = z0; iz < z1; ++iz) {
        T vz = T(0), pzr = T(0);
        if (DIM == 3 && iz < g.nz) {
            vz = v[j + sZ];
            pzr = pz[j] + tau * (vz - vc);
        }
        const T pxo = px[j];  // old value of the link (j, j + 1) (0 in the slot j_x = n_x)
        const T vl = __shfl_up_sync(kAll, vc, 1), vr = __shfl_down_sync(kAll, vc, 1);
        const T pl = __shfl_up_sync(kAll, pxo, 1);
        const T vxm = hx0 ? (lane > 0 ? vl : v[j - 1]) : T(0);
        const T vxp = hx1 ? (lane < 31 ? vr : v[j + 1]) : T(0);
        const T pxlo = hx0 ? (lane > 0 ? pl : px[j - 1]) : T(0);
        const T pxr = hx1 ? pxo + tau * (vxp - vc) : T(0);
        const T pxl = hx0 ? pxlo + tau * (vc - vxm) : T(0);
        const T pyr = hy1 ? py[j] + tau * (v[j + g.sx] - vc) : T(0);
        const T pyl = hy0 ? py[j - g.sx] + tau * (vc - v[j - g.sx]) : T(0);
        T div = (pxl - pxr) * rx + (pyl - pyr) * ry;
        int nb = nbxy;
        if (DIM == 3) {
            div += (pzl - pzr) * (T)inv_w(iz, g.nz);
            nb += ((iz == 0) & (int)((g.abc >> 4) & 1u)) + ((iz == g.nz) & (int)((g.abc >> 5) & 1u));
        }
        const T k = __ldcs(kap + j);  // streamed: the fields are what the next step re-reads
        T out = T(0);
        if (k != T(0)) {
            const T beta = (T)nb * sqrt(k);
            T rhs = (T(1) - beta) * vc - sig * k * div;
            if (SRC) rhs += (T)(S[2 * j] * cs + S[2 * j + 1] * sn);
            out = nb == 0 ? rhs : rhs / (T(1) + beta);
        }
        if (valid) {
            if (ACC) {
                acc[2 * j] += (double)vc * ca;
                acc[2 * j + 1] += (double)vc * sa;
            }
            qx[j] = pxr;
            qy[j] = pyr;
            if (DIM == 3) qz[j] = pzr;
            w[j] = out;
        }
        if (DIM == 3) {
            pzl = pzr;
            vc = vz;
            j += sZ;
        }
    }
}

// FP64 state -> stepping precision; MODE 0 a copy (0 on missing links and Dirichlet nodes),
// MODE 1 the adjoint's entry variables
// (q, u) = (p, v / (1 + beta)) (the input already E-scaled), MODE 2 the same from an unscaled
// cotangent: (pbar / W_e, vbar / (M (1 + beta))).
template <typename T, int MODE>
__global__ void __launch_bounds__(kFT) k_fo_load(const double* __restrict__ src, T* __restrict__ dst,
                                                 const double* __restrict__ kap64, const double* __restrict__ mass,
                                                 Geom g) {
    const long long n = (long long)(g.dim + 1) * g.np;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
        const Elem r = elem(g, e);
        double x = src[e];
        if (MODE == 0) {
            const bool keep = r.comp < g.dim ? link_mass(g, r.comp, r.ix, r.iy, r.iz) > 0.0 : kap64[r.j] != 0.0;
            dst[e] = keep ? (T)x : T(0);
            continue;
        }
        if (r.comp < g.dim) {
            if (MODE == 2) {
                const double we = link_mass(g, r.comp, r.ix, r.iy, r.iz);
                x = we > 0.0 ? x / we : 0.0;
            }
        } else {
            const double k = kap64[r.j];
            if (k == 0.0) {
                x = 0.0;
            } else {
                const double beta = num_abc(g, r.ix, r.iy, r.iz) * sqrt(k);
                if (MODE == 2) x /= mass[r.j];
                x /= 1.0 + beta;
            }
        }
        dst[e] = (T)x;
    }
}

// End of a forward period.  MODE 0: e = s_N - s_0 and J = (e, e)_E / 2 into sc[SC_J], with s_0
// rounded to the stepping precision (the state the period started from).
// MODE 1: out = s_N (FP64).
template <typename T, int MODE>
__global__ void __launch_bounds__(kFT) k_fo_end(const T* __restrict__ sN, const double* __restrict__ s0,
                                                double* __restrict__ out, const double* __restrict__ mass, Geom g,
                                                Red red) {
    const long long n = (long long)(g.dim + 1) * g.np;
    double acc[1] = {0.0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
        if (MODE == 1) {
            out[e] = (double)sN[e];
            continue;
        }
        const double d = (double)sN[e] - (double)(T)s0[e];  // against the copy the period started from
        out[e] = d;
        acc[0] += e_weight(g, mass, elem(g, e)) * d * d;
    }
    if (MODE == 0 && grid_sum<1>(acc, red.partials, red.ticket) && threadIdx.x == 0) red.sc[SC_J] = 0.5 * acc[0];
}

// End of the backward period.  MODE 0 (CG): g = P* e - e from the final (q, u) and
// (g, d)_E into sc[SC_GD].  MODE 1 (plain transpose): out = E (q, (1 + beta) u).
template <typename T, int MODE>
__global__ void __launch_bounds__(kFT) k_fo_adj_end(const T* __restrict__ s, const double* __restrict__ e_in,
                                                    const double* __restrict__ d, double* __restrict__ out,
                                                    const double* __restrict__ kap64, const double* __restrict__ mass,
                                                    Geom g, Red red) {
    const long long n = (long long)(g.dim + 1) * g.np;
    double acc[1] = {0.0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
        const Elem r = elem(g, e);
        double x = (double)s[e];
        double wgt;
        if (r.comp < g.dim) {
            wgt = link_mass(g, r.comp, r.ix, r.iy, r.iz);
        } else {
            const double k = kap64[r.j];
            x = k == 0.0 ? 0.0 : x * (1.0 + num_abc(g, r.ix, r.iy, r.iz) * sqrt(k));
            wgt = mass[r.j];
        }
        if (MODE == 1) {
            out[e] = wgt * x;
            continue;
        }
        const double gv = wgt > 0.0 ? x - e_in[e] : 0.0;
        out[e] = gv;
        acc[0] += wgt * gv * d[e];
    }
    if (MODE == 0 && grid_sum<1>(acc, red.partials, red.ticket) && threadIdx.x == 0) red.sc[SC_GD] = acc[0];
}

// (4) r = d = g; gamma = gamma0 = (g, g)_E.
__global__ void __launch_bounds__(kFT) k_fo_cg_init(const double* __restrict__ gr, double* __restrict__ r,
                                                    double* __restrict__ d, const double* __restrict__ mass, Geom g,
                                                    Red red) {
    const long long n = (long long)(g.dim + 1) * g.np;
    double acc[1] = {0.0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
        const double x = gr[e];
        r[e] = x;
        d[e] = x;
        acc[0] += e_weight(g, mass, elem(g, e)) * x * x;
    }
    if (grid_sum<1>(acc, red.partials, red.ticket) && threadIdx.x == 0) {
        red.sc[SC_GAMMA] = acc[0];
        red.sc[SC_GAMMA0] = acc[0];
        red.sc[SC_REL] = acc[0] > 0.0 ? 1.0 : 0.0;
        red.sc[SC_STATUS] = isfinite(acc[0]) ? 0.0 : 1.0;
    }
}

// 5.3-5.6: alpha = gamma / (g, d)_E, s -= alpha d, r -= alpha g, gamma_new = (r, r)_E.  A
// non-positive or non-finite (g, d)_E (rounding of the FP32 periods at their precision floor)
// leaves s and r unchanged and sets the status.
__global__ void __launch_bounds__(kFT) k_fo_cg_update(double* __restrict__ s, double* __restrict__ r,
                                                      const double* __restrict__ d, const double* __restrict__ gr,
                                                      const double* __restrict__ mass, Geom g, Red red) {
    const double gamma = red.sc[SC_GAMMA];
    const double gd = red.sc[SC_GD];
    const bool breakdown = !(gd > 0.0) || !isfinite(gd);
    const double alpha = breakdown ? 0.0 : gamma / gd;
    const long long n = (long long)(g.dim + 1) * g.np;
    double acc[1] = {0.0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
        s[e] -= alpha * d[e];
        const double x = r[e] - alpha * gr[e];
        r[e] = x;
        acc[0] += e_weight(g, mass, elem(g, e)) * x * x;
    }
    if (grid_sum<1>(acc, red.partials, red.ticket) && threadIdx.x == 0) {
        const double gnew = acc[0];
        red.sc[SC_ALPHA] = alpha;
        red.sc[SC_GAMMA_NEW] = gnew;
        red.sc[SC_BETA] = gamma > 0.0 ? gnew / gamma : 0.0;
        const double g0 = red.sc[SC_GAMMA0];
        red.sc[SC_REL] = g0 > 0.0 ? sqrt(fmax(gnew, 0.0) / g0) : 0.0;
        if (breakdown) red.sc[SC_STATUS] = 1.0;
        if (!isfinite(gnew)) red.sc[SC_STATUS] = 2.0;
    }
}

// 5.7: d = r + beta d; gamma = gamma_new.
__global__ void __launch_bounds__(kFT) k_fo_cg_direction(const double* __restrict__ r, double* __restrict__ d,
                                                         long long n, double* __restrict__ sc) {
    const double beta = sc[SC_BETA];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) d[e] = r[e] + beta * d[e];
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) sc[SC_GAMMA] = sc[SC_GAMMA_NEW];
}

// Step (6) by Eq. mix_solution, discrete-exact: Im U = v / wt, Re P = (2 p + dt G v) / (2 cos(w dt/2)),
// Re U = [(kappa h / dt^2) sum_a (ReP_a(j - e_a) - ReP_a(j)) / w_a + wh (2 beta / dt) Im U - S_re / dt^2] / wt^2.
__global__ void __launch_bounds__(kFT) k_fo_recover(const double* __restrict__ s, const double* __restrict__ kap64,
                                                    const double* __restrict__ S, double* __restrict__ u, Geom g,
                                                    double dt, double wt, double wh, double c_half) {
    const long long np = g.np;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const double* v = s + (long long)g.dim * np;
    const double gdt = dt / g.h;
    const double inv2c = 1.0 / (2.0 * c_half);
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < np; j += stride) {
        const double k = kap64[j];
        if (k == 0.0) {
            u[2 * j] = 0.0;
            u[2 * j + 1] = 0.0;
            continue;
        }
        const long long t = j / g.sx;
        const int ix = (int)(j - t * g.sx);
        const int iz = (int)(t / g.sy);
        const int iy = (int)(t - (long long)iz * g.sy);
        const int i[3] = {ix, iy, iz};
        const int nn[3] = {g.nx, g.ny, g.nz};
        const long long str[3] = {1, g.sx, (long long)g.sx * g.sy};
        const double vc = v[j];
        double div = 0.0;
        for (int a = 0; a < g.dim; ++a) {
            const double* p = s + (long long)a * np;
            double rr = 0.0, rl = 0.0;
            if (i[a] < nn[a]) rr = (2.0 * p[j] + gdt * (v[j + str[a]] - vc)) * inv2c;
            if (i[a] > 0) rl = (2.0 * p[j - str[a]] + gdt * (vc - v[j - str[a]])) * inv2c;
            div += (rl - rr) * inv_w(i[a], nn[a]);
        }
        const double im = vc / wt;
        const double beta = num_abc(g, ix, iy, iz) * sqrt(k);
        const double re = (k * g.h / (dt * dt) * div + wh * (2.0 * beta / dt) * im - S[2 * j] / (dt * dt)) / (wt * wt);
        u[2 * j] = re;
        u[2 * j + 1] = im;
    }
}

// Step (6) by Eq. TH_FILTERED_MIXED_SOLUTION: U = (2 i / (N wt)) acc, acc = sum v^n e^{i w t_n}.
__global__ void k_fo_filter_final(long long np, double* __restrict__ u, double scale) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < np; j += stride) {
        const double re = u[2 * j], im = u[2 * j + 1];
        u[2 * j] = -scale * im;
        u[2 * j + 1] = scale * re;
    }
}

template <typename T, int DIM>
void step_launch(const Geom& g, const T* a, T* b, const T* kap, const double* S, double cs, double sn, double tau,
                 double sig, int zc, double* acc, double ca, double sa, cudaStream_t st) {
    note_launch(1);
    const dim3 grid = fo_grid(g, DIM == 3 ? zc : 1);
    if (S && acc)
        k_fo_step<T, DIM, true, true><<<grid, kFT, 0, st>>>(a, b, kap, S, cs, sn, (T)tau, (T)sig, g, zc, acc, ca, sa);
    else if (S)
        k_fo_step<T, DIM, true, false><<<grid, kFT, 0, st>>>(a, b, kap, S, cs, sn, (T)tau, (T)sig, g, zc, acc, ca, sa);
    else
        k_fo_step<T, DIM, false, false><<<grid, kFT, 0, st>>>(a, b, kap, S, cs, sn, (T)tau, (T)sig, g, zc, acc, ca,
                                                               sa);
}

}  // namespace

namespace detail {

constexpr int kZcFO = 16;

template <typename T>
const T* fo_kap(const cmcg_handle* H) {
    return std::is_same<T, float>::value ? (const T*)H->kap32 : (const T*)H->kap64;
}

template <typename T>
void fo_step(cmcg_handle* H, const T* a, T* b, bool src, int n, bool backward, double* acc, double theta = 1.0) {
    const Geom& g = H->g;
    const double t = (n + 0.5) * H->dt;  // the source is T-periodic: n may count past one period
    const double cs = src ? theta * cos(H->omega * t) / H->dt : 0.0;
    const double sn = src ? theta * sin(H->omega * t) / H->dt : 0.0;
    const double tn = n * H->dt;
    const double ca = acc ? cos(H->omega * tn) : 0.0, sa = acc ? sin(H->omega * tn) : 0.0;
    const double tau = (backward ? -1.0 : 1.0) * H->dt / g.h;
    const double sig = (backward ? -1.0 : 1.0) * g.h / H->dt;
    const double* S = src ? H->S : nullptr;
    if (g.dim == 3)
        step_launch<T, 3>(g, a, b, fo_kap<T>(H), S, cs, sn, tau, sig, kZcFO, acc, ca, sa, H->st);
    else
        step_launch<T, 2>(g, a, b, fo_kap<T>(H), S, cs, sn, tau, sig, 1, acc, ca, sa, H->st);
}

// Forward period from the FP64 state s0.  mode 0: out = Pi(s0) - s0 and J; mode 1: out = Pi(s0).
// acc (optional, forced FP64 periods only) accumulates v^n e^{i w t_n}.
template <typename T>
void fo_forward(cmcg_handle* H, const double* s0, bool src, int mode, double* out, double* acc) {
    const Geom& g = H->g;
    const long long n = (long long)(g.dim + 1) * g.np;
    T* a = (T*)H->fo_a;
    T* b = (T*)H->fo_b;
    note_launch(1);
    k_fo_load<T, 0><<<fo_vec_blocks(n), kFT, 0, H->st>>>(s0, a, H->kap64, H->mass, g);
    const int slot = timing_begin(H, std::is_same<T, float>::value, H->N);
    for (int k = 0; k < H->N; ++k) {
        fo_step<T>(H, a, b, src, k, false, acc);
        std::swap(a, b);
    }
    timing_end(H, slot);
    note_launch(1);
    if (mode == 0)
        k_fo_end<T, 0><<<fo_vec_blocks(n), kFT, 0, H->st>>>(a, s0, out, H->mass, g, H->red());
    else
        k_fo_end<T, 1><<<fo_vec_blocks(n), kFT, 0, H->st>>>(a, s0, out, H->mass, g, H->red());
    H->periods += 1;
}

// Backward (adjoint) period.  mode 0: from the mismatch e (an E-scaled cotangent),
// out = P* e - e and (out, d)_E into sc[SC_GD]; mode 1: out = P^T y (plain transpose) for an
// unscaled cotangent y.
template <typename T>
void fo_backward(cmcg_handle* H, const double* y, const double* d, int mode, double* out) {
    const Geom& g = H->g;
    const long long n = (long long)(g.dim + 1) * g.np;
    T* a = (T*)H->fo_a;
    T* b = (T*)H->fo_b;
    note_launch(1);
    if (mode == 0)
        k_fo_load<T, 1><<<fo_vec_blocks(n), kFT, 0, H->st>>>(y, a, H->kap64, H->mass, g);
    else
        k_fo_load<T, 2><<<fo_vec_blocks(n), kFT, 0, H->st>>>(y, a, H->kap64, H->mass, g);
    const int slot = timing_begin(H, std::is_same<T, float>::value, H->N);
    for (int k = 0; k < H->N; ++k) {
        fo_step<T>(H, a, b, false, k, true, nullptr);
        std::swap(a, b);
    }
    timing_end(H, slot);
    note_launch(1);
    if (mode == 0)
        k_fo_adj_end<T, 0><<<fo_vec_blocks(n), kFT, 0, H->st>>>(a, y, d, out, H->kap64, H->mass, g, H->red());
    else
        k_fo_adj_end<T, 1><<<fo_vec_blocks(n), kFT, 0, H->st>>>(a, y, d, out, H->kap64, H->mass, g, H->red());
    H->periods += 1;
}

// Steps 5.1-5.8 of the CMCG Algorithm on the first-order state, from r = d = g already set
// (k_fo_cg_init): J^' by a forward and a backward period (Eq. mixJ_deriative_2), no Riesz
// solve.  Updates the iterate x.  Stops at rel <= tol, after max_iter iterations, when
// (g, d)_E stops being positive (status 1: the FP32 periods' rounding floor), or when the
// residual has grown a hundredfold above its smallest value (FP32 periods only).  Returns a
// CMCG status (CMCG_ERR_DIVERGED on a non-finite residual); *it, *rel report the run.
template <typename T>
int fo_cg_iterate(cmcg_handle* H, double* x, double tol, int max_iter, int* it_out, double* rel_out) {
    const Geom& g = H->g;
    const long long n = (long long)(g.dim + 1) * g.np;
    // relative to the reference in SC_GAMMA0 (the start gradient's, or the zero guess's after a run-up)
    double rel = H->hsc[SC_GAMMA0] > 0.0 ? sqrt(std::max(H->hsc[SC_GAMMA], 0.0) / H->hsc[SC_GAMMA0]) : 0.0;
    double best = rel;
    int it = 0;
    if (rel > tol) {
        for (it = 1; it <= max_iter; ++it) {
            // 5.1 homogeneous forward and backward period from d
            fo_forward<T>(H, H->fo_d, false, 0, H->fo_e, nullptr);
            fo_backward<T>(H, H->fo_e, H->fo_d, 0, H->fo_g);
            // 5.3-5.6
            note_launch(1);
            k_fo_cg_update<<<fo_vec_blocks(n), kFT, 0, H->st>>>(x, H->fo_r, H->fo_d, H->fo_g, H->mass, g, H->red());
            // 5.7
            note_launch(1);
            k_fo_cg_direction<<<fo_vec_blocks(n), kFT, 0, H->st>>>(H->fo_r, H->fo_d, n, H->sc);
            if (sync_read(H) != CMCG_OK) return CMCG_ERR_CUDA;
            if (H->hsc[SC_STATUS] == 2.0) {
                *it_out = it;
                *rel_out = rel;
                return CMCG_ERR_DIVERGED;
            }
            if (H->hsc[SC_STATUS] != 0.0) break;  // (g, d)_E <= 0: x is the last good iterate
            rel = H->hsc[SC_REL];
            best = std::min(best, rel);
            if (rel <= tol) break;  // 5.8
            if (std::is_same<T, float>::value && rel > 100.0 * best) break;
        }
        if (it > max_iter) it = max_iter;
    }
    *it_out = it;
    *rel_out = rel;
    return rel <= tol ? CMCG_OK : CMCG_NOT_CONVERGED;
}

// (1)-(4): x = 0, the gradient with the sources at x in stepping precision T, r = d = g.
template <typename T>
int fo_cg_start(cmcg_handle* H, double* x) {
    const Geom& g = H->g;
    const long long n = (long long)(g.dim + 1) * g.np;
    cudaMemsetAsync(x, 0, sizeof(double) * n, H->st);
    fo_forward<T>(H, x, true, 0, H->fo_e, nullptr);
    fo_backward<T>(H, H->fo_e, H->fo_e, 0, H->fo_g);
    note_launch(1);
    k_fo_cg_init<<<fo_vec_blocks(n), kFT, 0, H->st>>>(H->fo_g, H->fo_r, H->fo_d, H->mass, g, H->red());
    return sync_read(H) == CMCG_OK ? CMCG_OK : CMCG_ERR_CUDA;
}

// Initial run-up (Sec. 4.2.3) on the first-order state: the forced staggered leapfrog from rest for
// `periods` periods with the sources ramped in by theta_tr over [0, periods T]; the state at
// t = periods T goes to out (FP64).
template <typename T>
void fo_runup(cmcg_handle* H, int periods, double* out) {
    const Geom& g = H->g;
    const long long n = (long long)(g.dim + 1) * g.np;
    T* a = (T*)H->fo_a;
    T* b = (T*)H->fo_b;
    cudaMemsetAsync(a, 0, sizeof(T) * n, H->st);
    const long long total = (long long)periods * H->N;
    const double ttr = total * H->dt;
    for (long long k = 0; k < total; ++k) {
        fo_step<T>(H, a, b, true, (int)(k % H->N), false, nullptr, ramp((k + 0.5) * H->dt, ttr));
        std::swap(a, b);
    }
    note_launch(1);
    k_fo_end<T, 1><<<fo_vec_blocks(n), kFT, 0, H->st>>>(a, out, out, H->mass, g, H->red());
    H->periods += periods;
}

// With a run-up: the zero-guess gradient's gamma (the tolerance reference, and J0), then the
// run-up state into x and its gradient with r = d = g, and SC_GAMMA0 set to the reference.
// Without: x = 0 and its gradient.  Returns the number of run-up periods (or a negative status).
template <typename T>
int fo_start_with_runup(cmcg_handle* H, double* x, cmcg_stats* st) {
    const Geom& g = H->g;
    const long long n = (long long)(g.dim + 1) * g.np;
    if (fo_cg_start<T>(H, x) != CMCG_OK) return CMCG_ERR_CUDA;
    st->J0 = H->hsc[SC_J];
    const int ell = runup_count(H);
    if (ell <= 0) return 0;
    const double gamma_zero = H->hsc[SC_GAMMA0];
    fo_runup<T>(H, ell, x);
    fo_forward<T>(H, x, true, 0, H->fo_e, nullptr);
    fo_backward<T>(H, H->fo_e, H->fo_e, 0, H->fo_g);
    note_launch(1);
    k_fo_cg_init<<<fo_vec_blocks(n), kFT, 0, H->st>>>(H->fo_g, H->fo_r, H->fo_d, H->mass, g, H->red());
    cudaMemcpyAsync(H->sc + SC_GAMMA0, &gamma_zero, sizeof(double), cudaMemcpyHostToDevice, H->st);
    if (sync_read(H) != CMCG_OK) return CMCG_ERR_CUDA;
    return ell;
}

template <typename T>
int fo_cg(cmcg_handle* H, double tol, cmcg_stats* st) {
    const int ell = fo_start_with_runup<T>(H, H->fo_s, st);
    if (ell < 0) return ell;
    st->runup_periods = ell;
    int it = 0;
    double rel = 1.0;
    const int rc = fo_cg_iterate<T>(H, H->fo_s, tol, H->opt.max_iter, &it, &rel);
    st->iterations = it;
    st->outer_iterations = 1;
    st->rel_residual = rel;
    return rc;
}

// CMCG_MIXED: FP64 defect correction around FP32 CG.  Each outer step evaluates the gradient
// with the sources at s in FP64 (the true residual), then solves for the correction with FP32
// periods from zero to the relative tolerance inner_tol (tightened so as not to stop the outer
// loop short of tol) and adds it to s.  rel is relative to the first outer gradient (s = 0).
int fo_mixed(cmcg_handle* H, double tol, cmcg_stats* st) {
    const Geom& g = H->g;
    const long long n = (long long)(g.dim + 1) * g.np;
    cudaMemsetAsync(H->fo_s, 0, sizeof(double) * n, H->st);
    double gamma_ref = -1.0, rel = 1.0;
    int total = 0, outer = 0;
    const int max_outer = 50;
    const int ell = runup_count(H);
    if (ell > 0) {
        // the tolerance reference is the FP64 gradient of the zero guess; then an FP32 run-up
        fo_forward<double>(H, H->fo_s, true, 0, H->fo_e, nullptr);
        fo_backward<double>(H, H->fo_e, H->fo_e, 0, H->fo_g);
        note_launch(1);
        k_fo_cg_init<<<fo_vec_blocks(n), kFT, 0, H->st>>>(H->fo_g, H->fo_r, H->fo_d, H->mass, g, H->red());
        if (sync_read(H) != CMCG_OK) return CMCG_ERR_CUDA;
        gamma_ref = H->hsc[SC_GAMMA0];
        st->J0 = H->hsc[SC_J];
        fo_runup<float>(H, ell, H->fo_s);
        st->runup_periods = ell;
    }
    for (outer = 0; outer < max_outer; ++outer) {
        fo_forward<double>(H, H->fo_s, true, 0, H->fo_e, nullptr);
        fo_backward<double>(H, H->fo_e, H->fo_e, 0, H->fo_g);
        note_launch(1);
        k_fo_cg_init<<<fo_vec_blocks(n), kFT, 0, H->st>>>(H->fo_g, H->fo_r, H->fo_d, H->mass, g, H->red());
        if (sync_read(H) != CMCG_OK) return CMCG_ERR_CUDA;
        const double gam = H->hsc[SC_GAMMA0];
        if (!(gam == gam) || gam < 0) return CMCG_ERR_DIVERGED;
        if (gamma_ref < 0) {
            gamma_ref = gam;
            st->J0 = H->hsc[SC_J];
        }
        rel = gamma_ref > 0 ? sqrt(gam / gamma_ref) : 0.0;
        if (rel <= tol || total >= H->opt.max_iter) break;
        const double inner = std::min(0.5, std::max(H->opt.inner_tol, 0.5 * tol / std::max(rel, 1e-300)));
        int it = 0;
        double irel = 1.0;
        cudaMemsetAsync(H->fo_x, 0, sizeof(double) * n, H->st);
        const int rc = fo_cg_iterate<float>(H, H->fo_x, inner, H->opt.max_iter - total, &it, &irel);
        if (rc < 0) return rc;
        total += it;
        launch_axpy(n, 1.0, H->fo_x, H->fo_s, H->st);
        if (it == 0) break;  // no progress possible
    }
    st->iterations = total;
    st->outer_iterations = outer;
    st->rel_residual = rel;
    if (cuda_status() != CMCG_OK) return CMCG_ERR_CUDA;
    return rel <= tol ? CMCG_OK : CMCG_NOT_CONVERGED;
}

int fo_recover(cmcg_handle* H, double* u) {
    const Geom& g = H->g;
    if (H->opt.flags & CMCG_FLAG_FILTER) {
        // one forced FP64 period from s, accumulating v^n e^{i w t_n}
        cudaMemsetAsync(u, 0, sizeof(double) * 2 * g.np, H->st);
        fo_forward<double>(H, H->fo_s, true, 1, H->fo_e, u);
        note_launch(1);
        k_fo_filter_final<<<fo_vec_blocks(g.np), kFT, 0, H->st>>>(g.np, u, 2.0 / (H->N * H->wt));
    } else {
        note_launch(1);
        k_fo_recover<<<fo_vec_blocks(g.np), kFT, 0, H->st>>>(H->fo_s, H->kap64, H->S, u, g, H->dt, H->wt, H->wh,
                                                             cos(0.5 * H->omega * H->dt));
    }
    if (cudaStreamSynchronize(H->st) != cudaSuccess) return CMCG_ERR_CUDA;
    return cuda_status();
}

void fo_J(cmcg_handle* H) { fo_forward<double>(H, H->fo_s, true, 0, H->fo_e, nullptr); }

int fo_solve(cmcg_handle* H, double tol, cmcg_stats* st) {
    if (H->opt.precision == CMCG_FP64) return fo_cg<double>(H, tol, st);
    if (H->opt.precision == CMCG_FP32) return fo_cg<float>(H, tol, st);
    return fo_mixed(H, tol, st);
}

int fo_period(cmcg_handle* H, const double* s0, bool src, double* out) {
    if (H->opt.precision == CMCG_FP64)
        fo_forward<double>(H, s0, src, 1, out, nullptr);
    else
        fo_forward<float>(H, s0, src, 1, out, nullptr);
    return cuda_status();
}

int fo_adjoint(cmcg_handle* H, const double* y, double* out) {
    if (H->opt.precision == CMCG_FP64)
        fo_backward<double>(H, y, y, 1, out);
    else
        fo_backward<float>(H, y, y, 1, out);
    return cuda_status();
}

}  // namespace detail
}  // namespace cmcg
