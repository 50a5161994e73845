// Host runtime and C ABI of libcmcg: handle, workspace carve-up, the forward / adjoint period
// drivers, the Riesz (MG-PCG) driver, and the CMCG Algorithm of Sec. 2.3 with its CG
// recurrences on the device (the host reads one convergence word per iteration).
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <atomic>
#include <chrono>
#include <type_traits>

#include "cmcg.h"
#include "common.cuh"
#include "kernels.h"
#include "solver.h"

using namespace cmcg;

namespace cmcg {
static std::atomic<long long> g_launches{0};
void note_launch(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace cmcg

namespace {


struct Carver {
    char* base;
    size_t off = 0;
    template <typename T>
    T* take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

}  // namespace


namespace cmcg {
namespace detail {

bool valid_grid(const cmcg_grid* gr) {
    if (!gr) return false;
    if (gr->dim != 2 && gr->dim != 3) return false;
    if (!(gr->h > 0) || !isfinite(gr->h)) return false;
    if (gr->order != 2 && gr->order != 4) return false;
    for (int a = 0; a < gr->dim; ++a)
        if (gr->n[a] < 2 || gr->n[a] > (1 << 20)) return false;
    long long np = 1;
    for (int a = 0; a < gr->dim; ++a) np *= (long long)(gr->n[a] + 1);
    return np < (1ll << 31);
}

Geom make_geom(const cmcg_grid* gr, unsigned abc) {
    Geom g{};
    g.dim = gr->dim;
    g.nx = gr->n[0];
    g.ny = gr->n[1];
    g.nz = gr->dim == 3 ? gr->n[2] : 0;
    g.sx = g.nx + 1;
    g.sy = g.ny + 1;
    g.sz = g.nz + 1;
    g.np = (long long)g.sx * g.sy * g.sz;
    g.h = gr->h;
    g.abc = abc;
    return g;
}

void fill_defaults(cmcg_options* o) {
    if (o->max_iter <= 0) o->max_iter = 10000;
    if (!(o->riesz_tol > 0)) o->riesz_tol = 1e-12;
    if (o->riesz_max_iter <= 0) o->riesz_max_iter = 60;
    if (!(o->inner_tol > 0)) o->inner_tol = 1e-3;
}

// Multigrid level geometries: every axis n -> ceil(n/2) while all axes keep >= 2 intervals.
// The coarse spacing is the mean of the per-axis spacings n_f h / n_c (equal for square grids
// and for even n; the preconditioner tolerates the small anisotropy otherwise).
int mg_geometries(const Geom& fine, Geom* out) {
    int n = 0;
    out[n++] = fine;
    while (n < kMaxLevels) {
        const Geom& p = out[n - 1];
        const bool big = p.nx >= 4 && p.ny >= 4 && (p.dim == 2 || p.nz >= 4);
        if (!big || p.np <= 64) break;
        Geom c = p;
        c.nx = (p.nx + 1) / 2;
        c.ny = (p.ny + 1) / 2;
        c.nz = p.dim == 3 ? (p.nz + 1) / 2 : 0;
        c.sx = c.nx + 1;
        c.sy = c.ny + 1;
        c.sz = c.nz + 1;
        c.np = (long long)c.sx * c.sy * c.sz;
        double hs = p.nx * p.h / c.nx + p.ny * p.h / c.ny;
        if (p.dim == 3) hs += p.nz * p.h / c.nz;
        c.h = hs / p.dim;
        out[n++] = c;
    }
    return n;
}

// Workspace layout.  The same function sizes (base == nullptr) and carves the workspace.
size_t layout(cmcg_handle* H, const Geom& g, const cmcg_options& o, char* base) {
    Carver c{base};
    const size_t np = (size_t)g.np;
    H->kap64 = c.take<double>(np);
    H->mass = c.take<double>(np);
    H->minv = c.take<double>(np);
    H->mask = c.take<unsigned char>(np);
    H->kap32 = o.precision != CMCG_FP64 ? c.take<float>(np + 4) : nullptr;  // + 16 B for bulk copies
    H->S = c.take<double>(2 * np);
    // FP32 steps read the source in FP32 (GB300 runs FP64 arithmetic at a small fraction of the
    // FP32 rate: an FP64 source term would make a forced FP32 step ALU-bound)
    // (conditions on the options, never on a carved pointer: sizing runs with base == nullptr)
    const bool f32_copies = o.precision != CMCG_FP64 && !(o.flags & CMCG_FLAG_FIRST_ORDER);
    H->S32 = f32_copies ? c.take<float>(2 * np + 4) : nullptr;
    H->mass32 = f32_copies ? c.take<float>(np) : nullptr;
    H->minv32 = f32_copies ? c.take<float>(np) : nullptr;
    H->scol = g.dim == 3 && !(o.flags & CMCG_FLAG_FIRST_ORDER) ? c.take<unsigned char>((size_t)g.sx * g.sy) : nullptr;
    if (o.flags & CMCG_FLAG_FIRST_ORDER) {
        // first-order state (p, v): CG vectors and the two stepping buffers; no Riesz map
        const size_t ns = (size_t)(g.dim + 1) * np;
        double** fo[] = {&H->fo_s, &H->fo_r, &H->fo_d, &H->fo_e, &H->fo_g, &H->fo_x};
        for (double** p : fo) *p = c.take<double>(ns);
        H->fo_a = c.take<double>(ns);
        H->fo_b = c.take<double>(ns);
        H->first_order = true;
        H->nlev = 0;
        H->stage = (o.flags & CMCG_FLAG_HOST_IO) ? c.take<double>(2 * np) : nullptr;
        long long nb = std::max<long long>(kMaxBlocksReduce, plane_blocks(g, kZcEnds));
        H->partials = c.take<double>((size_t)8 * nb);
        H->tickets = c.take<unsigned>(kNumTickets);
        H->sc = c.take<double>(SC_COUNT);
        return c.off + 256;
    }
    H->ya = c.take<double>(np);
    H->yb = c.take<double>(np);
    H->tmp = c.take<double>(np);
    double** cg[] = {&H->w0, &H->w1, &H->r0, &H->r1, &H->rh0, &H->rh1, &H->d0,
                     &H->d1, &H->gh0, &H->gh1, &H->gt0, &H->gt1, &H->z0, &H->z1};
    for (double** p : cg) *p = c.take<double>(np);
    if (o.precision == CMCG_MIXED) {
        H->wo0 = c.take<double>(np);
        H->wo1 = c.take<double>(np);
    }
    H->pr = c.take<double>(np);
    H->pp = c.take<double>(np);
    H->pAp = c.take<double>(np);
    H->pzd = c.take<double>(np);
    Geom lg[kMaxLevels];
    H->nlev = mg_geometries(g, lg);
    for (int l = 0; l < H->nlev; ++l) {
        MGLevel& L = H->lv[l];
        L.g = lg[l];
        const size_t n = (size_t)lg[l].np;
        L.mask = l == 0 ? H->mask : c.take<unsigned char>(n);
        L.x = c.take<float>(n);
        L.x2 = c.take<float>(n);
        L.b = c.take<float>(n);
        L.r = c.take<float>(n);
    }
    H->stage = (o.flags & CMCG_FLAG_HOST_IO) ? c.take<double>(2 * np) : nullptr;
    long long nb = std::max<long long>(kMaxBlocksReduce, plane_blocks(g, kZcEnds));
    H->partials = c.take<double>((size_t)8 * nb);
    H->tickets = c.take<unsigned>(kNumTickets);
    H->sc = c.take<double>(SC_COUNT);
    return c.off + 256;
}

int cuda_status() { return cudaGetLastError() == cudaSuccess ? CMCG_OK : CMCG_ERR_CUDA; }

// ---- L2 residency of kappa (CMCG_FLAG_L2_KAPPA) ----------------------------------------------
// The persisting-L2 set-aside is a per-process device limit: raised while any handle uses it,
// restored (and the persisting lines released) when the last one is destroyed.
static std::mutex g_l2_mu;
static int g_l2_users = 0;
static size_t g_l2_prev_limit = 0;

void l2_kappa_begin(cmcg_handle* H) {
    const cudaStream_t st = H->st;
    if (!H->kap32 || st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread) return;
    int dev = 0, max_persist = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, dev) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    const size_t bytes = sizeof(float) * (size_t)H->g.np;
    if (max_persist <= 0 || bytes > (size_t)max_persist) return;
    std::lock_guard<std::mutex> lock(g_l2_mu);
    size_t cur = 0;
    if (cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    if (g_l2_users == 0) g_l2_prev_limit = cur;
    if (cur < bytes && cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, bytes) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    cudaStreamAttrValue attr = {};
    attr.accessPolicyWindow.base_ptr = (void*)H->kap32;
    attr.accessPolicyWindow.num_bytes = bytes;
    attr.accessPolicyWindow.hitRatio = 1.0f;
    attr.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
    attr.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    if (cudaStreamSetAttribute(st, cudaStreamAttributeAccessPolicyWindow, &attr) != cudaSuccess) {
        cudaGetLastError();
        if (g_l2_users == 0) cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, g_l2_prev_limit);
        return;
    }
    g_l2_users += 1;
    H->l2_kappa = true;
}

void l2_kappa_end(cmcg_handle* H) {
    if (!H->l2_kappa) return;
    cudaStreamSynchronize(H->st);
    cudaStreamAttrValue attr = {};
    attr.accessPolicyWindow.num_bytes = 0;  // no window
    cudaStreamSetAttribute(H->st, cudaStreamAttributeAccessPolicyWindow, &attr);
    std::lock_guard<std::mutex> lock(g_l2_mu);
    if (--g_l2_users == 0) {
        cudaCtxResetPersistingL2Cache();
        cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, g_l2_prev_limit);
    }
    cudaGetLastError();
    H->l2_kappa = false;
}

void source_updated(cmcg_handle* H) {
    if (H->S32) launch_to_float(2 * H->g.np, H->S, H->S32, H->st);
    if (H->scol) launch_source_columns(H->g, H->S, H->scol, H->st);
}

// Fold completed event pairs into the per-precision step times.
// A pair without an elapsed time is skipped, and the error it raised is cleared unless an
// earlier one is pending.
void collect_timing(cmcg_handle* H) {
    const cudaError_t pending = cudaPeekAtLastError();
    for (int p = 0; p < H->ev_used; ++p) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, H->ev[2 * p], H->ev[2 * p + 1]) == cudaSuccess) {
            H->step_s[H->ev_fp32[p] ? 1 : 0] += 1e-3 * ms;
            H->step_n[H->ev_fp32[p] ? 1 : 0] += H->ev_steps[p];
        } else if (pending == cudaSuccess) {
            cudaGetLastError();
        }
    }
    H->ev_used = 0;
}

int sync_read(cmcg_handle* H) {
    cudaMemcpyAsync(H->hsc, H->sc, sizeof(double) * SC_COUNT, cudaMemcpyDeviceToHost, H->st);
    if (cudaStreamSynchronize(H->st) != cudaSuccess) return CMCG_ERR_CUDA;
    if (H->timing) collect_timing(H);
    return cuda_status();
}

// True while the handle's stream is being captured into a CUDA graph.
static bool capturing(cmcg_handle* H) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(H->st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cs != cudaStreamCaptureStatusNone;
}

// Inside a capture an event record becomes a graph node only when marked external; a replay
// then records the event like a plain launch would.
static void record_event(cmcg_handle* H, cudaEvent_t e) {
    if (capturing(H))
        cudaEventRecordWithFlags(e, H->st, cudaEventRecordExternal);
    else
        cudaEventRecord(e, H->st);
}

// Event pair around a period's step loop (only with CMCG_FLAG_TIMING).  Returns the slot.
int timing_begin(cmcg_handle* H, bool fp32, int steps) {
    if (!H->timing) return -1;
    if (H->ev_used == 4) {  // all slots busy: wait for them (never inside a capture)
        if (capturing(H)) return -1;
        cudaStreamSynchronize(H->st);
        collect_timing(H);
    }
    const int p = H->ev_used++;
    H->ev_fp32[p] = fp32;
    H->ev_steps[p] = steps;
    record_event(H, H->ev[2 * p]);
    return p;
}

void timing_end(cmcg_handle* H, int p) {
    if (p >= 0) record_event(H, H->ev[2 * p + 1]);
}

// ---- period drivers ------------------------------------------------------------------------
// A period is begin (start kernel), N-1 leapfrog steps, end (end kernel).  The pieces are
// separate so that the multi-solve engine can run the step loops of many solves in one
// batched kernel.
template <typename T>
PeriodBuffers fwd_begin(cmcg_handle* H, const double* w0, const double* w1, bool src, bool w0f_ready) {
    const Geom& g = H->g;
    const int zce = g.dim == 3 ? kZcEnds : 1;
    const T* kap = std::is_same<T, float>::value ? (const T*)H->kap32 : (const T*)H->kap64;
    PeriodBuffers b;
    b.cur = H->yb;
    b.prev = H->ya;
    // T-precision copy of w0 for the endpoint stencils (FP32: in the temp buffer, which the
    // forward period does not otherwise use)
    b.w0t = w0;
    const bool v32 = std::is_same<T, float>::value && H->vec32_active;  // w0, w1 hold floats
    if (std::is_same<T, float>::value && !v32) {
        float* w0f = (float*)H->tmp;
        if (!w0f_ready) launch_to_float(g.np, w0, w0f, H->st);
        b.w0t = w0f;
    }
    launch_start<T>(g, H->order, (const T*)b.w0t, w1, (T*)b.prev, (T*)b.cur, kap, src ? H->S : nullptr, H->dt,
                    zce, H->st, v32);
    return b;
}

// z-planes per thread of the one-step kernels; negative selects the variant that processes two
// planes per loop iteration (tile[3] == 3), kZcFlat the FP32 vector form (tile[3] == 5)
// tile[3] == 0 takes the scheme the autotuner found fastest on every measured class: the
// z-pair kernel on 3D 7- and 13-point grids, the vector form on 2D 5-point grids (FP64 steps
// fall back to their one-step kernels).
int step_zc(const cmcg_handle* H) {
    const int scheme = H->opt.tile[3];
    if (H->order == 2 && (scheme == 5 || (scheme == 0 && H->g.dim == 2))) return kZcFlat;
    if (H->g.dim != 3) return 1;
    const int zc = H->opt.tile[0] > 0 ? H->opt.tile[0] : kZcStep3D;
    if (H->order == 4) return (scheme == 3 || scheme == 0) ? -zc : zc;  // the 13-point z-pair kernel
    if (H->order != 2 || (scheme != 3 && scheme != 0)) return zc;
    return H->opt.tile[2] == 4 ? -(zc + kZk4) : -zc;  // tile[2]: planes per loop iteration (2 or 4)
}

// FP32 3D 7-point homogeneous steps run in pairs through the two-step kernel, whose outputs go
// to the spare halves of the (double-sized) wave buffers.
template <typename T>
bool use_pairs(const cmcg_handle* H, bool src) {
    return H->opt.tile[3] == 2 && std::is_same<T, float>::value && !src && step2_supported(H->g, H->order);
}

// One leapfrog step cur -> prev (in place).  FP32 3D 7-point steps without a source go through
// the bulk-copy kernel when tile[3] == 4 (tile[1] = band rows, tile[0] = planes per CTA).
template <typename T>
void step_one(cmcg_handle* H, const T* cur, T* prev, const T* kap, const T* S, double cs, double sn, int flags,
              int zc) {
    if (std::is_same<T, float>::value && H->opt.tile[3] == 6 && H->order == 2 && H->g.dim == 3) {
        // operands staged by asynchronous copies: tile[1] rows per band, tile[0] planes per CTA,
        // tile[2] planes in flight (any step, forced or not)
        if (launch_step_async(H->g, (const float*)cur, (float*)prev, (const float*)kap, (const float*)S, cs, sn, flags,
                              H->opt.tile[1], H->opt.tile[0], H->opt.tile[2], H->st) == cudaSuccess)
            return;
        cudaGetLastError();
    }
    if (std::is_same<T, float>::value && H->opt.tile[3] == 4 && H->order == 2 && !(flags & kStepSrc)) {
        int ty = 0, zb = 0;
        if (step_bulk_plan(H->g, H->opt.tile[1], H->opt.tile[0], &ty, &zb)) {
            launch_step_bulk(H->g, (const float*)cur, (float*)prev, (const float*)kap, flags, ty, zb, H->sc, H->st);
            return;
        }
    }
    launch_step<T>(H->g, H->order, cur, prev, kap, S, cs, sn, flags, zc, H->st, H->scol);
}

// `count` homogeneous steps from b (in pairs where possible, else one by one).
template <typename T>
void plain_steps(cmcg_handle* H, PeriodBuffers& b, int count) {
    const Geom& g = H->g;
    const int zc = step_zc(H);
    const T* kap = std::is_same<T, float>::value ? (const T*)H->kap32 : (const T*)H->kap64;
    if (use_pairs<T>(H, false) && count >= 2) {
        float* spare[2] = {(float*)H->ya + g.np, (float*)H->yb + g.np};
        // the spare halves are whichever two of the four float fields cur/prev are not
        float* fields[4] = {(float*)H->ya, (float*)H->yb, spare[0], spare[1]};
        int k = 0;
        for (float* f : fields)
            if (f != (float*)b.cur && f != (float*)b.prev && k < 2) spare[k++] = f;
        const int tp = timing_begin(H, true, count / 2);
        while (count >= 2) {
            launch_step2(g, (const float*)b.prev, (const float*)b.cur, (const float*)kap, spare[0], spare[1],
                         H->opt.tile[1], H->opt.tile[2], H->opt.tile[0], H->st);
            float* old_prev = (float*)b.prev;
            float* old_cur = (float*)b.cur;
            b.prev = spare[0];
            b.cur = spare[1];
            spare[0] = old_prev;
            spare[1] = old_cur;
            count -= 2;
        }
        timing_end(H, tp);
    }
    if (count <= 0) return;
    const int tp = use_pairs<T>(H, false) ? -1 : timing_begin(H, std::is_same<T, float>::value, count);
    for (int n = 0; n < count; ++n) {
        step_one<T>(H, (const T*)b.cur, (T*)b.prev, kap, nullptr, 0.0, 0.0, 0, zc);
        std::swap(b.cur, b.prev);
    }
    timing_end(H, tp);
}

template <typename T>
void fwd_steps(cmcg_handle* H, PeriodBuffers& b, bool src) {
    const int zc = step_zc(H);
    const T* kap = std::is_same<T, float>::value ? (const T*)H->kap32 : (const T*)H->kap64;
    if (!src) {
        plain_steps<T>(H, b, H->N - 1);
        return;
    }
    const T* S = step_source<T>(H);
    const int tp = timing_begin(H, std::is_same<T, float>::value, H->N - 1);
    for (int n = 1; n < H->N; ++n) {
        const double th = H->omega * n * H->dt;
        step_one<T>(H, (const T*)b.cur, (T*)b.prev, kap, S, cos(th), sin(th), kStepSrc, zc);
        std::swap(b.cur, b.prev);
    }
    timing_end(H, tp);
}

// mode 0: z = E (Pi(w) - w) into (out0, out1) and J into sc[SC_J]; mode 1: (y(T), y_t(T)).
template <typename T>
void fwd_end(cmcg_handle* H, const PeriodBuffers& b, const double* w1, bool src, int mode, double* out0,
             double* out1) {
    const Geom& g = H->g;
    const int zce = g.dim == 3 ? kZcEnds : 1;
    const T* kap = std::is_same<T, float>::value ? (const T*)H->kap32 : (const T*)H->kap64;
    const double thN = H->omega * H->N * H->dt;
    const int m = fp32_handoff<T>(mode) ? (H->vec32_active ? 3 : 2) : mode;
    launch_end<T>(g, H->order, m, (const T*)b.cur, (const T*)b.prev, (const T*)b.w0t, w1, kap, step_mass<T>(H),
                  src ? H->S : nullptr, cos(thN), sin(thN), out0, out1, H->red(), H->dt, zce, H->st);
    H->periods += 1;
}

template <typename T>
void forward_period(cmcg_handle* H, const double* w0, const double* w1, bool src, int mode, double* out0,
                    double* out1, bool w0f_ready) {
    Range range("cmcg forward period");
    PeriodBuffers b = fwd_begin<T>(H, w0, w1, src, w0f_ready);
    fwd_steps<T>(H, b, src);
    fwd_end<T>(H, b, w1, src, mode, out0, out1);
}

// Adjoint (transposed) period of the cotangents (a, b).
template <typename T>
PeriodBuffers adj_begin(cmcg_handle* H, const double* a, const double* bb, int mode) {
    const Geom& g = H->g;
    const int zce = g.dim == 3 ? kZcEnds : 1;
    const T* kap = std::is_same<T, float>::value ? (const T*)H->kap32 : (const T*)H->kap64;
    PeriodBuffers b;
    b.cur = H->ya;
    b.prev = H->yb;
    b.w0t = nullptr;
    if constexpr (std::is_same<T, float>::value) {
        if (fp32_handoff<T>(mode)) {  // t = D^-1 z1 came with z0 from the forward end
            launch_adj_start<float, float>(g, H->order, (const float*)a, (const float*)bb, H->mass32, kap,
                                           (float*)b.cur, (float*)b.prev, H->dt, zce, H->st);
            return b;
        }
    }
    T* t = (T*)H->tmp;
    launch_adj_prep<T>(g, bb, step_mass<T>(H), kap, t, zce, H->st);
    launch_adj_start<T>(g, H->order, a, t, step_mass<T>(H), kap, (T*)b.cur, (T*)b.prev, H->dt, zce, H->st);
    return b;
}

// Step flags of the k-th of the N-1 adjoint steps.
int adj_step_flags(int k, int N) {
    int flags = 0;
    if (k == 0) flags |= kStepPrevScaled;
    if (k == N - 2) flags |= kStepNoDiv;
    return flags;
}

template <typename T>
void adj_steps(cmcg_handle* H, PeriodBuffers& b) {
    const int zc = step_zc(H);
    const T* kap = std::is_same<T, float>::value ? (const T*)H->kap32 : (const T*)H->kap64;
    const int n = H->N - 1;  // steps k = 0 .. N-2; the first and the last have their own variants
    auto single = [&](int k) {
        step_one<T>(H, (const T*)b.cur, (T*)b.prev, kap, nullptr, 0.0, 0.0, adj_step_flags(k, H->N), zc);
        std::swap(b.cur, b.prev);
    };
    if (use_pairs<T>(H, false)) {
        single(0);
        if (n >= 3) plain_steps<T>(H, b, n - 2);
        if (n >= 2) single(n - 1);
        return;
    }
    const int tp = timing_begin(H, std::is_same<T, float>::value, n);
    for (int k = 0; k < n; ++k) single(k);
    timing_end(H, tp);
}

// mode 1: q = P^T (a, b) into (o0, o1).  mode 0: ghat = P^T z - z into (o0, o1),
// g~1 = ghat1 / M into gt1, and the reductions ghat . d -> sc[SC_GD], sum ghat0 -> sc[SC_GSUM].
template <typename T>
void adj_end(cmcg_handle* H, const PeriodBuffers& b, const double* a, const double* bb, int mode, const double* d0,
             const double* d1, double* o0, double* o1, double* gt1) {
    const Geom& g = H->g;
    const int zce = g.dim == 3 ? kZcEnds : 1;
    const T* kap = std::is_same<T, float>::value ? (const T*)H->kap32 : (const T*)H->kap64;
    const int m = fp32_handoff<T>(mode) ? (H->vec32_active ? 3 : 2) : mode;
    launch_adj_final<T>(g, H->order, m, (const T*)b.cur, (const T*)b.prev, step_mass<T>(H), kap, H->minv, a, bb, d0, d1, o0,
                        o1, gt1, H->red(), H->dt, zce, H->st);
    H->periods += 1;
}

template <typename T>
void adjoint_period(cmcg_handle* H, const double* a, const double* bb, int mode, const double* d0, const double* d1,
                    double* o0, double* o1, double* gt1) {
    Range range("cmcg adjoint period");
    PeriodBuffers b = adj_begin<T>(H, a, bb, mode);
    adj_steps<T>(H, b);
    adj_end<T>(H, b, a, bb, mode, d0, d1, o0, o1, gt1);
}

// ---- initial run-up (Sec. 4.2.3) ---------------------------------------------------------------
// Run-up periods: runup_periods itself when positive; -k = the periods waves at the slowest
// speed need to cross the domain's diagonal k times, ceil(k diam / (T c_min)).
int runup_count(const cmcg_handle* H) {
    if (H->opt.runup_periods > 0) return H->opt.runup_periods;
    if (H->opt.runup_periods == 0) return 0;
    double d2 = (double)H->g.nx * H->g.nx + (double)H->g.ny * H->g.ny + (double)H->g.nz * H->g.nz;
    const double diam = H->g.h * sqrt(d2);
    const double crossings = -(double)H->opt.runup_periods;
    return std::max(1, (int)ceil(crossings * diam / (H->T * H->cmin) - 1e-9));
}

// theta_tr(t) = (2 - sin(pi t / (2 t_tr))) sin(pi t / (2 t_tr)) for t <= t_tr, 1 after.
double ramp(double t, double ttr) {
    if (t >= ttr) return 1.0;
    const double s = sin(0.5 * kPi * t / ttr);
    return (2.0 - s) * s;
}

// Integrate the wave equation from rest for `periods` periods with the ramped sources and
// return (y, y_t) at t = periods T in (w0, w1).
template <typename T>
void runup(cmcg_handle* H, int periods, double* w0, double* w1) {
    Range range("cmcg run-up");
    const Geom& g = H->g;
    const int zc = step_zc(H);
    const int zce = g.dim == 3 ? kZcEnds : 1;
    const T* kap = std::is_same<T, float>::value ? (const T*)H->kap32 : (const T*)H->kap64;
    T* cur = (T*)H->yb;
    T* prev = (T*)H->ya;
    // y^0 = 0 and y^1 = 0: at rest, and the ramp vanishes at t = 0
    cudaMemsetAsync(cur, 0, sizeof(T) * g.np, H->st);
    cudaMemsetAsync(prev, 0, sizeof(T) * g.np, H->st);
    const long long total = (long long)periods * H->N;
    const double ttr = periods * H->T;
    for (long long n = 1; n < total; ++n) {
        const double t = n * H->dt;
        const double th = ramp(t, ttr);
        step_one<T>(H, cur, prev, kap, step_source<T>(H), th * cos(H->omega * t), th * sin(H->omega * t), kStepSrc,
                    zc);
        std::swap(cur, prev);
    }
    const double tN = total * H->dt;
    launch_end<T>(g, H->order, 1, cur, prev, (const T*)nullptr, nullptr, kap, step_mass<T>(H), H->S,
                  ramp(tN, ttr) * cos(H->omega * tN), ramp(tN, ttr) * sin(H->omega * tN), w0, w1, H->red(), H->dt,
                  zce, H->st);
    H->periods += periods;
}

// The FP32 run-up split around a step loop that runs elsewhere (the engine's batched
// kernel): the start sets both wave buffers to rest (y^n in yb, y^{n-1} in ya at step 1); the
// finish reads the state after periods N - 1 steps and writes (y, y_t) at t = periods T.
void runup_start_f32(cmcg_handle* H) {
    cudaMemsetAsync(H->yb, 0, sizeof(float) * H->g.np, H->st);
    cudaMemsetAsync(H->ya, 0, sizeof(float) * H->g.np, H->st);
}

void runup_finish_f32(cmcg_handle* H, int periods, double* w0, double* w1) {
    const Geom& g = H->g;
    const long long total = (long long)periods * H->N;
    const bool odd = ((total - 1) & 1) != 0;  // the buffers swap roles after every step
    const float* cur = (const float*)(odd ? H->ya : H->yb);
    const float* prev = (const float*)(odd ? H->yb : H->ya);
    const double ttr = periods * H->T, tN = total * H->dt;
    launch_end<float>(g, H->order, 1, cur, prev, (const float*)nullptr, nullptr, H->kap32, step_mass<float>(H), H->S,
                      ramp(tN, ttr) * cos(H->omega * tN), ramp(tN, ttr) * sin(H->omega * tN), w0, w1, H->red(),
                      H->dt, g.dim == 3 ? kZcEnds : 1, H->st);
    H->periods += periods;
}

// ---- Riesz map: FP64 flexible PCG with a FP32 multigrid V-cycle --------------------------
float jacobi_omega(const Geom& g) { return g.dim == 3 ? 6.0f / 7.0f : 0.8f; }

int coarse_sweeps(const Geom& g) {
    const int nmax = std::max(g.nx, std::max(g.ny, g.nz));
    return std::min(512, std::max(32, 8 * nmax * nmax));
}

void vcycle(cmcg_handle* H, int l) {
    MGLevel& L = H->lv[l];
    const float om = jacobi_omega(L.g);
    if (l == H->blk_level) {
        const BlockLevels& B = H->blk;
        launch_mg_block_vcycle(B, L.b, L.x, om, 2, coarse_sweeps(B.g[B.n - 1]), H->st);
        return;
    }
    if (l == H->nlev - 1) {  // coarsest level too large for one block: Jacobi sweeps
        launch_mg_jacobi(L, nullptr, L.x, L.b, om, true, H->st);
        for (int s = 0; s < 7; ++s) {
            launch_mg_jacobi(L, L.x, L.x2, L.b, om, false, H->st);
            std::swap(L.x, L.x2);
        }
        return;
    }
    const int nu = 2;
    launch_mg_jacobi(L, nullptr, L.x, L.b, om, true, H->st);
    for (int s = 1; s < nu; ++s) {
        launch_mg_jacobi(L, L.x, L.x2, L.b, om, false, H->st);
        std::swap(L.x, L.x2);
    }
    MGLevel& C = H->lv[l + 1];
    launch_mg_residual(L, L.x, L.b, L.r, H->st);
    launch_mg_restrict(L, L.r, C, C.b, H->st);
    vcycle(H, l + 1);
    launch_mg_prolong_add(C, C.x, L, L.x, H->st);
    for (int s = 0; s < nu; ++s) {
        launch_mg_jacobi(L, L.x, L.x2, L.b, om, false, H->st);
        std::swap(L.x, L.x2);
    }
}

void precondition(cmcg_handle* H, const double* r) {
    launch_to_float(H->g.np, r, H->lv[0].b, H->st);
    vcycle(H, 0);
}

// K s = rhs (K singular without Dirichlet nodes: rhs projected, s with W-mean zero).
int riesz_solve(cmcg_handle* H, const double* rhs, double* x, int* iters_out) {
    Range range("cmcg riesz MG-PCG");
    const Geom& g = H->g;
    const long long n = g.np;
    const bool project = !H->has_dir;
    const double tol = H->opt.riesz_tol;
    Red red = H->red();
    launch_pcg_project(g, rhs, H->pr, H->mask, H->volume, red, project, H->st);
    launch_fill(x, n, 0.0, H->st);
    precondition(H, H->pr);
    launch_pcg_dots_after_precond(n, H->pr, H->lv[0].x, nullptr, H->pzd, red, H->st);
    launch_pcg_p_update(n, H->pp, H->pzd, red, true, H->st);
    int it = 0;
    bool converged = false;
    double bb = -1.0;
    // the previous solve's iteration count, less a margin, runs without host checks
    const int blind = std::max(0, std::min(H->riesz_guess - 2, H->opt.riesz_max_iter - 1));
    for (it = 1; it <= H->opt.riesz_max_iter; ++it) {
        launch_applyK(g, H->order, H->mask, H->pp, H->pAp, H->pp, red, SC_P_PAP, H->st);
        launch_pcg_xr_update(n, x, H->pr, H->pp, H->pAp, red, H->st);
        if (it <= blind) {
            precondition(H, H->pr);
            launch_pcg_dots_after_precond(n, H->pr, H->lv[0].x, H->pAp, H->pzd, red, H->st);
            launch_pcg_p_update(n, H->pp, H->pzd, red, false, H->st);
            continue;
        }
        int rc = sync_read(H);
        if (rc != CMCG_OK) return rc;
        bb = H->hsc[SC_P_BB];
        const double rr = H->hsc[SC_P_RR];
        if (!(rr == rr)) return CMCG_ERR_DIVERGED;
        if (bb == 0.0 || rr <= tol * tol * bb) {
            converged = true;
            break;
        }
        precondition(H, H->pr);
        launch_pcg_dots_after_precond(n, H->pr, H->lv[0].x, H->pAp, H->pzd, red, H->st);
        launch_pcg_p_update(n, H->pp, H->pzd, red, false, H->st);
    }
    if (project) launch_mean_remove(g, x, H->volume, red, H->st);
    if (converged) H->riesz_guess = it;
    H->riesz_iters += std::min(it, H->opt.riesz_max_iter);
    if (iters_out) *iters_out = std::min(it, H->opt.riesz_max_iter);
    int rc = cuda_status();
    if (rc != CMCG_OK) return rc;
    return converged ? CMCG_OK : CMCG_NOT_CONVERGED;
}

// ---- CMCG ---------------------------------------------------------------------------------
// Gradient of J at (w0, w1) (with the sources if src): ghat -> (gh0, gh1), g~ -> (gt0, gt1),
// z -> (z0, z1); J -> sc[SC_J].
template <typename T>
int gradient(cmcg_handle* H, const double* w0, const double* w1, bool src, const double* dd0, const double* dd1,
             bool riesz, bool w0f_ready) {
    forward_period<T>(H, w0, w1, src, 0, H->z0, H->z1, w0f_ready);
    adjoint_period<T>(H, H->z0, H->z1, 0, dd0, dd1, H->gh0, H->gh1, riesz ? H->gt1 : nullptr);
    if (!riesz) return CMCG_OK;
    int rc = riesz_solve(H, H->gh0, H->gt0, nullptr);
    return rc < 0 ? rc : CMCG_OK;
}

bool inexact(const cmcg_handle* H) { return (H->opt.flags & CMCG_FLAG_INEXACT_RIESZ) != 0; }

// Approximate Riesz map z = B rhat into (r0, r1): one V-cycle on rhat0 (W-mean removed when K
// is singular), M^-1 rhat1; reduces gamma = z . rhat (and the Polak-Ribiere beta unless first).
// lowp: inside a solve with FP32 periods, the pointwise work and the dots run in FP32.
void apply_B(cmcg_handle* H, bool first, bool lowp, bool b_ready) {
    Range range("cmcg riesz V-cycle");
    const Geom& g = H->g;
    Red red = H->red();
    const bool v32 = H->vec32_active;  // rhat, ghat and z are FP32 vectors
    if (!b_ready) {
        if (v32) cudaMemcpyAsync(H->lv[0].b, H->rh0, sizeof(float) * g.np, cudaMemcpyDeviceToDevice, H->st);
        else launch_to_float(g.np, H->rh0, H->lv[0].b, H->st);
    }
    vcycle(H, 0);
    if (!H->has_dir) launch_wsum_float(g, H->lv[0].x, red, H->st);
    launch_fcg_dots(g, H->lv[0].x, H->volume, !H->has_dir, lowp || v32, H->rh0, H->rh1,
                    v32 ? (const double*)H->minv32 : H->minv, H->gh0, H->gh1, H->r0, H->r1, red, first, H->st, v32);
    H->riesz_iters += 1;
}

// Start of an inner solve on FP32 CG vectors: rhat = float(ghat) from the FP64 gradient,
// z = B rhat and gamma0 (apply_B), d = z; leaves vec32_active set.
void begin_vec32_inner(cmcg_handle* H) {
    const long long n = H->g.np;
    launch_to_float(n, H->gh0, (float*)H->rh0, H->st);
    launch_to_float(n, H->gh1, (float*)H->rh1, H->st);
    H->vec32_active = true;
    apply_B(H, true, true);
    cudaMemcpyAsync(H->d0, H->r0, sizeof(float) * n, cudaMemcpyDeviceToDevice, H->st);
    cudaMemcpyAsync(H->d1, H->r1, sizeof(float) * n, cudaMemcpyDeviceToDevice, H->st);
}

// W += w: the inner correction (FP32 vectors on a vec32 handle) into the FP64 iterate.
void add_correction(cmcg_handle* H, double* W0, double* W1) {
    const long long n = H->g.np;
    if (H->vec32) {
        launch_add_float(n, (const float*)H->w0, W0, H->st);
        launch_add_float(n, (const float*)H->w1, W1, H->st);
    } else {
        launch_axpy(n, 1.0, H->w0, W0, H->st);
        launch_axpy(n, 1.0, H->w1, W1, H->st);
    }
}

// One CG iteration captured as a CUDA graph.  Capture needs a created stream that is not
// already being captured; any failure leaves the caller on plain launches.  A replay advances
// the host-side counters (periods, Riesz maps, launches) by what the captured iteration would
// have added.  With step timing the event records are graph nodes: a replay re-records the
// same slots, and the host bookkeeping of those slots (precision, step count) is restored
// from the capture.  If the first replay's events give no elapsed time, the graph is dropped
// and timing goes on with plain launches.
struct IterationGraph {
    cudaGraphExec_t exec = nullptr;
    long long periods = 0, riesz = 0, launches = 0;
    int ev_used = 0;
    bool ev_fp32[4] = {};
    int ev_steps[4] = {};
    long long timed_replays = 0;
    template <typename F>
    void capture(cmcg_handle* H, F body) {
        cudaStream_t st = H->st;
        if (st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread || capturing(H)) return;
        if (H->timing && H->ev_used != 0) {  // captured slots start at 0
            if (cudaStreamSynchronize(st) != cudaSuccess) return;
            collect_timing(H);
        }
        const long long p0 = H->periods, r0 = H->riesz_iters, l0 = launch_count();
        if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        body();
        cudaGraph_t g = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(st, &g);
        periods = H->periods - p0;
        riesz = H->riesz_iters - r0;
        launches = launch_count() - l0;
        ev_used = H->ev_used;
        for (int p = 0; p < ev_used; ++p) {
            ev_fp32[p] = H->ev_fp32[p];
            ev_steps[p] = H->ev_steps[p];
        }
        H->periods = p0;  // nothing ran yet
        H->riesz_iters = r0;
        H->ev_used = 0;
        note_launch(-launches);
        if (ce == cudaSuccess && g && cudaGraphInstantiate(&exec, g, 0) != cudaSuccess) exec = nullptr;
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
    }
    bool replay(cmcg_handle* H) {
        if (!exec) return false;
        if (H->timing && ev_used > 0) {
            if (timed_replays == 1 && H->step_n[0] + H->step_n[1] == steps_before) {
                drop();  // the graph's event records gave no elapsed time
                return false;
            }
            if (H->ev_used != 0) {
                cudaStreamSynchronize(H->st);
                collect_timing(H);
            }
            if (timed_replays == 0) steps_before = H->step_n[0] + H->step_n[1];
        }
        if (cudaGraphLaunch(exec, H->st) != cudaSuccess) {
            cudaGetLastError();
            drop();
            return false;
        }
        if (H->timing) {
            H->ev_used = ev_used;
            for (int p = 0; p < ev_used; ++p) {
                H->ev_fp32[p] = ev_fp32[p];
                H->ev_steps[p] = ev_steps[p];
            }
            ++timed_replays;
        }
        H->periods += periods;
        H->riesz_iters += riesz;
        ++H->graph_replays;
        note_launch(launches);
        return true;
    }
    void drop() {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
    }
    ~IterationGraph() { drop(); }

  private:
    long long steps_before = 0;
};

// Flexible CG (Polak-Ribiere) on the current gradient in (gh0, gh1) with z = B rhat;
// iterate accumulated into (w0, w1) (v -= alpha d).
template <typename T>
int fcg_loop(cmcg_handle* H, double tol, int max_iter, int* iters, double* rel_out) {
    const long long n = H->g.np;
    Red red = H->red();
    const bool f32 = std::is_same<T, float>::value;
    const bool v32 = f32 && H->vec32;  // the inner solve of mixed precision: FP32 CG vectors
    struct Reset {  // vec32_active holds only while this loop enqueues work
        cmcg_handle* h;
        ~Reset() { h->vec32_active = false; }
    } reset{H};
    if (v32) {
        begin_vec32_inner(H);
    } else {
        cudaMemcpyAsync(H->rh0, H->gh0, sizeof(double) * n, cudaMemcpyDeviceToDevice, H->st);
        cudaMemcpyAsync(H->rh1, H->gh1, sizeof(double) * n, cudaMemcpyDeviceToDevice, H->st);
        apply_B(H, true, f32);
        cudaMemcpyAsync(H->d0, H->r0, sizeof(double) * n, cudaMemcpyDeviceToDevice, H->st);
        cudaMemcpyAsync(H->d1, H->r1, sizeof(double) * n, cudaMemcpyDeviceToDevice, H->st);
    }
    int rc = sync_read(H);
    if (rc != CMCG_OK) return rc;
    if (H->hsc[SC_STATUS] != 0.0) return CMCG_ERR_DIVERGED;
    double rel = H->hsc[SC_REL];
    H->hist.push_back(rel * H->hist_scale);
    int it = 0;
    // FP32 periods read float(d0) (with FP32 vectors d0 itself); the direction update writes it
    // for the next iteration, and the dual-residual update writes float(rhat0) for the V-cycle
    float* d0f = f32 && !v32 ? (float*)H->tmp : nullptr;
    if (d0f) launch_to_float(n, H->d0, d0f, H->st);
    auto body = [&]() {
        gradient<T>(H, H->d0, H->d1, false, H->d0, H->d1, false, f32);  // 5.1: ghat_d = H d
        launch_fcg_update(n, H->w0, H->w1, H->rh0, H->rh1, H->d0, H->d1, H->gh0, H->gh1, red, H->st, H->lv[0].b,
                          v32);
        apply_B(H, false, f32, true);                                      // 5.2 on the residual
        launch_cg_direction(n, H->r0, H->r1, H->d0, H->d1, red, H->st, d0f, v32);  // 5.7
    };
    // The iteration's launches and arguments do not change (its scalars live on the device), so
    // it is captured once as a CUDA graph and replayed: on small grids the host's launch rate,
    // not the GPU, sets the pace of a plain loop.
    IterationGraph graph;
    if (rel > tol && max_iter > 1) graph.capture(H, body);
    if (rel > tol) {
        for (it = 1; it <= max_iter; ++it) {
            if (!graph.replay(H)) body();
            rc = sync_read(H);
            if (rc != CMCG_OK) return rc;
            if (H->hsc[SC_STATUS] != 0.0) return CMCG_ERR_DIVERGED;
            rel = H->hsc[SC_REL];
            H->hist.push_back(rel * H->hist_scale);
            if (rel <= tol) break;
        }
        if (it > max_iter) it = max_iter;
    }
    *iters = it;
    *rel_out = rel;
    return rel <= tol ? CMCG_OK : CMCG_NOT_CONVERGED;
}

// gamma = ||g~||_E^2 of the gradient currently in (gh, gt) (exact Riesz) or z = B ghat.
int gradient_norm(cmcg_handle* H, double* gamma) {
    const long long n = H->g.np;
    Red red = H->red();
    if (inexact(H)) {
        cudaMemcpyAsync(H->rh0, H->gh0, sizeof(double) * n, cudaMemcpyDeviceToDevice, H->st);
        cudaMemcpyAsync(H->rh1, H->gh1, sizeof(double) * n, cudaMemcpyDeviceToDevice, H->st);
        apply_B(H, true, false);
        launch_scalar_residual(n, H->r0, H->r1, H->rh0, H->rh1, red, SC_R7, H->st);
    } else {
        launch_scalar_residual(n, H->gt0, H->gt1, H->gh0, H->gh1, red, SC_R7, H->st);
    }
    const int rc = sync_read(H);
    if (rc != CMCG_OK) return rc;
    *gamma = H->hsc[SC_R7];
    return (*gamma == *gamma && *gamma >= 0) ? CMCG_OK : CMCG_ERR_DIVERGED;
}

// With a warm start (cmcg_solve_warm) or a run-up: the zero-guess gradient norm (the
// tolerance reference), then the start state into (w0, w1): the given field's periodic
// initial state, or the run-up state.  Otherwise: (w0, w1) = 0 and gamma_zero = -1.
template <typename T>
int initial_guess(cmcg_handle* H, double* w0, double* w1, double* gamma_zero, cmcg_stats* stats) {
    const long long n = H->g.np;
    launch_fill(w0, n, 0.0, H->st);
    launch_fill(w1, n, 0.0, H->st);
    *gamma_zero = -1.0;
    if (H->warm) {
        stats->runup_periods = 0;
        int rc = gradient<T>(H, w0, w1, true, w0, w1, !inexact(H));
        if (rc < 0) return rc;
        rc = gradient_norm(H, gamma_zero);
        if (rc != CMCG_OK) return rc;
        launch_warm_start(n, H->warm, H->kap64, H->wh, w0, w1, H->st);
        return cuda_status();
    }
    const int ell = runup_count(H);
    stats->runup_periods = ell;
    if (ell <= 0) return CMCG_OK;
    int rc = gradient<T>(H, w0, w1, true, w0, w1, !inexact(H));
    if (rc < 0) return rc;
    rc = gradient_norm(H, gamma_zero);
    if (rc != CMCG_OK) return rc;
    runup<T>(H, ell, w0, w1);
    return cuda_status();
}

// CG loop of Steps (4)-(5) on the current gradient (gh, gt) with homogeneous periods in
// precision T; iterate accumulated into (w0, w1) (v -= alpha d).
template <typename T>
int cg_loop(cmcg_handle* H, double tol, int max_iter, int* iters, double* rel_out) {
    if (inexact(H)) return fcg_loop<T>(H, tol, max_iter, iters, rel_out);
    const long long n = H->g.np;
    Red red = H->red();
    launch_cg_init(n, H->gt0, H->gt1, H->gh0, H->gh1, H->r0, H->r1, H->rh0, H->rh1, H->d0, H->d1, red, H->st);
    int rc = sync_read(H);
    if (rc != CMCG_OK) return rc;
    if (H->hsc[SC_STATUS] != 0.0) return CMCG_ERR_DIVERGED;
    double rel = H->hsc[SC_REL];
    H->hist.push_back(rel * H->hist_scale);
    int it = 0;
    if (rel > tol) {
        for (it = 1; it <= max_iter; ++it) {
            // 5.1: homogeneous forward + adjoint period from d; 5.2: Riesz
            rc = gradient<T>(H, H->d0, H->d1, false, H->d0, H->d1, true);
            if (rc < 0) return rc;
            // 5.3-5.6
            launch_cg_update(n, H->w0, H->w1, H->r0, H->r1, H->rh0, H->rh1, H->d0, H->d1, H->gt0, H->gt1, H->gh0,
                             H->gh1, -1.0, red, H->st);
            // 5.7
            launch_cg_direction(n, H->r0, H->r1, H->d0, H->d1, red, H->st);
            // 5.8
            rc = sync_read(H);
            if (rc != CMCG_OK) return rc;
            if (H->hsc[SC_STATUS] != 0.0) return CMCG_ERR_DIVERGED;
            rel = H->hsc[SC_REL];
            H->hist.push_back(rel * H->hist_scale);
            if (rel <= tol) break;
        }
        if (it > max_iter) it = max_iter;
    }
    *iters = it;
    *rel_out = rel;
    return rel <= tol ? CMCG_OK : CMCG_NOT_CONVERGED;
}

template <typename T>
int solve_plain(cmcg_handle* H, double tol, cmcg_stats* stats) {
    // (1) v = 0 or the run-up state; (2)-(3) gradient with the sources and its Riesz map
    double gamma_zero = -1.0;
    int rc = initial_guess<T>(H, H->w0, H->w1, &gamma_zero, stats);
    if (rc != CMCG_OK) return rc;
    rc = gradient<T>(H, H->w0, H->w1, true, H->w0, H->w1, !inexact(H));
    if (rc < 0) return rc;
    double scale = 1.0;  // rel w.r.t. this start -> rel w.r.t. the zero guess
    if (gamma_zero > 0) {
        double g_init = 0.0;
        rc = gradient_norm(H, &g_init);
        if (rc != CMCG_OK) return rc;
        scale = sqrt(g_init / gamma_zero);
    } else {
        rc = sync_read(H);
        if (rc != CMCG_OK) return rc;
    }
    stats->J0 = H->hsc[SC_J];
    int iters = 0;
    double rel = 1.0;
    if (scale <= tol) {
        H->hist.push_back(scale);
        stats->iterations = 0;
        stats->rel_residual = scale;
        return CMCG_OK;
    }
    H->hist_scale = scale;
    rc = cg_loop<T>(H, tol / scale, H->opt.max_iter, &iters, &rel);
    stats->iterations = iters;
    stats->rel_residual = rel * scale;
    return rc;
}

// CMCG_MIXED: defect correction.  Outer: FP64 gradient at the FP64 iterate W; inner: CG with
// FP32 periods on the correction, started from that gradient, to inner_tol; W += correction.
int solve_mixed(cmcg_handle* H, double tol, cmcg_stats* stats) {
    const long long n = H->g.np;
    Red red = H->red();
    double gamma_ref = -1.0;
    int rc0 = initial_guess<float>(H, H->wo0, H->wo1, &gamma_ref, stats);
    if (rc0 != CMCG_OK) return rc0;
    int total = 0, outer = 0;
    double rel = 1.0;
    int rc = CMCG_OK;
    const int max_outer = 50;
    for (outer = 0; outer < max_outer; ++outer) {
        rc = gradient<double>(H, H->wo0, H->wo1, true, H->wo0, H->wo1, !inexact(H));
        if (rc < 0) return rc;
        if (inexact(H)) {
            cudaMemcpyAsync(H->rh0, H->gh0, sizeof(double) * n, cudaMemcpyDeviceToDevice, H->st);
            cudaMemcpyAsync(H->rh1, H->gh1, sizeof(double) * n, cudaMemcpyDeviceToDevice, H->st);
            apply_B(H, true, false);
            launch_scalar_residual(n, H->r0, H->r1, H->rh0, H->rh1, red, SC_R7, H->st);
        } else {
            launch_scalar_residual(n, H->gt0, H->gt1, H->gh0, H->gh1, red, SC_R7, H->st);
        }
        rc = sync_read(H);
        if (rc != CMCG_OK) return rc;
        const double gam = H->hsc[SC_R7];
        if (!(gam == gam) || gam < 0) return CMCG_ERR_DIVERGED;
        if (outer == 0) {
            if (gamma_ref <= 0) gamma_ref = gam;
            stats->J0 = H->hsc[SC_J];
        }
        rel = gamma_ref > 0 ? sqrt(gam / gamma_ref) : 0.0;
        // the FP64 residual replaces the inner solve's last estimate
        if (H->hist.empty()) H->hist.push_back(rel);
        else H->hist.back() = rel;
        if (rel <= tol || total >= H->opt.max_iter) break;
        // inner solve: relative tolerance inner_tol, but not below what the outer needs
        const double inner = std::max(H->opt.inner_tol, 0.5 * tol / std::max(rel, 1e-300));
        launch_fill(H->w0, n, 0.0, H->st);
        launch_fill(H->w1, n, 0.0, H->st);
        int it = 0;
        double irel = 1.0;
        H->hist_scale = rel;
        H->hist.pop_back();  // the inner loop records its start, which is this FP64 residual
        rc = cg_loop<float>(H, std::min(inner, 0.5), H->opt.max_iter - total, &it, &irel);
        if (rc < 0) return rc;
        total += it;
        add_correction(H, H->wo0, H->wo1);
    }
    // the returned iterate lives in (w0, w1)
    cudaMemcpyAsync(H->w0, H->wo0, sizeof(double) * n, cudaMemcpyDeviceToDevice, H->st);
    cudaMemcpyAsync(H->w1, H->wo1, sizeof(double) * n, cudaMemcpyDeviceToDevice, H->st);
    stats->iterations = total;
    stats->outer_iterations = outer;
    stats->rel_residual = rel;
    if (cuda_status() != CMCG_OK) return CMCG_ERR_CUDA;
    return rel <= tol ? CMCG_OK : CMCG_NOT_CONVERGED;
}

// Step (6): U = v0 + i v1 / omega_hat from (w0, w1), then the compatibility-condition shift
//   lambda = (1.F + wt^2 1.M u + i wh 1.B u) / (wt^2 sum M + i wh sum B)
// when there is no Dirichlet node.
// lambda of the discrete compatibility condition (K - wt^2 M - i wh B)(u - lambda) = F^ from
// the sums 1.F^, 1.M u, 1.B u in hsc[SC_R0..+5]; subtracts it from u (device).
void compat_shift(cmcg_handle* h, double* u, double* lre, double* lim) {
    const double* r = h->hsc + SC_R0;
    const double wt2 = h->wt * h->wt;
    const double nre = r[0] + wt2 * r[2] - h->wh * r[5];
    const double nim = r[1] + wt2 * r[3] + h->wh * r[4];
    const double dre = wt2 * h->sumM, dim = h->wh * h->sumB;
    const double den = dre * dre + dim * dim;
    *lre = (nre * dre + nim * dim) / den;
    *lim = (nim * dre - nre * dim) / den;
    launch_shift(h->g.np, u, h->kap64, *lre, *lim, h->st);
}

int recover(cmcg_handle* h, double* u, cmcg_stats* st) {
    launch_recover(h->g, h->w0, h->w1, h->wh, h->S, h->kap64, h->mass, u, h->red(), h->st);
    if (sync_read(h) != CMCG_OK) return CMCG_ERR_CUDA;
    double lre = 0.0, lim = 0.0;
    if (!h->has_dir) compat_shift(h, u, &lre, &lim);
    if (cudaStreamSynchronize(h->st) != cudaSuccess) return CMCG_ERR_CUDA;
    if (cuda_status() != CMCG_OK) return CMCG_ERR_CUDA;
    st->lambda_re = lre;
    st->lambda_im = lim;
    return CMCG_OK;
}

// Step (6) by the fundamental-frequency filter of Sec. 2.2 instead of the compatibility
// condition: one forced FP64 period from (w0, w1), accumulating
// U = (1/N) sum_n (y^n + (i/wh) v^n) e^{i w t_n} in u.  The filter removes lambda and the
// T-periodic eigenmodes; a linearly growing part eta t of the minimiser survives as a constant.
// It vanishes when there are absorbing faces or Dirichlet nodes; in the pure Neumann case it is
// removed with the discrete compatibility condition (the discrete form of Eq. cc_neumann_eta),
// and its value is returned in stats lambda.
int filter_recover(cmcg_handle* h, double* u, cmcg_stats* st) {
    const Geom& g = h->g;
    const int zc = g.dim == 3 ? kZcStep3D : 1;
    launch_filter_init(g.np, h->w0, h->w1, h->kap64, 1.0 / h->wh, u, h->st);
    PeriodBuffers b = fwd_begin<double>(h, h->w0, h->w1, true);
    const double cv = 1.0 / (2.0 * h->dt * h->wh);
    for (int n = 1; n < h->N; ++n) {
        const double t = n * h->dt, c = cos(h->omega * t), sn = sin(h->omega * t);
        launch_step_filter(g, h->order, (const double*)b.cur, (double*)b.prev, h->kap64, h->S, c, sn, u, c, sn, cv, zc,
                           h->st);
        std::swap(b.cur, b.prev);
    }
    launch_scale_complex(g.np, u, 1.0 / h->N, h->st);
    h->periods += 1;
    st->lambda_re = st->lambda_im = 0.0;
    if (!h->has_dir && g.abc == 0u) {
        launch_compat_sums(g, u, h->S, h->kap64, h->mass, h->red(), h->st);
        if (sync_read(h) != CMCG_OK) return CMCG_ERR_CUDA;
        compat_shift(h, u, &st->lambda_re, &st->lambda_im);
    }
    if (cudaStreamSynchronize(h->st) != cudaSuccess) return CMCG_ERR_CUDA;
    return cuda_status();
}

// Steps (1)-(6) with the source S already in the workspace; U into u (device).
int solve_prepared(cmcg_handle* h, double tol, double* u, cmcg_stats* st, bool want_J) {
    Range range("cmcg solve");
    memset(st, 0, sizeof(*st));
    const long long launches0 = launch_count();
    h->step_s[0] = h->step_s[1] = 0.0;
    h->step_n[0] = h->step_n[1] = 0;
    h->ev_used = 0;
    h->riesz_iters = 0;
    h->periods = 0;
    h->graph_replays = 0;
    h->hist.clear();
    h->hist_scale = 1.0;
    const long long n = h->g.np;
    int rc;
    if (h->first_order) {
        // Sec. 3: CMCG on the first-order state, J^ at the result, step (6)
        rc = fo_solve(h, tol, st);
        if (rc < 0) return rc;
        const long long periods_solve = h->periods;
        if (want_J) {
            fo_J(h);
            if (sync_read(h) != CMCG_OK) return CMCG_ERR_CUDA;
            st->J_final = h->hsc[SC_J];
        }
        if (fo_recover(h, u) != CMCG_OK) return CMCG_ERR_CUDA;
        st->steps_per_period = h->N;
        st->dt = h->dt;
        st->omega_tilde = h->wt;
        st->omega_hat = h->wh;
        st->periods = (int)periods_solve;
        st->point_updates = periods_solve * (long long)h->N * n;
        st->kernel_launches = launch_count() - launches0;
        if (h->timing) collect_timing(h);
        st->step_seconds_fp64 = h->step_s[0];
        st->step_seconds_fp32 = h->step_s[1];
        st->step_launches_fp64 = h->step_n[0];
        st->step_launches_fp32 = h->step_n[1];
        return rc;
    }
    if (h->opt.flags & CMCG_FLAG_NO_CG) {
        // do-nothing: the run-up's final state is the answer
        const int ell = runup_count(h);
        st->runup_periods = ell;
        if (h->opt.precision == CMCG_FP64)
            runup<double>(h, ell, h->w0, h->w1);
        else
            runup<float>(h, ell, h->w0, h->w1);
        rc = cuda_status();
    } else if (h->opt.precision == CMCG_FP64)
        rc = solve_plain<double>(h, tol, st);
    else if (h->opt.precision == CMCG_FP32)
        rc = solve_plain<float>(h, tol, st);
    else
        rc = solve_mixed(h, tol, st);
    if (rc < 0) return rc;
    const long long periods_solve = h->periods;
    // J at the returned iterate (FP64 period with the sources)
    if (want_J) {
        forward_period<double>(h, h->w0, h->w1, true, 0, h->z0, h->z1);
        if (sync_read(h) != CMCG_OK) return CMCG_ERR_CUDA;
        st->J_final = h->hsc[SC_J];
    }
    // (6) recovery: the compatibility-condition shift, or the filter of Sec. 2.2
    if (h->opt.flags & CMCG_FLAG_FILTER) {
        if (filter_recover(h, u, st) != CMCG_OK) return CMCG_ERR_CUDA;
    } else if (recover(h, u, st) != CMCG_OK) {
        return CMCG_ERR_CUDA;
    }
    st->steps_per_period = h->N;
    st->dt = h->dt;
    st->omega_tilde = h->wt;
    st->omega_hat = h->wh;
    st->periods = (int)periods_solve;
    st->riesz_iterations = (int)h->riesz_iters;
    st->point_updates = periods_solve * (long long)h->N * n;
    st->kernel_launches = launch_count() - launches0;
    if (h->timing) collect_timing(h);
    st->step_seconds_fp64 = h->step_s[0];
    st->step_seconds_fp32 = h->step_s[1];
    st->step_launches_fp64 = h->step_n[0];
    st->step_launches_fp32 = h->step_n[1];
    st->graph_replays = h->graph_replays;
    return rc;
}


template PeriodBuffers fwd_begin<float>(cmcg_handle*, const double*, const double*, bool, bool);
template PeriodBuffers fwd_begin<double>(cmcg_handle*, const double*, const double*, bool, bool);
template void fwd_end<float>(cmcg_handle*, const PeriodBuffers&, const double*, bool, int, double*, double*);
template void fwd_end<double>(cmcg_handle*, const PeriodBuffers&, const double*, bool, int, double*, double*);
template PeriodBuffers adj_begin<float>(cmcg_handle*, const double*, const double*, int);
template PeriodBuffers adj_begin<double>(cmcg_handle*, const double*, const double*, int);
template void adj_end<float>(cmcg_handle*, const PeriodBuffers&, const double*, const double*, int, const double*,
                             const double*, double*, double*, double*);
template void adj_end<double>(cmcg_handle*, const PeriodBuffers&, const double*, const double*, int, const double*,
                              const double*, double*, double*, double*);
template void runup<float>(cmcg_handle*, int, double*, double*);
template int gradient<double>(cmcg_handle*, const double*, const double*, bool, const double*, const double*, bool,
                               bool);
template int gradient<float>(cmcg_handle*, const double*, const double*, bool, const double*, const double*, bool,
                              bool);
template void forward_period<double>(cmcg_handle*, const double*, const double*, bool, int, double*, double*, bool);

}  // namespace detail
}  // namespace cmcg

using namespace cmcg::detail;

// ---- period on caller-provided scratch (used by the allocation-free entry point) --------
namespace cmcg {

// Carve of the scratch a stand-alone FP64 period needs: coefficients, source, the two wave
// buffers, masked copies of the initial data, reduction slots.
static size_t scratch_layout(cmcg_handle* H, const Geom& g, char* base) {
    Carver c{base};
    const size_t np = (size_t)g.np;
    H->kap64 = c.take<double>(np);
    H->mass = c.take<double>(np);
    H->mask = c.take<unsigned char>(np);
    H->kap32 = nullptr;
    H->S = c.take<double>(2 * np);
    H->ya = c.take<double>(np);
    H->yb = c.take<double>(np);
    H->z0 = c.take<double>(np);
    H->z1 = c.take<double>(np);
    long long nb = std::max<long long>(kMaxBlocksReduce, plane_blocks(g, kZcEnds));
    H->partials = c.take<double>((size_t)8 * nb);
    H->tickets = c.take<unsigned>(kNumTickets);
    H->sc = c.take<double>(SC_COUNT);
    return c.off + 256;
}

int wave_period_in_scratch(const cmcg_grid* grid, const double* c, double omega, const cmcg_bc* bc,
                           double dt_target, const double* u0, const double* v0, const double* f, const double* g,
                           double* uT, double* vT, char* scratch, size_t scratch_bytes, cudaStream_t st) {
    if (!valid_grid(grid) || !c || !bc || !u0 || !v0 || !uT || !vT || !scratch) return CMCG_ERR_INVALID_ARG;
    if (!(omega > 0) || !isfinite(omega) || dt_target < 0 || !isfinite(dt_target)) return CMCG_ERR_INVALID_ARG;
    unsigned abc = 0, dir = 0;
    for (int fc = 0; fc < 2 * grid->dim; ++fc) {
        const int code = bc->face[fc];
        if (code == CMCG_BC_ABC) abc |= 1u << fc;
        else if (code == CMCG_BC_DIRICHLET) dir |= 1u << fc;
        else if (code != CMCG_BC_NEUMANN) return CMCG_ERR_INVALID_ARG;
    }
    cmcg_handle H;
    H.g = make_geom(grid, abc);
    H.order = grid->order;
    H.opt.precision = CMCG_FP64;
    fill_defaults(&H.opt);  // the same option defaults as a created handle
    H.st = st;
    H.omega = omega;
    H.T = 2.0 * kPi / omega;
    if (scratch_layout(&H, H.g, nullptr) > scratch_bytes) return CMCG_ERR_WORKSPACE;
    scratch_layout(&H, H.g, scratch);
    double host_sc[SC_COUNT];
    H.hsc = host_sc;
    // the scratch keeps the previous call's contents: clear the reduction slots
    cudaMemsetAsync(H.tickets, 0, sizeof(unsigned) * kNumTickets, st);
    cudaMemsetAsync(H.sc, 0, sizeof(double) * SC_COUNT, st);
    cudaMemsetAsync(H.sc + 6, 0xFF, sizeof(double), st);  // c_min starts at the largest key, as in cmcg_create
    launch_setup_coeffs(H.g, c, bc->dirichlet_mask, dir, 1.0, H.kap64, nullptr, H.mass, H.mask, H.red(), st);
    if (sync_read(&H) != CMCG_OK) return CMCG_ERR_CUDA;
    if (host_sc[3] != 0.0) return CMCG_ERR_INVALID_ARG;
    H.has_dir = host_sc[4] > 0.0;
    uint64_t bits;
    memcpy(&bits, &host_sc[5], sizeof(bits));
    double cmax;
    memcpy(&cmax, &bits, sizeof(cmax));
    if (H.has_dir && H.order == 4) return CMCG_ERR_UNSUPPORTED;
    const double dtt = dt_target > 0 ? dt_target : 0.5 * grid->h / (sqrt((double)grid->dim) * cmax);
    H.N = (int)ceil(H.T / dtt - 1e-9);
    if (H.N < 2) H.N = 2;
    H.dt = H.T / H.N;
    const double rho = (grid->order == 2 ? 4.0 * grid->dim : 16.0 * grid->dim / 3.0) / (grid->h * grid->h);
    if (H.dt * H.dt * cmax * cmax * rho >= 4.0) return CMCG_ERR_CFL;
    cudaMemsetAsync(H.sc, 0, sizeof(double) * SC_COUNT, st);
    launch_setup_coeffs(H.g, c, bc->dirichlet_mask, dir, H.dt, H.kap64, nullptr, H.mass, H.mask, H.red(), st);
    const bool src = f || g;
    const int zce = H.g.dim == 3 ? kZcEnds : 1;
    if (src) launch_make_source(H.g, f, g, H.kap64, H.S, zce, false, st);
    launch_mask_copy(H.g, u0, H.kap64, H.z0, st);
    launch_mask_copy(H.g, v0, H.kap64, H.z1, st);
    forward_period<double>(&H, H.z0, H.z1, src, 1, uT, vT);
    if (cudaStreamSynchronize(st) != cudaSuccess) return CMCG_ERR_CUDA;
    return cuda_status();
}

}  // namespace cmcg

// ======================================================================================
extern "C" {

size_t cmcg_workspace_size(const cmcg_grid* grid, const cmcg_options* opts) {
    if (!valid_grid(grid)) return 0;
    cmcg_options o{};
    if (opts) o = *opts;
    if (o.precision < CMCG_FP64 || o.precision > CMCG_MIXED) return 0;
    cmcg_handle tmp;
    Geom g = make_geom(grid, 0);
    return layout(&tmp, g, o, nullptr);
}

int cmcg_create(const cmcg_grid* grid, const double* c, double omega, const cmcg_bc* bc, const cmcg_options* opts,
                void* workspace, size_t ws_bytes, void* stream, cmcg_handle** out) {
    if (!out) return CMCG_ERR_INVALID_ARG;
    *out = nullptr;
    if (!valid_grid(grid) || !c || !bc || !workspace || !(omega > 0) || !isfinite(omega))
        return CMCG_ERR_INVALID_ARG;
    if (((uintptr_t)workspace & 255u) != 0) return CMCG_ERR_INVALID_ARG;
    cmcg_options o{};
    if (opts) o = *opts;
    if (o.precision < CMCG_FP64 || o.precision > CMCG_MIXED) return CMCG_ERR_INVALID_ARG;
    if (o.flags & ~(CMCG_FLAG_HOST_IO | CMCG_FLAG_TIMING | CMCG_FLAG_INEXACT_RIESZ | CMCG_FLAG_FILTER |
                    CMCG_FLAG_NO_CG | CMCG_FLAG_FIRST_ORDER | CMCG_FLAG_L2_KAPPA))
        return CMCG_ERR_INVALID_ARG;
    if ((o.flags & CMCG_FLAG_NO_CG) && o.runup_periods == 0) return CMCG_ERR_INVALID_ARG;
    if ((o.flags & CMCG_FLAG_FIRST_ORDER) &&
        (grid->order != 2 ||
         (o.flags & (CMCG_FLAG_INEXACT_RIESZ | CMCG_FLAG_NO_CG))))
        return CMCG_ERR_UNSUPPORTED;
    if (o.dt < 0 || !isfinite(o.dt)) return CMCG_ERR_INVALID_ARG;
    fill_defaults(&o);
    unsigned abc = 0, dir = 0;
    for (int f = 0; f < 2 * grid->dim; ++f) {
        const int code = bc->face[f];
        if (code == CMCG_BC_ABC) abc |= 1u << f;
        else if (code == CMCG_BC_DIRICHLET) dir |= 1u << f;
        else if (code != CMCG_BC_NEUMANN) return CMCG_ERR_INVALID_ARG;
    }
    const size_t need = cmcg_workspace_size(grid, &o);
    if (ws_bytes < need) return CMCG_ERR_WORKSPACE;

    cmcg_handle* H = new cmcg_handle();
    H->g = make_geom(grid, abc);
    H->order = grid->order;
    H->opt = o;
    H->st = (cudaStream_t)stream;
    H->omega = omega;
    H->T = 2.0 * kPi / omega;
    // carving must take exactly what sizing promised (a layout that depended on a carved
    // pointer would carve past the caller's workspace)
    if (layout(H, H->g, o, (char*)workspace) != need) {
        delete H;
        return CMCG_ERR_WORKSPACE;
    }
    H->volume = 1.0;
    for (int a = 0; a < grid->dim; ++a) H->volume *= grid->n[a] * grid->h;
    if (cudaMallocHost((void**)&H->hsc, sizeof(double) * SC_COUNT) != cudaSuccess) {
        delete H;
        return CMCG_ERR_CUDA;
    }
    H->timing = (o.flags & CMCG_FLAG_TIMING) != 0;
    H->vec32 = o.precision == CMCG_MIXED && (o.flags & CMCG_FLAG_INEXACT_RIESZ) && !(o.flags & CMCG_FLAG_FIRST_ORDER);
    if (H->timing)
        for (int e = 0; e < 8; ++e) cudaEventCreate(&H->ev[e]);
    auto fail = [&](int code) {
        if (H->timing)
            for (int e = 0; e < 8; ++e) cudaEventDestroy(H->ev[e]);
        cudaFreeHost(H->hsc);
        delete H;
        return code;
    };
    cudaMemsetAsync(H->tickets, 0, sizeof(unsigned) * kNumTickets, H->st);
    cudaMemsetAsync(H->sc, 0, sizeof(double) * SC_COUNT, H->st);
    cudaMemsetAsync(H->sc + 6, 0xFF, sizeof(double), H->st);
    // pass 1 (dt = 1): validity, sums, c_max, c_min
    launch_setup_coeffs(H->g, c, bc->dirichlet_mask, dir, 1.0, H->kap64, H->kap32, H->mass, H->mask, H->red(), H->st);
    if (sync_read(H) != CMCG_OK) return fail(CMCG_ERR_CUDA);
    if (H->hsc[3] != 0.0) return fail(CMCG_ERR_INVALID_ARG);
    H->sumM = H->hsc[0];
    H->sumB = H->hsc[1];
    H->sumW = H->hsc[2];
    H->has_dir = H->hsc[4] > 0.0;
    uint64_t bits;
    memcpy(&bits, &H->hsc[5], sizeof(bits));
    double cmax;
    memcpy(&cmax, &bits, sizeof(cmax));
    memcpy(&bits, &H->hsc[6], sizeof(bits));
    memcpy(&H->cmin, &bits, sizeof(double));
    if (H->has_dir && H->order == 4) return fail(CMCG_ERR_UNSUPPORTED);
    if (H->has_dir && H->sumW <= 0) return fail(CMCG_ERR_INVALID_ARG);
    if (o.runup_periods < -64 || o.runup_periods > 100000) return fail(CMCG_ERR_INVALID_ARG);
    if (o.tile[0] < 0 || o.tile[0] > 512 || o.tile[1] < 0 || o.tile[1] > 512 || o.tile[2] < 0 || o.tile[2] > 60 ||
        o.tile[3] < 0 || o.tile[3] > 6)
        return fail(CMCG_ERR_INVALID_ARG);
    // time step: N = ceil(T / dt_target - 1e-9), dt = T / N
    const double dt_target = o.dt > 0 ? o.dt : 0.5 * grid->h / (sqrt((double)grid->dim) * cmax);
    H->N = (int)ceil(H->T / dt_target - 1e-9);
    if (H->N < 2) H->N = 2;
    H->dt = H->T / H->N;
    const double rho = (grid->order == 2 ? 4.0 * grid->dim : 16.0 * grid->dim / 3.0) / (grid->h * grid->h);
    if (H->dt * H->dt * cmax * cmax * rho >= 4.0) return fail(CMCG_ERR_CFL);
    H->wt = 2.0 / H->dt * sin(omega * H->dt / 2.0);
    H->wh = sin(omega * H->dt) / H->dt;
    // pass 2 with the final dt
    cudaMemsetAsync(H->sc, 0, sizeof(double) * SC_COUNT, H->st);
    launch_setup_coeffs(H->g, c, bc->dirichlet_mask, dir, H->dt, H->kap64, H->kap32, H->mass, H->mask, H->red(),
                        H->st);
    for (int l = 1; l < H->nlev; ++l) launch_mg_coarsen_mask(H->lv[l - 1], H->lv[l], H->st);
    if (!H->has_dir)
        for (int l = 0; l < H->nlev; ++l) H->lv[l].mask = nullptr;
    launch_reciprocal(H->g.np, H->mass, H->minv, H->st);
    if (H->mass32) {
        launch_to_float(H->g.np, H->mass, H->mass32, H->st);
        launch_to_float(H->g.np, H->minv, H->minv32, H->st);
    }
    H->blk_level = -1;
    for (int l = 0; l < H->nlev; ++l)
        if (H->lv[l].g.np <= mg_block_max_nodes()) {
            H->blk_level = l;
            break;
        }
    if (H->blk_level >= 0) {
        H->blk.n = std::min(H->nlev - H->blk_level, kBlockLevelsMax);
        for (int i = 0; i < H->blk.n; ++i) {
            H->blk.g[i] = H->lv[H->blk_level + i].g;
            H->blk.mask[i] = H->lv[H->blk_level + i].mask;
        }
    }
    if (sync_read(H) != CMCG_OK) return fail(CMCG_ERR_CUDA);
    if (o.flags & CMCG_FLAG_L2_KAPPA) l2_kappa_begin(H);
    *out = H;
    return CMCG_OK;
}

int cmcg_destroy(cmcg_handle* h) {
    if (!h) return CMCG_ERR_INVALID_ARG;
    l2_kappa_end(h);
    if (h->timing)
        for (int e = 0; e < 8; ++e) cudaEventDestroy(h->ev[e]);
    cudaFreeHost(h->hsc);
    delete h;
    return CMCG_OK;
}

int cmcg_get_history(const cmcg_handle* h, double* rel_host, int capacity, int* count) {
    if (!h || !count || capacity < 0 || (capacity > 0 && !rel_host)) return CMCG_ERR_INVALID_ARG;
    const int n = (int)std::min<size_t>(h->hist.size(), (size_t)INT32_MAX);
    for (int k = 0; k < n && k < capacity; ++k) rel_host[k] = h->hist[k];
    *count = n;
    return CMCG_OK;
}

int cmcg_get_info(const cmcg_handle* h, cmcg_info* info) {
    if (!h || !info) return CMCG_ERR_INVALID_ARG;
    info->steps_per_period = h->N;
    info->dt = h->dt;
    info->omega_tilde = h->wt;
    info->omega_hat = h->wh;
    info->num_nodes = h->g.np;
    info->mg_levels = h->nlev;
    info->has_dirichlet = h->has_dir ? 1 : 0;
    return CMCG_OK;
}

int cmcg_wave_period(cmcg_handle* h, const double* u0, const double* v0, const double* f, const double* g,
                     double* uT, double* vT) {
    if (!h || !u0 || !v0 || !uT || !vT) return CMCG_ERR_INVALID_ARG;
    if (h->first_order) return CMCG_ERR_UNSUPPORTED;
    const bool src = f || g;
    if (src) launch_make_source(h->g, f, g, h->kap64, h->S, h->g.dim == 3 ? kZcEnds : 1, false, h->st);
    if (src) source_updated(h);
    launch_mask_copy(h->g, u0, h->kap64, h->z0, h->st);
    launch_mask_copy(h->g, v0, h->kap64, h->z1, h->st);
    if (h->opt.precision == CMCG_FP32)
        forward_period<float>(h, h->z0, h->z1, src, 1, uT, vT);
    else
        forward_period<double>(h, h->z0, h->z1, src, 1, uT, vT);
    if (cudaStreamSynchronize(h->st) != cudaSuccess) return CMCG_ERR_CUDA;
    return cuda_status();
}

int cmcg_adjoint_period(cmcg_handle* h, const double* a, const double* b, double* q0, double* q1) {
    if (!h || !a || !b || !q0 || !q1) return CMCG_ERR_INVALID_ARG;
    if (h->first_order) return CMCG_ERR_UNSUPPORTED;
    launch_mask_copy(h->g, a, h->kap64, h->z0, h->st);
    launch_mask_copy(h->g, b, h->kap64, h->z1, h->st);
    if (h->opt.precision == CMCG_FP32)
        adjoint_period<float>(h, h->z0, h->z1, 1, nullptr, nullptr, q0, q1, nullptr);
    else
        adjoint_period<double>(h, h->z0, h->z1, 1, nullptr, nullptr, q0, q1, nullptr);
    if (cudaStreamSynchronize(h->st) != cudaSuccess) return CMCG_ERR_CUDA;
    return cuda_status();
}

int cmcg_riesz(cmcg_handle* h, const double* rhs, double* s) {
    if (!h || !rhs || !s) return CMCG_ERR_INVALID_ARG;
    if (h->first_order) return CMCG_ERR_UNSUPPORTED;
    int rc = riesz_solve(h, rhs, s, nullptr);
    if (cudaStreamSynchronize(h->st) != cudaSuccess) return CMCG_ERR_CUDA;
    return rc;
}

int cmcg_bulk_wait_selftest(int spin_limit, void* stream) {
    if (spin_limit < 1) return CMCG_ERR_INVALID_ARG;
    return bulk_wait_selftest(spin_limit, (cudaStream_t)stream);
}

int cmcg_check_status(long long* count, long long* site, long long* index) {
    if (cudaDeviceSynchronize() != cudaSuccess) return CMCG_ERR_CUDA;
    long long total = 0, first_site = -1, first_index = 0;
    for (auto read : {check_read_wave, check_read_riesz, check_read_pair}) {
        long long w[3];
        read(w);
        if (w[0] > 0 && first_site < 0) {
            first_site = w[1];
            first_index = w[2];
        }
        total += w[0];
    }
    if (count) *count = total;
    if (site) *site = first_site;
    if (index) *index = first_index;
    if (cudaGetLastError() != cudaSuccess) return CMCG_ERR_CUDA;
#ifdef CMCG_CHECKED
    return CMCG_OK;
#else
    return CMCG_ERR_UNSUPPORTED;
#endif
}

int cmcg_fo_period(cmcg_handle* h, const double* s0, const double* f, const double* g, double* sT) {
    if (!h || !s0 || !sT) return CMCG_ERR_INVALID_ARG;
    if (!h->first_order) return CMCG_ERR_UNSUPPORTED;
    const bool src = f || g;
    if (src) launch_make_source(h->g, f, g, h->kap64, h->S, h->g.dim == 3 ? kZcEnds : 1, false, h->st);
    if (src) source_updated(h);
    if (fo_period(h, s0, src, sT) != CMCG_OK) return CMCG_ERR_CUDA;
    if (cudaStreamSynchronize(h->st) != cudaSuccess) return CMCG_ERR_CUDA;
    return cuda_status();
}

int cmcg_fo_adjoint_period(cmcg_handle* h, const double* y, double* out) {
    if (!h || !y || !out) return CMCG_ERR_INVALID_ARG;
    if (!h->first_order) return CMCG_ERR_UNSUPPORTED;
    if (fo_adjoint(h, y, out) != CMCG_OK) return CMCG_ERR_CUDA;
    if (cudaStreamSynchronize(h->st) != cudaSuccess) return CMCG_ERR_CUDA;
    return cuda_status();
}

int cmcg_solve(cmcg_handle* h, const double* f, const double* g, double tol, double* u, cmcg_stats* stats) {
    if (!h || !u || !(tol > 0)) return CMCG_ERR_INVALID_ARG;
    const auto t0 = std::chrono::steady_clock::now();
    if (f || g)
        launch_make_source(h->g, f, g, h->kap64, h->S, h->g.dim == 3 ? kZcEnds : 1, false, h->st);
    else
        launch_fill(h->S, 2 * h->g.np, 0.0, h->st);
    source_updated(h);
    cmcg_stats local{};
    cmcg_stats* st = stats ? stats : &local;
    const int rc = solve_prepared(h, tol, u, st, stats != nullptr);
    st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return rc;
}

int cmcg_solve_warm(cmcg_handle* h, const double* f, const double* g, double tol, double* u, cmcg_stats* stats) {
    if (!h || !u || !(tol > 0)) return CMCG_ERR_INVALID_ARG;
    if (h->first_order || (h->opt.flags & CMCG_FLAG_NO_CG)) return CMCG_ERR_UNSUPPORTED;
    h->warm = u;  // read by the first gradient's set-up, before u is written
    const int rc = cmcg_solve(h, f, g, tol, u, stats);
    h->warm = nullptr;
    return rc;
}

int cmcg_solve_host(cmcg_handle* h, const double* f_host, const double* g_host, double tol, double* u_host,
                    cmcg_stats* stats) {
    if (!h || !u_host || !h->stage || !(tol > 0)) return CMCG_ERR_INVALID_ARG;
    const auto t0 = std::chrono::steady_clock::now();
    const long long n = h->g.np;
    const size_t bytes = sizeof(double) * 2 * (size_t)n;
    const int zce = h->g.dim == 3 ? kZcEnds : 1;
    // S = kappa h^2 (f + (2 nb / h) g), built through the one staging buffer
    launch_fill(h->S, 2 * n, 0.0, h->st);
    if (f_host) {
        cudaMemcpyAsync(h->stage, f_host, bytes, cudaMemcpyHostToDevice, h->st);
        launch_make_source(h->g, h->stage, nullptr, h->kap64, h->S, zce, true, h->st);
    }
    if (g_host) {
        cudaMemcpyAsync(h->stage, g_host, bytes, cudaMemcpyHostToDevice, h->st);
        launch_make_source(h->g, nullptr, h->stage, h->kap64, h->S, zce, true, h->st);
    }
    source_updated(h);
    if (cuda_status() != CMCG_OK) return CMCG_ERR_CUDA;
    cmcg_stats local{};
    cmcg_stats* st = stats ? stats : &local;
    const int rc = solve_prepared(h, tol, h->stage, st, stats != nullptr);
    if (rc < 0) return rc;
    cudaMemcpyAsync(u_host, h->stage, bytes, cudaMemcpyDeviceToHost, h->st);
    if (cudaStreamSynchronize(h->st) != cudaSuccess) return CMCG_ERR_CUDA;
    st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return rc;
}

const char* cmcg_status_string(int s) {
    switch (s) {
        case CMCG_OK: return "ok";
        case CMCG_NOT_CONVERGED: return "not converged";
        case CMCG_ERR_INVALID_ARG: return "invalid argument";
        case CMCG_ERR_CFL: return "CFL condition violated";
        case CMCG_ERR_WORKSPACE: return "workspace too small";
        case CMCG_ERR_UNSUPPORTED: return "unsupported combination";
        case CMCG_ERR_CUDA: return "CUDA error";
        case CMCG_ERR_DIVERGED: return "diverged (non-finite or non-positive CG scalar)";
        case CMCG_ERR_DEVICE_TIMEOUT: return "device-side wait timed out";
        default: return "unknown status";
    }
}

}  // extern "C"
