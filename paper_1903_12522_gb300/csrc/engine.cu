// Multi-solve engine: many CMCG solves (different grids, frequencies, sources) advance
// together, one CG iteration per tick.
//
// Each admitted solve sits in a slot with its own handle (workspace, resident CG state).  A
// tick enqueues, for every active slot, its next unit of work:
//   - OUTER (CMCG_MIXED): W += w; FP64 gradient of J at W with the sources; z = B rhat; w = 0;
//     d = z  (the defect-correction residual, Sec. 2.3 steps (2)-(4) in FP64);
//   - INIT  (CMCG_FP32): w = 0; FP32 gradient with the sources; z = B rhat; d = z;
//   - INNER: one flexible-CG iteration with FP32 periods (Steps 5.1-5.7).
// The FP32 leapfrog step loops of all INNER slots run in ONE batched persistent kernel per
// period (forward, then adjoint); everything else is per-slot launches.  The tick is captured
// as a CUDA graph and replayed while the set of (slot, unit, submission number) triples stays
// the same; releasing a slot drops a cached graph that includes it.  After each tick the host
// reads every slot's convergence word and moves slots between units; a finished slot gets its
// recovery (Step (6)) and is released.
#include <string.h>

#include <algorithm>
#include <chrono>
#include <vector>

#include "cmcg.h"
#include "engine_sig.h"
#include "solver.h"

using namespace cmcg;
using namespace cmcg::detail;

namespace {

// U_RUNUP: the initial run-up (Sec. 4.2.3) of a mixed-precision slot, between its first outer
// unit (the zero guess, which sets the tolerance reference) and its second.
enum Unit { U_FREE = 0, U_INIT32, U_OUTER, U_INNER, U_DONE, U_RUNUP };

struct EngineSlot {
    cmcg_handle* h = nullptr;
    long long submission = 0;  // the engine's submission number of this solve (never reused)
    double* u = nullptr;
    double tol = 0;
    int unit = U_FREE;
    int status = CMCG_OK;
    int iters = 0, inner_iters = 0, outer = 0;
    long long periods = 0, riesz = 0;  // counted per tick (graph replays skip the launch-time counters)
    double gamma_ref = -1, rel = 1, inner_tol = 1e-3;
    int runup = 0;  // run-up periods still to run (mixed precision only)
    long long launches0 = 0;
    std::chrono::steady_clock::time_point t0;
    cmcg_stats st{};
};

}  // namespace

struct cmcg_engine {
    cudaStream_t st = nullptr;
    int max_slots = 0;
    std::vector<EngineSlot> slots;
    // device
    BatchItem* items_dev = nullptr;  // [3 * max_slots]: forward, adjoint, then run-up items
    unsigned* bar = nullptr;         // barrier counter + generation
    int* err = nullptr;              // barrier time-out flag
    int* err_host = nullptr;         // pinned
    int grid = 0;      // blocks of the batched step kernel (at most the co-resident maximum)
    int grid_max = 0;  // co-resident maximum
    int grid_forced = 0;  // blocks of the batched run-up kernel (its co-resident maximum)
    int zc3 = kZcStep3D;  // z-planes per work item of 3D grids in the batched kernel
    bool use_graph = true;
    // graph cache
    cudaGraphExec_t exec = nullptr;
    TickSignature signature;       // configuration of the cached graph
    TickSignature last_signature;  // configuration of the previous tick
    long long submissions = 0;     // solves submitted so far (the last submission number)
    long long graph_launches = 0;
    long long ticks = 0, graph_builds = 0;
    cudaError_t last_error = cudaSuccess;  // the CUDA error behind the last CMCG_ERR_CUDA
    // side streams: per-solve kernels of different solves run concurrently between the batched
    // launches (fork/join by events; under capture these become parallel graph branches)
    static constexpr int kSide = 8;
    cudaStream_t side[kSide] = {};
    cudaEvent_t fork = nullptr, join[kSide] = {};
};

namespace {

size_t engine_layout(cmcg_engine* e, int max_slots, char* base) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        off = (off + 255) & ~(size_t)255;
        char* p = base ? base + off : nullptr;
        off += bytes;
        return p;
    };
    char* items = take(sizeof(BatchItem) * 3 * (size_t)max_slots);
    char* bar = take(sizeof(unsigned) * 4);
    char* err = take(sizeof(int) * 4);
    if (e) {
        e->items_dev = (BatchItem*)items;
        e->bar = (unsigned*)bar;
        e->err = (int*)err;
    }
    return off + 256;
}

BatchItem make_item(cmcg_handle* h, const PeriodBuffers& b, bool adjoint, int zc3) {
    BatchItem it{};
    it.g = h->g;
    it.kap = h->kap32;
    it.buf0 = (float*)b.cur;
    it.buf1 = (float*)b.prev;
    it.order = h->order;
    it.nsteps = h->N - 1;
    it.adjoint = adjoint ? 1 : 0;
    it.zc = h->g.dim == 3 ? zc3 : 1;
    const long long plane = (long long)h->g.sx * h->g.sy;
    it.blocks_xy = (int)((plane + 255) / 256);
    it.vec4 = h->g.dim == 2 && h->order == 2 && step_vec4_ok(h->g, it.buf0, it.buf1, it.kap);
    if (it.vec4) it.blocks_xy = (int)((((h->g.np + 3) >> 2) + 255) / 256);
    it.blocks = it.blocks_xy * ((h->g.sz + it.zc - 1) / it.zc);
    return it;
}

// The run-up of a slot as one item of the batched run-up kernel: the forced ramped steps
// n = 1 .. periods N - 1 from rest (step n = s + 1 of the item), y^1 in yb and y^0 in ya at
// the first step, as in the one-solve run-up.
BatchItem make_runup_item(cmcg_handle* h, int periods, int zc3) {
    PeriodBuffers b{h->yb, h->ya, nullptr};
    BatchItem it = make_item(h, b, false, zc3);
    it.nsteps = (int)((long long)periods * h->N - 1);
    it.S = h->S32;
    it.scol = h->scol;
    it.steps_per_period = h->N;
    it.runup_steps = periods * h->N;
    return it;
}

PeriodBuffers after_steps(PeriodBuffers b, int nsteps) {
    if (nsteps & 1) std::swap(b.cur, b.prev);
    return b;
}

// The per-slot prologue of a unit that ends with "z = B rhat, d = z" (OUTER, INIT32).  On a
// handle with FP32 CG vectors (mixed precision) the inner vectors start as floats; gamma0, the
// outer residual, is then reduced in FP32 from float(rhat) (rhat is the current residual, so
// its rounding is relative to its own size).
void reset_direction(cmcg_handle* h) {
    const long long n = h->g.np;
    if (h->vec32) {
        begin_vec32_inner(h);
        h->vec32_active = false;
        return;
    }
    cudaMemcpyAsync(h->rh0, h->gh0, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->st);
    cudaMemcpyAsync(h->rh1, h->gh1, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->st);
    apply_B(h, true, false);
    cudaMemcpyAsync(h->d0, h->r0, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->st);
    cudaMemcpyAsync(h->d1, h->r1, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->st);
}

void fork_sides(cmcg_engine* e) {
    cudaEventRecord(e->fork, e->st);
    for (int k = 0; k < cmcg_engine::kSide; ++k) cudaStreamWaitEvent(e->side[k], e->fork, 0);
}

void join_sides(cmcg_engine* e) {
    for (int k = 0; k < cmcg_engine::kSide; ++k) {
        cudaEventRecord(e->join[k], e->side[k]);
        cudaStreamWaitEvent(e->st, e->join[k], 0);
    }
}

// Run f(h) with the handle's launches on side stream k (the handle's own stream is restored).
template <typename F>
void on_side(cmcg_engine* e, cmcg_handle* h, int k, F f) {
    cudaStream_t own = h->st;
    h->st = e->side[k % cmcg_engine::kSide];
    f(h);
    h->st = own;
}

// Enqueue one tick on the engine's stream (also used while capturing).
cudaError_t enqueue_tick(cmcg_engine* e, const std::vector<int>& act) {
    cudaMemsetAsync(e->err, 0, sizeof(int), e->st);
    fork_sides(e);
    std::vector<int> inner, runups;
    int lane = 0;
    for (int s : act) {
        EngineSlot& sl = e->slots[s];
        if (sl.unit == U_OUTER) {
            on_side(e, sl.h, lane++, [](cmcg_handle* h) {
                const long long n = h->g.np;
                add_correction(h, h->wo0, h->wo1);
                gradient<double>(h, h->wo0, h->wo1, true, h->wo0, h->wo1, false);
                launch_fill(h->w0, n, 0.0, h->st);
                launch_fill(h->w1, n, 0.0, h->st);
                reset_direction(h);
            });
        } else if (sl.unit == U_INIT32) {
            on_side(e, sl.h, lane++, [](cmcg_handle* h) {
                const long long n = h->g.np;
                launch_fill(h->w0, n, 0.0, h->st);
                launch_fill(h->w1, n, 0.0, h->st);
                gradient<float>(h, h->w0, h->w1, true, h->w0, h->w1, false);
                reset_direction(h);
            });
        } else if (sl.unit == U_RUNUP) {
            runups.push_back(s);
            on_side(e, sl.h, lane++, [](cmcg_handle* h) { runup_start_f32(h); });
        } else if (sl.unit == U_INNER) {
            inner.push_back(s);
        }
    }
    if (!runups.empty()) {
        // every run-up slot's forced steps in one cooperative launch (items uploaded before the
        // tick), then each slot's end state into its FP64 iterate
        const int r = (int)runups.size();
        int total = 0, maxs = 0;
        for (int s : runups) {
            const BatchItem it = make_runup_item(e->slots[s].h, e->slots[s].runup, e->zc3);
            total += it.blocks;
            maxs = std::max(maxs, it.nsteps);
        }
        join_sides(e);
        cudaError_t ce = launch_batch_steps(e->items_dev + 2 * e->max_slots, r, total, maxs, e->bar, e->err,
                                            e->grid_forced, e->st, true);
        if (ce != cudaSuccess) return ce;
        fork_sides(e);
        for (int i = 0; i < r; ++i) {
            const int periods = e->slots[runups[i]].runup;
            on_side(e, e->slots[runups[i]].h, lane + i,
                    [periods](cmcg_handle* h) { runup_finish_f32(h, periods, h->wo0, h->wo1); });
        }
        lane += r;
    }
    if (!inner.empty()) {
        const int m = (int)inner.size();
        std::vector<PeriodBuffers> fb(m), ab(m);
        // forward periods from d: start kernels, one batched step loop, end kernels
        int total = 0, maxs = 0;
        std::vector<BatchItem> items(2 * (size_t)m);
        for (int i = 0; i < m; ++i) {
            cmcg_handle* h = e->slots[inner[i]].h;
            on_side(e, h, lane + i, [&](cmcg_handle* hh) {
                hh->vec32_active = hh->vec32;
                fb[i] = fwd_begin<float>(hh, hh->d0, hh->d1, false);
                hh->vec32_active = false;
            });
            items[i] = make_item(h, fb[i], false, e->zc3);
            items[i].offset = total;
            total += items[i].blocks;
            maxs = std::max(maxs, items[i].nsteps);
        }
        join_sides(e);  // the cooperative kernel runs alone: all its blocks are co-resident
        cudaError_t ce = launch_batch_steps(e->items_dev, m, total, maxs, e->bar, e->err, e->grid, e->st);
        if (ce != cudaSuccess) return ce;
        fork_sides(e);
        int total_a = 0, maxa = 0;
        for (int i = 0; i < m; ++i) {
            cmcg_handle* h = e->slots[inner[i]].h;
            on_side(e, h, lane + i, [&](cmcg_handle* hh) {
                hh->vec32_active = hh->vec32;
                fwd_end<float>(hh, after_steps(fb[i], hh->N - 1), hh->d1, false, 0, hh->z0, hh->z1);
                ab[i] = adj_begin<float>(hh, hh->z0, hh->z1, 0);
                hh->vec32_active = false;
            });
            items[m + i] = make_item(h, ab[i], true, e->zc3);
            items[m + i].offset = total_a;
            total_a += items[m + i].blocks;
            maxa = std::max(maxa, items[m + i].nsteps);
        }
        join_sides(e);
        ce = launch_batch_steps(e->items_dev + e->max_slots, m, total_a, maxa, e->bar, e->err, e->grid, e->st);
        if (ce != cudaSuccess) return ce;
        fork_sides(e);
        for (int i = 0; i < m; ++i) {
            cmcg_handle* h = e->slots[inner[i]].h;
            on_side(e, h, lane + i, [&](cmcg_handle* hh) {
                const long long n = hh->g.np;
                hh->vec32_active = hh->vec32;
                adj_end<float>(hh, after_steps(ab[i], hh->N - 1), hh->z0, hh->z1, 0, hh->d0, hh->d1, hh->gh0, hh->gh1,
                               nullptr);
                launch_fcg_update(n, hh->w0, hh->w1, hh->rh0, hh->rh1, hh->d0, hh->d1, hh->gh0, hh->gh1, hh->red(),
                                  hh->st, hh->lv[0].b, hh->vec32);
                apply_B(hh, false, true, true);
                launch_cg_direction(n, hh->r0, hh->r1, hh->d0, hh->d1, hh->red(), hh->st, nullptr, hh->vec32);
                hh->vec32_active = false;
            });
        }
        // the descriptors are uploaded before the tick (upload_items)
    }
    join_sides(e);
    for (int s : act) {
        cmcg_handle* h = e->slots[s].h;
        cudaMemcpyAsync(h->hsc, h->sc, sizeof(double) * SC_COUNT, cudaMemcpyDeviceToHost, e->st);
    }
    cudaMemcpyAsync(e->err_host, e->err, sizeof(int), cudaMemcpyDeviceToHost, e->st);
    return cudaGetLastError();
}

// Batch descriptors of the INNER slots (forward and adjoint) and of the RUNUP slots: the
// buffer roles at step 0 are fixed per handle (fwd and run-up: cur = yb, prev = ya; adjoint:
// cur = ya, prev = yb), so they can be uploaded before the tick and stay valid across graph
// replays.
void upload_items(cmcg_engine* e, const std::vector<int>& act) {
    std::vector<BatchItem> items(3 * (size_t)e->max_slots);
    int m = 0, tf = 0, ta = 0, r = 0, tr = 0;
    for (int s : act) {
        EngineSlot& sl = e->slots[s];
        if (sl.unit == U_RUNUP) {
            BatchItem& it = items[2 * (size_t)e->max_slots + r++];
            it = make_runup_item(sl.h, sl.runup, e->zc3);
            it.offset = tr;
            tr += it.blocks;
            continue;
        }
        if (sl.unit != U_INNER) continue;
        cmcg_handle* h = sl.h;
        PeriodBuffers f{h->yb, h->ya, nullptr}, a{h->ya, h->yb, nullptr};
        items[m] = make_item(h, f, false, e->zc3);
        items[m].offset = tf;
        tf += items[m].blocks;
        items[e->max_slots + m] = make_item(h, a, true, e->zc3);
        items[e->max_slots + m].offset = ta;
        ta += items[e->max_slots + m].blocks;
        ++m;
    }
    cudaMemcpyAsync(e->items_dev, items.data(), sizeof(BatchItem) * 3 * (size_t)e->max_slots, cudaMemcpyHostToDevice,
                    e->st);
    cudaStreamSynchronize(e->st);
}

// Drop the cached graph if it includes slot s: the graph holds that solve's device pointers
// and its pinned status mirror, which the caller may free once the slot is released.
void drop_graph_of_slot(cmcg_engine* e, int s) {
    if (e->exec && e->signature.names_slot(s)) {
        cudaGraphExecDestroy(e->exec);
        e->exec = nullptr;
        e->signature.clear();
    }
    if (e->last_signature.names_slot(s)) e->last_signature.clear();
}

int finish_slot(cmcg_engine* e, int s) {
    EngineSlot& sl = e->slots[s];
    cmcg_handle* h = sl.h;
    const long long n = h->g.np;
    if (h->opt.precision == CMCG_MIXED) {
        cudaMemcpyAsync(h->w0, h->wo0, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->st);
        cudaMemcpyAsync(h->w1, h->wo1, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->st);
    }
    if (recover(h, sl.u, &sl.st) != CMCG_OK) return CMCG_ERR_CUDA;
    sl.st.iterations = sl.iters;
    sl.st.outer_iterations = sl.outer;
    sl.st.rel_residual = sl.rel;
    sl.st.steps_per_period = h->N;
    sl.st.dt = h->dt;
    sl.st.omega_tilde = h->wt;
    sl.st.omega_hat = h->wh;
    sl.st.periods = (int)sl.periods;
    sl.st.riesz_iterations = (int)sl.riesz;
    sl.st.point_updates = sl.periods * (long long)h->N * n;
    sl.st.kernel_launches = launch_count() - sl.launches0;
    sl.st.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - sl.t0).count();
    sl.unit = U_DONE;
    return CMCG_OK;
}

}  // namespace

extern "C" {

size_t cmcg_engine_workspace_size(int max_slots) {
    if (max_slots <= 0 || max_slots > 4096) return 0;
    return engine_layout(nullptr, max_slots, nullptr);
}

int cmcg_engine_create(int max_slots, void* workspace, size_t ws_bytes, void* stream, int flags,
                       cmcg_engine** out) {
    if (!out || max_slots <= 0 || max_slots > 4096 || !workspace) return CMCG_ERR_INVALID_ARG;
    if (((uintptr_t)workspace & 255u) != 0 || (flags & ~CMCG_ENGINE_NO_GRAPH)) return CMCG_ERR_INVALID_ARG;
    *out = nullptr;
    if (ws_bytes < cmcg_engine_workspace_size(max_slots)) return CMCG_ERR_WORKSPACE;
    cmcg_engine* e = new cmcg_engine();
    e->st = (cudaStream_t)stream;
    e->max_slots = max_slots;
    e->slots.resize(max_slots);
    // stream capture needs a created stream: on the legacy default stream run plain launches
    e->use_graph = (flags & CMCG_ENGINE_NO_GRAPH) == 0 && stream != nullptr;
    engine_layout(e, max_slots, (char*)workspace);
    if (cudaMallocHost((void**)&e->err_host, sizeof(int)) != cudaSuccess) {
        delete e;
        return CMCG_ERR_CUDA;
    }
    cudaMemsetAsync(e->bar, 0, sizeof(unsigned) * 4, e->st);
    cudaMemsetAsync(e->err, 0, sizeof(int) * 4, e->st);
    e->grid = e->grid_max = batch_steps_max_blocks(false);
    e->grid_forced = batch_steps_max_blocks(true);
    bool ok = cudaEventCreateWithFlags(&e->fork, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; k < cmcg_engine::kSide; ++k) {
        ok = ok && cudaStreamCreateWithFlags(&e->side[k], cudaStreamNonBlocking) == cudaSuccess;
        ok = ok && cudaEventCreateWithFlags(&e->join[k], cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok || cudaStreamSynchronize(e->st) != cudaSuccess || e->grid <= 0 || e->grid_forced <= 0) {
        for (int k = 0; k < cmcg_engine::kSide; ++k) {
            if (e->side[k]) cudaStreamDestroy(e->side[k]);
            if (e->join[k]) cudaEventDestroy(e->join[k]);
        }
        if (e->fork) cudaEventDestroy(e->fork);
        cudaFreeHost(e->err_host);
        delete e;
        return CMCG_ERR_CUDA;
    }
    *out = e;
    return CMCG_OK;
}

int cmcg_engine_set_shape(cmcg_engine* e, int blocks_per_sm, int z_planes) {
    if (!e || blocks_per_sm < 0 || z_planes < 0 || z_planes > 256) return CMCG_ERR_INVALID_ARG;
    for (const EngineSlot& sl : e->slots)
        if (sl.unit != U_FREE && sl.unit != U_DONE) return CMCG_ERR_INVALID_ARG;  // only while idle
    int sms = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        return CMCG_ERR_CUDA;
    e->grid = blocks_per_sm == 0 ? e->grid_max : std::min(e->grid_max, blocks_per_sm * sms);
    e->zc3 = z_planes == 0 ? kZcStep3D : z_planes;
    if (e->exec) {
        cudaGraphExecDestroy(e->exec);
        e->exec = nullptr;
    }
    e->signature.clear();
    e->last_signature.clear();
    return CMCG_OK;
}

int cmcg_engine_destroy(cmcg_engine* e) {
    if (!e) return CMCG_ERR_INVALID_ARG;
    if (e->exec) cudaGraphExecDestroy(e->exec);
    cudaStreamSynchronize(e->st);
    for (int k = 0; k < cmcg_engine::kSide; ++k) {
        cudaStreamSynchronize(e->side[k]);
        cudaStreamDestroy(e->side[k]);
        cudaEventDestroy(e->join[k]);
    }
    cudaEventDestroy(e->fork);
    cudaFreeHost(e->err_host);
    delete e;
    return CMCG_OK;
}

int cmcg_engine_submit(cmcg_engine* e, cmcg_handle* h, const double* f, const double* g, double tol, double* u) {
    if (!e || !h || !u || !(tol > 0)) return CMCG_ERR_INVALID_ARG;
    if (h->st != e->st || h->opt.precision == CMCG_FP64 || !(h->opt.flags & CMCG_FLAG_INEXACT_RIESZ) ||
        (h->opt.flags & (CMCG_FLAG_FILTER | CMCG_FLAG_NO_CG | CMCG_FLAG_FIRST_ORDER)))
        return CMCG_ERR_UNSUPPORTED;
    if (h->opt.precision != CMCG_MIXED && runup_count(h) > 0) return CMCG_ERR_UNSUPPORTED;
    int s = -1;
    for (int i = 0; i < e->max_slots; ++i) {
        if (e->slots[i].h == h && e->slots[i].unit != U_FREE) return CMCG_ERR_INVALID_ARG;  // handle busy
        if (s < 0 && e->slots[i].unit == U_FREE) s = i;
    }
    if (s < 0) return CMCG_ERR_WORKSPACE;  // no free slot
    drop_graph_of_slot(e, s);
    EngineSlot& sl = e->slots[s];
    sl = EngineSlot();
    sl.h = h;
    sl.submission = ++e->submissions;
    sl.u = u;
    sl.tol = tol;
    sl.t0 = std::chrono::steady_clock::now();
    sl.launches0 = launch_count();
    sl.runup = h->opt.precision == CMCG_MIXED ? runup_count(h) : 0;
    h->riesz_iters = 0;
    h->periods = 0;
    if (f || g)
        launch_make_source(h->g, f, g, h->kap64, h->S, h->g.dim == 3 ? kZcEnds : 1, false, h->st);
    else
        launch_fill(h->S, 2 * h->g.np, 0.0, h->st);
    source_updated(h);
    if (h->opt.precision == CMCG_MIXED) {
        launch_fill(h->wo0, h->g.np, 0.0, h->st);
        launch_fill(h->wo1, h->g.np, 0.0, h->st);
        launch_fill(h->w0, h->g.np, 0.0, h->st);
        launch_fill(h->w1, h->g.np, 0.0, h->st);
        sl.unit = U_OUTER;
    } else {
        sl.unit = U_INIT32;
    }
    if (cudaGetLastError() != cudaSuccess) return CMCG_ERR_CUDA;
    return s;
}

int cmcg_engine_tick(cmcg_engine* e, int* finished, int max_finished, int* n_finished) {
    cmcg::Range range("cmcg engine tick");
    if (!e || !n_finished || (max_finished > 0 && !finished)) return CMCG_ERR_INVALID_ARG;
    *n_finished = 0;
    std::vector<int> act;
    for (int i = 0; i < e->max_slots; ++i) {
        const int u = e->slots[i].unit;
        if (u == U_INIT32 || u == U_OUTER || u == U_INNER || u == U_RUNUP) act.push_back(i);
    }
    if (act.empty()) return CMCG_OK;
    // configuration signature: (slot, unit, submission number) of every active slot
    TickSignature sig;
    for (int s : act) sig.add(s, e->slots[s].unit, e->slots[s].submission);
    // the batch descriptors follow the configuration of every tick (a cached graph reads them)
    const bool changed = sig != e->last_signature;
    if (changed) upload_items(e, act);
    e->last_signature = sig;
    const bool same = e->exec != nullptr && sig == e->signature;
    // capture a configuration only once it has held for two ticks: a solve that changes unit
    // every few ticks would otherwise pay a graph build each time
    if (e->use_graph && (same || !changed)) {
        if (!same) {
            if (e->exec) {
                cudaGraphExecDestroy(e->exec);
                e->exec = nullptr;
            }
            cudaGraph_t graph = nullptr;
            cudaError_t ce0 = cudaStreamBeginCapture(e->st, cudaStreamCaptureModeThreadLocal);
            if (ce0 != cudaSuccess) {
                e->last_error = ce0;
                return CMCG_ERR_CUDA;
            }
            const long long before = launch_count();
            const cudaError_t ce = enqueue_tick(e, act);
            const cudaError_t ce2 = cudaStreamEndCapture(e->st, &graph);
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            if (cudaStreamIsCapturing(e->st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
                cudaGraph_t g2 = nullptr;
                cudaStreamEndCapture(e->st, &g2);  // never leave the stream capturing
                if (g2) cudaGraphDestroy(g2);
            }
            if (ce != cudaSuccess || ce2 != cudaSuccess || !graph) {
                e->last_error = ce != cudaSuccess ? ce : (ce2 != cudaSuccess ? ce2 : cudaErrorUnknown);
                if (graph) cudaGraphDestroy(graph);
                cudaGetLastError();
                return CMCG_ERR_CUDA;
            }
            const cudaError_t ce3 = cudaGraphInstantiate(&e->exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ce3 != cudaSuccess) {
                e->last_error = ce3;
                e->exec = nullptr;
                return CMCG_ERR_CUDA;
            }
            e->signature = sig;
            e->graph_launches = launch_count() - before;  // kernels one replay runs
            e->graph_builds += 1;
        } else {
            note_launch(e->graph_launches);
        }
        const cudaError_t ce = cudaGraphLaunch(e->exec, e->st);
        if (ce != cudaSuccess) {
            e->last_error = ce;
            return CMCG_ERR_CUDA;
        }
    } else {
        const cudaError_t ce = enqueue_tick(e, act);
        if (ce != cudaSuccess) {
            e->last_error = ce;
            return CMCG_ERR_CUDA;
        }
    }
    const cudaError_t cs = cudaStreamSynchronize(e->st);
    if (cs != cudaSuccess) {
        e->last_error = cs;
        return CMCG_ERR_CUDA;
    }
    e->ticks += 1;
    const bool timeout = *e->err_host != 0;
    for (int s : act) {
        EngineSlot& sl = e->slots[s];
        cmcg_handle* h = sl.h;
        const double* sc = h->hsc;
        bool done = false;
        if (sl.unit == U_RUNUP) {  // the run-up state is the next outer unit's iterate
            sl.periods += sl.runup;
            sl.st.runup_periods = sl.runup;
            sl.runup = 0;
            sl.unit = U_OUTER;
            continue;
        }
        sl.periods += 2;  // every other unit runs one forward and one adjoint period
        sl.riesz += 1;    // and one approximate Riesz map
        if (timeout && sl.unit == U_INNER) {
            sl.status = CMCG_ERR_DEVICE_TIMEOUT;
            done = true;
        } else if (sc[SC_STATUS] != 0.0) {
            sl.status = CMCG_ERR_DIVERGED;
            done = true;
        } else if (sl.unit == U_OUTER) {
            const double gam = sc[SC_GAMMA0];
            if (sl.outer == 0) {
                sl.gamma_ref = gam;
                sl.st.J0 = sc[SC_J];
            }
            sl.outer += 1;
            sl.rel = sl.gamma_ref > 0 ? sqrt(std::max(gam, 0.0) / sl.gamma_ref) : 0.0;
            if (sl.rel <= sl.tol) {
                sl.status = CMCG_OK;
                done = true;
            } else if (sl.runup > 0) {
                sl.unit = U_RUNUP;  // the zero guess set the reference; now the run-up
            } else if (sl.iters >= h->opt.max_iter || sl.outer > 50) {
                sl.status = CMCG_NOT_CONVERGED;
                done = true;
            } else {
                sl.inner_tol = std::min(0.5, std::max(h->opt.inner_tol, 0.5 * sl.tol / sl.rel));
                sl.inner_iters = 0;
                sl.unit = U_INNER;
            }
        } else if (sl.unit == U_INIT32) {
            sl.st.J0 = sc[SC_J];
            sl.rel = sc[SC_REL];
            if (sl.rel <= sl.tol) {
                sl.status = CMCG_OK;
                done = true;
            } else {
                sl.unit = U_INNER;
            }
        } else {  // U_INNER
            sl.iters += 1;
            sl.inner_iters += 1;
            const double r = sc[SC_REL];
            if (h->opt.precision == CMCG_MIXED) {
                if (r <= sl.inner_tol || sl.iters >= h->opt.max_iter) sl.unit = U_OUTER;
            } else {
                sl.rel = r;
                if (r <= sl.tol) {
                    sl.status = CMCG_OK;
                    done = true;
                } else if (sl.iters >= h->opt.max_iter) {
                    sl.status = CMCG_NOT_CONVERGED;
                    done = true;
                }
            }
        }
        if (done) {
            if (sl.status >= 0 && finish_slot(e, s) != CMCG_OK) sl.status = CMCG_ERR_CUDA;
            sl.unit = U_DONE;
            if (*n_finished < max_finished) finished[*n_finished] = s;
            *n_finished += 1;
        }
    }
    return timeout ? CMCG_ERR_DEVICE_TIMEOUT : CMCG_OK;
}

int cmcg_engine_result(cmcg_engine* e, int slot, cmcg_stats* stats) {
    if (!e || slot < 0 || slot >= e->max_slots || e->slots[slot].unit != U_DONE) return CMCG_ERR_INVALID_ARG;
    EngineSlot& sl = e->slots[slot];
    if (stats) *stats = sl.st;
    const int status = sl.status;
    sl = EngineSlot();
    // the caller may now destroy the handle and free its workspace: no cached graph may
    // still point at them
    drop_graph_of_slot(e, slot);
    return status;
}

int cmcg_engine_active(const cmcg_engine* e) {
    if (!e) return CMCG_ERR_INVALID_ARG;
    int n = 0;
    for (const EngineSlot& sl : e->slots)
        n += (sl.unit == U_INIT32 || sl.unit == U_OUTER || sl.unit == U_INNER || sl.unit == U_RUNUP) ? 1 : 0;
    return n;
}

int cmcg_engine_info(const cmcg_engine* e, long long* ticks, long long* graph_builds) {
    if (!e) return CMCG_ERR_INVALID_ARG;
    if (ticks) *ticks = e->ticks;
    if (graph_builds) *graph_builds = e->graph_builds;
    return CMCG_OK;
}

const char* cmcg_engine_cuda_error(const cmcg_engine* e) {
    if (!e) return "invalid engine";
    return cudaGetErrorName(e->last_error);
}

int cmcg_engine_barrier_selftest(cmcg_engine* e, long long spin_limit) {
    if (!e || spin_limit <= 0 || spin_limit > (1ll << 24)) return CMCG_ERR_INVALID_ARG;
    cudaMemsetAsync(e->bar + 2, 0, sizeof(unsigned) * 2, e->st);
    cudaMemsetAsync(e->err + 1, 0, sizeof(int), e->st);
    if (launch_barrier_selftest(e->bar + 2, e->err + 1, spin_limit, e->st) != cudaSuccess) return CMCG_ERR_CUDA;
    int flag = 0;
    cudaMemcpyAsync(&flag, e->err + 1, sizeof(int), cudaMemcpyDeviceToHost, e->st);
    if (cudaStreamSynchronize(e->st) != cudaSuccess) return CMCG_ERR_CUDA;
    return flag ? CMCG_ERR_DEVICE_TIMEOUT : CMCG_OK;
}

}  // extern "C"
