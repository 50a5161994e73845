// Internal: the solver handle and the host-side pieces shared by the single-solve entry
// points (api.cu) and the multi-solve engine (engine.cu).
#pragma once
#include <type_traits>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "cmcg.h"
#include "common.cuh"
#include "kernels.h"

namespace cmcg {
constexpr int kMaxLevels = 16;
constexpr int kZcStep3D = 16;  // z-planes per thread in the leapfrog step (3D)
constexpr int kZcEnds = 8;     // z-planes per thread in the period endpoint kernels
constexpr double kPi = 3.14159265358979323846;
}  // namespace cmcg

using namespace cmcg;  // internal header: the handle's members use the library's types

struct cmcg_handle {
    Geom g{};
    int order = 2;
    cmcg_options opt{};
    cudaStream_t st = nullptr;
    double omega = 0, T = 0, dt = 0, wt = 0, wh = 0, volume = 0;
    int N = 0;
    bool has_dir = false;
    double sumM = 0, sumB = 0, sumW = 0, cmin = 1;
    // coefficients
    double *kap64 = nullptr, *mass = nullptr, *minv = nullptr, *S = nullptr;
    float* kap32 = nullptr;
    float* S32 = nullptr;  // FP32 copy of S, the source of FP32 leapfrog steps (FP32 / mixed)
    float *mass32 = nullptr, *minv32 = nullptr;  // FP32 copies of M and M^-1 (FP32 / mixed)
    unsigned char* scol = nullptr;  // 3D: columns with source inside the grid (launch_source_columns)
    unsigned char* mask = nullptr;
    const double* warm = nullptr;  // cmcg_solve_warm: the start field U (complex, interleaved) of this solve
    // wave buffers (sized for double; FP32 stepping uses the first half) + FP64 temp
    void *ya = nullptr, *yb = nullptr;
    double* tmp = nullptr;
    // CG state
    double *w0, *w1, *r0, *r1, *rh0, *rh1, *d0, *d1, *gh0, *gh1, *gt0, *gt1, *z0, *z1;
    double *wo0 = nullptr, *wo1 = nullptr;  // CMCG_MIXED outer iterate
    // Riesz PCG
    double *pr, *pp, *pAp, *pzd;
    MGLevel lv[kMaxLevels];
    int nlev = 0;
    int blk_level = -1;       // first level run inside one thread block (-1: none)
    BlockLevels blk{};
    int riesz_guess = 0;      // PCG iterations of the previous Riesz solve
    // first-order formulation (CMCG_FLAG_FIRST_ORDER): CG vectors on the state (p, v) of
    // (dim + 1) N_p doubles, and the two stepping buffers (sized for double)
    double *fo_s = nullptr, *fo_r = nullptr, *fo_d = nullptr, *fo_e = nullptr, *fo_g = nullptr, *fo_x = nullptr;
    void *fo_a = nullptr, *fo_b = nullptr;
    bool first_order = false;
    // host staging
    double* stage = nullptr;
    // reductions
    double* partials = nullptr;
    unsigned* tickets = nullptr;
    double* sc = nullptr;
    double* hsc = nullptr;  // pinned host mirror of sc
    // FP32 CG vectors: a mixed-precision handle with the V-cycle Riesz map keeps the vectors of
    // its inner (FP32-period) flexible CG -- w, rhat, d, ghat, z -- as floats in the first half
    // of their buffers; vec32_active is set while such an inner iteration is being enqueued
    bool vec32 = false;
    bool vec32_active = false;
    bool l2_kappa = false;  // CMCG_FLAG_L2_KAPPA took effect (window set on st, set-aside held)
    // residual history of the last solve: sqrt(gamma_k / gamma_0) per CG iteration, relative to
    // the zero initial guess (hist_scale converts a loop's own relative residual)
    std::vector<double> hist;
    double hist_scale = 1.0;
    // counters of the current call
    long long riesz_iters = 0;
    long long periods = 0;
    long long graph_replays = 0;
    // CMCG_FLAG_TIMING: event pairs around the step loops of the periods since the last sync
    bool timing = false;
    cudaEvent_t ev[8] = {};
    int ev_used = 0;
    bool ev_fp32[4] = {};
    int ev_steps[4] = {};
    double step_s[2] = {0, 0};     // [fp64, fp32]
    long long step_n[2] = {0, 0};
    Red red() const { return Red{partials, tickets, sc}; }
};

namespace cmcg {
namespace detail {

// The two leapfrog buffers of a period in flight: cur holds y^n, prev y^{n-1}; w0t is the
// stepping-precision copy of the initial displacement (forward periods).
struct PeriodBuffers {
    void* cur;
    void* prev;
    const void* w0t;
};

int cuda_status();
// After every change of S: refresh its FP32 copy (FP32 and mixed-precision handles).
void source_updated(cmcg_handle* H);
// The lumped mass M in precision T (what the period kernels of that precision read).
template <typename T>
const T* step_mass(const cmcg_handle* H) {
    if constexpr (std::is_same<T, float>::value) return H->mass32;
    else return H->mass;
}
// The source array of leapfrog steps in precision T.
template <typename T>
const T* step_source(const cmcg_handle* H) {
    if constexpr (std::is_same<T, float>::value) return H->S32;
    else return H->S;
}
int sync_read(cmcg_handle* H);
bool inexact(const cmcg_handle* H);
// b_ready: the finest level's right-hand side already holds float(rhat0) (written by the
// flexible-CG update), so the conversion pass is skipped.
void apply_B(cmcg_handle* H, bool first, bool lowp, bool b_ready = false);
// FP32 CG vectors (H->vec32): start of an inner solve from the FP64 gradient (rhat, z = B rhat,
// gamma0, d = z as floats; sets vec32_active), and W += w of the finished inner solve.
void begin_vec32_inner(cmcg_handle* H);
void add_correction(cmcg_handle* H, double* W0, double* W1);
int adj_step_flags(int k, int N);
// Gradient periods (mode 0) in FP32 hand z from the forward end to the adjoint period as
// floats in the z buffers: z0, and t = D^-1 z1 (D = M (1 + beta)) in place of z1.
template <typename T>
constexpr bool fp32_handoff(int mode) {
    return std::is_same<T, float>::value && mode == 0;
}
// w0f_ready (FP32): the temp buffer already holds float(w0) (written by the CG direction update).
template <typename T>
PeriodBuffers fwd_begin(cmcg_handle* H, const double* w0, const double* w1, bool src, bool w0f_ready = false);
template <typename T>
void fwd_end(cmcg_handle* H, const PeriodBuffers& b, const double* w1, bool src, int mode, double* out0,
             double* out1);
// mode as for adj_end: with the FP32 hand-off (mode 0, T = float) a and bb are its float z0 and t.
template <typename T>
PeriodBuffers adj_begin(cmcg_handle* H, const double* a, const double* bb, int mode);
template <typename T>
void adj_end(cmcg_handle* H, const PeriodBuffers& b, const double* a, const double* bb, int mode, const double* d0,
             const double* d1, double* o0, double* o1, double* gt1);
// riesz: also the exact Riesz map of the gradient (needs g~1 = ghat1 / M, written only then).
template <typename T>
int gradient(cmcg_handle* H, const double* w0, const double* w1, bool src, const double* dd0, const double* dd1,
             bool riesz, bool w0f_ready = false);
template <typename T>
void forward_period(cmcg_handle* H, const double* w0, const double* w1, bool src, int mode, double* out0,
                    double* out1, bool w0f_ready = false);
// Step (6): U from (w0, w1) into u and the compatibility-condition shift; fills st's
// lambda fields.  Synchronises the stream.
int recover(cmcg_handle* h, double* u, cmcg_stats* st);
int timing_begin(cmcg_handle* H, bool fp32, int steps);
// Run-up (Sec. 4.2.3): its number of periods, and the source ramp theta_tr(t) over [0, ttr].
int runup_count(const cmcg_handle* H);
// The run-up itself: (y, y_t) at t = periods T into (w0, w1).
template <typename T>
void runup(cmcg_handle* H, int periods, double* w0, double* w1);
// The FP32 run-up around a step loop run elsewhere: buffers at rest (yb = y^1, ya = y^0), then
// after periods N - 1 steps (y, y_t) at t = periods T into (w0, w1).
void runup_start_f32(cmcg_handle* H);
void runup_finish_f32(cmcg_handle* H, int periods, double* w0, double* w1);
double ramp(double t, double ttr);
void timing_end(cmcg_handle* H, int p);

// First-order formulation (first_order.cu).  fo_solve runs steps (1)-(5) on the state in
// fo_s; fo_recover writes U (step (6), Eq. mix_solution or, with CMCG_FLAG_FILTER, Eq.
// TH_FILTERED_MIXED_SOLUTION) and synchronises; fo_J evaluates J^ at fo_s into sc[SC_J];
// fo_period / fo_adjoint are one forward period (with the sources when src) and the plain
// transpose of the homogeneous period.
int fo_solve(cmcg_handle* H, double tol, cmcg_stats* st);
int fo_recover(cmcg_handle* H, double* u);
void fo_J(cmcg_handle* H);
int fo_period(cmcg_handle* H, const double* s0, bool src, double* out);
int fo_adjoint(cmcg_handle* H, const double* y, double* out);

}  // namespace detail
// Named NVTX range over a host scope (a solve, a period, a Riesz map, an engine tick): the
// profilers group the kernels launched inside it (ncu --nvtx --nvtx-include "cmcg <name>/";
// no slash inside a name, which ncu reads as nesting).  Kernels of a captured iteration graph
// launch at its replay, outside these host ranges.  Without an attached tool the push and pop
// cost a branch each.
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

}  // namespace cmcg
