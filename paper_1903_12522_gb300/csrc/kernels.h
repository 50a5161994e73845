// Host-side launcher declarations of libcmcg's kernels (internal).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace cmcg {


// Reduction context: per-block partials, a ticket counter and the device scalar slots.
struct Red {
    double* partials;
    unsigned* ticket;
    double* sc;
};

enum StepFlags { kStepSrc = 1, kStepPrevScaled = 2, kStepNoDiv = 4 };
// Added to the (negated) planes-per-thread of a step launch: four z-planes per loop iteration.
constexpr int kZk4 = 1 << 12;
// Planes-per-thread value that selects the FP32 3D 7-point step in vector form (one aligned
// float4 of the flat node index per thread; FP64 and other stencils take their default kernel).
constexpr int kZcFlat = 1 << 20;

// Process-wide count of kernels launched by this library (every launcher records its launches).
void note_launch(long long k);
// Compiled-in bounds checks (CMCG_CHECKED builds): (count, first site, first index) of the
// failed checks in each translation unit since the last read; the read clears them.
void check_read_wave(long long* out);
void check_read_riesz(long long* out);
void check_read_pair(long long* out);
long long launch_count();

// ---- wave.cu --------------------------------------------------------------------------
template <typename T>
// S: the source dt^2 M^-1 F^ (complex interleaved) in the stepping precision T; scol (3D,
// nullable): per (x, y) column, nonzero if S is nonzero at some node with 0 < z < nz (the
// 3D 7-point kernels then read S on the other columns' z-faces only)
void launch_step(const Geom& g, int order, const T* cur, T* prev, const T* kap, const T* S, double cs,
                 double sn, int flags, int zc, cudaStream_t st, const unsigned char* scol = nullptr);
// scol of S (3D): one byte per (x, y) column
void launch_source_columns(const Geom& g, const double* S, unsigned char* scol, cudaStream_t st);
template <typename T>
// w1_float (T = float): w1 points to floats (the FP32 CG vectors of a mixed-precision inner solve)
void launch_start(const Geom& g, int order, const T* w0t, const double* w1, T* y0, T* y1, const T* kap,
                  const double* S, double dt, int zc, cudaStream_t st, bool w1_float = false);
// mode 0: z = E (Pi(w) - w) and J; mode 1: (y(T), y_t(T)); mode 2 (T = float only): mode 0
// with z0 and t = D^-1 z1 written as floats into out0 and out1 (the FP32 hand-off to the
// adjoint period: launch_adj_start with a = z0 and t, then launch_adj_final mode 2); mode 3
// (T = float only): mode 2 with w1 pointing to floats (FP32 CG vectors).
template <typename T>
void launch_end(const Geom& g, int order, int mode, const T* yN, const T* yNm1, const T* w0t, const double* w1,
                const T* kap, const T* mass, const double* S, double cs, double sn, double* out0, double* out1,
                Red red, double dt, int zc, cudaStream_t st);
template <typename T>
void launch_adj_prep(const Geom& g, const double* b, const T* mass, const T* kap, T* t, int zc,
                     cudaStream_t st);
// a: double, or (T = float) float for the FP32 hand-off.
template <typename T, typename A>
void launch_adj_start(const Geom& g, int order, const A* a, const T* t, const T* mass, const T* kap,
                      T* cur, T* prev, double dt, int zc, cudaStream_t st);
// mode 0: gradient (gt1 may be null); mode 1: q; mode 2 (T = float only): mode 0 reading the
// FP32 hand-off (z0, t) through z0 and z1; mode 3 (T = float only): mode 2 with d0, d1, o0, o1
// pointing to floats (FP32 CG vectors).
template <typename T>
void launch_adj_final(const Geom& g, int order, int mode, const T* s, const T* u1, const T* mass, const T* kap,
                      const double* minv, const double* z0, const double* z1, const double* d0, const double* d1,
                      double* o0, double* o1, double* gt1, Red red, double dt, int zc, cudaStream_t st);
// Two leapfrog steps per launch (step_pair.cu; 3D 7-point, FP32, homogeneous): (A = y^{n-1},
// B = y^n) -> (C = y^{n+1}, D = y^{n+2}); the four buffers must be distinct.  zc: z-planes per
// block (0: 16); ty: interior tile height (0: fewest tiles); depth: planes staged ahead (1..3,
// 0: 2).
bool step2_supported(const Geom& g, int order);
void launch_step2(const Geom& g, const float* A, const float* B, const float* kap, float* C, float* D, int zc,
                  int ty, int depth, cudaStream_t st);

// Batched persistent step loop (wave.cu): one cooperative launch runs the FP32 step loops of
// many solves.  offset = prefix sum of blocks over the preceding items.
struct BatchItem {
    Geom g;
    const float* kap;
    float* buf0;  // y^n at step 0
    float* buf1;  // y^{n-1} at step 0
    int order, nsteps, adjoint, zc, blocks_xy, blocks, offset;
    int vec4;  // 2D 5-point: work items are 256 aligned float4 chunks of the flat index
    // run-up items (forced steps): FP32 source, 3D source columns, steps per period N and
    // the run-up's steps l N; step n = s + 1 has phase omega t_n = 2 pi (n mod N) / N and
    // ramp theta_tr(t_n) = (2 - r) r with r = sin(pi n / (2 l N))
    const float* S;
    const unsigned char* scol;
    int steps_per_period, runup_steps;
};
bool step_vec4_ok(const Geom& g, const void* cur, const void* prev, const void* kap);
// forced: the run-up kernel (forced, ramped steps) instead of the period step loops
int batch_steps_max_blocks(bool forced = false);
cudaError_t launch_batch_steps(const BatchItem* items, int nitems, int total_blocks, int max_steps, unsigned* bar,
                               int* err, int grid, cudaStream_t st, bool forced = false);
cudaError_t launch_barrier_selftest(unsigned* bar, int* err, long long spin_limit, cudaStream_t st);
// Fundamental-frequency filter (Sec. 2.2) fused into a forced FP64 forward period.
void launch_filter_init(long long n, const double* w0, const double* w1, const double* kap64, double inv_wh,
                        double* acc, cudaStream_t st);
void launch_step_filter(const Geom& g, int order, const double* cur, double* prev, const double* kap,
                        const double* S, double cs, double sn, double* acc, double fc, double fs, double cv, int zc,
                        cudaStream_t st);
void launch_scale_complex(long long n, double* u, double s, cudaStream_t st);
void launch_make_source(const Geom& g, const double* f, const double* gb, const double* kap64, double* S, int zc,
                        bool accumulate, cudaStream_t st);
long long plane_blocks(const Geom& g, int zc);

// ---- step_bulk.cu -----------------------------------------------------------------------
// FP32 3D 7-point leapfrog step with TMA bulk-copy staging (homogeneous; flags 0, PREV_SCALED,
// NO_DIV).  step_bulk_plan picks the band height ty and the planes per CTA zc (requests <= 0 mean
// automatic) and returns false when the grid does not fit the kernel.  The fields must have 16
// bytes of readable memory past their last node.  A timed-out wait sets sc[SC_DEVERR].
int step_bulk_smem(int sx, int ty);
// Runs the bulk kernel's bounded mbarrier wait on a phase that never completes; returns
// CMCG_ERR_DEVICE_TIMEOUT when the wait runs out as it must (CMCG_OK would mean it did not).
int bulk_wait_selftest(int spin_limit, cudaStream_t st);
bool step_bulk_plan(const Geom& g, int ty_req, int zc_req, int* ty, int* zc);
// FP32 3D 7-point step with its operands staged in shared memory by asynchronous copies
// (step_async.cu): ty rows per band, zc planes per CTA (0 = automatic), depth = planes in
// flight (2 or 3).  Any step flags.  cudaErrorInvalidValue if the grid does not suit it.
cudaError_t launch_step_async(const Geom& g, const float* cur, float* prev, const float* kap, const float* S,
                              double cs, double sn, int flags, int ty, int zc, int depth, cudaStream_t st);
bool step_async_plan(const Geom& g, int ty_req, int zc_req, int depth, int* ty, int* zc, size_t* smem, int* cap_c,
                     int* cap_p);
void launch_step_bulk(const Geom& g, const float* cur, float* prev, const float* kap, int flags, int ty, int zc,
                      double* sc, cudaStream_t st);

// ---- linalg.cu ------------------------------------------------------------------------
// Setup: kappa = c^2 dt^2 / h^2 (0 on Dirichlet nodes), M = W / c^2 (0 on Dirichlet nodes),
// optional FP32 copy of kappa, Dirichlet byte mask.  sc[0..5) = (sum M, sum B, sum W over
// active nodes, invalid c count, Dirichlet count); sc[5] = bits of max c (zero it first).
void launch_setup_coeffs(const Geom& g, const double* c, const unsigned char* user_mask, unsigned face_dir,
                         double dt, double* kap64, float* kap32, double* mass, unsigned char* mask, Red red,
                         cudaStream_t st);
void launch_mask_copy(const Geom& g, const double* in, const double* kap64, double* out, cudaStream_t st);
void launch_fill(double* p, long long n, double v, cudaStream_t st);
// (w0, w1) = (Re u, wh Im u) on active nodes, 0 on Dirichlet nodes (kap64 = 0); u interleaved.
void launch_warm_start(long long n, const double* u, const double* kap64, double wh, double* w0, double* w1,
                       cudaStream_t st);

// CG recurrences (Step (4) and Steps 5.3-5.8), scalars on the device.
void launch_cg_init(long long n, const double* gt0, const double* gt1, const double* gh0, const double* gh1,
                    double* r0, double* r1, double* rh0, double* rh1, double* d0, double* d1, Red red,
                    cudaStream_t st);
void launch_cg_update(long long n, double* w0, double* w1, double* r0, double* r1, double* rh0, double* rh1,
                      const double* d0, const double* d1, const double* gt0, const double* gt1, const double* gh0,
                      const double* gh1, double sign, Red red, cudaStream_t st);
// d0f (optional): also float(d0).  f32vec: r and d point to floats (FP32 CG vectors).
void launch_cg_direction(long long n, const double* r0, const double* r1, double* d0, double* d1, Red red,
                         cudaStream_t st, float* d0f = nullptr, bool f32vec = false);
// Reductions on the solution for the compatibility-condition shift: sums of
// (F re, F im, (M u) re, (M u) im, (B u) re, (B u) im) into sc[SC_R0..SC_R5].
void launch_recover(const Geom& g, const double* w0, const double* w1, double omega_hat, const double* S,
                    const double* kap64, const double* mass, double* u, Red red, cudaStream_t st);
void launch_axpy(long long n, double a, const double* x, double* y, cudaStream_t st);
void launch_reciprocal(long long n, const double* m, double* out, cudaStream_t st);
// Flexible CG with an approximate Riesz map (one multigrid V-cycle).
// bf (optional): also float(rhat0), the V-cycle's right-hand side.
// f32vec: every vector argument points to floats (FP32 CG vectors of a mixed-precision inner solve).
void launch_fcg_update(long long n, double* w0, double* w1, double* rh0, double* rh1, const double* d0,
                       const double* d1, const double* gh0, const double* gh1, Red red, cudaStream_t st,
                       float* bf = nullptr, bool f32vec = false);
// y += x, x in FP32.
void launch_add_float(long long n, const float* x, double* y, cudaStream_t st);
// lowp: FP32 arithmetic with compensated FP32 partial sums (inside an FP32-period solve);
// f32vec: rh, gh, z and minv point to floats (implies lowp).
void launch_fcg_dots(const Geom& g, const float* zf, double volume, bool remove_mean, bool lowp, const double* rh0,
                     const double* rh1, const double* minv, const double* gh0, const double* gh1, double* z0,
                     double* z1, Red red, bool first, cudaStream_t st, bool f32vec = false);
void launch_wsum_float(const Geom& g, const float* x, Red red, cudaStream_t st);
void launch_shift(long long n, double* u, const double* kap64, double lre, double lim, cudaStream_t st);
// Sums of the compatibility condition for a complex field u: 1.F^, 1.M u, 1.B u -> sc[SC_R0..+5].
void launch_compat_sums(const Geom& g, const double* u, const double* S, const double* kap64, const double* mass,
                        Red red, cudaStream_t st);
void launch_scalar_residual(long long n, const double* r0, const double* r1, const double* rh0,
                            const double* rh1, Red red, int slot, cudaStream_t st);

// ---- riesz.cu -------------------------------------------------------------------------
struct MGLevel {
    Geom g;
    unsigned char* mask;  // Dirichlet bytes (nullptr if the problem has none)
    float *x, *x2, *b, *r;
};
void launch_mg_coarsen_mask(const MGLevel& fine, const MGLevel& coarse, cudaStream_t st);
void launch_mg_jacobi(const MGLevel& L, const float* xin, float* xout, const float* b, float omega, bool zero_init,
                      cudaStream_t st);
void launch_mg_residual(const MGLevel& L, const float* x, const float* b, float* r, cudaStream_t st);
void launch_mg_restrict(const MGLevel& fine, const float* rf, const MGLevel& coarse, float* bc, cudaStream_t st);
void launch_mg_prolong_add(const MGLevel& coarse, const float* xc, const MGLevel& fine, float* xf, cudaStream_t st);
// Coarse end of the V-cycle in one thread block (levels up to kBlockLevelsMax, total nodes
// within the shared-memory budget).
constexpr int kBlockLevelsMax = 8;
constexpr int kBlockMaxNodes = 6000;  // nodes of the first in-block level
struct BlockLevels {
    int n;
    Geom g[kBlockLevelsMax];
    const unsigned char* mask[kBlockLevelsMax];
};
void launch_mg_block_vcycle(const BlockLevels& lv, const float* b, float* x, float omega, int nu, int coarse_sweeps,
                            cudaStream_t st);
size_t mg_block_smem_bytes(const BlockLevels& lv);
int mg_block_max_nodes();
// FP64 PCG pieces on the fine level
void launch_applyK(const Geom& g, int order, const unsigned char* mask, const double* x, double* y,
                   const double* dotwith, Red red, int slot, cudaStream_t st);
void launch_to_float(long long n, const double* in, float* out, cudaStream_t st);
void launch_pcg_project(const Geom& g, const double* in, double* out, const unsigned char* mask, double volume,
                        Red red, bool project, cudaStream_t st);
void launch_pcg_dots_after_precond(long long n, const double* r, const float* z, const double* Ap, double* zd,
                                   Red red, cudaStream_t st);
void launch_pcg_xr_update(long long n, double* x, double* r, const double* p, const double* Ap, Red red,
                          cudaStream_t st);
void launch_pcg_p_update(long long n, double* p, const double* zd, Red red, bool first, cudaStream_t st);
void launch_mean_remove(const Geom& g, double* x, double volume, Red red, cudaStream_t st);
void launch_reduce_sum(long long n, const double* x, Red red, int slot, cudaStream_t st);

}  // namespace cmcg
