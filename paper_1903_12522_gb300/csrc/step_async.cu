// FP32 leapfrog step, 3D 7-point, with its operands staged in shared memory by per-thread
// asynchronous copies (cp.async, 16 bytes each) in a pipeline several planes deep.  Same
// arithmetic, in the same order, as k_step3d7 in wave.cu (homogeneous, forced, and the
// adjoint variants PREV_SCALED / NO_DIV):
//
//   y^{n+1} = [2 y^n - kappa Lt y^n + src - (1 - beta) y^{n-1}] / (1 + beta)   (over y^{n-1})
//
// Work split: a CTA owns a band of ty full x-rows (y0 .. y0+ty-1) and marches z over planes
// z0 .. z1-1; each thread keeps the same nodes of the band on every plane, with their values
// on planes z-1 and z in registers (the z-neighbours).  Per plane the CTA stages
//   cur   rows y0-1 .. y0+ty (clipped to the grid) of plane z+1        ring of D+2 slots
//   prev  rows y0 .. y0+ty-1 of plane z                                ring of D+1 slots
//   kappa rows y0 .. y0+ty-1 of plane z                                ring of D+1 slots
// issued D planes ahead of their use.  The rows of a band are one contiguous range of a
// plane, so each is copied as the 16-byte-aligned superset of that range (at most 3 floats
// either side), which every FP32 field's allocation slack covers, and indexed from the start's
// remainder.  Mirror neighbours at y = -1 and y = ny + 1 are the mirrored rows, which the
// staged range holds; at z = -1 and z = nz + 1 they are the register copies of planes 1 and
// nz - 1.  The output goes straight to global memory: a node's y^{n-1} was staged D planes
// before the node is written, and no other CTA reads it.
//
// Pipeline per plane z: wait for this thread's copy group of plane z, a CTA barrier (every
// thread's copies are visible, and every thread has finished plane z-1, so the slots that
// held plane z-1 are free), issue the group of plane z+D into those slots, compute plane z.
// No wait spins: cp.async.wait_group and __syncthreads complete by themselves.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace cmcg {
namespace {

constexpr int kAT = 256;     // threads per CTA
constexpr int kNodeMax = 5;  // band nodes per thread and plane (ty * sx <= 5 * 256)
constexpr size_t kSmemCap = 200 * 1024;  // dynamic shared memory per CTA at most

__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Stage rows [r0, r1] of plane p of field f (row length sx) into slot s: the 16-byte-aligned
// superset of the range; returns nothing, the remainder is recomputed by the reader.
__device__ __forceinline__ void stage_rows(float* s, const float* __restrict__ f, long long p, long long sZ, int sx,
                                           int r0, int r1) {
    const long long start = p * sZ + (long long)r0 * sx;
    const long long end = p * sZ + (long long)(r1 + 1) * sx;  // one past the last float
    const long long a0 = start & ~3ll;
    const int chunks = (int)((end - a0 + 3) >> 2);
    for (int k = threadIdx.x; k < chunks; k += kAT) cp_async16(s + 4 * k, f + a0 + 4 * k);
}

template <int FLAGS, int D>
__global__ void __launch_bounds__(kAT) k_step3d7_async(const float* __restrict__ cur, float* __restrict__ prev_out,
                                                       const float* __restrict__ kap, const float* __restrict__ S,
                                                       double cs, double sn, Geom g, int ty, int zc, int cap_c,
                                                       int cap_p) {
    extern __shared__ __align__(16) float smem[];
    constexpr int RC = D + 2, RP = D + 1;
    float* s_cur = smem;
    float* s_prev = s_cur + RC * cap_c;
    float* s_kap = s_prev + RP * cap_p;

    const int sx = g.sx;
    const long long sZ = (long long)sx * g.sy;
    const int y0 = (int)blockIdx.x * ty;
    const int y1 = min(y0 + ty, g.sy);  // one past the band's last row
    const int z0 = (int)blockIdx.y * zc;
    const int z1 = min(z0 + zc, g.sz);
    if (y0 >= g.sy || z0 >= z1) return;  // uniform over the CTA
    const int lo = max(y0 - 1, 0), hi = min(y1, g.sy - 1);  // cur rows staged
    const int nb_nodes = (y1 - y0) * sx;

    // this thread's band nodes: q = tid + 256 i, row y0 + q / sx, column q % sx
    int qc[kNodeMax];   // index within the staged cur rows (from row lo)
    int info[kNodeMax];  // bit 0: x = 0, 1: x = nx, 2: y = 0, 3: y = ny; bits 4..: absorbing faces
    int nn = 0;
#pragma unroll
    for (int i = 0; i < kNodeMax; ++i) {
        const int q = threadIdx.x + kAT * i;
        qc[i] = 0;
        info[i] = 0;
        if (q < nb_nodes) {
            const int r = y0 + q / sx, x = q - (q / sx) * sx;
            qc[i] = (r - lo) * sx + x;
            int nbxy = 0;
            nbxy += (x == 0) & (int)(g.abc & 1u);
            nbxy += (x == g.nx) & (int)((g.abc >> 1) & 1u);
            nbxy += (r == 0) & (int)((g.abc >> 2) & 1u);
            nbxy += (r == g.ny) & (int)((g.abc >> 3) & 1u);
            info[i] = (x == 0) | ((x == g.nx) << 1) | ((r == 0) << 2) | ((r == g.ny) << 3) | (nbxy << 4);
            nn = i + 1;
        }
    }
    const int row_off = (y0 - lo) * sx;  // band node q sits at qc - row_off in the prev / kappa rows

    auto issue = [&](int zc_plane, int zp_plane) {
        // cur plane zc_plane (if it exists and is needed), prev / kappa plane zp_plane (if < z1)
        if (zc_plane <= g.nz && zc_plane <= z1)
            stage_rows(s_cur + (zc_plane % RC) * cap_c, cur, zc_plane, sZ, sx, lo, hi);
        if (zp_plane < z1) {
            stage_rows(s_prev + (zp_plane % RP) * cap_p, prev_out, zp_plane, sZ, sx, y0, y1 - 1);
            stage_rows(s_kap + (zp_plane % RP) * cap_p, kap, zp_plane, sZ, sx, y0, y1 - 1);
        }
        cp_commit();
    };

    // prologue: cur plane z0, then the groups of the virtual planes z0-D .. z0-1
    stage_rows(s_cur + (z0 % RC) * cap_c, cur, z0, sZ, sx, lo, hi);
    cp_commit();
#pragma unroll
    for (int v = 1; v <= D; ++v) issue(z0 + v, z0 + v - 1);  // virtual plane z0 - D + v - 1

    // z-neighbour below plane z0 (mirror at z = 0: plane 1), read directly
    float zm[kNodeMax];
    {
        const int pb = z0 > 0 ? z0 - 1 : 1;
#pragma unroll
        for (int i = 0; i < kNodeMax; ++i) {
            zm[i] = 0.f;
            if (i < nn) zm[i] = cur[(long long)pb * sZ + (long long)lo * sx + qc[i]];
        }
    }

    for (int z = z0; z < z1; ++z) {
        cp_wait<D - 1>();
        __syncthreads();
        issue(z + 1 + D, z + D);
        const long long base_c = (long long)z * sZ + (long long)lo * sx;
        const int rc0 = (int)(base_c & 3ll);  // remainder of plane z's staged cur rows
        const long long base_n = (long long)(z + 1) * sZ + (long long)lo * sx;
        const int rc1 = (int)(base_n & 3ll);
        const long long base_p = (long long)z * sZ + (long long)y0 * sx;
        const int rp = (int)(base_p & 3ll);
        const float* c0 = s_cur + (z % RC) * cap_c + rc0;
        const float* c1 = s_cur + ((z + 1) % RC) * cap_c + rc1;
        const float* pv = s_prev + (z % RP) * cap_p + rp;
        const float* kv = s_kap + (z % RP) * cap_p + rp;
        const int nbz = ((z == 0) & (int)((g.abc >> 4) & 1u)) + ((z == g.nz) & (int)((g.abc >> 5) & 1u));
#pragma unroll
        for (int i = 0; i < kNodeMax; ++i) {
            if (i < nn) {
                const int q = qc[i];
                const int f = info[i];
                const float y = c0[q];
                const float zp = z < g.nz ? c1[q] : zm[i];
                const float xm = c0[q + ((f & 1) ? 1 : -1)];
                const float xp = c0[q + ((f & 2) ? -1 : 1)];
                const float ym = c0[q + ((f & 4) ? sx : -sx)];
                const float yp = c0[q + ((f & 8) ? -sx : sx)];
                const float L = 6.f * y - (((xm + xp) + (ym + yp)) + (zm[i] + zp));
                const int qp = q - row_off;
                const float k = kv[qp];
                const float yq = pv[qp];
                float rhs = 2.f * y - k * L;
                const long long j = base_p + qp;
                if (FLAGS & kStepSrc) rhs += S[2 * j] * (float)cs + S[2 * j + 1] * (float)sn;
                const int nb = (f >> 4) + nbz;
                float out;
                if (nb == 0) {
                    out = rhs - yq;
                } else {
                    const float beta = (float)nb * sqrtf(k);
                    const float vv = rhs - ((FLAGS & kStepPrevScaled) ? yq : (1.f - beta) * yq);
                    out = (FLAGS & kStepNoDiv) ? vv : vv / (1.f + beta);
                }
                prev_out[j] = out;
                zm[i] = y;
            }
        }
    }
    cp_wait<0>();  // leave no copy in flight
}

template <int FLAGS, int D>
cudaError_t launch_async_t(const Geom& g, const float* cur, float* prev, const float* kap, const float* S, double cs,
                           double sn, int ty, int zc, int cap_c, int cap_p, size_t smem, cudaStream_t st) {
    // the attribute belongs to the function on the current device; setting it is a host call
    const cudaError_t e =
        cudaFuncSetAttribute(k_step3d7_async<FLAGS, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)((g.sy + ty - 1) / ty), (unsigned)((g.sz + zc - 1) / zc));
    k_step3d7_async<FLAGS, D><<<grid, kAT, smem, st>>>(cur, prev, kap, S, cs, sn, g, ty, zc, cap_c, cap_p);
    return cudaGetLastError();
}

}  // namespace

// Plan of the staged step for a grid: rows per band (ty) and planes per CTA (zc), from the
// requests (0 = automatic); false if the grid does not suit the kernel (a band row must fit
// the per-thread node budget).
bool step_async_plan(const Geom& g, int ty_req, int zc_req, int depth, int* ty, int* zc, size_t* smem, int* cap_c,
                     int* cap_p) {
    if (g.dim != 3 || g.sx > kNodeMax * kAT || g.np >= (1ll << 40)) return false;
    const int D = depth == 3 ? 3 : 2;
    int t = ty_req > 0 ? ty_req : std::max(1, std::min(4, (kNodeMax * kAT) / g.sx));
    t = std::min(t, std::max(1, (kNodeMax * kAT) / g.sx));
    t = std::min(t, g.sy);
    const int cc = ((t + 2) * g.sx + 8 + 3) & ~3;  // staged cur rows + alignment slack, 16-byte slots
    const int cp = (t * g.sx + 8 + 3) & ~3;
    const size_t bytes = sizeof(float) * ((size_t)(D + 2) * cc + 2 * (size_t)(D + 1) * cp);
    if (bytes > kSmemCap) return false;
    int z = zc_req;
    if (z <= 0) {
        // one wave: bands x z-chunks at most the resident CTA count (a second, partial wave
        // would take as long as the first)
        int dev = 0, sms = 148, per = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        per = std::max(1, std::min(8, (int)((228 * 1024) / (bytes + 1024))));
        per = std::min(per, (64 * 1024) / (kAT * 64));  // registers: at most 64 per thread
        const long long bands = (g.sy + t - 1) / t;
        const long long want = (long long)sms * per;
        const long long chunks = std::max(1ll, want / bands);
        z = (int)std::max(2ll, (g.sz + chunks - 1) / chunks);
    }
    *ty = t;
    *zc = std::min(z, g.sz);
    *smem = bytes;
    *cap_c = cc;
    *cap_p = cp;
    return true;
}

cudaError_t launch_step_async(const Geom& g, const float* cur, float* prev, const float* kap, const float* S,
                              double cs, double sn, int flags, int ty_req, int zc_req, int depth, cudaStream_t st) {
    int ty = 0, zc = 0, cap_c = 0, cap_p = 0;
    size_t smem = 0;
    if (!step_async_plan(g, ty_req, zc_req, depth, &ty, &zc, &smem, &cap_c, &cap_p)) return cudaErrorInvalidValue;
    note_launch(1);
#define CMCG_ASYNC(F, DD) launch_async_t<F, DD>(g, cur, prev, kap, S, cs, sn, ty, zc, cap_c, cap_p, smem, st)
    const bool d3 = depth == 3;
    switch (flags) {
        case 0: return d3 ? CMCG_ASYNC(0, 3) : CMCG_ASYNC(0, 2);
        case kStepSrc: return d3 ? CMCG_ASYNC(kStepSrc, 3) : CMCG_ASYNC(kStepSrc, 2);
        case kStepPrevScaled: return d3 ? CMCG_ASYNC(kStepPrevScaled, 3) : CMCG_ASYNC(kStepPrevScaled, 2);
        case kStepNoDiv: return d3 ? CMCG_ASYNC(kStepNoDiv, 3) : CMCG_ASYNC(kStepNoDiv, 2);
        case kStepPrevScaled | kStepNoDiv:
            return d3 ? CMCG_ASYNC(kStepPrevScaled | kStepNoDiv, 3) : CMCG_ASYNC(kStepPrevScaled | kStepNoDiv, 2);
        default: return cudaErrorInvalidValue;
    }
#undef CMCG_ASYNC
}

}  // namespace cmcg
