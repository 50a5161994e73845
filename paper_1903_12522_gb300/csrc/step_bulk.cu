// FP32 leapfrog step, 3D 7-point, with its operands staged in shared memory by the TMA unit
// (cp.async.bulk, mbarrier completion).  Same arithmetic, in the same order, as k_step3d7 in
// wave.cu (the homogeneous step and its adjoint variants PREV_SCALED / NO_DIV):
//
//   y^{n+1} = [2 y^n - kappa Lt y^n - (1 - beta) y^{n-1}] / (1 + beta)      (written over y^{n-1})
//
// Work split: a CTA owns a band of ty full x-rows (y0 .. y1-1) and marches z over planes
// z0 .. z1-1.  The rows of a band are one contiguous range of a plane, so each plane's operands
// come in as one bulk copy per field:
//   cur ring, kNC = 5 slots : rows y0-1 .. y1 of planes z-1, z, z+1 and the two planes in flight
//   prev / kappa rings, kNP = 3 slots : rows y0 .. y1-1 of planes z, z+1, z+2
// A bulk copy starts and ends on 16-byte boundaries, so each copies the aligned superset of its
// range (at most 3 floats either side) and the kernel indexes from the start's remainder.
// Mirror neighbours at the faces (y = -1, y = ny + 1, z = -1, z = nz + 1) are read from the
// mirrored row / plane, which the staged ranges contain.
//
// One thread (tid 0) initialises the barriers and issues every copy; lane 0 of each warp waits
// on a slot's barrier (bounded spin) and a warp barrier then releases its lanes.  After a
// plane, a CTA barrier frees the slots of plane z-1 (cur) and plane z (prev/kappa), which are
// refilled with planes z+4 and z+3.  If a
// wait runs out, the kernel records CMCG_ERR_DEVICE_TIMEOUT in sc[SC_DEVERR], waits (again
// bounded) for the copies it issued, and returns.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>

#include "common.cuh"
#include "kernels.h"

namespace cmcg {
namespace {

constexpr int kBT = 512;                  // threads per CTA
constexpr int kNC = 5;                    // cur ring slots (two planes in flight)
constexpr int kNP = 3;                    // prev / kappa ring slots
constexpr int kBarBytes = 128;            // barrier + flag header of the shared memory
constexpr int kWaitLimit = 1 << 22;       // try_wait polls before a wait counts as timed out
constexpr int kSmemBudget = 112 * 1024;   // per CTA, so that two CTAs fit on an SM

__host__ __device__ __forceinline__ int round4(int x) { return (x + 3) & ~3; }

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// global -> shared bulk copy completing on the barrier (a CTA is its own cluster here)
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int limit = kWaitLimit) {
    for (int i = 0; i < limit; ++i)
        if (mbar_try(bar, parity)) return true;
    return false;
}

// Self-test of the bounded wait: phase 0 of a fresh barrier never completes (nothing arrives),
// so the wait must run out and report a time-out.
__global__ void k_bulk_wait_selftest(int limit, int* out) {
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        fence_mbar_init();
    }
    __syncthreads();
    const bool ok = mbar_wait(smem_u32(&bar), 0u, limit);
    if (threadIdx.x == 0) *out = ok ? 0 : CMCG_ERR_DEVICE_TIMEOUT;
}

__device__ int g_selftest_out;

__device__ __forceinline__ int mirror_z(int q, int nz) { return q < 0 ? -q : (q > nz ? 2 * nz - q : q); }

template <int FLAGS>
__global__ void __launch_bounds__(kBT) k_step3d7_bulk(const float* __restrict__ cur, float* __restrict__ prev_out,
                                                      const float* __restrict__ kap, Geom g, int ty, int zc,
                                                      int cur_cap, int p_cap, double* __restrict__ sc) {
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(smem);  // kNC cur + kNP prev/kappa
    volatile int* s_abort = reinterpret_cast<volatile int*>(smem + 8 * (kNC + kNP));
    float* s_cur = reinterpret_cast<float*>(smem + kBarBytes);
    float* s_prev = s_cur + (size_t)kNC * cur_cap;
    float* s_kap = s_prev + (size_t)kNP * p_cap;

    const int tid = threadIdx.x;
    const int sx = g.sx;
    const long long plane = (long long)sx * g.sy;
    const int y0 = (int)blockIdx.x * ty;
    const int y1 = min(y0 + ty, g.sy);
    const int z0 = (int)blockIdx.y * zc;
    const int z1 = min(z0 + zc, g.sz);
    if (y0 >= g.sy || z0 >= z1) return;  // uniform over the CTA
    const int lo = max(y0 - 1, 0), hi = min(y1, g.sy - 1);  // cur rows staged
    const int ncur = hi - lo + 1, nrow = y1 - y0;

    // remainders of the staged ranges' starts (floats past the 16-byte boundary)
    auto cur_off = [&](int q) { return (int)(((long long)mirror_z(q, g.nz) * plane + (long long)lo * sx) & 3LL); };
    auto p_off = [&](int q) { return (int)(((long long)q * plane + (long long)y0 * sx) & 3LL); };

    // producer (tid 0 only): cur plane q (virtual, mirrored at the z faces) into its slot
    auto issue_cur = [&](int q) {
        const int s = (q - (z0 - 1)) % kNC;
        const long long start = (long long)mirror_z(q, g.nz) * plane + (long long)lo * sx;
        const long long a = start & ~3LL, b = (start + (long long)ncur * sx + 3) & ~3LL;
        const uint32_t bar = smem_u32(&bars[s]);
        const uint32_t bytes = (uint32_t)(4 * (b - a));
        mbar_expect_tx(bar, bytes);
        bulk_g2s(smem_u32(s_cur + (size_t)s * cur_cap), cur + a, bytes, bar);
    };
    auto issue_p = [&](int q) {
        const int s = (q - z0) % kNP;
        const long long start = (long long)q * plane + (long long)y0 * sx;
        const long long a = start & ~3LL, b = (start + (long long)nrow * sx + 3) & ~3LL;
        const uint32_t bar = smem_u32(&bars[kNC + s]);
        const uint32_t bytes = (uint32_t)(4 * (b - a));
        mbar_expect_tx(bar, 2u * bytes);
        bulk_g2s(smem_u32(s_prev + (size_t)s * p_cap), prev_out + a, bytes, bar);
        bulk_g2s(smem_u32(s_kap + (size_t)s * p_cap), kap + a, bytes, bar);
    };
    auto cur_bar = [&](int q) { return smem_u32(&bars[(q - (z0 - 1)) % kNC]); };
    auto cur_par = [&](int q) { return (uint32_t)(((q - (z0 - 1)) / kNC) & 1); };
    auto p_bar = [&](int q) { return smem_u32(&bars[kNC + (q - z0) % kNP]); };
    auto p_par = [&](int q) { return (uint32_t)(((q - z0) / kNP) & 1); };

    if (tid == 0) {
        for (int i = 0; i < kNC + kNP; ++i) mbar_init(smem_u32(&bars[i]), 1);
        *s_abort = 0;
        fence_mbar_init();
    }
    __syncthreads();
    // planes issued so far (tid 0): cur up to cq (virtual planes z0-1 .. z1), prev/kappa up to pq
    int cq = z0 - 2, pq = z0 - 1;
    if (tid == 0) {
        for (int q = z0 - 1; q <= min(z0 + kNC - 2, z1); ++q) issue_cur(q), cq = q;
        for (int q = z0; q < min(z0 + kNP, z1); ++q) issue_p(q), pq = q;
    }

    // ABC faces through the band's rows and columns
    const unsigned abc = g.abc;
    const int ax0 = (int)(abc & 1u), ax1 = (int)((abc >> 1) & 1u), ay0 = (int)((abc >> 2) & 1u),
              ay1 = (int)((abc >> 3) & 1u), az0 = (int)((abc >> 4) & 1u), az1 = (int)((abc >> 5) & 1u);
    const int nout = nrow * sx;

    const int lane = tid & 31;
    for (int z = z0; z < z1; ++z) {
        if (lane == 0) {
            const bool ready = mbar_wait(cur_bar(z - 1), cur_par(z - 1)) && mbar_wait(cur_bar(z), cur_par(z)) &&
                               mbar_wait(cur_bar(z + 1), cur_par(z + 1)) && mbar_wait(p_bar(z), p_par(z));
            if (!ready) *s_abort = 1;
        }
        __syncwarp();  // orders lane 0's completed waits before the other lanes' reads
        if (*s_abort) {
            // skip the plane; the CTA barrier below ends the march
        } else {
            const float* cm = s_cur + (size_t)((z - 1 - (z0 - 1)) % kNC) * cur_cap + cur_off(z - 1);
            const float* cc = s_cur + (size_t)((z - (z0 - 1)) % kNC) * cur_cap + cur_off(z);
            const float* cp = s_cur + (size_t)((z + 1 - (z0 - 1)) % kNC) * cur_cap + cur_off(z + 1);
            const int po = p_off(z);
            const float* pv = s_prev + (size_t)((z - z0) % kNP) * p_cap + po;
            const float* kv = s_kap + (size_t)((z - z0) % kNP) * p_cap + po;
            float* out_row = prev_out + (long long)z * plane + (long long)y0 * sx;
            const int nbz = (z == 0 ? az0 : 0) + (z == g.nz ? az1 : 0);
            int x = tid, yy = 0;
            while (x >= sx) x -= sx, ++yy;
            for (int i = tid; i < nout; i += kBT) {
                const int y = y0 + yy;
                const int rc = (y - lo) * sx + x;
                const float yc = cc[rc];
                const float xm = cc[rc + (x > 0 ? -1 : 1)];
                const float xp = cc[rc + (x < g.nx ? 1 : -1)];
                const float ym = cc[rc + (y > 0 ? -sx : sx)];
                const float yp = cc[rc + (y < g.ny ? sx : -sx)];
                const float L = 6.0f * yc - ((xm + xp) + (ym + yp) + (cm[rc] + cp[rc]));
                const int rp = yy * sx + x;
                const float k = kv[rp];
                const float ypv = pv[rp];
                const float rhs = 2.0f * yc - k * L;
                const int nb = nbz + (x == 0 ? ax0 : 0) + (x == g.nx ? ax1 : 0) + (y == 0 ? ay0 : 0) +
                               (y == g.ny ? ay1 : 0);
                float o;
                if (nb == 0) {
                    o = rhs - ypv;
                } else {
                    const float beta = (float)nb * sqrtf(k);
                    const float v = rhs - ((FLAGS & kStepPrevScaled) ? ypv : (1.0f - beta) * ypv);
                    o = (FLAGS & kStepNoDiv) ? v : v / (1.0f + beta);
                }
                out_row[rp] = o;
                x += kBT;
                while (x >= sx) x -= sx, ++yy;
            }
        }
        __syncthreads();
        if (*s_abort) break;
        if (tid == 0) {
            fence_proxy_async();  // this CTA's reads of the freed slots precede the refills
            if (z + kNC - 1 <= z1) issue_cur(z + kNC - 1), cq = z + kNC - 1;
            if (z + kNP < z1) issue_p(z + kNP), pq = z + kNP;
        }
    }
    if (*s_abort && tid == 0) {
        sc[SC_DEVERR] = (double)CMCG_ERR_DEVICE_TIMEOUT;
        // let every copy this CTA issued land before its shared memory is released
        for (int q = max(z0 - 1, cq - kNC + 1); q <= cq; ++q) mbar_wait(cur_bar(q), cur_par(q));
        for (int q = max(z0, pq - kNP + 1); q <= pq; ++q) mbar_wait(p_bar(q), p_par(q));
    }
}

int g_num_sms = 0;

int num_sms() {
    if (g_num_sms == 0) {
        int dev = 0, n = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        g_num_sms = n > 0 ? n : 1;
    }
    return g_num_sms;
}

template <int FLAGS>
void set_smem_attr() {
    static std::atomic<int> done{0};
    if (!done.load(std::memory_order_acquire)) {
        cudaFuncSetAttribute(k_step3d7_bulk<FLAGS>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBudget);
        done.store(1, std::memory_order_release);
    }
}

}  // namespace

int bulk_wait_selftest(int spin_limit, cudaStream_t st) {
    int* out = nullptr;
    if (cudaGetSymbolAddress((void**)&out, g_selftest_out) != cudaSuccess) return CMCG_ERR_CUDA;
    note_launch(1);
    k_bulk_wait_selftest<<<1, 32, 0, st>>>(spin_limit, out);
    int h = 0;
    if (cudaMemcpyAsync(&h, out, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return CMCG_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return CMCG_ERR_CUDA;
    return h;
}

int step_bulk_smem(int sx, int ty) {
    const int cur_cap = round4((ty + 2) * sx + 8), p_cap = round4(ty * sx + 8);
    return kBarBytes + 4 * (kNC * cur_cap + 2 * kNP * p_cap);
}

bool step_bulk_plan(const Geom& g, int ty_req, int zc_req, int* ty, int* zc) {
    if (g.dim != 3 || g.sz < 2 || g.sy < 2) return false;
    int t = ty_req;
    if (t <= 0) {
        t = 0;
        for (int c : {8, 6, 4, 3, 2})
            if (step_bulk_smem(g.sx, c) <= kSmemBudget) {
                t = c;
                break;
            }
        if (t == 0) return false;
    }
    if (t < 1 || step_bulk_smem(g.sx, t) > kSmemBudget) return false;
    int z = zc_req;
    if (z <= 0) {
        // one wave: bands x z-chunks close to the resident CTA count (two per SM)
        const int bands = (g.sy + t - 1) / t;
        const int resident = 2 * num_sms();
        const int chunks = std::max(1, resident / bands);
        z = (g.sz + chunks - 1) / chunks;
        if (z < 2) z = 2;
    }
    *ty = t;
    *zc = z;
    return true;
}

void launch_step_bulk(const Geom& g, const float* cur, float* prev, const float* kap, int flags, int ty, int zc,
                      double* sc, cudaStream_t st) {
    note_launch(1);
    const int cur_cap = round4((ty + 2) * g.sx + 8), p_cap = round4(ty * g.sx + 8);
    const int smem = step_bulk_smem(g.sx, ty);
    const dim3 grid((unsigned)((g.sy + ty - 1) / ty), (unsigned)((g.sz + zc - 1) / zc));
    switch (flags) {
        case 0:
            set_smem_attr<0>();
            k_step3d7_bulk<0><<<grid, kBT, smem, st>>>(cur, prev, kap, g, ty, zc, cur_cap, p_cap, sc);
            break;
        case kStepPrevScaled:
            set_smem_attr<kStepPrevScaled>();
            k_step3d7_bulk<kStepPrevScaled><<<grid, kBT, smem, st>>>(cur, prev, kap, g, ty, zc, cur_cap, p_cap, sc);
            break;
        case kStepNoDiv:
            set_smem_attr<kStepNoDiv>();
            k_step3d7_bulk<kStepNoDiv><<<grid, kBT, smem, st>>>(cur, prev, kap, g, ty, zc, cur_cap, p_cap, sc);
            break;
        case kStepPrevScaled | kStepNoDiv:
            set_smem_attr<kStepPrevScaled | kStepNoDiv>();
            k_step3d7_bulk<kStepPrevScaled | kStepNoDiv>
                <<<grid, kBT, smem, st>>>(cur, prev, kap, g, ty, zc, cur_cap, p_cap, sc);
            break;
        default:
            break;
    }
}

}  // namespace cmcg
