// Two leapfrog steps per launch (temporal blocking, depth 2): 3D 7-point, FP32, homogeneous
// steps of Eq. WE (Sec. 4.3.1), (A = y^{n-1}, B = y^n) -> (C = y^{n+1}, D = y^{n+2}).
//
// A block owns the interior tile [tx TX, tx TX + TX) x [ty TY, ty TY + TY) of every plane of
// its z-chunk [z0, z1) and marches z.  Its columns are the tile plus a 2-node halo, at most
// kPairCols per thread (column i = thread + r * kPairThreads, x fastest); a column outside the
// grid holds its mirror node's values (ghost-point Neumann), so the stencil needs no face test.
// Operands are staged in shared memory by per-thread asynchronous copies (cp.async, 4 bytes:
// the columns of a tile row need not be 16-byte aligned) P planes ahead of their use, in rings
//   rY: y^n on the 2-halo region, P + 2 planes;  rA, rK: y^{n-1} and kappa on the 1-halo
//   region, P + 1 planes each,
// and the first step's result goes to sL[k & 1], y^{n+1}(k) on the 1-halo region (computed
// redundantly on the halo ring with the mirror node's coefficients there, so that it equals
// the mirror value).  Iteration k: wait for this thread's copies of plane k, one __syncthreads
// (every thread's copies are visible and every thread is done with iteration k - 1, whose
// ring slots are free), issue the copies of plane k + P (y^n: k + 1 + P) into those slots,
// compute y^{n+1}(k) on the 1-halo region and y^{n+2}(k - 1) on the interior.  The z-neighbours
// y^n(k - 1), y^n(k) and y^{n+1}(k - 2 .. k) of a column stay in its thread's registers.
// Every value is the one-step update, the same expression in the same order as the one-step
// kernels, applied twice.  Outputs go to two further buffers, because neighbouring blocks
// still read the inputs on their halos.  DRAM traffic per node: read y^{n-1}, y^n, kappa,
// write y^{n+1}, y^{n+2}: 20 B for two updates against 32 B for two single steps.  No wait
// spins: cp.async.wait_group and __syncthreads complete by themselves.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace cmcg {

namespace {

constexpr int kPairThreads = 256;
constexpr int kPairCols = 4;                          // columns per thread
constexpr int kPairArea = kPairThreads * kPairCols;   // 2-halo region, columns

__device__ __forceinline__ int mirror_ix(int i, int n) { return i < 0 ? -i : (i > n ? 2 * n - i : i); }

__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// One homogeneous leapfrog update (FP32): y^{n+1} = [2 y^n - (1 - beta) y^{n-1} - kappa Lt y^n] / (1 + beta).
__device__ __forceinline__ float leap(float yc, float lap, float kk, float yp, int nb) {
    const float rhs = 2.f * yc - kk * lap;
    if (nb == 0) return rhs - yp;
    const float beta = (float)nb * sqrtf(kk);
    return (rhs - (1.f - beta) * yp) / (1.f + beta);
}

template <int P>
constexpr size_t pair_smem_bytes() {
    return sizeof(float) * (size_t)kPairArea * ((P + 2) + 2 * (P + 1) + 2);
}

template <int P>
__global__ void __launch_bounds__(kPairThreads)
    k_step3d7_pair(const float* __restrict__ A, const float* __restrict__ B, const float* __restrict__ kap,
                   float* __restrict__ C, float* __restrict__ D, Geom g, int TX, int TY, int tiles_x, int zc) {
    constexpr int RY = P + 2, RA = P + 1, RK = P + 1;
    extern __shared__ __align__(16) float smem[];
    float* rY = smem;
    float* rA = rY + RY * kPairArea;
    float* rK = rA + RA * kPairArea;
    float* sL = rK + RK * kPairArea;
    const int W = TX + 4, H = TY + 4;
    const int tyi = blockIdx.x / tiles_x, txi = blockIdx.x - tyi * tiles_x;
    const int gx0 = txi * TX - 2, gy0 = tyi * TY - 2;  // origin of the 2-halo region
    const int z0 = blockIdx.y * zc, z1 = min(z0 + zc, g.sz);
    const int nz = g.nz;
    const long long sxy = (long long)g.sx * g.sy;
    const int tid = threadIdx.x;
    if (!CMCG_RANGE_OK(z0, z1 - 1, g.sz, kSitePairGlobal)) return;  // uniform over the block

    // Column r of this thread: in-plane offset of its (mirror) node, -1 outside the region;
    // role bit 0: 1-halo region (computes y^{n+1}), bit 1: interior (computes y^{n+2}, stores);
    // bits 2..4: absorbing xy faces through the node.
    int ph[kPairCols], role[kPairCols];
#pragma unroll
    for (int r = 0; r < kPairCols; ++r) {
        const int i = tid + r * kPairThreads;
        ph[r] = -1;
        role[r] = 0;
        const int ly = i / W, lx = i - ly * W;
        const int gx = gx0 + lx, gy = gy0 + ly;
        if (i < W * H && gx <= g.nx + 2 && gy <= g.ny + 2) {
            const int px = mirror_ix(gx, g.nx), py = mirror_ix(gy, g.ny);
            ph[r] = px + g.sx * py;
            const bool h1 = lx >= 1 && ly >= 1 && lx <= W - 2 && ly <= H - 2 && gx <= g.nx + 1 && gy <= g.ny + 1;
            const bool in = lx >= 2 && ly >= 2 && lx <= W - 3 && ly <= H - 3 && gx <= g.nx && gy <= g.ny;
            const int nb = ((px == 0) & (int)(g.abc & 1u)) + ((px == g.nx) & (int)((g.abc >> 1) & 1u)) +
                           ((py == 0) & (int)((g.abc >> 2) & 1u)) + ((py == g.ny) & (int)((g.abc >> 3) & 1u));
            role[r] = (h1 ? 1 : 0) | (in ? 2 : 0) | (nb << 2);
            // checked build: the node lies in its plane, and a first-step column's neighbours
            // lie in the staged region
            if (!CMCG_RANGE_OK(ph[r], ph[r], sxy, kSitePairGlobal) ||
                ((role[r] & 1) && !CMCG_RANGE_OK(i - W, i + W, W * H, kSitePairShared))) {
                ph[r] = -1;
                role[r] = 0;
            }
        }
    }
    const int zabc0 = (int)((g.abc >> 4) & 1u), zabc1 = (int)((g.abc >> 5) & 1u);
    // y^{n+1} is needed on planes z0-1 .. z1 (mirrored at the faces), so y^n on z0-2 .. z1+1
    const int kb = max(z0 - 1, 0), ke = min(z1, nz);

    // copies of y^n plane py (virtual index, mirrored) and of y^{n-1}, kappa plane pa, where needed
    auto stage_y = [&](int py) {
        if (py > ke + 1) return;
        const float* src = B + (long long)mirror_ix(py, nz) * sxy;
        float* dst = rY + (py % RY) * kPairArea + tid;
#pragma unroll
        for (int r = 0; r < kPairCols; ++r)
            if (ph[r] >= 0) cp_async4(dst + r * kPairThreads, src + ph[r]);
    };
    auto stage_ak = [&](int pa) {
        if (pa > ke) return;
        const long long o = (long long)pa * sxy;
        float* da = rA + (pa % RA) * kPairArea + tid;
        float* dk = rK + (pa % RK) * kPairArea + tid;
#pragma unroll
        for (int r = 0; r < kPairCols; ++r) {
            if (role[r] & 1) {
                cp_async4(da + r * kPairThreads, A + o + ph[r]);
                cp_async4(dk + r * kPairThreads, kap + o + ph[r]);
            }
        }
    };
    // prologue: the groups of the virtual iterations kb - P .. kb - 1 (the first also stages y^n(kb))
    stage_y(kb);
#pragma unroll
    for (int v = 0; v < P; ++v) {
        stage_y(kb + 1 + v);
        stage_ak(kb + v);
        cp_commit();
    }
    // z-neighbours of the 1-halo columns: y^n(kb - 1) (mirrored) and y^n(kb), read directly
    float ym[kPairCols], yc[kPairCols], kq[kPairCols], lm[kPairCols], lc[kPairCols];
    {
        const float* Bm = B + (long long)mirror_ix(kb - 1, nz) * sxy;
        const float* Bc = B + (long long)kb * sxy;
#pragma unroll
        for (int r = 0; r < kPairCols; ++r) {
            ym[r] = yc[r] = kq[r] = lm[r] = lc[r] = 0.f;
            if (role[r] & 1) {
                ym[r] = __ldg(Bm + ph[r]);
                yc[r] = __ldg(Bc + ph[r]);
            }
        }
    }
    for (int k = kb; k <= z1; ++k) {
        cp_wait<P - 1>();
        __syncthreads();
        stage_y(k + 1 + P);
        stage_ak(k + P);
        cp_commit();
        float ln[kPairCols], kk[kPairCols], yn[kPairCols];
#pragma unroll
        for (int r = 0; r < kPairCols; ++r) ln[r] = kk[r] = yn[r] = 0.f;
        if (k <= ke) {  // first step: y^{n+1}(k) on the 1-halo region
            const int nbz = ((k == 0) & zabc0) + ((k == nz) & zabc1);
            const bool own = k >= z0 && k < z1;
            const float* Yk = rY + (k % RY) * kPairArea;
            const float* Yn = rY + ((k + 1) % RY) * kPairArea;
            const float* Ak = rA + (k % RA) * kPairArea;
            const float* Kk = rK + (k % RK) * kPairArea;
            float* Lk = sL + (k & 1) * kPairArea;
            const long long ok = (long long)k * sxy;
#pragma unroll
            for (int r = 0; r < kPairCols; ++r) {
                if (!(role[r] & 1)) continue;
                const int i = tid + r * kPairThreads;
                yn[r] = Yn[i];
                kk[r] = Kk[i];
                const float sxy_ = (Yk[i - 1] + Yk[i + 1]) + (Yk[i - W] + Yk[i + W]);
                const float lap = 6.f * yc[r] - (sxy_ + (ym[r] + yn[r]));
                ln[r] = leap(yc[r], lap, kk[r], Ak[i], (role[r] >> 2) + nbz);
                Lk[i] = ln[r];
                if (own && (role[r] & 2)) C[ok + ph[r]] = ln[r];
            }
        }
        const int q = k - 1;
        if (q >= z0) {  // second step: y^{n+2}(q) on the interior (q < z1 since k <= z1)
            const int nbz = ((q == 0) & zabc0) + ((q == nz) & zabc1);
            const float* Lq = sL + (q & 1) * kPairArea;
            const long long oq = (long long)q * sxy;
#pragma unroll
            for (int r = 0; r < kPairCols; ++r) {
                if (!(role[r] & 2)) continue;
                const int i = tid + r * kPairThreads;
                const float below = q == 0 ? ln[r] : lm[r];  // mirror of plane 1 at the bottom face
                const float above = k > nz ? lm[r] : ln[r];  // mirror of plane nz - 1 at the top face
                const float sxy_ = (Lq[i - 1] + Lq[i + 1]) + (Lq[i - W] + Lq[i + W]);
                const float lap = 6.f * lc[r] - (sxy_ + (below + above));
                D[oq + ph[r]] = leap(lc[r], lap, kq[r], ym[r], (role[r] >> 2) + nbz);
            }
        }
#pragma unroll
        for (int r = 0; r < kPairCols; ++r) {
            ym[r] = yc[r];
            yc[r] = yn[r];
            kq[r] = kk[r];
            lm[r] = lc[r];
            lc[r] = ln[r];
        }
    }
    cp_wait<0>();  // leave no copy in flight
}

struct PairShape {
    int TX, TY, tiles_x, tiles_y, zc, chunks;
};

template <int P>
void pair_smem_limit() {  // the attribute belongs to the function on the current device
    static bool done = false;
    if (!done) {
        cudaFuncSetAttribute(k_step3d7_pair<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pair_smem_bytes<P>());
        cudaGetLastError();
        done = true;
    }
}

// Tile: the interior TX x TY with (TX + 4)(TY + 4) <= kPairArea that needs the fewest tiles
// (ty_req > 0 fixes TY).  z-chunk: zc_req > 0, else 16 planes, the fastest of 16, 32, 64 and
// one wave of resident blocks (52) on a 257^3 grid.
PairShape pair_shape(const Geom& g, int zc_req, int ty_req) {
    PairShape s{};
    long long best = -1;
    if (ty_req > 60) ty_req = 60;
    const int ty_lo = ty_req > 0 ? ty_req : 4, ty_hi = ty_req > 0 ? ty_req : 60;
    for (int ty = ty_lo; ty <= ty_hi; ++ty) {
        const int tx = kPairArea / (ty + 4) - 4;
        if (tx < 1) continue;
        const long long tiles = (long long)((g.sx + tx - 1) / tx) * ((g.sy + ty - 1) / ty);
        if (best < 0 || tiles < best || (tiles == best && tx > s.TX)) {
            best = tiles;
            s.TX = tx;
            s.TY = ty;
        }
    }
    s.tiles_x = (g.sx + s.TX - 1) / s.TX;
    s.tiles_y = (g.sy + s.TY - 1) / s.TY;
    const int zc = zc_req > 0 ? zc_req : 16;
    s.zc = std::max(1, std::min(zc, g.sz));
    s.chunks = (g.sz + s.zc - 1) / s.zc;
    return s;
}

template <int P>
void launch_pair(const Geom& g, const float* A, const float* B, const float* kap, float* C, float* D, int zc, int ty,
                 cudaStream_t st) {
    pair_smem_limit<P>();
    const PairShape s = pair_shape(g, zc, ty);
    const dim3 grid((unsigned)(s.tiles_x * s.tiles_y), (unsigned)s.chunks);
    k_step3d7_pair<P><<<grid, kPairThreads, pair_smem_bytes<P>(), st>>>(A, B, kap, C, D, g, s.TX, s.TY, s.tiles_x,
                                                                          s.zc);
}

}  // namespace

bool step2_supported(const Geom& g, int order) {
    return g.dim == 3 && order == 2 && g.nx >= 2 && g.ny >= 2 && g.nz >= 2;
}

void launch_step2(const Geom& g, const float* A, const float* B, const float* kap, float* C, float* D, int zc,
                  int ty, int depth, cudaStream_t st) {
    note_launch(1);
    if (depth == 1)
        launch_pair<1>(g, A, B, kap, C, D, zc, ty, st);
    else if (depth == 3)
        launch_pair<3>(g, A, B, kap, C, D, zc, ty, st);
    else
        launch_pair<2>(g, A, B, kap, C, D, zc, ty, st);
}

}  // namespace cmcg

namespace cmcg {
CMCG_CHECK_TU(pair)
}  // namespace cmcg
