// cmcg_wave_period_static: one FP64 wave period that allocates nothing.
//
// Some callers cannot call cudaMalloc: a plug-in running inside a host application that owns
// the whole device-memory budget, or a real-time loop that must not take cudaMalloc's
// implicit device-wide synchronisation.  They still pass inputs and outputs; the period's
// scratch (coefficients, source, the two leapfrog buffers, masked initial data, reduction
// slots) lives in the file-scope device array below, of fixed size.
#include <mutex>

#include "cmcg.h"
#include "common.cuh"

namespace cmcg {
int wave_period_in_scratch(const cmcg_grid* grid, const double* c, double omega, const cmcg_bc* bc,
                           double dt_target, const double* u0, const double* v0, const double* f, const double* g,
                           double* uT, double* vT, char* scratch, size_t scratch_bytes, cudaStream_t st);
}

namespace {

constexpr long long kStaticMaxNodes = 1ll << 18;  // 262,144 nodes
constexpr size_t kStaticBytes = (size_t)18 << 20;  // 18 MiB: 65 B per node + reduction slots
constexpr int kMaxDevices = 64;

// Shared by every call on a device; holds the last call's contents.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

}  // namespace

extern "C" int cmcg_wave_period_static(const cmcg_grid* grid, const double* c, double omega, const cmcg_bc* bc,
                                       double dt, const double* u0, const double* v0, const double* f,
                                       const double* g, double* uT, double* vT, void* stream) {
    if (!grid || grid->dim < 2 || grid->dim > 3) return CMCG_ERR_INVALID_ARG;
    long long np = 1;
    for (int a = 0; a < grid->dim; ++a) {
        if (grid->n[a] < 2 || grid->n[a] > (1 << 20)) return CMCG_ERR_INVALID_ARG;
        np *= (long long)(grid->n[a] + 1);
    }
    if (np > kStaticMaxNodes) return CMCG_ERR_WORKSPACE;  // larger than the static scratch
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CMCG_ERR_CUDA;
    void* base = nullptr;
    {
        // once per device, with that device current: the device address of the array (a host
        // reference to g_static_scratch is only a host-side stand-in)
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return CMCG_ERR_CUDA;
            g_scratch_ptr[dev] = p;
        }
        base = g_scratch_ptr[dev];
    }
    return cmcg::wave_period_in_scratch(grid, c, omega, bc, dt, u0, v0, f, g, uT, vT, (char*)base, kStaticBytes,
                                        (cudaStream_t)stream);
}
