// energy_noalloc.cu -- total energy of caller-provided spin states, computed
// without allocating any device memory.
//
// Who needs this: callers that cannot call cudaMalloc.  Examples are code that
// runs under a device-memory budget owned by someone else (a framework's
// caching allocator or a serving process that reserves all device memory up
// front and hands out slices of it), and latency-critical loops where a
// cudaMalloc/cudaFree would synchronise the device.  Such callers own their
// input and output buffers and cannot give the library a workspace.
//
// The field scratch that mc_energy keeps in its lattice handle lives here in a
// file-scope device array of fixed size instead.  Every GPU that loads the
// library holds this array until the process exits.
#include <cstdio>
#include <mutex>

#include "internal.cuh"

namespace dipmc {

namespace {

// Capacity of the field scratch: R * 3 * L * L FP32 values (4 MiB).
constexpr size_t kScratchFloats = size_t(1) << 20;
// The field kernel runs one grid row per state (gridDim.y), at most 65535 rows.
constexpr int kMaxStates = 65535;

static __device__ __align__(256) float g_field_scratch[kScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
float *g_scratch_addr[kMaxDevices] = {};  // device address of g_field_scratch, per device

// The energy sums of the lattice handles' energy kernel (cta_replica_energy),
// reading the couplings as [R][4] = (J, C_D, K2, K4).
__global__ void __launch_bounds__(256) k_energy_couplings(int L, const float *__restrict__ spins,
                                                          const float *__restrict__ h,
                                                          const float *__restrict__ couplings,
                                                          double *E) {
    const int N = L * L, r = blockIdx.x;
    const float *c = couplings + 4 * (size_t)r;
    const double e = cta_replica_energy(L, spins + (size_t)r * 3 * N, h + (size_t)r * 3 * N, c[0], c[1], c[2], c[3]);
    if (threadIdx.x == 0) E[r] = e;
}

}  // namespace
}  // namespace dipmc

using namespace dipmc;

extern "C" int mc_energy_noalloc(int L, int R, const float *W32, const float *spins,
                                 const float *couplings, double *energy, void *stream) {
    if (L < 2 || L > 4096)
        return set_last_error(MC_EINVAL, "mc_energy_noalloc: need 2 <= L <= 4096");
    if (R < 1 || R > kMaxStates)
        return set_last_error(MC_EINVAL, "mc_energy_noalloc: need 1 <= R <= 65535 (one grid row per state)");
    if (!W32 || !spins || !couplings || !energy)
        return set_last_error(MC_EINVAL, "mc_energy_noalloc: null buffer");
    const size_t need = (size_t)R * 3 * (size_t)L * (size_t)L;
    if (need > kScratchFloats) {
        char msg[256];
        snprintf(msg, sizeof msg,
                 "mc_energy_noalloc: R*3*L*L = %zu field values exceed the fixed scratch of %zu "
                 "(4 MiB); pass at most %zu replicas of this L per call",
                 need, kScratchFloats, kScratchFloats / (3 * (size_t)L * (size_t)L));
        return set_last_error(MC_EINVAL, msg);
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_last_error(MC_ECUDA, "mc_energy_noalloc: cudaGetDevice failed");
    if (dev < 0 || dev >= kMaxDevices) return set_last_error(MC_EINVAL, "mc_energy_noalloc: device index too large");
    float *scratch = nullptr;
    {
        // First call on this device: look up the array's device address (host
        // code cannot use the symbol itself).
        std::lock_guard<std::mutex> lock(g_setup_mu);
        if (!g_scratch_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_field_scratch);
            if (e != cudaSuccess) {
                char msg[256];
                snprintf(msg, sizeof msg, "mc_energy_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
                return set_last_error(MC_ECUDA, msg);
            }
            g_scratch_addr[dev] = static_cast<float *>(p);
        }
        scratch = g_scratch_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    // The field kernel writes every one of the R*3*L*L values before the energy
    // kernel reads them, so nothing left by an earlier call is ever read.
    e = launch_full_field(L, R, W32, spins, scratch, st);
    if (e != cudaSuccess) return set_last_error(MC_ECUDA, "mc_energy_noalloc: field kernel launch failed");
    k_energy_couplings<<<R, 256, 0, st>>>(L, spins, scratch, couplings, energy);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_last_error(MC_ECUDA, "mc_energy_noalloc: energy kernel launch failed");
    return MC_OK;
}
