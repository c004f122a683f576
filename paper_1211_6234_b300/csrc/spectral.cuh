// spectral.cuh -- sub-lattice spectral field path (internal).
#pragma once

#include "internal.cuh"

namespace dipmc {

struct SpecConfig {
    int L, l, R;
    uint2 key;
    uint32_t t;             // sweep counter (when t_dev is null)
    const uint32_t *t_dev;  // device sweep counter at the start of the call (graph replays)
    int k;                  // sub-step within the sweep
    int it;                 // sweep index within the call
    int nsweeps_call;       // sweeps of the call (trace stride)
    int proposal;
    float cap_c1;
    int schedule;
    int esplit;             // chunks of the cell-offset sum (partial spectra)
    int skip_prev;          // field: leave out the previous sub-step's offset (its term comes from the update)
    int extra_in;           // update: the partial spectra have one more chunk (that term)
    int extra_out;          // update: write the next sub-step's term of the updated offset
    uint32_t mC, mn;        // ceil(2^32 / C), ceil(2^32 / n): exact x / C and x / n for x * C, x * n < 2^32
};

inline uint32_t fastdiv_magic(uint32_t d) { return (uint32_t)(((1ull << 32) + d - 1) / d); }

struct SpecBuffers {
    const float *W32 = nullptr;          // [4][N]: W~(0) for the self term
    float *spins = nullptr;              // [R][3][N]
    const RepParams *params = nullptr;   // [R]
    ObsAcc *obs = nullptr;               // [R] (accepted count)
    float *trace = nullptr;              // optional
    const SlotState *slots = nullptr;    // optional [R]: packed launch
    const float2 *T = nullptr;           // [l^2][4][n]: transforms of the W~ sub-lattice sequences
    float2 *S = nullptr;                 // [R][l^2][3][n]: transforms of the spin sub-lattices
    float2 *Hpart = nullptr;             // [esplit + 1][R][3][n]: partial field spectra of this sub-step
    float2 *Hnext = nullptr;             // the same for the next sub-step (double buffer)
    int *off = nullptr;                  // [R][l^2]: offsets of the sweep's sub-steps (-1: idle slot)
};

bool spectral_supported(int L, int l);
int spectral_esplit(int L, int l, int R, int nsm);
size_t spectral_S_elems(int L, int R);
// both partial-spectrum buffers: 2 x (esplit + 1) x R x 3 x n
size_t spectral_part_elems(int L, int l, int R, int esplit);
// T from W~ (FP64 separable DFTs, rounded to FP32 complex).
cudaError_t launch_spec_table(int L, int l, const double *W64, float2 *T, cudaStream_t st);
// S of every cell offset from the spins.
cudaError_t launch_spec_init(int L, int l, int R, const float *spins, float2 *S, cudaStream_t st);
// Offsets of all sub-steps of sweep cfg.it for every replica (once per sweep).
cudaError_t launch_spec_offsets(const SpecConfig &c, const SpecBuffers &b, cudaStream_t st);
// One sub-step is launch_spec_field (partial field spectra at the sub-step's
// sites: contraction over cell offsets) then launch_spec_update (per replica the
// inverse transform, the update and the new S of the updated offset).
cudaError_t launch_spec_field(const SpecConfig &c, const SpecBuffers &b, cudaStream_t st);
cudaError_t launch_spec_update(const SpecConfig &c, const SpecBuffers &b, cudaStream_t st);

}  // namespace dipmc
