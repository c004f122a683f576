// spectral.cuh -- sub-lattice spectral field path (internal).
#pragma once

#include "internal.cuh"

namespace dipmc {

struct SpecConfig {
    int L, l, R;
    uint2 key;
    uint32_t t;             // sweep counter (when t_dev is null)
    const uint32_t *t_dev;  // device sweep counter at the start of the call (graph replays)
    int k;                  // first sub-step of the window within the sweep
    int it;                 // sweep index within the call
    int nsweeps_call;       // sweeps of the call (trace stride)
    int proposal;
    float cap_c1;
    int schedule;
    int esplit;             // chunks of the cell-offset sum (partial spectra)
    int wlen;               // sub-steps of this window (<= wmax)
    int wmax;               // window capacity (Hw stride)
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
    const float2 *T = nullptr;           // [4][l^2][4][n]: transforms of the W~ sub-lattice sequences, wrap phase applied
    float2 *S = nullptr;                 // [R][l^2][3][n]: transforms of the spin sub-lattices
    float2 *Hw = nullptr;                // [esplit][R][wmax][3][n]: partial field spectra of the window's offsets
    int *off = nullptr;                  // [R][l^2]: offsets of the sweep's sub-steps (-1: idle slot)
};

bool spectral_supported(int L, int l);
// sub-steps of a window (the update keeps the window's changes of S in shared memory)
int spectral_window(int L, int l);
int spectral_esplit(int L, int l, int R, int nsm);
size_t spectral_S_elems(int L, int R);
// the window's partial field spectra: esplit x R x wmax x 3 x n
size_t spectral_part_elems(int L, int l, int R, int esplit);
// T from W~ (FP64 separable DFTs, rounded to FP32 complex): T[sg][d][c][K] =
// omega^(K.sigma) T_d^c(K) for the four wraps sigma = (sg % 2, sg / 2).
cudaError_t launch_spec_table(int L, int l, const double *W64, float2 *T, cudaStream_t st);
// S of every cell offset from the spins.
cudaError_t launch_spec_init(int L, int l, int R, const float *spins, float2 *S, cudaStream_t st);
// Offsets of all sub-steps of sweep cfg.it for every replica (once per sweep).
cudaError_t launch_spec_offsets(const SpecConfig &c, const SpecBuffers &b, cudaStream_t st);
// A window of sub-steps is launch_spec_wfield (partial field spectra of the
// window's offsets from the spectra at its start: contraction over cell offsets)
// then launch_spec_wupdate (per replica, sub-step by sub-step: the window's earlier
// changes of S added to the spectra, the inverse transform, the update and the new
// S of the updated offset).
cudaError_t launch_spec_wfield(const SpecConfig &c, const SpecBuffers &b, cudaStream_t st);
cudaError_t launch_spec_wupdate(const SpecConfig &c, const SpecBuffers &b, cudaStream_t st);

}  // namespace dipmc
