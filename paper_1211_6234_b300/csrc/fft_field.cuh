// fft_field.cuh -- declarations of the FFT field and the FFT sweep path (fft_field.cu).
#pragma once

#include "internal.cuh"

namespace dipmc {

struct FftStepConfig {
    int L, l, R;
    uint2 key;
    uint32_t t;          // sweep counter (when t_dev is null)
    const uint32_t *t_dev;  // device sweep counter at the start of the call (graph replays)
    int k;               // sub-step within the sweep
    int it;              // sweep index within the call (trace position)
    int nsweeps_call;    // sweeps of the call (trace stride)
    int proposal;
    float cap_c1;
    int schedule;
};

struct FftStepBuffers {
    const float *W32;          // [4][N]
    float *spins;              // [R][3][N]
    const float *field;        // [R][3][N], field of the state before the sub-step
    const RepParams *params;   // [R]
    ObsAcc *obs;               // [R] (accepted count)
    float *trace;              // optional
    const SlotState *slots;    // optional [R]: packed launch (per-replica key, counter, sweeps)
};

bool fft_supported(int L);
size_t fft_scratch_bytes(int L, int R);
cudaError_t launch_build_what(int L, const double *W64, float *What, cudaStream_t st);
// Full field of all R replicas into field[R][3][N]; scratch holds fft_scratch_bytes.
cudaError_t launch_fft_field(int L, int R, const float *spins, const float *What, float2 *scratch, float *field,
                             cudaStream_t st);
cudaError_t launch_fft_update(const FftStepConfig &c, const FftStepBuffers &b, cudaStream_t st);
// Observables of every replica; with slots, only replicas whose own sweep count
// (t0 + it + 1) is a multiple of measure_every and that are active at sweep `it`.
cudaError_t launch_fft_observe(int L, int R, const float *spins, const float *field, const RepParams *P,
                               double *energy, ObsAcc *obs, double *theta2, const SlotState *slots, int it,
                               int measure_every, const EnergyHist &hist, cudaStream_t st);
// attempted += add for every replica; with slots, += min(nsweeps_call, slot sweeps) * N.
cudaError_t launch_add_attempted(ObsAcc *obs, int R, long long add, const SlotState *slots, int nsweeps_call,
                                 long long N, cudaStream_t st);

}  // namespace dipmc
