// incremental.cuh -- sweep path with the field kept at every site (internal).
#pragma once

#include "internal.cuh"

namespace dipmc {

struct IncrConfig {
    int L, l, R;
    uint2 key;
    uint32_t t0;          // sweep counter of the launch's first sweep
    int nsweeps;          // sweeps of this launch
    int it0;              // index of the launch's first sweep within the call
    int nsweeps_call;     // sweeps of the call (trace stride)
    int measure_every;
    int proposal;
    float cap_c1;
    int schedule;
};

struct IncrBuffers {
    const float *W32 = nullptr;          // [4][N]
    float *spins = nullptr;              // [R][3][N]
    const float *field = nullptr;        // [R][3][N]: the field of the spins at the launch's start
    const RepParams *params = nullptr;   // [R]
    double *energy = nullptr;            // [R]: energy of the last measured sweep
    ObsAcc *obs = nullptr;
    double *theta2 = nullptr;
    float *trace = nullptr;
    EnergyHist hist;
};

bool incremental_supported(int L, int l);
cudaError_t launch_sweep_incremental(const IncrConfig &c, const IncrBuffers &b, cudaStream_t st);

}  // namespace dipmc
