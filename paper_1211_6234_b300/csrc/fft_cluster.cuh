// fft_cluster.cuh -- declarations of the cluster-resident transform path (fft_cluster.cu).
#pragma once

#include "internal.cuh"

namespace dipmc {

// CTAs of one replica's cluster.
constexpr int kClusterCtas = 16;

struct ClusterSweepArgs {
    int L, l, R;
    uint2 key;
    uint32_t t;                 // sweep counter (when t_dev is null)
    const uint32_t *t_dev;      // device sweep counter at the start of the call (graph replays)
    int it;                     // sweep index within the call (trace position)
    int nsweeps_call;           // sweeps of the call (trace stride)
    int proposal;
    float cap_c1;
    int schedule;
    const float *What;          // [4][K2][L]: real transform of W~ (xx, xy, yy, zz), kx in [0, L/2]
    const float2 *Shat;         // [R][3][K2][L]: transform of the spins at the sweep's start
    float *spins;               // [R][3][L][L]
    const float *W32;           // [4][L][L] (W~(0): self-image term)
    const RepParams *params;    // [R]
    ObsAcc *obs;                // [R] (accepted counts)
    float *trace;               // optional [R][nsweeps_call][l^2][n][MC_TRACE_W]
};

// The path serves (L, l) when L % 16 == 0, C = L / l is a power of two <= 16, the
// cluster's shared memory fits, and the device runs clusters of 16 CTAs of it.
bool cluster_supported(int L, int l);
// Device bytes of the transform buffers of R replicas (Shat and the row scratch).
size_t cluster_scratch_bytes(int L, int R);
// Real transform of W~ (FP64 sums from W64), [4][K2][L] FP32.
cudaError_t launch_cluster_what(int L, const double *W64, float *What, cudaStream_t st);
// Transform of the spins of every replica into Shat ([R][3][K2][L]); rowbuf holds
// [R][3][L][K2] complex FP32 between the row and column passes.
cudaError_t launch_cluster_transform(int L, int R, const float *spins, float2 *rowbuf, float2 *Shat, cudaStream_t st);
// One sweep of every replica (one cluster of kClusterCtas CTAs per replica).
cudaError_t launch_cluster_sweep(const ClusterSweepArgs &a, cudaStream_t st);

}  // namespace dipmc
