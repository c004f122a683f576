// window.cuh -- declarations of the windowed sweep (window.cu, tc_field.cu).
#pragma once

#include <cuda_bf16.h>

#include "internal.cuh"

namespace dipmc {

struct WindowConfig {
    int L, l, R;
    uint2 key;
    uint32_t t;          // sweep counter of this sweep (when t_dev is null)
    const uint32_t *t_dev;  // device sweep counter at the start of the call (graph replays)
    int it;              // index of this sweep within the call (trace position)
    int nsweeps_call;    // sweeps of the call (trace stride)
    int w;               // window index within the sweep
    int B;               // sub-steps per window (divides l^2)
    int proposal;        // 0 cap, 1 sphere
    float cap_c1;        // 1 - cos(cone)
    int schedule;        // 0 permutation, 1 draw
    int measure;         // sample observables after this window (last window of a measured sweep)
    int stale_mode;      // 0: stale = full field [R][3][N]; 2: the split-K partial tiles of the
                         // tensor-core field (part, tile_first), rows b*Sw + s
    int NT, mtiles;      // stale_mode 2: replicas per N-tile, M-tiles of 128 rows
    int layout;          // warp roles of the permutation-schedule sub-steps (mc_tuning.steps_layout):
                         // 0 decider warp 0, helpers 1..7; 1 decider warp 0, warp 4 (the
                         // decider's sub-partition partner) idle during the blocks, helpers the
                         // other six; 2 as 1, but CTAs r with (r / nsm) odd decide on warp 2
                         // (partner warp 6 idle), so that two CTAs sharing an SM decide on
                         // different sub-partitions
    int nsm;             // SMs of the device (layout 2)
    int gpc;             // replicas a CTA (1 or 2; set by launch_window_steps)
    unsigned smem_group; // shared-memory bytes of one replica (set by launch_window_steps)
};

struct WindowBuffers {
    const float *W32;             // [4][N]
    float *spins;                 // [R][3][N] FP32
    __nv_bfloat16 *spins_hi;      // [R][3][N] bf16(s) (may be null)
    __nv_bfloat16 *spins_lo;      // [R][3][N] bf16(s - hi)
    const RepParams *params;      // [R]
    double *energy;               // [R]
    ObsAcc *obs;                  // [R]
    double *theta2;               // [R][N]
    float *trace;                 // optional
    const float *stale;           // see stale_mode
    const float *part;            // stale_mode 2: [units][NT][128] partial tiles, row fastest
    const int *tile_first;        // stale_mode 2: [ntiles * mtiles + 1] first unit of tile (nt, mt)
    const float4 *wq;             // [wq_table_elems(L)]: W~ on the minimum-image quarter, (xx, xy, yy, zz),
                                  // [(L/2+1)^2]; for even L then the sub-lattice spectra of W~ for
                                  // l = L/2, [L/4+1][L/4+1][4] (wq_table_elems)
    EnergyHist hist;              // optional energy histogram
    unsigned long long *cycles;   // optional [4]: SM clock cycles summed over CTAs of the blocks, the
                                  // set-up before them and the tail after them, and the blocks run
    int *error;                   // stale_mode 2, 3: set to 3 when the set-up's bulk copy of the spins
                                  // did not complete within its bound (the replica's window is skipped)
};

size_t window_smem_bytes(int L, int Sw, int n);
// Dynamic shared memory of a sub-step CTA that still leaves room for two per SM.
constexpr size_t kWindowSmemTwoCtas = 112 * 1024;
// Dynamic shared memory of a CTA that carries two replicas' sub-steps.
constexpr size_t kWindowSmemTwoGroups = 224 * 1024;
// float4 entries of the W~ tables of the windowed path: the minimum-image quarter
// [(L/2+1)^2] and, for even L, after it the table U of the 2 x 2 sub-lattice spectra
// at l = L/2: U_d(kappa) = sum_P (-1)^(kappa.P) W~(d + l P) for 0 <= dx, dy <= l/2 and
// kappa = kx + 2 ky, entry (dy (l/2+1) + dx) * 4 + kappa.
size_t wq_table_elems(int L);
// Fills both tables from the FP32 W~ (wq holds wq_table_elems(L) entries).
cudaError_t launch_build_wq(int L, const float *W32, float4 *wq, cudaStream_t st);
cudaError_t launch_set_u32(uint32_t *dst, uint32_t v, cudaStream_t st);
bool window_supported(int L, int l, int B);
cudaError_t launch_window_steps(const WindowConfig &c, const WindowBuffers &b, cudaStream_t st);
cudaError_t launch_spins_to_bf16(size_t count, const float *s, __nv_bfloat16 *hi, __nv_bfloat16 *lo,
                                 cudaStream_t st);

}  // namespace dipmc
