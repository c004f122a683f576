// tc_field.cuh -- declarations of the tensor-core window field (tc_field.cu).
#pragma once

#include <cuda_bf16.h>

#include "internal.cuh"

namespace dipmc {

// One CTA of k_tc_field: an M-tile of 128 rows (b*Sw + s), an N-tile of
// replicas, and a range of 64-wide K blocks of that tile's contraction.
struct TcUnit {
    int mtile, ntile, kb_begin, kb_end;
};

struct TcFieldArgs {
    int L, Sw, R, NT, ldh, tmem_cols;
    const TcUnit *units;                 // [nunits]
    const int *wsite;                    // [Sw] window sites
    const __nv_bfloat16 *wsh;            // tc_wsh_elems(L): shifted hi/lo copies of W~
    const __nv_bfloat16 *spins_hi;       // [R][3][N]
    const __nv_bfloat16 *spins_lo;       // [R][3][N]
    float *H0;                           // [R][ldh] (+=)
    int *error;                          // set to 1 if a bounded wait gave up
};

size_t tc_wsh_elems(int L);
bool tc_supported(int L, int l, int B);
size_t tc_smem_bytes();
cudaError_t launch_build_wsh(int L, const double *W64, __nv_bfloat16 *wsh, cudaStream_t st);
cudaError_t launch_window_sites(int L, int l, uint2 key, uint32_t t, const uint32_t *t_dev, int it, int schedule,
                                int k0, int B, int *wsite, cudaStream_t st);
// Fills units[] for a window of Sw sites and R replicas; returns the number of
// units (CTAs) or -1 if max_units is too small.
int tc_plan(int L, int Sw, int R, int nsm, TcUnit *units, int max_units, int *NT, int *tmem_cols);
cudaError_t launch_tc_field(const TcFieldArgs &a, int nunits, cudaStream_t st);

}  // namespace dipmc
