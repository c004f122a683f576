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
    int L, Sw, R, NT, tmem_cols;
    // spec2 = 1 (L = 2l, S_w = 256): the operands are the sub-lattice spectra of
    // the window's offsets instead of the Toeplitz rows of its sites -- rows
    // (kappa, b, j) for the 4 frequencies kappa of the 2 x 2 cell grid, output
    // component b and window offset j; K = (a, e') over the l^2 cell offsets; wsh
    // holds the signed doubled spectra of W~ (tc_t2_elems) and spins_hi/lo the
    // spin spectra [R][kappa][a][e'] (launch_spec2_init).
    int spec2;
    const TcUnit *units;                 // [nunits]
    // the window's sites (computed in the kernel): sub-steps k0 .. k0 + Sw/n - 1 of sweep
    // t (t_dev[0] + it when t_dev is set, else t_host) under the given schedule
    int l, schedule, it, k0;
    uint2 key;
    uint32_t t_host;
    const uint32_t *t_dev;
    const __nv_bfloat16 *wsh;            // tc_wsh_elems(L): shifted hi/lo copies of W~
    const __nv_bfloat16 *spins_hi;       // [R][3][N]
    const __nv_bfloat16 *spins_lo;       // [R][3][N]
    int *error;                          // set to 1 if a bounded wait gave up, 2 if the stages are misaligned
    float *part;                         // [nunits][NT][128]: each unit's partial tile, row fastest
    const int *tile_first;               // [ntiles * mtiles + 1]: first unit of tile (nt, mt)
    int mtiles, ntiles;
};

size_t tc_wsh_elems(int L);
// Spectral operand mode (L = 2l, l % 8 == 0, a 256- or 512-site window).
bool tc_spec2_supported(int L, int l, int Sw);
size_t tc_t2_elems(int l);
// t2[c][kappa][comp][sy][hl][dy][i]: bf16 hi/lo of the signed, doubled spectrum of W~
// (see tc_field.cu), shifted by c = 0..7 along i.
cudaError_t launch_build_t2(int L, const double *W64, __nv_bfloat16 *t2, cudaStream_t st);
// Spin spectra S'[r][kappa][a][e'] of every cell offset, bf16 hi/lo.
cudaError_t launch_spec2_init(int L, int R, const float *spins, __nv_bfloat16 *hi, __nv_bfloat16 *lo, cudaStream_t st);
bool tc_supported(int L, int l, int B);
size_t tc_smem_bytes();
cudaError_t launch_build_wsh(int L, const double *W64, __nv_bfloat16 *wsh, cudaStream_t st);
// Fills units[] for a window of Sw sites and R replicas; returns the number of
// units (CTAs) or -1 if max_units is too small.
// Work plan: units ordered by (N-tile, M-tile, K range); tile_first (host,
// ntiles * mtiles + 1 entries) gets the first unit of each tile.
// kblocks > 0 fixes the K-blocks per unit (else the fewest whose units fit one wave);
// ntile > 0 caps the replicas per N-tile (a multiple of 16, at most 256).
int tc_plan(int L, int Sw, int R, int nsm, TcUnit *units, int max_units, int *NT, int *tmem_cols,
            int *tile_first, int *mtiles, int *ntiles, bool spec2 = false, int kblocks = 0, int ntile = 0);
// TMA maps of the bf16 spin arrays (opaque 64-byte-aligned buffers of tc_map_bytes()).
size_t tc_map_bytes();
int tc_encode_map(void *map, const __nv_bfloat16 *spins, int L, int R, int NT);
cudaError_t launch_tc_field(const TcFieldArgs &a, int nunits, const void *map_hi, const void *map_lo, cudaStream_t st);

}  // namespace dipmc
