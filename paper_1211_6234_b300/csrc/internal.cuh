// internal.cuh -- shared device/host definitions of libdipmc (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dipmc.h"

namespace dipmc {

// ----------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
// as 1, 2, 3", SC'11): ten rounds of two 32x32 -> 64 multiplies (words 0, 2),
// a word permutation and a Weyl key schedule.
// ----------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
#ifdef __CUDA_ARCH__
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
#else
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x, p1 = (uint64_t)0xCD9E8D57u * c.z;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
#endif
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

enum : uint32_t { kTagAttempt = 1u << 24, kTagPerm = 2u << 24, kTagDraw = 3u << 24, kTagInit = 4u << 24 };

enum : int { kPropCap = 0, kPropSphere = 1, kPropFlip = 2 };

// Uniform in [0, 1) with 24 random bits (exact in FP32).
__device__ __forceinline__ float u24f(uint32_t w) { return (float)(w >> 8) * 5.9604644775390625e-8f; }

// Feistel round function of the sweep schedule (any function gives a bijection).
__host__ __device__ __forceinline__ uint32_t feistel_f(uint32_t x, uint32_t rk) {
    uint32_t y = (x ^ rk) * 0x9E3779B1u;
    return y ^ (y >> 15);
}

// Offset index v = oy*l + ox for sub-step k of a sweep.
// kind 0: 4-round balanced Feistel permutation of [0, 4^h) (2^h >= l) keyed by the
// sweep's round keys rk, cycle-walked back into [0, l^2).
// kind 1: uniform draw per sub-step (Philox word scaled by l^2).
__host__ __device__ __forceinline__ uint32_t perm_offset(uint4 rk, int h, uint32_t ll, uint32_t k) {
    const uint32_t mask = h ? ((1u << h) - 1u) : 0u;
    uint32_t v = k;
    const uint32_t guard_max = 1u << (2 * h);
    for (uint32_t guard = 0; guard <= guard_max; ++guard) {
        uint32_t lo = v & mask, hi = (v >> h) & mask, nl;
        nl = hi ^ (feistel_f(lo, rk.x) & mask); hi = lo; lo = nl;
        nl = hi ^ (feistel_f(lo, rk.y) & mask); hi = lo; lo = nl;
        nl = hi ^ (feistel_f(lo, rk.z) & mask); hi = lo; lo = nl;
        nl = hi ^ (feistel_f(lo, rk.w) & mask); hi = lo; lo = nl;
        v = (hi << h) | lo;
        if (v < ll) return v;
    }
    return 0;  // unreachable: the walk stays in k's cycle of a bijection
}

__host__ __device__ __forceinline__ int ceil_log2_u(uint32_t v) {
    int b = 0;
    while ((1u << b) < v) ++b;
    return b;
}

// Lattice site visited by slot s of a window that starts at sub-step k0 of sweep t:
// sub-step k0 + s / n, cell s % n of the C x C grid of its offset (Sec. 3.1 update
// sites), as x | y << 16.  rk = philox({t, 0, 0, kTagPerm}, key) under the
// permutation schedule (schedule 0); the draw schedule draws the offset per sub-step.
__device__ __forceinline__ int window_site_xy(int l, int C, uint2 key, uint32_t t, int schedule, uint4 rk, int k0,
                                              int s) {
    const int n = C * C, j = s / n, d = s - j * n, k = k0 + j;
    const uint32_t ll = (uint32_t)(l * l);
    uint32_t v;
    if (schedule == 0) {
        v = perm_offset(rk, ceil_log2_u((uint32_t)l), ll, (uint32_t)k);
    } else {
        const uint4 o = philox(make_uint4(t, (uint32_t)k, 0u, kTagDraw), key);
        v = (uint32_t)(((unsigned long long)o.x * (unsigned long long)ll) >> 32);
    }
    const int qx = (int)(v % (uint32_t)l) + l * (d % C), qy = (int)(v / (uint32_t)l) + l * (d / C);
    return qx | (qy << 16);
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may start while the previous kernel of its stream drains; it
// must wait for that kernel (and, transitively, everything before it) before
// touching memory the stream's earlier kernels write.  Without the launch
// attribute both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launch with programmatic stream serialization (the kernel must call pdl_wait
// before its first access to memory that earlier work of the stream writes).
template <typename... Exp, typename... Act>
cudaError_t launch_pdl(void (*k)(Exp...), dim3 grid, int threads, size_t smem, cudaStream_t st, Act... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

// Orthonormal pair perpendicular to a unit vector n (Duff, Burgess, Christensen,
// Hery, Kensler, Liani, Villemin, "Building an orthonormal basis, revisited",
// JCGT 2017), continuous except across n_z = 0.
__device__ __forceinline__ void perp_basis_unit(float nx, float ny, float nz, float3 &b1, float3 &b2) {
    const float sign = copysignf(1.0f, nz);
    const float a = -1.0f / (sign + nz);
    const float b = nx * ny * a;
    b1 = make_float3(1.0f + sign * nx * nx * a, sign * b, -sign * nx);
    b2 = make_float3(b, sign + ny * ny * a, -ny);
}

// Proposal S for the current spin s (Sec. 3.1 proposal): kind 2 the complete
// reversal of Appendix B, kind 1 uniform on S^2 (z = 2 u1 - 1, azimuth from
// cps, sps), otherwise uniform on the cap of half-angle cone around s with
// 1 - cos(alpha) = u1 (1 - cos cone) = u1 cap_c1 (formed without cancellation),
// renormalised.
__device__ __forceinline__ float3 propose_spin(int kind, float cap_c1, float s0, float s1, float s2, float u1,
                                               float cps, float sps) {
    if (kind == kPropFlip) return make_float3(-s0, -s1, -s2);
    if (kind == kPropSphere) {
        const float z = 2.0f * u1 - 1.0f;
        const float rr = sqrtf(fmaxf(0.0f, (1.0f - z) * (1.0f + z)));
        return make_float3(rr * cps, rr * sps, z);
    }
    const float omc = u1 * cap_c1;
    const float ca = 1.0f - omc;
    const float sa = sqrtf(fmaxf(0.0f, omc * (2.0f - omc)));
    float3 b1, b2;
    perp_basis_unit(s0, s1, s2, b1, b2);
    float S0 = ca * s0 + sa * (cps * b1.x + sps * b2.x);
    float S1 = ca * s1 + sa * (cps * b1.y + sps * b2.y);
    float S2 = ca * s2 + sa * (cps * b1.z + sps * b2.z);
    const float inv = 1.0f / sqrtf(S0 * S0 + S1 * S1 + S2 * S2);
    return make_float3(S0 * inv, S1 * inv, S2 * inv);
}

// Per-replica couplings as the kernels read them.
struct RepParams {
    float J, CD, K2, K4, T;
    float pad[3];
};

constexpr int kNB = 24;  // binning levels: blocks of 2^k samples, k < kNB

// Device accumulators of one replica (FP64).
struct ObsAcc {
    double psum[MC_NOBS][kNB];  // running sum of the current block at level k
    double bsum[MC_NOBS][kNB];  // sum of completed block means
    double bsq[MC_NOBS][kNB];   // sum of squared completed block means
    long long pcnt[kNB];        // samples in the current block at level k
    long long bcnt[kNB];        // completed blocks at level k
    long long nsamples;
    long long accepted;
    long long attempted;
    long long pad;
};

// One measurement sample x into binning level k (blocks of 2^k samples): the level's
// running block sum takes x, and when the block is complete its mean (the sum times the
// exact 2^-k) joins the sums of block means and of their squares.  Levels are
// independent, so kNB threads may push one level each; k == 0 also counts the sample.
__device__ __forceinline__ void obs_push_level(ObsAcc &A, const double x[MC_NOBS], int k) {
    const long long pc = A.pcnt[k] + 1;
    const bool done = pc == (1LL << k);
    const double inv = __longlong_as_double((long long)(1023 - k) << 52);   // 2^-k
    double ps[MC_NOBS], bs[MC_NOBS], bq[MC_NOBS];
#pragma unroll
    for (int o = 0; o < MC_NOBS; ++o) {   // the loads of the level first, so they overlap
        ps[o] = A.psum[o][k];
        bs[o] = A.bsum[o][k];
        bq[o] = A.bsq[o][k];
    }
#pragma unroll
    for (int o = 0; o < MC_NOBS; ++o) {
        const double p = ps[o] + x[o];
        if (done) {
            const double mean = p * inv;
            A.bsum[o][k] = bs[o] + mean;
            A.bsq[o][k] = bq[o] + mean * mean;
            A.psum[o][k] = 0.0;
        } else {
            A.psum[o][k] = p;
        }
    }
    if (done) {
        A.bcnt[k] += 1;
        A.pcnt[k] = 0;
    } else {
        A.pcnt[k] = pc;
    }
    if (k == 0) A.nsamples += 1;
}

// The same sample into every level, by one thread: the arithmetic of obs_push_level
// element by element (no staged loads, so the one thread holds few registers).
__device__ __forceinline__ void obs_push(ObsAcc &A, const double x[MC_NOBS]) {
    A.nsamples += 1;
#pragma unroll 1
    for (int k = 0; k < kNB; ++k) {
        A.pcnt[k] += 1;
        const bool done = A.pcnt[k] == (1LL << k);
        const double inv = 1.0 / (double)(1LL << k);
        for (int o = 0; o < MC_NOBS; ++o) {
            A.psum[o][k] += x[o];
            if (done) {
                const double mean = A.psum[o][k] * inv;
                A.bsum[o][k] += mean;
                A.bsq[o][k] += mean * mean;
                A.psum[o][k] = 0.0;
            }
        }
        if (done) {
            A.bcnt[k] += 1;
            A.pcnt[k] = 0;
        }
    }
}

struct SweepConfig {
    int L, l, R;
    uint2 key;
    uint32_t t0;
    int nsweeps;
    int measure_every;
    int proposal;     // 0 cap, 1 sphere
    float cap_c1;     // 1 - cos(cone)
    int schedule;     // 0 permutation, 1 draw
};

// Sec. 4.1 stripe observables of one state from per-component wall counts
// n_h[a] = sum_i 1 - sgn(s_i^a s_{i+x}^a), n_v[a] (i+y), and sum_i |theta_i - pi/2|.
__device__ __forceinline__ float wall_term(float a, float b) {
    const float p = a * b;
    return 1.0f - (p > 0.0f ? 1.0f : (p < 0.0f ? -1.0f : 0.0f));
}

__device__ __forceinline__ void stripe_obs(double x[MC_NOBS], const double nh[3], const double nv[3], double cone,
                                           int N) {
    x[MC_OBS_WALL] = (nv[2] + nh[2]) / (4.0 * N);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double sum = nh[c] + nv[c];
        x[MC_OBS_OX + c] = sum > 0.0 ? fabs(nh[c] - nv[c]) / sum : 0.0;
    }
    x[MC_OBS_CONE] = 0.63661977236758134 * cone / N;   // 2/pi
}

// Histogram of E/N per replica: counts[R][nbins] over [lo, lo + nbins / scale).
struct EnergyHist {
    unsigned long long *counts = nullptr;
    double lo = 0.0, scale = 0.0;
    int nbins = 0;
};

__device__ __forceinline__ void hist_push(const EnergyHist &h, int r, double e) {
    if (!h.counts) return;
    const double b = (e - h.lo) * h.scale;
    if (b >= 0.0 && b < (double)h.nbins) atomicAdd(h.counts + (size_t)r * h.nbins + (int)b, 1ULL);
}

// Per-replica stream state of a packed launch: independent requests share one
// launch, each replica slot with its own Philox key, its own sweep counter t0,
// the replica index its counters use, and how many of the launch's sweeps it
// takes (0 = idle slot, left untouched).
struct SlotState {
    uint32_t key_lo, key_hi;
    uint32_t t0;
    int32_t nsweeps;
    uint32_t rid;
    uint32_t pad[3];
};

// One CTA of a grouped direct launch: lattices of different L (with the same
// C = L / l) share one launch, each CTA carrying its own geometry, stream state
// and buffers.  nft and nt are the field threads and the threads of the launch
// the replica would have on its own handle, so that the CTA's arithmetic (which
// cell offsets each thread sums, the order of every reduction) is the lone one.
struct SlotGeom {
    int L, l;
    int nft;                    // field threads of the lone launch: cell offset e = ftid + j * nft
    int nt;                     // threads of the lone launch: stride of the observable sums
    uint32_t key_lo, key_hi;    // Philox key
    uint32_t t0;                // sweep counter at the start of the launch
    uint32_t rid;               // replica index of the counters
    int nsweeps;                // sweeps of this CTA (<= the launch's)
    uint32_t mphase;            // observables after sweep it of the launch when (mphase + it + 1) % measure_every == 0
    const float *W32;           // [4][L*L]
    float *spins;               // [3][L*L] of this replica
    const RepParams *params;    // this replica's couplings
    double *energy;             // its tracked energy
    ObsAcc *obs;                // its accumulators (may be null)
    double *theta2;             // [L*L] (may be null)
};

struct SweepBuffers {
    const float *W32 = nullptr;         // [4][N]
    float *spins = nullptr;             // [R][3][N]
    const RepParams *params = nullptr;  // [R]
    double *energy = nullptr;           // [R] tracked energy (in: at t0, out: at t0+nsweeps)
    ObsAcc *obs = nullptr;              // [R]
    double *theta2 = nullptr;           // [R][N]
    float *trace = nullptr;             // optional [R][nsweeps][l^2][n][MC_TRACE_W]
    const SlotState *slots = nullptr;   // optional [R]: packed launch
    EnergyHist hist;                    // optional energy histogram
    const SlotGeom *geom = nullptr;     // optional [grid]: grouped direct launch (the fields above unused)
};

// Total energy of one replica (Sec. 4 energy with the ferromagnetic-exchange and
// E_A = -K2 z^2 - K4 z^4 readings) from its spins s [3][L][L] and field f = W~ * s
// [3][L][L]:  -J sum_bonds s_i.s_j + sum_i E_A(s_i) + (C_D / 2) sum_i s_i.h_i, each bond
// (i, i + x), (i, i + y) once, FP64 sums.  Called by every thread of one CTA (a
// multiple of 32 threads, at most 1024); the result is valid in thread 0.  The
// handle energy kernel and the allocation-free energy kernel both call it.
__device__ __forceinline__ double cta_replica_energy(int L, const float *__restrict__ s,
                                                     const float *__restrict__ f, double J, double CD,
                                                     double K2, double K4) {
    const int N = L * L;
    double ex = 0, an = 0, dp = 0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const int x = i % L, y = i / L;
        const int ixp = y * L + (x + 1 == L ? 0 : x + 1);
        const int iyp = (y + 1 == L ? 0 : y + 1) * L + x;
        const double a = s[i], b = s[N + i], c = s[2 * N + i];
        ex += a * ((double)s[ixp] + (double)s[iyp]) + b * ((double)s[N + ixp] + (double)s[N + iyp]) +
              c * ((double)s[2 * N + ixp] + (double)s[2 * N + iyp]);
        const double z2 = c * c;
        an += -K2 * z2 - K4 * z2 * z2;
        dp += a * (double)f[i] + b * (double)f[N + i] + c * (double)f[2 * N + i];
    }
    double tot = -J * ex + an + 0.5 * CD * dp;
    for (int off = 16; off; off >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, off);
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = tot;
    __syncthreads();
    double sum = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += red[w];
    return sum;
}

// Launchers (implemented in their .cu files).  Return a cudaError_t.
cudaError_t launch_wtilde(int L, int A, int tail, double *W64, float *W32, cudaStream_t st);
cudaError_t launch_cast_W(int L, const double *W64, float *W32, cudaStream_t st);
// W~ by the Ewald/Harris split, [6][L][L] (xx, xy, yy, zz, xz, yz), layers z apart.
cudaError_t launch_wtilde_ewald(int L, double z, double eta, double *W6, cudaStream_t st);
cudaError_t launch_take_plane(int L, const double *W6, double *W64, float *W32, cudaStream_t st);
cudaError_t launch_init_spins(int L, int R, uint2 key, int mode, float *spins, cudaStream_t st);
cudaError_t launch_full_field(int L, int R, const float *W32, const float *spins, float *h,
                              cudaStream_t st);
cudaError_t launch_energy(int L, int R, const float *spins, const float *h, const RepParams *p,
                          double *E, cudaStream_t st);
// eta (Sec. 4.1) of `count` replicas from their per-site sums of (theta - pi/2)^2.
cudaError_t launch_eta(int N, int count, const double *theta2, const ObsAcc *obs, double *eta, cudaStream_t st);
// Returns cudaErrorNotSupported when no direct-kernel instance fits (L, l).
cudaError_t launch_sweep_direct(const SweepConfig &c, const SweepBuffers &b, int threads_hint,
                                cudaStream_t st);
bool direct_supported(int L, int l);
// Threads and cell offsets per field thread (EPT) of the direct launch a handle
// of R replicas of (L, l) gets; false if the direct kernel does not serve (L, l).
bool direct_lone_shape(int L, int l, int R, int *threads, int *ept);
// Dynamic shared memory of a direct CTA of (L, l) with `threads` threads.
size_t direct_smem_bytes(int L, int l, int threads);
// One launch over `count` CTAs of possibly different L (all with L / l == C), each
// described by geom_dev[i] (device memory); c.nsweeps is the largest per-CTA count
// and c.R is ignored.  threads = the largest lone thread count, max_ept the largest
// lone EPT, smem the largest direct_smem_bytes at `threads`.
cudaError_t launch_sweep_direct_grouped(int C, int max_ept, int threads, size_t smem, const SweepConfig &c,
                                        const SlotGeom *geom_dev, int count, cudaStream_t st);
// CTAs of such a grouped launch resident on the whole GPU at once (0: no instance).
int direct_grouped_resident(int C, int max_ept, int threads, size_t smem);
// CTAs of the direct kernel resident on the whole GPU for a packed launch of (L, l).
int direct_resident_ctas(int L, int l);

// Records a one-line error message for mc_last_error() and returns `code`.
int set_last_error(int code, const char *msg);

}  // namespace dipmc
