// window.cu -- the windowed sweep: the l^2 sub-steps of a sweep are processed in
// windows of B consecutive sub-steps.  At the start of a window the dipole
// field at all S_w = B*n sites the window will visit is taken from one bulk
// evaluation on the state at the window's start (the "stale" field: a fat
// contraction over all replicas, done by the tensor-core kernel, or the FP32
// full field for validation).  The B sub-steps then run in order, each exactly
// as the simultaneous-flip update of Sec. 3.1/3.2 prescribes; the field of a
// window site is its stale value plus the exact change from every move
// accepted earlier in the window:
//     h_q = h_q(stale) + sum_{p accepted since the window start} W~(q - p) (S_p - s_p).
// This is the same field the direct path computes, up to rounding.
//
// k_window_steps: eight warps per replica (one CTA, or one half of a CTA that
// carries two).  Spins live in shared memory for the window (three planes); the
// replica's first warp takes the decisions of blocks of 16 sites
// on its own; warps 1..7 push older moves into the window's later sites.  Under
// the permutation schedule a site's proposal is fixed at the window's start, so
// what the decider adds per sub-step is a sum of precomputed scalar pair energies;
// at L = 2l the pushes and the pair energies go through the 2 x 2 sub-lattice
// spectra of the moves and of W~ (the four cells o + l D of a sub-step's offset o).
#include <cuda_bf16.h>

#include "internal.cuh"
#include "window.cuh"

namespace dipmc {

namespace {

constexpr int kWThreads = 256;
constexpr int kBlockSites = 16; // sites per decider block (G = 16 / n sub-steps; at least one sub-step)
constexpr float kPiF = 3.14159265358979f;

// float4 entries of the W~ table in shared memory: the minimum-image quarter, or at
// n = 4 (L = 2l) the larger of it and the sub-lattice spectra U (the permutation
// schedule reads U, the other schedule the quarter; one layout serves both)
__host__ __device__ __forceinline__ int wtab_smem_elems(int L, int n) {
    const int hq = L / 2 + 1, hu = L / 4 + 1;
    return (n == 4 && 4 * hu * hu > hq * hq) ? 4 * hu * hu : hq * hq;
}

// Bulk global -> shared copies on an mbarrier (the set-up's tables and spins).  Waits are
// bounded: a copy that has not landed after kCopyWaitCycles is reported, not waited on forever.
constexpr long long kCopyWaitCycles = 1LL << 31;   // about one second at 2 GHz

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init_tx(uint64_t *m) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(m)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void bar_expect_tx(uint64_t *m, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(m)), "r"(bytes) : "memory");
}

// bytes: a multiple of 16; both addresses 16-byte aligned
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *m) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(m))
                 : "memory");
}

__device__ __forceinline__ bool bar_wait_bounded(uint64_t *m, uint32_t parity) {
    const long long t0 = clock64();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_addr(m)), "r"(parity)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > kCopyWaitCycles) return false;
    }
}


// W~ restricted to the minimum-image quarter 0 <= x, y <= L/2, as (xx, xy, yy, zz).
// The tensor is even in x and in y except xy, which is odd in each: a
// displacement (dx, dy) reads entry (|dx|, |dy|) and flips the sign of xy when
// exactly one of dx, dy is negative (xy vanishes on the axes and at L/2).
// W~(dx, dy) itself, (xx, xy, yy, zz), from the quarter table.
__device__ __forceinline__ float4 wq_get(const float4 *__restrict__ wq, int L, int dx, int dy) {
    const int h = L >> 1;
    if (dx < 0) dx += L;
    if (dy < 0) dy += L;
    float sgn = 1.0f;
    if (dx > h) { dx = L - dx; sgn = -sgn; }
    if (dy > h) { dy = L - dy; sgn = -sgn; }
    const float4 w = wq[dy * (h + 1) + dx];
    return make_float4(w.x, sgn * w.y, w.z, w.w);
}

__device__ __forceinline__ float3 wq_apply(const float4 *__restrict__ wq, int L, int dx, int dy, float3 d) {
    const int h = L >> 1;
    if (dx < 0) dx += L;
    if (dy < 0) dy += L;
    float sgn = 1.0f;
    if (dx > h) { dx = L - dx; sgn = -sgn; }
    if (dy > h) { dy = L - dy; sgn = -sgn; }
    const float4 w = wq[dy * (h + 1) + dx];
    const float xy = sgn * w.y;
    return make_float3(w.x * d.x + xy * d.y, xy * d.x + w.z * d.y, w.w * d.z);
}

// Scalar pair energy of two window sites i and p (x | y << 16 coordinates, flag bit
// ignored): the dipolar change C_D d_i.W~(q_i - q_p).d_p of site i's move once p has
// moved, plus, when `exch`, the exchange change -J m d_i.d_p, m = the number of lattice
// directions in which q_p neighbours q_i (Eq. 1 with both moves in place).
__device__ __forceinline__ float pair_energy(const float4 *__restrict__ wq, int L, int ai, int ap, float4 di,
                                             float4 dp, float CD, float J, bool exch) {
    const int dx = (ai & 0xFFFF) - (ap & 0xFFFF), dy = ((ai >> 16) & 0x7FFF) - ((ap >> 16) & 0x7FFF);
    const float3 w = wq_apply(wq, L, dx, dy, make_float3(dp.x, dp.y, dp.z));
    float e = CD * (di.x * w.x + di.y * w.y + di.z * w.z);
    if (exch) {
        const int ax = dx < 0 ? dx + L : dx, ay = dy < 0 ? dy + L : dy;
        int m = 0;
        if (ay == 0) m += (ax == 1) + (ax == L - 1);
        if (ax == 0) m += (ay == 1) + (ay == L - 1);
        if (m) e -= J * (float)m * (di.x * dp.x + di.y * dp.y + di.z * dp.z);
    }
    return e;
}

// The 2 x 2 sub-lattice spectra of W~ at L = 2l (table U, k_build_uq).  For a signed
// offset difference d (|dx|, |dy| < l) of two l x l cells, U_d(kappa) = sum_P
// (-1)^(kappa.P) W~(d + l P) is read at (|dx|, |dy|) folded into [0, l/2]: a negative
// component reflects W~ in that axis (xy changes sign; l P is its own negative modulo
// L), and a component a > l/2 is read at l - a, which reflects and shifts P by one in
// that axis (xy changes sign, and U(kappa) by (-1)^kappa_axis).
struct UFold {
    int base;        // float4 index of kappa = 0
    float sxy;       // sign of the xy component
    unsigned kneg;   // bit kappa set: U(kappa) changes sign
};
__device__ __forceinline__ UFold u_fold(int l, int dx, int dy) {
    const int hl = l >> 1;
    int ax = abs(dx), ay = abs(dy);
    int par = (dx < 0) ^ (dy < 0);
    unsigned kneg = 0u;
    if (ax > hl) { ax = l - ax; par ^= 1; kneg ^= 0xAu; }   // kappa with kx = 1: 1, 3
    if (ay > hl) { ay = l - ay; par ^= 1; kneg ^= 0xCu; }   // kappa with ky = 1: 2, 3
    return {(ay * (hl + 1) + ax) * 4, par ? -1.0f : 1.0f, kneg};
}
__device__ __forceinline__ float4 u_get(const float4 *__restrict__ uq, const UFold &f, int kap) {
    const float4 u = uq[f.base + kap];
    const float sg = ((f.kneg >> kap) & 1u) ? -1.0f : 1.0f;
    return make_float4(sg * u.x, sg * f.sxy * u.y, sg * u.z, sg * u.w);
}
// The fold of u_fold packed in one word: cell index << 4 | kneg | (xy sign bit), so
// that the lanes of a warp can share it (kneg uses bits 1..3: kappa = 0 never changes sign).
__device__ __forceinline__ int u_fold_word(int l, int dx, int dy) {
    const UFold f = u_fold(l, dx, dy);
    return ((f.base >> 2) << 4) | (int)f.kneg | (f.sxy < 0.0f ? 1 : 0);
}
__device__ __forceinline__ float4 u_get_word(const float4 *__restrict__ uq, int w, int kap) {
    const float4 u = uq[((w >> 4) << 2) + kap];
    const unsigned neg = ((unsigned)((w & 0xE) >> kap) & 1u) << 31;
    const unsigned negxy = neg ^ ((unsigned)(w & 1) << 31);
    return make_float4(__uint_as_float(__float_as_uint(u.x) ^ neg), __uint_as_float(__float_as_uint(u.y) ^ negxy),
                       __uint_as_float(__float_as_uint(u.z) ^ neg), __uint_as_float(__float_as_uint(u.w) ^ neg));
}
// W~ between lattice sites (xi, yi) and (xp, yp) of an L = 2l lattice from U: with
// d = o_i - o_p (offsets in the l x l cell) and P = D_i xor D_p (cells),
// W~(d + l P) = (1/4) sum_kappa (-1)^(kappa.P) U_d(kappa).
__device__ __forceinline__ float4 w_from_u(const float4 *__restrict__ uq, int l, int xi, int yi, int xp, int yp) {
    const int Dxi = xi >= l, Dyi = yi >= l, Dxp = xp >= l, Dyp = yp >= l;
    const UFold f = u_fold(l, (xi - l * Dxi) - (xp - l * Dxp), (yi - l * Dyi) - (yp - l * Dyp));
    const int P = (Dxi ^ Dxp) | ((Dyi ^ Dyp) << 1);
    float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int kap = 0; kap < 4; ++kap) {
        const float4 u = u_get(uq, f, kap);
        const float sg = (__popc(kap & P) & 1) ? -0.25f : 0.25f;
        w.x += sg * u.x;
        w.y += sg * u.y;
        w.z += sg * u.z;
        w.w += sg * u.w;
    }
    return w;
}

// PRE: the permutation schedule, where every site is visited once per sweep, so the
// proposal, its threshold and the field-free part of dE of every window site are fixed
// at the window's start.  The window's sub-steps then only add, to each site's dE, the
// pair energies of the moves accepted before it, and the decisions of a block of 16
// sites run as a chain of ballots over precomputed pair energies.  Otherwise (the
// with-replacement schedule, where a site may recur within a window) each decision
// proposes from the current spin and pulls the field vector of the block's moves.
template <int C, bool PRE>
__global__ void __launch_bounds__(2 * kWThreads, 1) k_window_steps(const WindowConfig cfg, const WindowBuffers buf) {
    constexpr int n = C * C;
    constexpr int NB = kBlockSites;   // sites per decider block
    constexpr int G = NB / n;         // sub-steps per block
    // permutation schedule at L = 2l: moves pushed, and pair energies tabulated, through
    // the 2 x 2 sub-lattice spectra (table U in place of the quarter of W~)
    constexpr bool SPX = PRE && C == 2;
    constexpr int kTab = 2 * NB / 4 * NB;   // float4 entries of one block's pair table
    constexpr int kDecItems = 64;           // of them taken by the decider warp after its decisions
    const int L = cfg.L, l = cfg.l, N = L * L, ll = l * l, B = cfg.B, Sw = B * n;
    // two replicas a CTA where shared memory allows (cfg.gpc == 2): replica group g takes the
    // even or the odd warps, so that each has two SM sub-partitions to itself and its decider
    // (the group's lowest warp) the first claim on them; below, tid and warp count within the
    // group (0..255, 0..7), and every barrier is the group's own
    const int g = cfg.gpc == 2 ? (int)((threadIdx.x >> 5) & 1) : 0;
    const int tid = cfg.gpc == 2 ? (int)(((threadIdx.x >> 6) << 5) | (threadIdx.x & 31)) : (int)threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int r = cfg.gpc * blockIdx.x + g;
    if (r >= cfg.R) return;   // the odd group of the last CTA when R is odd (it shares no barrier)
    auto gsync = [&]() {
        if (g) asm volatile("bar.sync 2, %0;" ::"n"(kWThreads) : "memory");
        else asm volatile("bar.sync 1, %0;" ::"n"(kWThreads) : "memory");
    };

    extern __shared__ float4 smem_all[];
    float4 *smem_w = smem_all + (size_t)g * (cfg.smem_group / sizeof(float4));
    const int hq = (L >> 1) + 1;
    float *sxyz = reinterpret_cast<float *>(smem_w);     // [3][N] spins (x, y, z planes)
    float4 *hcur = reinterpret_cast<float4 *>(sxyz + 3 * N);   // [Sw] !PRE: field of the window sites
                                                         // (stale + pushed moves); 3N floats keep it 16-byte aligned (N % 4 == 0)
    float *dacc = reinterpret_cast<float *>(hcur);       // PRE: [Sw] dE so far, without exchange and block pairs
    float4 *pS = hcur + Sw;                              // [Sw] proposal S, threshold -T ln u; after the decision w = dE
    float4 *pd = pS + Sw;                                // [Sw] delta = S - s, field-free part of dE
    float4 *wq = pd + Sw;                                // [wtab_smem_elems] minimum-image quarter of W~
                                                         // (SPX: the sub-lattice spectra U)
    float4 *s_mvb = wq + wtab_smem_elems(L, n);          // [2][NB] accepted moves of a block:
                                                         // (delta, x | y << 16), double-buffered by parity
                                                         // (SPX: lane 4u + kappa holds the 2 x 2 spectrum
                                                         // at kappa of sub-step u's moves)
    float4 *wpair = s_mvb + 2 * NB;                      // !PRE: [NB][NB] W~ between the sites of a block
    float4 *etab = wpair;                                // PRE: [2][2 NB / 4][NB] pair energies by block parity,
                                                         // four columns of a row per float4
    int *wxy = reinterpret_cast<int *>(wpair + NB * NB); // [Sw] site as x | y << 16 (bit 31: accepted);
                                                         // then stale_mode 3: [3 Sw] floats of split-K sums
    __shared__ int s_nmv_g[2][2];
    __shared__ double s_epart_g[2][32];
    __shared__ double s_energy_g[2];   // the tracked energy after this window (measured windows)
    __shared__ float s_mred_g[2][kWThreads / 32][12];
    // stale_mode 3: one bit per group of 16 cell offsets (one 32-byte sector of a spectra
    // plane) holding a move accepted in this window; 256 groups cover l <= 64
    constexpr int kSpecWords = 8;
    __shared__ uint32_t s_ck_g[2][kSpecWords];
    uint32_t *s_ck = s_ck_g[g];
    if (tid < kSpecWords) s_ck[tid] = 0u;
    int *s_nmv = s_nmv_g[g];
    double *s_epart = s_epart_g[g];
    double &s_energy = s_energy_g[g];
    float(*s_mred)[12] = s_mred_g[g];

    const RepParams P = buf.params[r];
    const uint2 key = cfg.key;
    const uint32_t t = cfg.t_dev ? *cfg.t_dev + (uint32_t)cfg.it : cfg.t;
    const int k0 = cfg.w * B;
    auto spin = [&](int q) -> float3 { return make_float3(sxyz[q], sxyz[N + q], sxyz[2 * N + q]); };
    auto set_spin = [&](int q, float a, float b, float c) {
        sxyz[q] = a;
        sxyz[N + q] = b;
        sxyz[2 * N + q] = c;
    };
    const float W0xx = __ldg(buf.W32), W0xy = __ldg(buf.W32 + N), W0yy = __ldg(buf.W32 + 2 * N), W0zz = __ldg(buf.W32 + 3 * N);

    // proposal, delta and the field-free part of dE (anisotropy + self-image) of site q
    auto propose = [&](int q, float u1, float cps, float sps, float4 &S, float4 &D) {
        const float3 sq = spin(q);
        float S0, S1, S2;
        {
            const float3 Sv = propose_spin(cfg.proposal, cfg.cap_c1, sq.x, sq.y, sq.z, u1, cps, sps);   // Sec. 3.1 proposal
            S0 = Sv.x;
            S1 = Sv.y;
            S2 = Sv.z;
        }
        const float dX = S0 - sq.x, dY = S1 - sq.y, dZ = S2 - sq.z;
        const float z0 = sq.z * sq.z, z1 = S2 * S2;
        const float dan = (-P.K2 * z1 - P.K4 * z1 * z1) - (-P.K2 * z0 - P.K4 * z0 * z0);
        const float self = W0xx * dX * dX + 2.0f * W0xy * dX * dY + W0yy * dY * dY + W0zz * dZ * dZ;
        S = make_float4(S0, S1, S2, 0.0f);
        D = make_float4(dX, dY, dZ, dan + 0.5f * P.CD * self);
    };
    const uint4 rk = PRE ? philox(make_uint4(t, 0u, 0u, kTagPerm), key) : make_uint4(0, 0, 0, 0);
    auto attempt_rng = [&](int s, int q) -> uint4 {
        const int k = k0 + s / n;
        return philox(make_uint4((uint32_t)q, (uint32_t)r, t, ((uint32_t)k & 0x00FFFFFFu) | kTagAttempt), key);
    };
    auto trace_row = [&](int s) -> float * {
        return buf.trace + ((((size_t)r * cfg.nsweeps_call + cfg.it) * ll + (k0 + s / n)) * n + s % n) * MC_TRACE_W;
    };
    // neighbour sum of site (qx, qy) from the spins in shared memory
    auto nbr_sum = [&](int qx, int qy) -> float3 {
        const int q = qy * L + qx;
        const int xp = (qx + 1 == L) ? q - qx : q + 1;
        const int xm = (qx == 0) ? q + L - 1 : q - 1;
        const int yp = (qy + 1 == L) ? qx : q + L;
        const int ym = (qy == 0) ? q + N - L : q - L;
        const float3 a = spin(xp), bb = spin(xm), c = spin(yp), dd = spin(ym);
        return make_float3((a.x + bb.x) + (c.x + dd.x), (a.y + bb.y) + (c.y + dd.y), (a.z + bb.z) + (c.z + dd.z));
    };

    // stale_mode 3 (spectra of the window's offsets, L = 2l): the field of site
    // 4j + d, d = Dx + 2 Dy, is (1/4) sum_kappa (-1)^(kappa.D) H_j(kappa); it is staged
    // in shared memory (PRE: after dacc; otherwise in hcur) before the per-site set-up
    float *hst = dacc + Sw;
    auto staged = [&](int s) -> float3 {
        if (PRE) return make_float3(hst[3 * s], hst[3 * s + 1], hst[3 * s + 2]);
        const float4 h = hcur[s];
        return make_float3(h.x, h.y, h.z);
    };
    // the stale field at window site s (lattice site q)
    auto stale_at = [&](int s, int q) -> float3 {
        if (cfg.stale_mode == 3) return staged(s);
        if (cfg.stale_mode == 0) {
            const float *f = buf.stale + (size_t)r * 3 * N;
            return make_float3(f[q], f[N + q], f[2 * N + q]);
        }
        // stale_mode 2: row b*Sw + s of this replica's column is the sum of the split-K
        // partial tiles of its output tile, in unit order (the tensor-core field's reduction)
        const int nt = r / cfg.NT, col = r - nt * cfg.NT;
        const float *pc[3];
        int cnt[3];
        float h[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int bb = 0; bb < 3; ++bb) {
            const int row = bb * Sw + s, mt = row >> 7, rr = row & 127;
            const int u0 = buf.tile_first[nt * cfg.mtiles + mt], u1 = buf.tile_first[nt * cfg.mtiles + mt + 1];
            pc[bb] = buf.part + ((size_t)u0 * cfg.NT + col) * 128 + rr;
            cnt[bb] = u1 - u0;
        }
        const size_t ustride = (size_t)cfg.NT * 128;
        const int cmax = max(cnt[0], max(cnt[1], cnt[2]));
        // four partial tiles of each row in flight; summed in unit order
        for (int j0 = 0; j0 < cmax; j0 += 4) {
            float v[3][4];
#pragma unroll
            for (int bb = 0; bb < 3; ++bb)
#pragma unroll
                for (int j = 0; j < 4; ++j) v[bb][j] = (j0 + j < cnt[bb]) ? __ldcg(pc[bb] + (size_t)(j0 + j) * ustride) : 0.f;
#pragma unroll
            for (int bb = 0; bb < 3; ++bb)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (j0 + j < cnt[bb]) h[bb] += v[bb][j];
        }
        return make_float3(h[0], h[1], h[2]);
    };

    const long long cyc0 = clock64();   // the kernel's start on this SM (for buf.cycles)
    long long cyc1 = 0, cyc2 = 0;
    // ---- window set-up.  Before the previous kernel of the stream has finished:
    // the tensor table and the window's sites (they depend on the sweep counter
    // only); then the state, stale field and proposals.
    pdl_trigger();
    // the spins, and under PRE the proposals (they depend on the spins at the window's start
    // and the counter-based draws only), before the wait when the previous kernel is the
    // tensor-core field kernel (stale_mode 2, 3): it lets this kernel launch only once it is
    // past its own wait on the sub-step kernel before it, so every writer of the spins has
    // completed.  The W~ table and the spins then come by two bulk copies (async proxy, read
    // through L2) that thread 0 issues first and waits for.
    const bool early = cfg.stale_mode >= 2;
    const float *gs = buf.spins + (size_t)r * 3 * N;
    const float4 *gwq = SPX ? buf.wq + hq * hq : buf.wq;
    const int nwq = SPX ? 4 * ((l >> 1) + 1) * ((l >> 1) + 1) : hq * hq;   // float4 of the table
    __shared__ uint64_t s_cbar_g[2][2];   // per group: the spins, the table
    __shared__ int s_cok_g[2];
    if (early && tid == 0) {
        bar_init_tx(&s_cbar_g[g][0]);
        bar_init_tx(&s_cbar_g[g][1]);
        bar_expect_tx(&s_cbar_g[g][0], (uint32_t)(12 * N));
        bulk_g2s(sxyz, gs, (uint32_t)(12 * N), &s_cbar_g[g][0]);
        bar_expect_tx(&s_cbar_g[g][1], (uint32_t)(16 * nwq));
        bulk_g2s(wq, gwq, (uint32_t)(16 * nwq), &s_cbar_g[g][1]);
    }
    __shared__ float4 s_wl_g[2][4];   // SPX: W~(l P), P = Px + 2 Py (the cells of one offset)
    float4 *s_wl = s_wl_g[g];
    if (SPX && tid < 4) {
        const int g = l * (tid >> 1) * L + l * (tid & 1);
        s_wl[tid] = make_float4(__ldg(buf.W32 + g), __ldg(buf.W32 + N + g), __ldg(buf.W32 + 2 * N + g),
                                __ldg(buf.W32 + 3 * N + g));
    }
    if (!early) {
#pragma unroll 4
        for (int i = tid; i < nwq; i += kWThreads) wq[i] = gwq[i];
    }
    // W~(q_i - q_p) v for lattice sites i = (xi, yi), p = (xp, yp)
    auto w_apply_sites = [&](int xi, int yi, int xp, int yp, float3 v) -> float3 {
        if constexpr (SPX) {
            const float4 w = w_from_u(wq, l, xi, yi, xp, yp);
            return make_float3(w.x * v.x + w.y * v.y, w.y * v.x + w.z * v.y, w.w * v.z);
        } else {
            return wq_apply(wq, L, xi - xp, yi - yp, v);
        }
    };
    for (int s = tid; s < Sw; s += kWThreads) wxy[s] = window_site_xy(l, C, key, t, cfg.schedule, rk, k0, s);
    // stale_mode 3: warp mt sums M-tile mt of this replica's column over the tile's units
    // (3 S_w / 128 M-tiles of 128 rows: six, or twelve at 512 sites); the work plan is
    // fixed when the buffers are set up
    const int st_mt = warp, st_f = lane;
    int st_u0 = 0, st_cnt = 0;
    if (cfg.stale_mode == 3 && st_mt < cfg.mtiles) {
        const int nt = r / cfg.NT;
        st_u0 = buf.tile_first[nt * cfg.mtiles + st_mt];
        st_cnt = buf.tile_first[nt * cfg.mtiles + st_mt + 1] - st_u0;
    }
    auto load_spins = [&]() {
#pragma unroll 8
        for (int i = tid; i < 3 * N / 4; i += kWThreads) smem_w[i] = reinterpret_cast<const float4 *>(gs)[i];
    };
    // proposal of window site s (lattice site q): pS = (S, -T ln u), pd = (delta, field-free dE)
    auto propose_site = [&](int s, int q) {
        const uint4 wds = attempt_rng(s, q);
        float sps, cps;
        sincospif(2.0f * u24f(wds.y), &sps, &cps);
        const float u = u24f(wds.z);
        float4 S, D;
        propose(q, u24f(wds.x), cps, sps, S, D);
        // accept iff u < exp(-dE/T)  <=>  dE < -T ln u   (u = 0: always)
        S.w = (u > 0.0f) ? -P.T * logf(u) : INFINITY;
        pS[s] = S;
        pd[s] = D;
    };
    if (early) {
        if (PRE) {
            // the draws first, while the copies land: pd[s] = (u1, cos, sin) of the proposal,
            // pS[s].w = -T ln u (same thread and site as below)
            for (int s = tid; s < Sw; s += kWThreads) {
                const int xy = wxy[s];
                const uint4 wds = attempt_rng(s, (xy >> 16) * L + (xy & 0xFFFF));
                float sps, cps;
                sincospif(2.0f * u24f(wds.y), &sps, &cps);
                const float u = u24f(wds.z);
                pS[s].w = (u > 0.0f) ? -P.T * logf(u) : INFINITY;
                pd[s] = make_float4(u24f(wds.x), cps, sps, 0.0f);
            }
        }
        if (tid == 0) {
            const bool ok = bar_wait_bounded(&s_cbar_g[g][0], 0u);
            if (!ok) {
                if (buf.error) atomicExch(buf.error, 3);
                bar_wait_bounded(&s_cbar_g[g][0], 0u);   // once more for the copies in flight
                bar_wait_bounded(&s_cbar_g[g][1], 0u);
            }
            s_cok_g[g] = ok ? 1 : 0;
        }
        gsync();
        if (!s_cok_g[g]) return;   // the whole group: results of this call are invalid (reported)
        if (PRE) {
            for (int s = tid; s < Sw; s += kWThreads) {
                const int xy = wxy[s];
                const float4 dr = pd[s];
                float4 S, D;
                propose((xy >> 16) * L + (xy & 0xFFFF), dr.x, dr.y, dr.z, S, D);
                S.w = pS[s].w;
                pS[s] = S;
                pd[s] = D;
            }
        }
    }
    pdl_wait();
    if (early && tid == 0 && !bar_wait_bounded(&s_cbar_g[g][1], 0u)) {
        // the table (needed from the first pair table on, after the barrier below): reported;
        // once more for the copy in flight
        if (buf.error) atomicExch(buf.error, 3);
        bar_wait_bounded(&s_cbar_g[g][1], 0u);
    }
    // the loads of the split-K partial tiles (stale_mode 3: lane f of warp mt takes rows
    // 4f .. 4f+3 of M-tile mt, one 16-byte load of each unit's 512-byte column segment)
    // and (late) of the spins go out together
    const bool st_on = cfg.stale_mode == 3 && st_mt < cfg.mtiles;
    const size_t ustride = (size_t)cfg.NT * 32;   // float4 per unit
    const float4 *pc = nullptr;
    constexpr int kPV = 8;    // units whose loads go out at once
    float4 pv[kPV];
    if (st_on) {
        const int col = r - (r / cfg.NT) * cfg.NT;
        pc = reinterpret_cast<const float4 *>(buf.part + ((size_t)st_u0 * cfg.NT + col) * 128) + st_f;
#pragma unroll
        for (int j = 0; j < kPV; ++j) pv[j] = (j < st_cnt) ? __ldcg(pc + (size_t)j * ustride) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (!early) load_spins();
    if (cfg.stale_mode == 3) {
        // split-K sums in unit order (the tensor-core field's reduction) into rs[row]
        // (3 S_w rows of scratch after the window's site list)
        float *rs = reinterpret_cast<float *>(wxy + Sw);
        if (st_on) {
            float4 h = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int j = 0; j < kPV; ++j)
                if (j < st_cnt) {
                    h.x += pv[j].x;
                    h.y += pv[j].y;
                    h.z += pv[j].z;
                    h.w += pv[j].w;
                }
            for (int j0 = kPV; j0 < st_cnt; j0 += 8) {
                float4 v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    v[j] = (j0 + j < st_cnt) ? __ldcg(pc + (size_t)(j0 + j) * ustride) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (j0 + j < st_cnt) {
                        h.x += v[j].x;
                        h.y += v[j].y;
                        h.z += v[j].z;
                        h.w += v[j].w;
                    }
            }
            reinterpret_cast<float4 *>(rs)[st_mt * 32 + st_f] = h;
        }
        // M-tiles beyond the eight warps (512-site windows: twelve): warp mt takes mt + 8, ...
        for (int mt = st_mt + kWThreads / 32; mt < cfg.mtiles; mt += kWThreads / 32) {
            const int nt = r / cfg.NT, col = r - nt * cfg.NT;
            const int u0 = buf.tile_first[nt * cfg.mtiles + mt], cnt = buf.tile_first[nt * cfg.mtiles + mt + 1] - u0;
            const float4 *pm = reinterpret_cast<const float4 *>(buf.part + ((size_t)u0 * cfg.NT + col) * 128) + st_f;
            float4 h = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int j0 = 0; j0 < cnt; j0 += 8) {
                float4 v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    v[j] = (j0 + j < cnt) ? __ldcg(pm + (size_t)(j0 + j) * ustride) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (j0 + j < cnt) {
                        h.x += v[j].x;
                        h.y += v[j].y;
                        h.z += v[j].z;
                        h.w += v[j].w;
                    }
            }
            reinterpret_cast<float4 *>(rs)[mt * 32 + st_f] = h;
        }
        gsync();
        // rows kappa*2B + b*B + j (b = x, y) and 2 S_w + (kappa/2)*2B + (kappa%2)*B + j (z), B = S_w/4
        const int B4 = Sw >> 2;
        for (int task = tid; task < 3 * B4; task += kWThreads) {
            const int j = task / 3, bb = task - 3 * j;
            float H[4];
#pragma unroll
            for (int kap = 0; kap < 4; ++kap)
                H[kap] = rs[bb < 2 ? kap * 2 * B4 + bb * B4 + j : 2 * Sw + (kap >> 1) * 2 * B4 + (kap & 1) * B4 + j];
#pragma unroll
            for (int d = 0; d < 4; ++d) {
                float h = 0.f;
#pragma unroll
                for (int kap = 0; kap < 4; ++kap) h += (((kap & 1) * (d & 1) + (kap >> 1) * (d >> 1)) & 1) ? -H[kap] : H[kap];
                h *= 0.25f;
                if (PRE) hst[3 * (4 * j + d) + bb] = h;
                else reinterpret_cast<float *>(hcur + 4 * j + d)[bb] = h;
            }
        }
    }
    gsync();
    for (int s = tid; s < Sw; s += kWThreads) {
        const int xy = wxy[s];
        const int q = (xy >> 16) * L + (xy & 0xFFFF);
        const float3 hs = stale_at(s, q);
        const float h0 = hs.x, h1 = hs.y, h2 = hs.z;
        if (PRE) {
            if (!early) propose_site(s, q);
            const float4 D = pd[s];
            dacc[s] = D.w + P.CD * (D.x * h0 + D.y * h1 + D.z * h2);
        } else {
            hcur[s] = make_float4(h0, h1, h2, 0.0f);
        }
    }
    if (tid == 0) {
        s_nmv[0] = 0;
        s_nmv[1] = 0;
    }
    gsync();

    long long n_acc = 0;
    const int nblk = B / G;
    if (tid == 0) cyc1 = clock64();
    // warp roles during the blocks (layout): the decider warp dw, an idle warp or none,
    // and the helpers, numbered hw = 0 .. nh-1
    const int dw = (PRE && cfg.layout == 2 && ((r / cfg.nsm) & 1)) ? 2 : 0;
    const bool spare = PRE && cfg.layout >= 1;
    const bool idle = spare && warp == dw + 4;
    const int hw = warp - (warp > dw ? 1 : 0) - (spare && warp > dw + 4 ? 1 : 0);
    const int kH = (spare ? kWThreads / 32 - 2 : kWThreads / 32 - 1) * 32;   // helper threads
    const int ht = hw * 32 + lane;                                           // helper thread index
    if constexpr (PRE) {
        // pair energies of block nb into etab[nb & 1]: row i is site nb*NB + i; columns
        // 0..NB-1 the sites of block nb-1 (dipolar part: their exchange acts through the
        // spins, which hold those moves by the time block nb decides), columns NB.. the
        // sites of the block's own earlier sub-steps (dipolar and exchange).  Entry e is
        // column e / NB of row e % NB, so a warp's lanes take one column pair.
        auto etab_fill = [&](int nb, int t0, int stride) {
            float *et = reinterpret_cast<float *>(etab + (nb & 1) * (2 * NB / 4) * NB);
#pragma unroll 2
            for (int e = t0; e < NB * 2 * NB; e += stride) {
                const int c = e / NB, i = e % NB;
                const int si = nb * NB + i;
                float v = 0.0f;
                if (c < NB) {
                    if (nb > 0) {
                        const int sp = (nb - 1) * NB + c;
                        v = pair_energy(wq, L, wxy[si], wxy[sp], pd[si], pd[sp], P.CD, P.J, false);
                    }
                } else if ((c - NB) / n < i / n) {
                    const int sp = nb * NB + (c - NB);
                    v = pair_energy(wq, L, wxy[si], wxy[sp], pd[si], pd[sp], P.CD, P.J, true);
                }
                et[((c >> 2) * NB + i) * 4 + (c & 3)] = v;
            }
        };
        // SPX: item it = g * NB + i of block nb's table, the four entries of row i and
        // column group g (the four cells D_p of one sub-step) as one float4: W~ between the
        // cells of the two sub-steps' offsets from U (four loads and one inverse 2 x 2
        // transform), the exchange as in pair_energy
        auto etab_item = [&](int nb, int it) -> float4 {
            const int g = it / NB, i = it - g * NB, ui = i / n, Di = i - ui * n;
            const bool prevb = g < G;
            if (prevb ? nb == 0 : (g - G) >= ui) return make_float4(0.f, 0.f, 0.f, 0.f);
            const int jr = nb * G + ui, jc = prevb ? (nb - 1) * G + g : nb * G + (g - G);
            const int orr = wxy[n * jr], oc = wxy[n * jc];
            const UFold f = u_fold(l, (orr & 0xFFFF) - (oc & 0xFFFF), ((orr >> 16) & 0x7FFF) - ((oc >> 16) & 0x7FFF));
            const float4 U0 = u_get(wq, f, 0), U1 = u_get(wq, f, 1), U2 = u_get(wq, f, 2), U3 = u_get(wq, f, 3);
            // 4 W~(d + l P), P = Px + 2 Py: sum_kappa (-1)^(kappa.P) U(kappa)
            const float4 a = make_float4(U0.x + U1.x, U0.y + U1.y, U0.z + U1.z, U0.w + U1.w);
            const float4 b = make_float4(U0.x - U1.x, U0.y - U1.y, U0.z - U1.z, U0.w - U1.w);
            const float4 c = make_float4(U2.x + U3.x, U2.y + U3.y, U2.z + U3.z, U2.w + U3.w);
            const float4 e = make_float4(U2.x - U3.x, U2.y - U3.y, U2.z - U3.z, U2.w - U3.w);
            const float4 Wp[4] = {make_float4(a.x + c.x, a.y + c.y, a.z + c.z, a.w + c.w),
                                  make_float4(b.x + e.x, b.y + e.y, b.z + e.z, b.w + e.w),
                                  make_float4(a.x - c.x, a.y - c.y, a.z - c.z, a.w - c.w),
                                  make_float4(b.x - e.x, b.y - e.y, b.z - e.z, b.w - e.w)};
            const float4 di = pd[n * jr + Di];
            const int ai = wxy[n * jr + Di];
            const float cd4 = 0.25f * P.CD;
            float v[4];   // v[Pp]: the entry of cell D_p = D_i xor Pp
#pragma unroll
            for (int Pp = 0; Pp < 4; ++Pp) {
                const int Dp = Di ^ Pp;
                const float4 W = Wp[Pp], dp = pd[n * jc + Dp];
                v[Pp] = cd4 * (di.x * (W.x * dp.x + W.y * dp.y) + di.y * (W.y * dp.x + W.z * dp.y) + di.z * (W.w * dp.z));
                if (!prevb) {
                    const int ap = wxy[n * jc + Dp];
                    const int dx = (ai & 0xFFFF) - (ap & 0xFFFF), dy = ((ai >> 16) & 0x7FFF) - ((ap >> 16) & 0x7FFF);
                    const int ax = dx < 0 ? dx + L : dx, ay = dy < 0 ? dy + L : dy;
                    int m = 0;
                    if (ay == 0) m += (ax == 1) + (ax == L - 1);
                    if (ax == 0) m += (ay == 1) + (ay == L - 1);
                    if (m) v[Pp] -= P.J * (float)m * (di.x * dp.x + di.y * dp.y + di.z * dp.z);
                }
            }
            // into cell order: entry D_p is v[D_i xor D_p]
            if (Di & 1) {
                float t = v[0]; v[0] = v[1]; v[1] = t;
                t = v[2]; v[2] = v[3]; v[3] = t;
            }
            if (Di & 2) {
                float t = v[0]; v[0] = v[2]; v[2] = t;
                t = v[1]; v[1] = v[3]; v[3] = t;
            }
            return make_float4(v[0], v[1], v[2], v[3]);
        };
        if constexpr (SPX) {
            for (int it = tid; it < kTab; it += kWThreads) etab[it] = etab_item(0, it);
        } else {
            etab_fill(0, tid, kWThreads);
        }
        gsync();
        // Blocks of G sub-steps (16 sites), one CTA barrier per block.  Warp 0 (the
        // decider) takes block b's decisions: a site's dE is its window-start value, plus
        // the pushed pair energies of the moves of blocks <= b-2, plus those of block b-1
        // and of the block's earlier sub-steps from the pair table, with the exchange of
        // all earlier moves through the current neighbour spins.  Warps 1.. (the helpers)
        // meanwhile push the moves of block b-1 into the sites of blocks >= b+1 and
        // tabulate block b+1's pair energies.
        unsigned pm = 0;   // accepted sites of the previous block (decider)
        // decider: the site data of its next block (fixed since the window's start) and
        // their neighbour sums (the decider alone writes spins during the blocks), taken
        // before the block barrier
        int nx_xy = 0;
        float4 nx_D = make_float4(0.f, 0.f, 0.f, 0.f), nx_S = nx_D;
        float3 nx_nb = make_float3(0.f, 0.f, 0.f);
        auto dec_prefetch = [&](int nb) {
            const int s = nb * NB + (lane & (NB - 1));
            nx_xy = wxy[s];
            nx_D = pd[s];
            nx_S = pS[s];
            nx_nb = nbr_sum(nx_xy & 0xFFFF, (nx_xy >> 16) & 0x7FFF);
        };
        if (warp == dw) dec_prefetch(0);
        for (int bk = 0; bk < nblk; ++bk) {
            const int cur = bk & 1, prv = cur ^ 1, base = bk * NB;
            if (warp == dw) {
                const int i = lane & (NB - 1);
                const int s = base + i;
                const float4 *er = etab + cur * (2 * NB / 4) * NB + i;
                float E[2 * NB];
#pragma unroll
                for (int c = 0; c < 2 * NB; c += 4) {
                    const float4 v = er[(c >> 2) * NB];
                    E[c] = v.x;
                    E[c + 1] = v.y;
                    E[c + 2] = v.z;
                    E[c + 3] = v.w;
                }
                const int xy = nx_xy;
                const int qx = xy & 0xFFFF, qy = (xy >> 16) & 0x7FFF, q = qy * L + qx;
                const float4 D = nx_D, S = nx_S;
                const float3 nb3 = nx_nb;
                float dE = dacc[s] - P.J * (D.x * nb3.x + D.y * nb3.y + D.z * nb3.z);
#pragma unroll
                for (int p = 0; p < NB; ++p)
                    if ((pm >> p) & 1u) dE += E[p];
                unsigned am = 0;
#pragma unroll
                for (int u = 0; u < G; ++u) {
                    const unsigned ball = __ballot_sync(0xffffffffu, lane < NB && i / n == u && dE < S.w);
                    am |= ball;
                    if (u + 1 < G) {
#pragma unroll
                        for (int d = 0; d < n; ++d)
                            if ((ball >> (u * n + d)) & 1u) dE += E[NB + u * n + d];
                    }
                }
                const bool act = lane < NB;
                const bool acc = act && ((am >> i) & 1u);
                if (act && buf.trace) {
                    // the field the decision saw: stale field plus every earlier accepted move
                    const float3 h0 = stale_at(s, q);
                    float hx = h0.x, hy = h0.y, hz = h0.z;
                    for (int p = 0; p < base + i; ++p) {
                        const int pxy = wxy[p];
                        const bool moved = p < base ? pxy < 0 : ((p - base) / n < i / n && ((am >> (p - base)) & 1u));
                        if (!moved) continue;
                        const float4 dp = pd[p];
                        const float3 w = w_apply_sites(qx, qy, pxy & 0xFFFF, (pxy >> 16) & 0x7FFF,
                                                       make_float3(dp.x, dp.y, dp.z));
                        hx += w.x;
                        hy += w.y;
                        hz += w.z;
                    }
                    const uint4 wds = attempt_rng(s, q);
                    float *tr = trace_row(s);
                    tr[0] = (float)q;
                    tr[1] = hx; tr[2] = hy; tr[3] = hz;
                    tr[4] = dE;
                    tr[5] = u24f(wds.z);
                    tr[6] = (float)acc;
                    tr[7] = S.x; tr[8] = S.y; tr[9] = S.z;
                }
                __syncwarp();
                if (act) {
                    reinterpret_cast<float *>(pS + s)[3] = dE;
                    if (acc) {
                        set_spin(q, S.x, S.y, S.z);
                        wxy[s] = xy | (int)0x80000000;
                        if constexpr (!SPX)
                            s_mvb[cur * NB + __popc(am & ((1u << lane) - 1u))] = make_float4(D.x, D.y, D.z, __int_as_float(xy));
                    }
                }
                if constexpr (SPX) {
                    // the block's moves as 2 x 2 spectra: lane 4u + kappa takes sum_D
                    // (-1)^(kappa.D) (accepted move of site 4u + D), a Walsh-Hadamard
                    // butterfly over the four lanes of sub-step u
                    float x = acc ? D.x : 0.f, y = acc ? D.y : 0.f, z = acc ? D.z : 0.f;
#pragma unroll
                    for (int bb = 1; bb <= 2; bb <<= 1) {
                        const float px = __shfl_xor_sync(0xffffffffu, x, bb);
                        const float py = __shfl_xor_sync(0xffffffffu, y, bb);
                        const float pz = __shfl_xor_sync(0xffffffffu, z, bb);
                        const bool up = lane & bb;
                        x = up ? px - x : x + px;
                        y = up ? py - y : y + py;
                        z = up ? pz - z : z + pz;
                    }
                    if (act) s_mvb[cur * NB + lane] = make_float4(x, y, z, 0.0f);
                }
                pm = am;
                if (lane == 0) {
                    s_nmv[cur] = __popc(am);
                    n_acc += __popc(am);
                }
                if (bk + 1 < nblk) {
                    __syncwarp();   // this block's spins before the next block's neighbour sums
                    dec_prefetch(bk + 1);
                    // SPX: items 0..kDecItems-1 of block b+1's pair table (the helpers take the rest)
                    if constexpr (SPX)
#pragma unroll
                        for (int it = lane; it < kDecItems; it += 32) etab[((bk + 1) & 1) * kTab + it] = etab_item(bk + 1, it);
                }
            } else if (!idle) {
                const int nprev = bk > 0 ? s_nmv[prv] : 0;
                if constexpr (SPX) {
                    // push the moves of block b-1 into the dE of the sites of blocks >= b+1
                    // through their spectra: item 4 j + kappa of target sub-step j (offset o)
                    // sums dH(kappa) = sum_u U_{o - e_u}(kappa) S_u(kappa) over the block's
                    // four sub-steps u (offsets e_u; lane kappa folds o - e_kappa and the four
                    // lanes of the target share the folds); an inverse 2 x 2 transform over the
                    // four lanes then leaves lane D with the field change of cell D,
                    // (1/4) sum_kappa (-1)^(kappa.D) dH(kappa), and lane D adds C_D d_D . dh
                    if (nprev > 0) {
                        const int j0 = (bk + 1) * G, nitem = n * (B - j0), kap = lane & 3;
                        const int os = wxy[n * ((bk - 1) * G + kap)];
                        const int osx = os & 0xFFFF, osy = (os >> 16) & 0x7FFF;
                        float4 Sk[G];
#pragma unroll
                        for (int u = 0; u < G; ++u) Sk[u] = s_mvb[prv * NB + n * u + kap];
                        for (int ib = hw * 32; ib < nitem; ib += kH) {   // warp-uniform
                            const int item = ib + lane;
                            const bool on = item < nitem;
                            const int jt = on ? j0 + (item >> 2) : j0;
                            const int ot = wxy[n * jt];
                            const int fw = u_fold_word(l, (ot & 0xFFFF) - osx, ((ot >> 16) & 0x7FFF) - osy);
                            float Hx = 0.f, Hy = 0.f, Hz = 0.f;
#pragma unroll
                            for (int u = 0; u < G; ++u) {
                                const int w = __shfl_sync(0xffffffffu, fw, (lane & ~3) | u);
                                const float4 Uv = u_get_word(wq, w, kap);
                                Hx += Uv.x * Sk[u].x + Uv.y * Sk[u].y;
                                Hy += Uv.y * Sk[u].x + Uv.z * Sk[u].y;
                                Hz += Uv.w * Sk[u].z;
                            }
#pragma unroll
                            for (int bb = 1; bb <= 2; bb <<= 1) {
                                const float px = __shfl_xor_sync(0xffffffffu, Hx, bb);
                                const float py = __shfl_xor_sync(0xffffffffu, Hy, bb);
                                const float pz = __shfl_xor_sync(0xffffffffu, Hz, bb);
                                const bool up = lane & bb;
                                Hx = up ? px - Hx : Hx + px;
                                Hy = up ? py - Hy : Hy + py;
                                Hz = up ? pz - Hz : Hz + pz;
                            }
                            if (on) {
                                const float4 Dv = pd[n * jt + kap];
                                dacc[n * jt + kap] += 0.25f * P.CD * (Dv.x * Hx + Dv.y * Hy + Dv.z * Hz);
                            }
                        }
                    }
                    // block b+1's pair energies 32.. on the helper threads from the last down
                    // (their pushes are the fewest)
                    const int it = ht - (kH - kTab);
                    if (bk + 1 < nblk && it >= kDecItems) etab[((bk + 1) & 1) * kTab + it] = etab_item(bk + 1, it);
                } else {
                // push the moves of block b-1 into the dE of the sites of blocks >= b+1
                if (nprev > 0) {
                    for (int s = base + NB + ht; s < Sw; s += kH) {
                        const int xy = wxy[s];
                        const int qx = xy & 0xFFFF, qy = (xy >> 16) & 0x7FFF;
                        const float4 D = pd[s];
                        float e = 0.0f;
                        // four moves at a time: their loads go out together (the sum keeps
                        // the order m = 0, 1, 2, ...)
                        int m = 0;
                        for (; m + 4 <= nprev; m += 4) {
                            float4 mv[4];
#pragma unroll
                            for (int u = 0; u < 4; ++u) mv[u] = s_mvb[prv * NB + m + u];
                            float3 w[4];
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                const int pxy = __float_as_int(mv[u].w);
                                w[u] = wq_apply(wq, L, qx - (pxy & 0xFFFF), qy - ((pxy >> 16) & 0x7FFF),
                                                make_float3(mv[u].x, mv[u].y, mv[u].z));
                            }
#pragma unroll
                            for (int u = 0; u < 4; ++u) e += D.x * w[u].x + D.y * w[u].y + D.z * w[u].z;
                        }
                        for (; m < nprev; ++m) {
                            const float4 mv = s_mvb[prv * NB + m];
                            const int pxy = __float_as_int(mv.w);
                            const float3 w = wq_apply(wq, L, qx - (pxy & 0xFFFF), qy - ((pxy >> 16) & 0x7FFF),
                                                      make_float3(mv.x, mv.y, mv.z));
                            e += D.x * w.x + D.y * w.y + D.z * w.z;
                        }
                        dacc[s] += P.CD * e;
                    }
                }
                if (bk + 1 < nblk) etab_fill(bk + 1, ht, kH);
                }
            }
            gsync();
        }
    } else {
        // Blocks of G sub-steps (16 sites), two CTA barriers per block.  At the start
        // of block b all warps add the moves of block b-1 to the fields of block b's
        // sites, which then hold the stale field plus every move before the block (the
        // moves of blocks <= b-2 were pushed there earlier by the helpers), and tabulate
        // W~ between each site of the block and the sites of its earlier sub-steps.
        // Then warp 0 (the decider) runs the block's sub-steps alone, pulling the moves
        // of the block's earlier sub-steps through that table (lanes split them, a
        // shuffle reduction sums them per site), while warps 1.. (the helpers) push the
        // moves of block b-1 into every site of blocks >= b+1.  Block move lists are
        // compact (accepted moves only) and double-buffered by parity.
        constexpr int LPS = 32 / n;                       // decider lanes per site
        const int dsite = lane / LPS, dsub = lane % LPS;  // decider lane -> (site, move subset)
        constexpr int tps = kWThreads / NB;               // threads per block site in the catch-up
        for (int bk = 0; bk < nblk; ++bk) {
            const int cur = bk & 1, prv = cur ^ 1;
            const int nprev = bk > 0 ? s_nmv[prv] : 0;
            if (G > 1) {
                // W~ between each site of the block and the sites of its earlier sub-steps
                const int base = bk * NB;
                for (int idx = tid; idx < NB * NB; idx += kWThreads) {
                    const int i = idx / NB, i2 = idx - i * NB;
                    if (i2 / n < i / n) {
                        const int a = wxy[base + i], c = wxy[base + i2];
                        wpair[idx] = wq_get(wq, L, (a & 0xFFFF) - (c & 0xFFFF), ((a >> 16) & 0x7FFF) - ((c >> 16) & 0x7FFF));
                    }
                }
            }
            if (nprev > 0) {
                // catch-up: the moves of block b-1 into the sites of block b
                const int site = tid / tps, g = tid - site * tps, s = bk * NB + site;
                const int xy = wxy[s];
                const int qx = xy & 0xFFFF, qy = (xy >> 16) & 0x7FFF;
                float3 cr = make_float3(0.f, 0.f, 0.f);
                for (int m = g; m < nprev; m += tps) {
                    const float4 mv = s_mvb[prv * NB + m];
                    const int pxy = __float_as_int(mv.w);
                    const float3 c = wq_apply(wq, L, qx - (pxy & 0xFFFF), qy - ((pxy >> 16) & 0x7FFF),
                                              make_float3(mv.x, mv.y, mv.z));
                    cr.x += c.x;
                    cr.y += c.y;
                    cr.z += c.z;
                }
                for (int off = 1; off < tps; off <<= 1) {
                    cr.x += __shfl_xor_sync(0xffffffffu, cr.x, off);
                    cr.y += __shfl_xor_sync(0xffffffffu, cr.y, off);
                    cr.z += __shfl_xor_sync(0xffffffffu, cr.z, off);
                }
                if (g == 0) {
                    float4 h = hcur[s];
                    h.x += cr.x;
                    h.y += cr.y;
                    h.z += cr.z;
                    hcur[s] = h;
                }
            }
            if (G > 1 || nprev > 0) gsync();
            if (warp == 0) {
                int ncur = 0;                                    // moves of this block so far (warp-uniform)
                for (int u = 0; u < G; ++u) {
                    const int j = bk * G + u;
                    const int s = j * n + dsite;
                    const int xy = wxy[s];
                    const int qx = xy & 0xFFFF, qy = (xy >> 16) & 0x7FFF, q = qy * L + qx;
                    // pull: moves of this block's earlier sub-steps (pd holds the move of an
                    // accepted site and zero for a rejected one), split over the site's lanes
                    float3 cr = make_float3(0.f, 0.f, 0.f);
                    const float4 *wrow = wpair + (u * n + dsite) * NB;
                    const int base = bk * NB;
                    for (int i2 = dsub; i2 < u * n; i2 += LPS) {
                        const float4 w = wrow[i2], mv = pd[base + i2];
                        cr.x += w.x * mv.x + w.y * mv.y;
                        cr.y += w.y * mv.x + w.z * mv.y;
                        cr.z += w.w * mv.z;
                    }
#pragma unroll
                    for (int off = 1; off < LPS; off <<= 1) {
                        cr.x += __shfl_xor_sync(0xffffffffu, cr.x, off);
                        cr.y += __shfl_xor_sync(0xffffffffu, cr.y, off);
                        cr.z += __shfl_xor_sync(0xffffffffu, cr.z, off);
                    }
                    int accept = 0;
                    float dX = 0.f, dY = 0.f, dZ = 0.f;
                    if (dsub == 0) {
                        float4 h = hcur[s];
                        h.x += cr.x;
                        h.y += cr.y;
                        h.z += cr.z;
                        const float3 nb3 = nbr_sum(qx, qy);
                        const uint4 wds = attempt_rng(s, q);
                        float sps, cps;
                        sincospif(2.0f * u24f(wds.y), &sps, &cps);
                        const float uu = u24f(wds.z);
                        float4 S, D;
                        propose(q, u24f(wds.x), cps, sps, S, D);
                        const float thr = (uu > 0.0f) ? -P.T * logf(uu) : INFINITY;
                        dX = D.x;
                        dY = D.y;
                        dZ = D.z;
                        const float dex = -P.J * (dX * nb3.x + dY * nb3.y + dZ * nb3.z);
                        const float dE = D.w + dex + P.CD * (dX * h.x + dY * h.y + dZ * h.z);
                        accept = dE < thr;
                        if (buf.trace) {
                            float *tr = trace_row(s);
                            tr[0] = (float)q;
                            tr[1] = h.x; tr[2] = h.y; tr[3] = h.z;
                            tr[4] = dE;
                            tr[5] = uu;
                            tr[6] = (float)accept;
                            tr[7] = S.x; tr[8] = S.y; tr[9] = S.z;
                        }
                        if (accept) {
                            set_spin(q, S.x, S.y, S.z);
                            wxy[s] = xy | (int)0x80000000;             // accepted
                        }
                        // the move (for the block's later sub-steps and the window-end bookkeeping)
                        pd[s] = accept ? make_float4(dX, dY, dZ, dE) : make_float4(0.f, 0.f, 0.f, 0.f);
                        pS[s] = make_float4(S.x, S.y, S.z, dE);
                    }
                    // append the accepted moves of this sub-step to the block's list, in site order
                    const unsigned ball = __ballot_sync(0xffffffffu, accept);
                    if (accept) {
                        const unsigned below = ball & ((1u << lane) - 1u);
                        s_mvb[cur * NB + ncur + __popc(below)] = make_float4(dX, dY, dZ, __int_as_float(xy));
                    }
                    ncur += __popc(ball);
                    __syncwarp();
                }
                if (lane == 0) {
                    s_nmv[cur] = ncur;
                    n_acc += ncur;
                }
            } else if (nprev > 0) {
                // helpers: push the moves of block b-1 into the sites of blocks >= b+1
                constexpr int kH = kWThreads - 32;
                for (int s = (bk + 1) * NB + (tid - 32); s < Sw; s += kH) {
                    const int xy = wxy[s];
                    const int qx = xy & 0xFFFF, qy = (xy >> 16) & 0x7FFF;
                    float4 h = hcur[s];
                    for (int m = 0; m < nprev; ++m) {
                        const float4 mv = s_mvb[prv * NB + m];
                        const int pxy = __float_as_int(mv.w);
                        const float3 c = wq_apply(wq, L, qx - (pxy & 0xFFFF), qy - ((pxy >> 16) & 0x7FFF),
                                                  make_float3(mv.x, mv.y, mv.z));
                        h.x += c.x;
                        h.y += c.y;
                        h.z += c.z;
                    }
                    hcur[s] = h;
                }
            }
            gsync();
        }
    }

    if (tid == 0) cyc2 = clock64();
    // ---- write the accepted moves back to global memory (FP32 and the bf16 split);
    // stale_mode 3 also marks the offset groups whose spectra change (S_w is a multiple of
    // 256 there, so every warp runs the loop whole)
    float *gd = buf.spins + (size_t)r * 3 * N;
    const int nck = (l * l) >> 4;   // stale_mode 3 (l % 8 == 0): groups of 16 offsets
    for (int s = tid; s < Sw; s += kWThreads) {
        const int xy = wxy[s];
        if (cfg.stale_mode == 3) {
            int c = -1;
            if (xy < 0) {
                const int x = xy & 0xFFFF, y = (xy >> 16) & 0x7FFF;
                const int ox = x >= l ? x - l : x, oy = y >= l ? y - l : y;
                c = (oy * l + (l - 1 - ox)) >> 4;
            }
            for (int w = 0; w < kSpecWords && 32 * w < nck; ++w) {
                const uint32_t m = __reduce_or_sync(0xffffffffu, (c >> 5) == w ? 1u << (c & 31) : 0u);
                if (lane == 0 && m) atomicOr(&s_ck[w], m);
            }
        }
        if (xy >= 0) continue;
        const int q = ((xy >> 16) & 0x7FFF) * L + (xy & 0xFFFF);
        const float3 v = spin(q);
        gd[q] = v.x;
        gd[N + q] = v.y;
        gd[2 * N + q] = v.z;
        if (buf.spins_hi && cfg.stale_mode != 3) {
            __nv_bfloat16 *hi = buf.spins_hi + (size_t)r * 3 * N;
            __nv_bfloat16 *lo = buf.spins_lo + (size_t)r * 3 * N;
            const float v3[3] = {v.x, v.y, v.z};
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) {
                const __nv_bfloat16 h16 = __float2bfloat16_rn(v3[cc]);
                hi[cc * N + q] = h16;
                lo[cc * N + q] = __float2bfloat16_rn(v3[cc] - __bfloat162float(h16));
            }
        }
    }
    // ---- exact energy change of the window: accepted dE plus, per sub-step, the
    // neglected cross terms C_D d_p.W~(q - p).d_q of its simultaneous moves (Sec. 3.2).
    // PRE: a thread per accepted site and per site pair of a sub-step; otherwise a thread
    // per sub-step
    double e_loc = 0.0;
    if (PRE) {
        float e_f = 0.0f;   // a few terms per thread
        for (int s = tid; s < Sw; s += kWThreads)
            if (wxy[s] < 0) e_f += pS[s].w;
        constexpr int npair = n * (n - 1) / 2;   // site pairs d > dp of a sub-step
        if constexpr (npair > 0) {
            for (int task = tid; task < B * npair; task += kWThreads) {
                const int j = task / npair;
                int d = 1, dp = task - j * npair;
                while (dp >= d) {
                    dp -= d;
                    ++d;
                }
                const int xy = wxy[j * n + d], pxy = wxy[j * n + dp];
                if (xy >= 0 || pxy >= 0) continue;
                const float4 m = pd[j * n + d], mp = pd[j * n + dp];
                float3 Wd;
                if constexpr (SPX) {
                    // cells d and dp of one offset: W~(l P), P = d xor dp
                    const float4 w = s_wl[d ^ dp];
                    Wd = make_float3(w.x * m.x + w.y * m.y, w.y * m.x + w.z * m.y, w.w * m.z);
                } else {
                    Wd = w_apply_sites(xy & 0xFFFF, (xy >> 16) & 0x7FFF, pxy & 0xFFFF, (pxy >> 16) & 0x7FFF,
                                       make_float3(m.x, m.y, m.z));
                }
                e_f += P.CD * (mp.x * Wd.x + mp.y * Wd.y + mp.z * Wd.z);
            }
        }
        // a few terms per thread, then 32 per warp in FP32; the warps' sums in FP64
        for (int off = 16; off; off >>= 1) e_f += __shfl_xor_sync(0xffffffffu, e_f, off);
        e_loc = (double)e_f;
    }
    for (int j = tid; !PRE && j < B; j += kWThreads) {
        float sub = 0.0f;
        for (int d = 0; d < n; ++d) {
            const int s = j * n + d;
            const int xy = wxy[s];
            if (xy >= 0) continue;
            const float4 m = pd[s];
            sub += pS[s].w;
            for (int dp = 0; dp < d; ++dp) {
                const int pxy = wxy[j * n + dp];
                if (pxy >= 0) continue;
                const float4 mp = pd[j * n + dp];
                const float3 Wd = wq_apply(wq, L, (xy & 0xFFFF) - (pxy & 0xFFFF),
                                           ((xy >> 16) & 0x7FFF) - ((pxy >> 16) & 0x7FFF), make_float3(m.x, m.y, m.z));
                sub += P.CD * (mp.x * Wd.x + mp.y * Wd.y + mp.z * Wd.z);
            }
        }
        e_loc += (double)sub;
    }
    if (!PRE)
        for (int off = 16; off; off >>= 1) e_loc += __shfl_xor_sync(0xffffffffu, e_loc, off);
    if (lane == 0) s_epart[warp] = e_loc;
    gsync();
    if (tid == 0) {
        double et = 0.0;
        for (int i = 0; i < kWThreads / 32; ++i) et += s_epart[i];
        // one adder per replica and launch: the reduction without a read-back is the
        // same sum; a measured window needs the value
        if (cfg.measure) {
            s_energy = buf.energy[r] + et;
            buf.energy[r] = s_energy;
        } else {
            atomicAdd(buf.energy + r, et);
        }
    }
    if (cfg.stale_mode == 3) {
        // ---- spectra S'[r][kappa][a][e'] (bf16 hi/lo) of every marked offset group after the
        // window's moves, F(kappa) = sum_D (-1)^(kappa.D) s(o + l D).  A thread takes two
        // adjacent offsets e', e' + 1 (columns ex, ex - 1 of one row) through all twelve
        // (kappa, a) planes, so eight threads fill one 32-byte sector of a plane; an unchanged
        // offset of a marked group is rewritten with the bits it already holds (same sum order)
        const int lsq = l * l;
        __nv_bfloat16 *hi = buf.spins_hi + (size_t)r * 12 * lsq, *lo = buf.spins_lo + (size_t)r * 12 * lsq;
        for (int task = tid; task < nck * 8; task += kWThreads) {
            const int c = task >> 3;
            if (c < 32 * kSpecWords && !((s_ck[c >> 5] >> (c & 31)) & 1u)) continue;
            const int ep = (c << 4) + ((task & 7) << 1);
            const int ey = ep / l, ex = l - 1 - (ep - ey * l);   // ex odd: e' + 1 sits at ex - 1
            float2 sv[3][4];
#pragma unroll
            for (int aa = 0; aa < 3; ++aa)
#pragma unroll
                for (int D = 0; D < 4; ++D)
                    sv[aa][D] = *reinterpret_cast<const float2 *>(sxyz + aa * N + (ey + l * (D >> 1)) * L + ex - 1 + l * (D & 1));
#pragma unroll
            for (int kap = 0; kap < 4; ++kap)
#pragma unroll
                for (int aa = 0; aa < 3; ++aa) {
                    float v0 = 0.0f, v1 = 0.0f;   // offsets e' (.y) and e' + 1 (.x)
#pragma unroll
                    for (int D = 0; D < 4; ++D) {
                        const bool neg = ((kap & 1) * (D & 1) + (kap >> 1) * (D >> 1)) & 1;
                        v0 += neg ? -sv[aa][D].y : sv[aa][D].y;
                        v1 += neg ? -sv[aa][D].x : sv[aa][D].x;
                    }
                    const __nv_bfloat16 h0 = __float2bfloat16_rn(v0), h1 = __float2bfloat16_rn(v1);
                    const size_t idx = (size_t)(kap * 3 + aa) * lsq + ep;
                    *reinterpret_cast<__nv_bfloat162 *>(hi + idx) = __halves2bfloat162(h0, h1);
                    *reinterpret_cast<__nv_bfloat162 *>(lo + idx) = __halves2bfloat162(
                        __float2bfloat16_rn(v0 - __bfloat162float(h0)), __float2bfloat16_rn(v1 - __bfloat162float(h1)));
                }
        }
    }
    if (cfg.measure) {
        gsync();
        float mv_[12] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        double *gt = buf.theta2 ? buf.theta2 + (size_t)r * N : nullptr;
        // two sites of a row a thread (L even): i and i + 1, their right neighbours i + 1 and
        // (ix + 2) mod L, and the sites below them, with the shared loads as pairs
#pragma unroll 2
        for (int i = 2 * tid; i < N; i += 2 * kWThreads) {
            const int iy = i / L, ix = i - iy * L;
            const int ir = iy * L + (ix + 2 == L ? 0 : ix + 2), id = (iy + 1 == L ? 0 : iy + 1) * L + ix;
            float2 va[3], vd[3];
            float vr[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                va[c] = *reinterpret_cast<const float2 *>(sxyz + c * N + i);
                vd[c] = *reinterpret_cast<const float2 *>(sxyz + c * N + id);
                vr[c] = sxyz[c * N + ir];
            }
            const float zr = (iy & 1) ? -1.0f : 1.0f;   // m1 + m2 - m3 - m4 (rows); columns: ix even
            mv_[0] += va[0].x + va[0].y;
            mv_[1] += va[1].x + va[1].y;
            mv_[2] += va[2].x + va[2].y;
            mv_[3] += zr * (va[2].x + va[2].y);
            mv_[4] += va[2].x - va[2].y;                 // m1 + m4 - m3 - m2 (columns)
            mv_[5] += wall_term(va[0].x, va[0].y) + wall_term(va[0].y, vr[0]);
            mv_[6] += wall_term(va[0].x, vd[0].x) + wall_term(va[0].y, vd[0].y);
            mv_[7] += wall_term(va[1].x, va[1].y) + wall_term(va[1].y, vr[1]);
            mv_[8] += wall_term(va[1].x, vd[1].x) + wall_term(va[1].y, vd[1].y);
            mv_[9] += wall_term(va[2].x, va[2].y) + wall_term(va[2].y, vr[2]);
            mv_[10] += wall_term(va[2].x, vd[2].x) + wall_term(va[2].y, vd[2].y);
            const float th0 = acosf(fminf(1.0f, fmaxf(-1.0f, va[2].x))) - 0.5f * kPiF;
            const float th1 = acosf(fminf(1.0f, fmaxf(-1.0f, va[2].y))) - 0.5f * kPiF;
            mv_[11] += fabsf(th0) + fabsf(th1);
            if (gt) {
                double2 *g2 = reinterpret_cast<double2 *>(gt + i);
                double2 v = *g2;
                v.x += (double)(th0 * th0);
                v.y += (double)(th1 * th1);
                *g2 = v;
            }
        }
#pragma unroll
        for (int c = 0; c < 12; ++c)
            for (int off = 16; off; off >>= 1) mv_[c] += __shfl_xor_sync(0xffffffffu, mv_[c], off);
        if (lane == 0)
#pragma unroll
            for (int c = 0; c < 12; ++c) s_mred[warp][c] = mv_[c];
        gsync();
        // the sample once, in FP64 across the lanes of one warp: lane c sums component c over
        // the warps; every quotient of the observables is one lane's share of a single
        // division, the three norms of a single square root; then lane k < kNB pushes the
        // sample into binning level k
        if (warp == 0 && buf.obs) {
            double smv = 0.0;
            if (lane < 12)
                for (int ww = 0; ww < kWThreads / 32; ++ww) smv += s_mred[ww][lane];
            double sm[12];
#pragma unroll
            for (int c = 0; c < 12; ++c) sm[c] = __shfl_sync(0xffffffffu, smv, c);
            const double Nd = (double)N;
            // lanes 0-4: M_x, M_y, M_z, M_h, M_v; 5: E/N; 6: wall density; 7-9: O_x, O_y, O_z
            // (n_h^a = sm[5 + 2a], n_v^a = sm[6 + 2a]); 10: cone angle
            const double nh = lane == 7 ? sm[5] : (lane == 8 ? sm[7] : sm[9]);
            const double nv = lane == 7 ? sm[6] : (lane == 8 ? sm[8] : sm[10]);
            const double osum = nh + nv;
            const bool ol = lane >= 7 && lane <= 9;
            double num = 0.0, den = 1.0;
            if (lane < 5) { num = smv; den = Nd; }
            else if (lane == 5) { num = s_energy; den = Nd; }
            else if (lane == 6) { num = sm[10] + sm[9]; den = 4.0 * Nd; }
            else if (ol) { num = fabs(nh - nv); den = osum > 0.0 ? osum : 1.0; }
            else if (lane == 10) { num = 0.63661977236758134 * sm[11]; den = Nd; }   // 2/pi
            double q = num / den;
            if (ol && !(osum > 0.0)) q = 0.0;
            const double Mx = __shfl_sync(0xffffffffu, q, 0), My = __shfl_sync(0xffffffffu, q, 1),
                         Mz = __shfl_sync(0xffffffffu, q, 2), Mh = __shfl_sync(0xffffffffu, q, 3),
                         Mv = __shfl_sync(0xffffffffu, q, 4);
            const double rad = lane == 0 ? Mx * Mx + My * My + Mz * Mz
                                         : (lane == 1 ? Mx * Mx + My * My : (lane == 2 ? Mh * Mh + Mv * Mv : 0.0));
            const double rt = sqrt(rad);
            double x[MC_NOBS];
            x[MC_OBS_ABS_M] = __shfl_sync(0xffffffffu, rt, 0);
            x[MC_OBS_MZ] = Mz;
            x[MC_OBS_ABS_MZ] = fabs(Mz);
            x[MC_OBS_MPAR] = __shfl_sync(0xffffffffu, rt, 1);
            x[MC_OBS_E] = __shfl_sync(0xffffffffu, q, 5);
            x[MC_OBS_MST] = __shfl_sync(0xffffffffu, rt, 2);
            x[MC_OBS_WALL] = __shfl_sync(0xffffffffu, q, 6);
            x[MC_OBS_OX] = __shfl_sync(0xffffffffu, q, 7);
            x[MC_OBS_OY] = __shfl_sync(0xffffffffu, q, 8);
            x[MC_OBS_OZ] = __shfl_sync(0xffffffffu, q, 9);
            x[MC_OBS_CONE] = __shfl_sync(0xffffffffu, q, 10);
            if (lane == 0) hist_push(buf.hist, r, x[MC_OBS_E]);
            if (lane < kNB) obs_push_level(buf.obs[r], x, lane);
        }
    }
    if (warp == dw && lane == 0 && buf.obs)
        atomicAdd(reinterpret_cast<unsigned long long *>(&buf.obs[r].accepted), (unsigned long long)n_acc);
    if (tid == 0 && buf.cycles) {
        atomicAdd(buf.cycles + 0, (unsigned long long)(cyc2 - cyc1));
        atomicAdd(buf.cycles + 1, (unsigned long long)(cyc1 - cyc0));
        atomicAdd(buf.cycles + 2, (unsigned long long)(clock64() - cyc2));
        atomicAdd(buf.cycles + 3, (unsigned long long)nblk);
    }
    if (tid == 0 && buf.obs)
        atomicAdd(reinterpret_cast<unsigned long long *>(&buf.obs[r].attempted), (unsigned long long)Sw);
}

__global__ void k_build_wq(int L, const float *__restrict__ W32, float4 *wq) {
    const int hq = L / 2 + 1, N = L * L;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= hq * hq) return;
    const int g = (i / hq) * L + (i % hq);
    wq[i] = make_float4(W32[g], W32[N + g], W32[2 * N + g], W32[3 * N + g]);
}

// The sub-lattice spectra of W~ for l = L/2 (the table U of the permutation-schedule
// sub-steps at L = 2l): U_d(kappa) = sum_P (-1)^(kappa.P) W~(d + l P), P in {0,1}^2,
// for 0 <= dx, dy <= l/2; one thread per entry, the four terms summed in FP64.
__global__ void k_build_uq(int L, const float *__restrict__ W32, float4 *uq) {
    const int l = L / 2, hu = l / 2 + 1, N = L * L;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 4 * hu * hu) return;
    const int kap = i & 3, cell = i >> 2, dx = cell % hu, dy = cell / hu;
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int P = 0; P < 4; ++P) {
        const double sg = (__popc(kap & P) & 1) ? -1.0 : 1.0;
        const int g = (dy + l * (P >> 1)) * L + dx + l * (P & 1);
        for (int c = 0; c < 4; ++c) a[c] += sg * (double)W32[c * N + g];
    }
    uq[i] = make_float4((float)a[0], (float)a[1], (float)a[2], (float)a[3]);
}

__global__ void k_spins_to_bf16(size_t count, const float *__restrict__ s, __nv_bfloat16 *hi, __nv_bfloat16 *lo) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float x = s[i];
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi[i] = h;
    lo[i] = __float2bfloat16_rn(x - __bfloat162float(h));
}

}  // namespace

size_t wq_table_elems(int L) {
    const size_t hq = (size_t)(L / 2 + 1), hu = (size_t)(L / 4 + 1);
    return hq * hq + (L % 2 == 0 ? 4 * hu * hu : 0);
}

size_t window_smem_bytes(int L, int Sw, int n) {
    const size_t N = (size_t)L * L;
    // blocks of kBlockSites sites (n <= kBlockSites)
    return sizeof(float) * 3 * N +
           sizeof(float4) * (3 * (size_t)Sw + (size_t)wtab_smem_elems(L, n) + 2 * kBlockSites + kBlockSites * kBlockSites) +
           sizeof(int) * (size_t)Sw + sizeof(float) * 3 * (size_t)Sw;   // sites, split-K sums
}

bool window_supported(int L, int l, int B) {
    if (l < 2 || L % l || L % 2) return false;   // even L: 16-byte aligned spin rows
    const int C = L / l;
    if (C != 1 && C != 2 && C != 4) return false;
    if (B < 1 || (l * l) % B) return false;
    // decider blocks of 16 sites: whole sub-steps
    const int n = C * C;
    if (B % (kBlockSites / n)) return false;
    return window_smem_bytes(L, B * C * C, C * C) <= 200 * 1024;
}

cudaError_t launch_window_steps(const WindowConfig &c0, const WindowBuffers &b, cudaStream_t st) {
    const int C = c0.L / c0.l;
    // two replicas a CTA (one on the even, one on the odd warps) when the replicas outnumber the
    // SMs, so that two would share an SM anyway, and both fit its shared memory; else one replica
    // a CTA, each alone on its SM while R <= SM count
    const size_t group = (window_smem_bytes(c0.L, c0.B * C * C, C * C) + 127) & ~(size_t)127;
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    WindowConfig c = c0;
    c.gpc = (c0.R > nsm && 2 * group <= kWindowSmemTwoGroups) ? 2 : 1;
    c.smem_group = (unsigned)group;
    const size_t smem = c.gpc * group;
    cudaError_t e;
#define LAUNCH1(CC, PRE)                                                                             \
    e = cudaFuncSetAttribute(k_window_steps<CC, PRE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    if (e != cudaSuccess) return e;                                                                  \
    {                                                                                                \
        cudaLaunchConfig_t lc{};                                                                     \
        lc.gridDim = dim3((c.R + c.gpc - 1) / c.gpc);                                                \
        lc.blockDim = dim3(kWThreads * c.gpc);                                                       \
        lc.dynamicSmemBytes = smem;                                                                  \
        lc.stream = st;                                                                              \
        cudaLaunchAttribute at[1];                                                                   \
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;                               \
        at[0].val.programmaticStreamSerializationAllowed = 1;                                        \
        lc.attrs = at;                                                                               \
        lc.numAttrs = 1;                                                                             \
        e = cudaLaunchKernelEx(&lc, k_window_steps<CC, PRE>, c, b);                                  \
        if (e != cudaSuccess) return e;                                                              \
    }
#define LAUNCH(CC)                                                                                   \
    if (c.schedule == 0) { LAUNCH1(CC, true) } else { LAUNCH1(CC, false) }
    if (C == 1) { LAUNCH(1) }
    else if (C == 2) { LAUNCH(2) }
    else if (C == 4) { LAUNCH(4) }
    else return cudaErrorNotSupported;
#undef LAUNCH
#undef LAUNCH1
    return cudaGetLastError();
}

__global__ void k_set_u32(uint32_t *dst, uint32_t v) { *dst = v; }

cudaError_t launch_set_u32(uint32_t *dst, uint32_t v, cudaStream_t st) {
    k_set_u32<<<1, 1, 0, st>>>(dst, v);
    return cudaGetLastError();
}

cudaError_t launch_build_wq(int L, const float *W32, float4 *wq, cudaStream_t st) {
    const int hq = L / 2 + 1;
    k_build_wq<<<(hq * hq + 127) / 128, 128, 0, st>>>(L, W32, wq);
    if (L % 2 == 0) {
        const int hu = L / 4 + 1;
        k_build_uq<<<(4 * hu * hu + 127) / 128, 128, 0, st>>>(L, W32, wq + (size_t)hq * hq);
    }
    return cudaGetLastError();
}

cudaError_t launch_spins_to_bf16(size_t count, const float *s, __nv_bfloat16 *hi, __nv_bfloat16 *lo, cudaStream_t st) {
    k_spins_to_bf16<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(count, s, hi, lo);
    return cudaGetLastError();
}

}  // namespace dipmc
