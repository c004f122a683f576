// fft_cluster.cu -- the sweep of one replica in a thread-block cluster that keeps
// the replica's 2D Fourier transform in its CTAs' shared memory.
//
// The field (Sec. 2.1, Eq. 2) is a circular convolution, h = W~ * s, so with the
// 2D DFT F(k) = sum_r f(r) e^{-2 pi i k.r / L}:  H^(k) = W^(k) S^(k) (W^ is real:
// W~ is even) and h(r) = (1/N) sum_k e^{2 pi i k.r / L} H^(k).  The sites of a
// sub-step are x_j = o_x + l j, y_i = o_y + l i, i, j < C = L / l (Sec. 3.1).
// Grouping ky by its residue r = ky mod C (e^{2 pi i ky l i / L} depends on r only):
//   P_c(kx, r)  = sum_{ky = r mod C} e^{2 pi i ky o_y / L} H^_c(kx, ky),
//   G_c(kx, y_i) = sum_r e^{2 pi i r i / C} P_c(kx, r),
// and, the spins being real, only kx in [0, L/2] is kept (weight 2 for 0 < kx < L/2):
//   h_c(x_j, y_i) = (1/N) sum_kx w(kx) Re[e^{2 pi i kx x_j / L} G_c(kx, y_i)].
// After the decisions the accepted moves d(i, j) update the transform exactly:
//   S^_c(kx, ky) += e^{-2 pi i ky o_y / L} B_c(kx, ky mod C),
//   B_c(kx, r)   = sum_i e^{-2 pi i r i / C} sum_j d_c(i, j) e^{-2 pi i kx x_j / L}.
// A sub-step is thus one pass over a CTA's columns of S^ for the field and one for
// the update, plus one cluster barrier, instead of a full 2D FFT convolution.
//
// A cluster of 16 CTAs per replica.  CTA c owns rows [c H, c H + H) of the spins
// (H = L / 16) and columns kx in [c K2 / 16, (c + 1) K2 / 16) of S^ and W^
// (K2 = L/2 + 1).  Per sub-step, with ONE cluster barrier:
//   1. every CTA: P over its columns, then G, then its columns' share of the field
//      at the n sites, into a share buffer of the sub-step's parity;  barrier;
//   2. every CTA takes all n decisions itself (the same inputs and arithmetic in
//      every CTA, so the same results): field = the 16 shares summed in rank
//      order, spins of the sites and their neighbours from the owning CTAs,
//      proposals and Metropolis decisions (every site from the state before the
//      step, Sec. 3.1, 3.2);
//   3. every CTA updates its columns of S^ with the moves; the owner of a site's
//      row writes the new spin.
// The spin rows are double-buffered by sub-step parity: sub-step k reads copy
// k % 2 (the state before it) while the owners bring copy (k + 1) % 2 up to date
// with the moves of sub-steps k - 1 and k, so no CTA writes what another may
// still be reading.
// S^ is a direct 2D DFT of the spins taken before each sweep, so the FP32 rounding
// of the updates accumulates over one sweep at most.
#include <cooperative_groups.h>

#include <map>
#include <mutex>
#include <tuple>

#include "fft_cluster.cuh"

namespace cg = cooperative_groups;

namespace dipmc {

namespace {

constexpr int kCT = 256;   // threads per CTA

// Shared-memory layout of one CTA (bytes from the dynamic base; 16-byte aligned).
struct CLayout {
    int L, l, C, n, H, K2, nk;   // nk: the most kx columns a CTA owns
    int LP;                      // column stride of S^ and W^: L + C, so that the C-strided
                                 // reads of a warp's column groups fall in distinct banks
    int sched_on;                // the sweep's offsets tabulated at the start (l^2 <= kSchedMax)
    size_t o_tw, o_sp, o_S, o_W, o_P, o_G, o_part, o_mv, o_sch, bytes;
};

constexpr int kSchedMax = 4096;

__host__ __device__ inline size_t up16(size_t b) { return (b + 15) & ~(size_t)15; }

__host__ __device__ inline CLayout clayout(int L, int l) {
    CLayout g{};
    g.L = L;
    g.l = l;
    g.C = L / l;
    g.n = g.C * g.C;
    g.H = L / kClusterCtas;
    g.K2 = L / 2 + 1;
    g.nk = (g.K2 + kClusterCtas - 1) / kClusterCtas;
    g.LP = L + g.C;
    g.sched_on = l * l <= kSchedMax;
    size_t o = 0;
    g.o_tw = o;   o = up16(o + sizeof(float2) * L);                          // e^{2 pi i m / L}
    g.o_sp = o;   o = up16(o + sizeof(float) * 2 * 3 * g.H * L);             // [2][3][H][L] own rows, by parity
    g.o_S = o;    o = up16(o + sizeof(float2) * 3 * g.nk * g.LP);            // [3][nk][LP] own columns of S^
    g.o_W = o;    o = up16(o + sizeof(float) * 4 * g.nk * g.LP);             // [4][nk][LP] own columns of W^
    g.o_P = o;    o = up16(o + sizeof(float2) * 3 * g.nk * g.C);             // [3][nk][C] P, then A
    g.o_G = o;    o = up16(o + sizeof(float2) * 3 * g.nk * g.C);             // [3][nk][C] G, then B
    g.o_part = o; o = up16(o + sizeof(float4) * 2 * g.n);                    // [2][n] field shares (x, y, z, -), by parity
    g.o_mv = o;   o = up16(o + sizeof(float4) * 2 * 2 * g.n);                // [2][n] (d, accepted), [2][n] S, by parity
    g.o_sch = o;  o = up16(o + (g.sched_on ? sizeof(uint16_t) * l * l : 0)); // [l^2] offsets of the sweep
    g.bytes = o;
    return g;
}

// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) { return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y); }

__global__ void __launch_bounds__(kCT, 1) k_cluster_sweep(const ClusterSweepArgs a) {
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int r = blockIdx.x / kClusterCtas;
    const int tid = threadIdx.x;
    const CLayout g = clayout(a.L, a.l);
    const int L = g.L, l = g.l, C = g.C, n = g.n, H = g.H, K2 = g.K2, nk = g.nk, N = L * L, ll = l * l;
    const int HL = H * L, LP = g.LP;
    const int mask = L - 1;   // L is a power of two
    extern __shared__ __align__(16) unsigned char smc[];
    float2 *tw = reinterpret_cast<float2 *>(smc + g.o_tw);
    float *sp = reinterpret_cast<float *>(smc + g.o_sp);            // copy b at sp + b * 3 HL
    float2 *Sh = reinterpret_cast<float2 *>(smc + g.o_S);
    float *Wh = reinterpret_cast<float *>(smc + g.o_W);
    float2 *Pb = reinterpret_cast<float2 *>(smc + g.o_P);
    float2 *Gb = reinterpret_cast<float2 *>(smc + g.o_G);
    float4 *part = reinterpret_cast<float4 *>(smc + g.o_part);      // copy b at part + b * n
    float4 *mvd = reinterpret_cast<float4 *>(smc + g.o_mv);         // [b][n]: (d, accepted)
    float4 *mvs = mvd + 2 * n;                                      // [b][n]: S
    uint16_t *sch = reinterpret_cast<uint16_t *>(smc + g.o_sch);
    __shared__ int s_off;

    const int kx0 = rank * K2 / kClusterCtas, kx1 = (rank + 1) * K2 / kClusterCtas, nkx = kx1 - kx0;
    const int y0 = rank * H;
    const RepParams P = a.params[r];
    const uint2 key = a.key;
    const uint32_t t = a.t_dev ? *a.t_dev + (uint32_t)a.it : a.t;
    const float *gs = a.spins + (size_t)r * 3 * N;
    const uint4 rk = a.schedule == 0 ? philox(make_uint4(t, 0u, 0u, kTagPerm), key) : make_uint4(0, 0, 0, 0);
    const int hbits = ceil_log2_u((uint32_t)l);
    auto offset_of = [&](int k) -> int {
        if (a.schedule == 0) return (int)perm_offset(rk, hbits, (uint32_t)ll, (uint32_t)k);
        const uint4 o = philox(make_uint4(t, (uint32_t)k, 0u, kTagDraw), key);
        return (int)(((unsigned long long)o.x * (unsigned long long)ll) >> 32);
    };

    // ---- set-up: twiddles, both copies of the own rows, own columns of S^ and W^, offsets
    for (int m = tid; m < L; m += kCT) {
        float sn, cs;
        sincospif(2.0f * (float)m / (float)L, &sn, &cs);
        tw[m] = make_float2(cs, sn);
    }
    for (int i = tid; i < 3 * HL; i += kCT) {
        const int c = i / HL, rem = i - c * HL;
        const float v = gs[(size_t)c * N + (size_t)y0 * L + rem];
        sp[i] = v;
        sp[3 * HL + i] = v;
    }
    for (int i = tid; i < 3 * nkx * L; i += kCT) {
        const int c = i / (nkx * L), rem = i - c * nkx * L, kl = rem / L, ky = rem - kl * L;
        Sh[(c * nk + kl) * LP + ky] = a.Shat[(((size_t)r * 3 + c) * K2 + kx0 + kl) * L + ky];
    }
    for (int i = tid; i < 4 * nkx * L; i += kCT) {
        const int c = i / (nkx * L), rem = i - c * nkx * L, kl = rem / L, ky = rem - kl * L;
        Wh[(c * nk + kl) * LP + ky] = a.What[((size_t)c * K2 + kx0 + kl) * L + ky];
    }
    if (g.sched_on)
        for (int k = tid; k < ll; k += kCT) sch[k] = (uint16_t)offset_of(k);
    for (int i = tid; i < 4 * n; i += kCT) mvd[i] = make_float4(0.f, 0.f, 0.f, 0.f);   // both parities, d and S
    const float W0xx = __ldg(a.W32), W0xy = __ldg(a.W32 + N), W0yy = __ldg(a.W32 + 2 * N), W0zz = __ldg(a.W32 + 3 * N);
    const float invN = 1.0f / (float)N;
    long long nacc = 0;
    int prev_off = 0;
    __syncthreads();

    for (int k = 0; k < ll; ++k) {
        const int b = k & 1;
        int v;
        if (g.sched_on) {
            v = sch[k];
        } else {
            if (tid == 0) s_off = offset_of(k);
            __syncthreads();
            v = s_off;
        }
        const int ox = v % l, oy = v / l;
        const float *spb = sp + b * 3 * HL;   // the state before this sub-step

        // ---- 1a. P_c(kx, r) over this CTA's columns
        for (int task = tid; task < 3 * nkx * C; task += kCT) {
            const int c = task / (nkx * C), rem = task - c * nkx * C, kl = rem / C, rr = rem - kl * C;
            float2 acc = make_float2(0.f, 0.f);
            if (c < 2) {
                const float2 *Sx = Sh + (0 * nk + kl) * LP, *Sy = Sh + (1 * nk + kl) * LP;
                const float *Wa = Wh + ((c == 0 ? 0 : 1) * nk + kl) * LP, *Wb = Wh + ((c == 0 ? 1 : 2) * nk + kl) * LP;
#pragma unroll 4
                for (int ky = rr; ky < L; ky += C) {
                    const float2 a0 = Sx[ky], a1 = Sy[ky];
                    const float w0 = Wa[ky], w1 = Wb[ky];
                    const float hx = w0 * a0.x + w1 * a1.x, hy = w0 * a0.y + w1 * a1.y;
                    const float2 e = tw[(ky * oy) & mask];
                    acc.x += hx * e.x - hy * e.y;
                    acc.y += hx * e.y + hy * e.x;
                }
            } else {
                const float2 *Sz = Sh + (2 * nk + kl) * LP;
                const float *Wz = Wh + (3 * nk + kl) * LP;
#pragma unroll 4
                for (int ky = rr; ky < L; ky += C) {
                    const float2 a2 = Sz[ky];
                    const float w3 = Wz[ky];
                    const float2 e = tw[(ky * oy) & mask];
                    acc.x += w3 * (a2.x * e.x - a2.y * e.y);
                    acc.y += w3 * (a2.x * e.y + a2.y * e.x);
                }
            }
            Pb[(c * nk + kl) * C + rr] = acc;
        }
        __syncthreads();
        // ---- 1b. G_c(kx, y_i) = sum_r e^{2 pi i r i / C} P_c(kx, r)
        for (int task = tid; task < 3 * nkx * C; task += kCT) {
            const int c = task / (nkx * C), rem = task - c * nkx * C, kl = rem / C, i = rem - kl * C;
            const float2 *Pr = Pb + (c * nk + kl) * C;
            float2 G = make_float2(0.f, 0.f);
            for (int rr = 0; rr < C; ++rr) {
                const float2 e = tw[(rr * i * l) & mask], p = Pr[rr];
                G.x += e.x * p.x - e.y * p.y;
                G.y += e.x * p.y + e.y * p.x;
            }
            Gb[(c * nk + kl) * C + i] = G;
        }
        __syncthreads();
        // ---- 1c. this CTA's share of the field at the n sites
        float4 *pb = part + b * n;
        for (int d = tid; d < n; d += kCT) {
            const int i = d / C, j = d - i * C;
            const int x = ox + l * j;
            float acc[3] = {0.f, 0.f, 0.f};
            for (int kl = 0; kl < nkx; ++kl) {
                const int kx = kx0 + kl;
                const float2 e = tw[(kx * x) & mask];
                const float wgt = (kx == 0 || 2 * kx == L) ? 1.0f : 2.0f;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float2 G = Gb[(c * nk + kl) * C + i];
                    acc[c] += wgt * (e.x * G.x - e.y * G.y);
                }
            }
            pb[d] = make_float4(acc[0] * invN, acc[1] * invN, acc[2] * invN, 0.0f);
        }
        // the draws of this CTA's deciding lanes do not depend on the state: before the barrier
        const int spl = n <= kCT / 4 ? 4 : 1;     // lanes per site in the decisions below
        float u1 = 0.f, uacc = 0.f, sps = 0.f, cps = 0.f, thr = 0.f;
        if (tid < n * spl && tid % spl == 0) {
            const int d = tid / spl, i = d / C, j = d - i * C;
            const int q = (oy + l * i) * L + ox + l * j;
            const uint4 wds = philox(make_uint4((uint32_t)q, (uint32_t)r, t, ((uint32_t)k & 0x00FFFFFFu) | kTagAttempt), key);
            u1 = u24f(wds.x);
            uacc = u24f(wds.z);
            sincospif(2.0f * u24f(wds.y), &sps, &cps);
            thr = (uacc > 0.0f) ? -P.T * logf(uacc) : INFINITY;
        }
        cl.sync();   // every CTA's shares of this sub-step are complete

        // ---- 2. all n decisions, in every CTA alike.  With n <= 64, four lanes share
        // a site's 16 shares (four ranks each, then a fixed two-step butterfly, the
        // same in every CTA); with more sites one lane takes a site's 16.
        float4 *md = mvd + b * n, *ms = mvs + b * n;
        int moved = 0;
        float h0 = 0.f, h1 = 0.f, h2 = 0.f;
        if (tid < n * spl) {
            const int d = tid / spl, part_i = tid - d * spl;
            for (int rk2 = part_i; rk2 < kClusterCtas; rk2 += spl) {
                const float4 sv = cl.map_shared_rank(pb, rk2)[d];
                h0 += sv.x;
                h1 += sv.y;
                h2 += sv.z;
            }
        }
        if (spl == 4) {
            // lanes 4d .. 4d+3 of a warp hold the four partial sums of site d
            h0 += __shfl_xor_sync(0xffffffffu, h0, 1);
            h1 += __shfl_xor_sync(0xffffffffu, h1, 1);
            h2 += __shfl_xor_sync(0xffffffffu, h2, 1);
            h0 += __shfl_xor_sync(0xffffffffu, h0, 2);
            h1 += __shfl_xor_sync(0xffffffffu, h1, 2);
            h2 += __shfl_xor_sync(0xffffffffu, h2, 2);
        }
        if (tid < n * spl && tid % spl == 0) {
            const int d = tid / spl, i = d / C, j = d - i * C;
            const int qx = ox + l * j, qy = oy + l * i, q = qy * L + qx;
            // the site and its neighbours from the CTAs owning their rows (copy b)
            const int ypg = (qy + 1) & mask, ymg = (qy + L - 1) & mask;
            const float *own = cl.map_shared_rank(spb, qy / H);
            const float *spp = cl.map_shared_rank(spb, ypg / H), *spm = cl.map_shared_rank(spb, ymg / H);
            const int yl = qy - (qy / H) * H, ypl = ypg - (ypg / H) * H, yml = ymg - (ymg / H) * H;
            const int xp = (qx + 1) & mask, xm = (qx + L - 1) & mask;
            const float s0 = own[yl * L + qx], s1 = own[HL + yl * L + qx], s2 = own[2 * HL + yl * L + qx];
            float nb[3];
#pragma unroll
            for (int c = 0; c < 3; ++c)
                nb[c] = (own[c * HL + yl * L + xp] + own[c * HL + yl * L + xm]) +
                        (spp[c * HL + ypl * L + qx] + spm[c * HL + yml * L + qx]);
            const float3 S = propose_spin(a.proposal, a.cap_c1, s0, s1, s2, u1, cps, sps);
            const float dX = S.x - s0, dY = S.y - s1, dZ = S.z - s2;
            const float dex = -P.J * (dX * nb[0] + dY * nb[1] + dZ * nb[2]);
            const float z0 = s2 * s2, z1 = S.z * S.z;
            const float dan = (-P.K2 * z1 - P.K4 * z1 * z1) - (-P.K2 * z0 - P.K4 * z0 * z0);
            const float self = W0xx * dX * dX + 2.0f * W0xy * dX * dY + W0yy * dY * dY + W0zz * dZ * dZ;
            const float dE = dex + dan + P.CD * ((dX * h0 + dY * h1 + dZ * h2) + 0.5f * self);
            const int accept = dE < thr;
            md[d] = accept ? make_float4(dX, dY, dZ, 1.0f) : make_float4(0.f, 0.f, 0.f, 0.f);
            ms[d] = make_float4(S.x, S.y, S.z, 0.0f);
            moved = accept;
            if (qy / H == rank) {   // this CTA owns the site's row
                nacc += accept;
                if (a.trace) {
                    float *tr = a.trace + ((((size_t)r * a.nsweeps_call + a.it) * ll + k) * n + d) * MC_TRACE_W;
                    tr[0] = (float)q;
                    tr[1] = h0; tr[2] = h1; tr[3] = h2;
                    tr[4] = dE;
                    tr[5] = uacc;
                    tr[6] = (float)accept;
                    tr[7] = S.x; tr[8] = S.y; tr[9] = S.z;
                }
            }
        }
        const int any = __syncthreads_or(moved);
        // ---- 3a. copy b ^ 1 of the own rows: the moves of sub-step k - 1, then of k.
        // A site that both sub-steps visit (the with-replacement schedule) has the
        // same index d in both, so one thread writes it twice in order.
        {
            float *spn = sp + (b ^ 1) * 3 * HL;
            if (tid < n) {
                const int d = tid, i = d / C, j = d - i * C;
                for (int pass = (k == 0 ? 1 : 0); pass < 2; ++pass) {
                    const int op = pass == 0 ? prev_off : v;
                    const int qy = op / l + l * i, qx = op % l + l * j;
                    const int pb2 = pass == 0 ? (b ^ 1) : b;
                    if (qy / H == rank && mvd[pb2 * n + d].w != 0.0f) {
                        const float4 sv = mvs[pb2 * n + d];
                        const int yl = qy - y0;
                        spn[yl * L + qx] = sv.x;
                        spn[HL + yl * L + qx] = sv.y;
                        spn[2 * HL + yl * L + qx] = sv.z;
                    }
                }
            }
        }
        if (any) {
            // ---- 3b. A_c(kx, i) = sum_j d_c(i, j) e^{-2 pi i kx x_j / L}
            for (int task = tid; task < 3 * nkx * C; task += kCT) {
                const int c = task / (nkx * C), rem = task - c * nkx * C, kl = rem / C, i = rem - kl * C;
                const int kx = kx0 + kl;
                float2 A = make_float2(0.f, 0.f);
                for (int j = 0; j < C; ++j) {
                    const float4 m = md[i * C + j];
                    const float dv = c == 0 ? m.x : (c == 1 ? m.y : m.z);
                    if (dv != 0.0f) {
                        const float2 e = tw[(kx * (ox + l * j)) & mask];
                        A.x += dv * e.x;
                        A.y -= dv * e.y;
                    }
                }
                Pb[(c * nk + kl) * C + i] = A;
            }
            __syncthreads();
            // ---- 3c. B_c(kx, r) = sum_i e^{-2 pi i r i / C} A_c(kx, i)
            for (int task = tid; task < 3 * nkx * C; task += kCT) {
                const int c = task / (nkx * C), rem = task - c * nkx * C, kl = rem / C, rr = rem - kl * C;
                const float2 *Ar = Pb + (c * nk + kl) * C;
                float2 B = make_float2(0.f, 0.f);
                for (int i = 0; i < C; ++i) {
                    const float2 u = cmulc(Ar[i], tw[(rr * i * l) & mask]);
                    B.x += u.x;
                    B.y += u.y;
                }
                Gb[(c * nk + kl) * C + rr] = B;
            }
            __syncthreads();
            // ---- 3d. S^_c(kx, ky) += e^{-2 pi i ky o_y / L} B_c(kx, ky mod C): each thread
            // keeps one ky (L divides the CTA's threads) and walks the (c, kx) columns
            {
                const int ky = tid & mask, grp = tid / L, ngrp = kCT / L;
                const float2 e = tw[(ky * oy) & mask];
                const int rr = ky & (C - 1);
                for (int c = 0; c < 3; ++c)
                    for (int kl = grp; kl < nkx; kl += ngrp) {
                        const float2 u = cmulc(Gb[(c * nk + kl) * C + rr], e);
                        float2 &sv = Sh[(c * nk + kl) * LP + ky];
                        sv.x += u.x;
                        sv.y += u.y;
                    }
            }
        }
        prev_off = v;
        __syncthreads();   // S^ and copy b ^ 1 are done before the next sub-step
    }
    cl.sync();   // no CTA leaves while another may still read its shared memory

    // ---- write back this CTA's rows (copy ll % 2: the state after the sweep); the accepted count
    const float *spf = sp + (ll & 1) * 3 * HL;
    float *gd = a.spins + (size_t)r * 3 * N;
    for (int i = tid; i < 3 * HL; i += kCT) {
        const int c = i / HL, rem = i - c * HL;
        gd[(size_t)c * N + (size_t)y0 * L + rem] = spf[i];
    }
    __syncthreads();
    // per-thread counts of the owned decisions
    for (int off = 16; off; off >>= 1) nacc += __shfl_xor_sync(0xffffffffu, nacc, off);
    if ((tid & 31) == 0 && nacc && a.obs)
        atomicAdd(reinterpret_cast<unsigned long long *>(&a.obs[r].accepted), (unsigned long long)nacc);
}

// Rows of the 2D DFT: R_c(kx, y) = sum_x f_c(x, y) e^{-2 pi i kx x / L}, kx in [0, L/2].
// One CTA per (row y, component c, replica).
__global__ void k_dft_rows(int L, int K2, int P, const float *__restrict__ f, float2 *__restrict__ rowbuf) {
    extern __shared__ float sdr[];
    float *row = sdr;
    float2 *tw = reinterpret_cast<float2 *>(sdr + L);
    const int y = blockIdx.x, c = blockIdx.y, r = blockIdx.z, mask = L - 1;
    const float *src = f + (((size_t)r * P + c) * L + y) * L;
    for (int x = threadIdx.x; x < L; x += blockDim.x) {
        row[x] = src[x];
        float sn, cs;
        sincospif(2.0f * (float)x / (float)L, &sn, &cs);
        tw[x] = make_float2(cs, sn);
    }
    __syncthreads();
    for (int kx = threadIdx.x; kx < K2; kx += blockDim.x) {
        float re = 0.f, im = 0.f;
        for (int x = 0; x < L; ++x) {
            const float2 e = tw[(kx * x) & mask];
            re += row[x] * e.x;
            im -= row[x] * e.y;
        }
        rowbuf[(((size_t)r * P + c) * L + y) * K2 + kx] = make_float2(re, im);
    }
}

// Columns: F_c(kx, ky) = sum_y R_c(kx, y) e^{-2 pi i ky y / L}.  One CTA per
// (column kx, component c, replica).
__global__ void k_dft_cols(int L, int K2, int P, const float2 *__restrict__ rowbuf, float2 *__restrict__ out) {
    extern __shared__ float2 sdc[];
    float2 *col = sdc, *tw = sdc + L;
    const int kx = blockIdx.x, c = blockIdx.y, r = blockIdx.z, mask = L - 1;
    for (int y = threadIdx.x; y < L; y += blockDim.x) {
        col[y] = rowbuf[(((size_t)r * P + c) * L + y) * K2 + kx];
        float sn, cs;
        sincospif(2.0f * (float)y / (float)L, &sn, &cs);
        tw[y] = make_float2(cs, sn);
    }
    __syncthreads();
    for (int ky = threadIdx.x; ky < L; ky += blockDim.x) {
        float2 acc = make_float2(0.f, 0.f);
        for (int y = 0; y < L; ++y) {
            const float2 u = cmulc(col[y], tw[(ky * y) & mask]);
            acc.x += u.x;
            acc.y += u.y;
        }
        out[(((size_t)r * P + c) * K2 + kx) * L + ky] = acc;
    }
}

// W^ (real: W~ is even) from the FP64 W~: one CTA per (column kx, component c),
// FP64 sums, rows into shared memory first, then the column transform.
__global__ void k_cluster_what(int L, int K2, const double *__restrict__ W64, float *__restrict__ What) {
    extern __shared__ double2 sdw[];
    double2 *Rk = sdw;
    const int kx = blockIdx.x, c = blockIdx.y, N = L * L;
    const double two_pi_over_L = 6.283185307179586476925286766559 / (double)L;
    for (int y = threadIdx.x; y < L; y += blockDim.x) {
        double re = 0.0, im = 0.0;
        for (int x = 0; x < L; ++x) {
            const double w = W64[(size_t)c * N + (size_t)y * L + x];
            double sn, cs;
            sincos(two_pi_over_L * (double)((kx * x) % L), &sn, &cs);
            re += w * cs;
            im -= w * sn;
        }
        Rk[y] = make_double2(re, im);
    }
    __syncthreads();
    for (int ky = threadIdx.x; ky < L; ky += blockDim.x) {
        double re = 0.0;
        for (int y = 0; y < L; ++y) {
            double sn, cs;
            sincos(two_pi_over_L * (double)((ky * y) % L), &sn, &cs);
            re += Rk[y].x * cs + Rk[y].y * sn;   // Re[R e^{-i theta}]
        }
        What[((size_t)c * K2 + kx) * L + ky] = (float)re;
    }
}

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

bool cluster_shape_ok(int L, int l) {
    if (!pow2(L) || L < kClusterCtas || L > kCT || l < 2 || l > L || L % l) return false;
    const int C = L / l;
    if (!pow2(C) || C > kClusterCtas) return false;
    return clayout(L, l).bytes <= 227 * 1024;
}

cudaLaunchConfig_t cluster_cfg(const CLayout &g, int R, cudaStream_t st, cudaLaunchAttribute *at) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(kClusterCtas * R);
    cfg.blockDim = dim3(kCT);
    cfg.dynamicSmemBytes = g.bytes;
    cfg.stream = st;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = kClusterCtas;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cfg;
}

cudaError_t set_attrs(size_t bytes) {
    cudaError_t e = cudaFuncSetAttribute(k_cluster_sweep, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_cluster_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

bool cluster_runs(int L, int l) {
    const CLayout g = clayout(L, l);
    if (set_attrs(g.bytes) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = cluster_cfg(g, 1, nullptr, at);
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, k_cluster_sweep, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return nc >= 1;
}

}  // namespace

bool cluster_supported(int L, int l) {
    if (!cluster_shape_ok(L, l)) return false;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    // the answer depends on the device and the layout only: cached per (device, L, l)
    static std::mutex mu;
    static std::map<std::tuple<int, int, int>, bool> known;
    const auto key = std::make_tuple(dev, L, l);
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = known.find(key);
        if (it != known.end()) return it->second;
    }
    const bool ok = cluster_runs(L, l);
    std::lock_guard<std::mutex> lk(mu);
    known[key] = ok;
    return ok;
}



size_t cluster_scratch_bytes(int L, int R) {
    const size_t K2 = (size_t)L / 2 + 1;
    return sizeof(float2) * (size_t)R * 3 * K2 * L * 2;   // Shat and the row scratch
}

cudaError_t launch_cluster_what(int L, const double *W64, float *What, cudaStream_t st) {
    const int K2 = L / 2 + 1;
    k_cluster_what<<<dim3(K2, 4), 256, sizeof(double2) * L, st>>>(L, K2, W64, What);
    return cudaGetLastError();
}

cudaError_t launch_cluster_transform(int L, int R, const float *spins, float2 *rowbuf, float2 *Shat, cudaStream_t st) {
    const int K2 = L / 2 + 1;
    k_dft_rows<<<dim3(L, 3, R), 128, sizeof(float) * L + sizeof(float2) * L, st>>>(L, K2, 3, spins, rowbuf);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_dft_cols<<<dim3(K2, 3, R), 256, sizeof(float2) * 2 * L, st>>>(L, K2, 3, rowbuf, Shat);
    return cudaGetLastError();
}

cudaError_t launch_cluster_sweep(const ClusterSweepArgs &a, cudaStream_t st) {
    if (!cluster_shape_ok(a.L, a.l)) return cudaErrorNotSupported;
    const CLayout g = clayout(a.L, a.l);
    cudaError_t e = set_attrs(g.bytes);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg = cluster_cfg(g, a.R, st, at);
    return cudaLaunchKernelEx(&cfg, k_cluster_sweep, a);
}

}  // namespace dipmc
