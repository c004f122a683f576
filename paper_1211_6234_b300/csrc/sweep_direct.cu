// sweep_direct.cu -- FP32 CUDA-core sweep: one CTA owns one replica for the
// whole launch (all sweeps, all sub-steps), with the spins resident in shared
// memory and the dipole tensor resident in registers.
//
// Field at the update sites (Sec. 3.1; the paper's dipole partial-sum kernel):
// with C = L/l the update sites of sub-step offset o are q = o + l*Dq, Dq in
// [0, C)^2.  Writing every source site as m = o + l*Dm + e with e in [0, l)^2,
//     h_q = sum_e sum_Dm W~(l*((Dq - Dm) mod C) - e) s_{o + l*Dm + e}.
// The tensor entries W~(l*D - e) do not depend on o, so each thread owns a fixed
// set of cell offsets e and keeps their C^2 x 4 tensor components in registers
// for the whole launch; per sub-step it only reads C^2 spins per e from shared
// memory and does 5 C^4 FMAs per e.  The per-thread partial fields are reduced
// across the CTA (warp reduce-scatter + one shared-memory pass).
//
// Update (Sec. 3.1 single-site kernel, Sec. 3.2 approximation): lane d < n of
// warp 0 owns site d, draws its proposal and acceptance uniform from Philox,
// computes dE from the pre-step state (exchange with the four neighbours,
// anisotropy, dipole via h and the self-image W~(0)), accepts iff
// u < exp(-dE/T) and writes the new spin in place.  Update sites are never
// nearest neighbours (l >= 2), so in-place writes cannot change another site's
// dE.  The energy is tracked exactly: sum of accepted dE plus the neglected
// cross terms C_D d_p.W~(p - q).d_q of the sub-step (Sec. 3.2, H3 - H1 - H2 + H0),
// accumulated in FP64.
#include "internal.cuh"

namespace dipmc {

namespace {

constexpr float kPiF = 3.14159265358979f;

// Reduce V per-thread values across a warp with recursive halving: after the
// call, lane `lane` holds the warp sum of value index vidx(lane) in v[0] of the
// group it belongs to; lanes with even index write their value.
// Values are processed in groups of 32 (P = values per group, power of 2 <= 32).
template <int P>
__device__ __forceinline__ float warp_reduce_scatter(float (&v)[P], int lane) {
    int cnt = P;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        if (cnt > 1) {
            const bool upper = (lane & off) != 0;
            const int half = cnt >> 1;
#pragma unroll
            for (int i = 0; i < P / 2; ++i) {
                if (i < half) {
                    const float send = upper ? v[i] : v[i + half];
                    const float keep = upper ? v[i + half] : v[i];
                    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
                }
            }
            cnt = half;
        } else {
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], off);
        }
    }
    return v[0];
}

// Value index held by `lane` after warp_reduce_scatter<P>.
template <int P>
__device__ __forceinline__ int reduce_scatter_index(int lane) {
    int idx = 0, cnt = P;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        if (cnt > 1) {
            const int half = cnt >> 1;
            if (lane & off) idx += half;
            cnt = half;
        }
    }
    return idx;
}

template <int P>
__device__ __forceinline__ int reduce_scatter_writer(int lane) {
    // the lanes that hold a finished sum are those whose bits below the last
    // halving stage are zero
    int cnt = P, last = 1;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        if (cnt > 1) { cnt >>= 1; last = off; }
    }
    return (lane & (last - 1)) == 0;
}

__host__ __device__ constexpr int pow2_at_least(int v) { return v <= 1 ? 1 : 2 * pow2_at_least((v + 1) / 2); }


// Sites whose proposals the permutation schedule draws together (all threads, at the start
// of every batch of sub-steps): a site is visited once per sweep, so its proposal depends
// only on its spin at the sweep's start.
constexpr int kPropBatch = 128;

template <int C, int EPT, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) k_sweep_direct(const SweepConfig cfg, const SweepBuffers buf) {
    constexpr int n = C * C;
    constexpr int V = 3 * n;                    // partial-field values per thread
    constexpr int G = (V + 31) / 32;            // groups of <= 32 values
    constexpr int PV = pow2_at_least(V < 32 ? V : 32);
    const int tid = threadIdx.x, NT = blockDim.x, lane = tid & 31, warp = tid >> 5, NW = NT >> 5;
    const int NWF = NW - 1;                     // field warps; warp 0 is the control warp
    const int ftid = tid - 32;
    const int r = blockIdx.x;
    // geometry, buffers and stream state of this replica: the lattice's own, its
    // slot's in a packed launch, or its descriptor's in a grouped launch
    const SlotGeom *G0 = buf.geom ? buf.geom + r : nullptr;
    const int L = G0 ? G0->L : cfg.L, l = G0 ? G0->l : cfg.l, N = L * L, ll = l * l;
    const int NTF = G0 ? G0->nft : NT - 32;     // field threads whose cell offsets this CTA sums
    const int NTO = G0 ? G0->nt : NT;           // threads of the observable sums
    const float *__restrict__ W32 = G0 ? G0->W32 : buf.W32;
    float *spins_r = G0 ? G0->spins : buf.spins + (size_t)r * 3 * N;
    const RepParams *par_r = G0 ? G0->params : buf.params + r;
    double *energy_r = G0 ? G0->energy : (buf.energy ? buf.energy + r : nullptr);
    ObsAcc *obs_r = G0 ? G0->obs : (buf.obs ? buf.obs + r : nullptr);
    double *theta2_r = G0 ? G0->theta2 : (buf.theta2 ? buf.theta2 + (size_t)r * N : nullptr);
    uint2 key = cfg.key;
    uint32_t t0 = cfg.t0, rid = (uint32_t)r, mphase = 0;
    int nsw = cfg.nsweeps;
    if (G0) {
        key = make_uint2(G0->key_lo, G0->key_hi);
        t0 = G0->t0;
        mphase = G0->mphase;
        rid = G0->rid;
        nsw = min(nsw, G0->nsweeps);
        if (nsw <= 0) return;
    } else if (buf.slots) {
        const SlotState sl = buf.slots[r];
        key = make_uint2(sl.key_lo, sl.key_hi);
        t0 = sl.t0;
        mphase = sl.t0;             // measure on the slot's own sweep count
        rid = sl.rid;
        nsw = min(nsw, (int)sl.nsweeps);
        if (nsw <= 0) return;       // idle slot: whole CTA leaves before any barrier
    }

    extern __shared__ float4 smem_f4[];
    float4 *s4 = smem_f4;                                         // [N] spins (x, y, z, 0)
    float *red = reinterpret_cast<float *>(s4 + N);               // [NWF][V] warp partial fields
    float *mred = red + NWF * V;                                  // [NW][12] magnetisation, staggered and wall sums
    float *wl = mred + NW * 12;                                   // [n][4] W~(l*D), D in [0,C)^2
    uint16_t *sched = reinterpret_cast<uint16_t *>(wl + n * 4);   // [ll] offsets of the sweep
    // [kPropBatch] proposals of a batch (schedule 0): (S, threshold), (delta, anisotropy +
    // self-image part of dE), the acceptance uniform; 16-byte aligned after the schedule
    const size_t pb_off = ((size_t)(reinterpret_cast<char *>(sched + ll) - reinterpret_cast<char *>(smem_f4)) + 15) & ~(size_t)15;
    float4 *pbS = reinterpret_cast<float4 *>(reinterpret_cast<char *>(smem_f4) + pb_off);
    float4 *pbX = pbS + kPropBatch;
    float *pbU = reinterpret_cast<float *>(pbX + kPropBatch);
    constexpr int KB = kPropBatch / n;                             // sub-steps per batch
    __shared__ ObsAcc acc_s;
    __shared__ double e_track_s;
    // control-warp state kept in shared memory so that it does not occupy
    // registers of the field threads (lane d < n: update site d)
    __shared__ float c_S[3][32], c_d[3][32], c_pre[32], c_thr[32], c_u[32];
    __shared__ int c_q[32];
    __shared__ float b_d[3][32], b_E[32];     // last decided sub-step, for the bookkeeping
    __shared__ double c_epart[32];
    __shared__ RepParams c_P;
    __shared__ float c_W0[4];

    // ---- load state: global SoA -> shared AoS
    const float *gs = spins_r;
    for (int i = tid; i < N; i += NT) s4[i] = make_float4(gs[i], gs[N + i], gs[2 * N + i], 0.0f);
    const bool measuring = cfg.measure_every > 0;
    // per-site sum of (theta - pi/2)^2, added in FP64 at every measured sweep so
    // that the result does not depend on how the sweeps are split into launches
    double *gt = theta2_r;
    if (tid < 4 * n) {
        const int D = tid >> 2, c = tid & 3;
        wl[tid] = W32[c * N + (l * (D / C)) * L + l * (D % C)];
    }
    if (tid == 0) {
        if (obs_r) acc_s = *obs_r;
        e_track_s = energy_r ? *energy_r : 0.0;
        c_P = *par_r;
    }
    if (tid < 4) c_W0[tid] = W32[tid * N];
    if (tid < 32) {
        c_epart[tid] = 0.0;
        b_d[0][tid] = b_d[1][tid] = b_d[2][tid] = b_E[tid] = 0.0f;
    }

    // ---- field threads: tensor slices of their cell offsets e (registers, whole launch)
    float w[EPT][n][4];
    int ex[EPT], ey[EPT];
#pragma unroll
    for (int j = 0; j < EPT; ++j) {
        const int e = ftid + j * NTF;
        const bool valid = warp > 0 && ftid < NTF && e < ll;
        ex[j] = valid ? e % l : 0;
        ey[j] = valid ? e / l : 0;
#pragma unroll
        for (int D = 0; D < n; ++D) {
            int rx = l * (D % C) - ex[j];
            int ry = l * (D / C) - ey[j];
            if (rx < 0) rx += L;
            if (ry < 0) ry += L;
            const int idx = ry * L + rx;
#pragma unroll
            for (int c = 0; c < 4; ++c) w[j][D][c] = valid ? W32[c * N + idx] : 0.0f;
        }
        if constexpr (C == 2) {
            // at C = 2 the field of cell d from the four cells m of offset o + e is the XOR
            // convolution sum_m W~(l (d xor m) - e) s_m, which the 2 x 2 Walsh-Hadamard
            // transform diagonalises: keep the slices' transform T(kappa) = sum_D (-1)^(kappa.D) W(D)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float a = w[j][0][c] + w[j][1][c], b = w[j][0][c] - w[j][1][c];
                const float cc = w[j][2][c] + w[j][3][c], dd = w[j][2][c] - w[j][3][c];
                w[j][0][c] = a + cc;
                w[j][1][c] = b + dd;
                w[j][2][c] = a - cc;
                w[j][3][c] = b - dd;
            }
        }
    }

    const int hbits = ceil_log2_u((uint32_t)l);
    bool pending = false;      // control warp: a decided sub-step awaits bookkeeping
    long long n_acc = 0;       // control warp lane 0: accepted moves
    __syncthreads();

    // sum of accepted dE plus the pair cross terms C_D d_p.W~(q - p).d_q of the
    // last decided sub-step (Sec. 3.2, H3 - H1 - H2 + H0); control warp only
    auto bookkeeping = [&]() {
        if (lane < n) {
            const int dxl = lane % C, dyl = lane / C;
            const float bX = b_d[0][lane], bY = b_d[1][lane], bZ = b_d[2][lane];
            float cross = 0.0f;
            for (int dp = 0; dp < lane; ++dp) {
                const int Dd = ((dxl - dp % C + C) % C) + C * ((dyl - dp / C + C) % C);
                const float xx = wl[4 * Dd], xy = wl[4 * Dd + 1], yy = wl[4 * Dd + 2], zz = wl[4 * Dd + 3];
                const float pX = b_d[0][dp], pY = b_d[1][dp], pZ = b_d[2][dp];
                cross += pX * (xx * bX + xy * bY) + pY * (xy * bX + yy * bY) + pZ * (zz * bZ);
            }
            c_epart[lane] += (double)b_E[lane] + (double)(c_P.CD * cross);
        }
        __syncwarp();
    };

    // Sec. 3.1 proposal of site q at sub-step kk of sweep t: the new spin and its delta,
    // the threshold -T ln u, the uniform u, and the field- and exchange-free part of dE
    // (anisotropy and the self-image term)
    auto proposal = [&](int q, int kk, uint32_t t, float3 &Sn, float3 &dS, float &thr, float &uacc, float &part) {
        const RepParams &P = c_P;
        const uint4 wds = philox(make_uint4((uint32_t)q, rid, t, ((uint32_t)kk & 0x00FFFFFFu) | kTagAttempt), key);
        const float u1 = u24f(wds.x);
        float sps, cps;
        sincospif(2.0f * u24f(wds.y), &sps, &cps);
        uacc = u24f(wds.z);
        const float4 sq = s4[q];
        Sn = propose_spin(cfg.proposal, cfg.cap_c1, sq.x, sq.y, sq.z, u1, cps, sps);
        dS = make_float3(Sn.x - sq.x, Sn.y - sq.y, Sn.z - sq.z);
        const float z0 = sq.z * sq.z, z1 = Sn.z * Sn.z;
        const float dan = (-P.K2 * z1 - P.K4 * z1 * z1) - (-P.K2 * z0 - P.K4 * z0 * z0);
        const float self = c_W0[0] * dS.x * dS.x + 2.0f * c_W0[1] * dS.x * dS.y + c_W0[2] * dS.y * dS.y + c_W0[3] * dS.z * dS.z;
        part = dan + 0.5f * P.CD * self;
        // accept iff u < exp(-dE/T)  <=>  dE < -T ln u   (u = 0: always)
        thr = (uacc > 0.0f) ? -P.T * logf(uacc) : INFINITY;
    };

    for (int it = 0; it < nsw; ++it) {
        const uint32_t t = t0 + (uint32_t)it;
        // ---- the sweep's schedule
        if (cfg.schedule == 0) {
            const uint4 rk = philox(make_uint4(t, 0u, 0u, kTagPerm), key);
            for (int k = tid; k < ll; k += NT) {
                const uint32_t v = perm_offset(rk, hbits, (uint32_t)ll, (uint32_t)k);
                sched[k] = (uint16_t)(((v / l) << 8) | (v % l));  // (oy, ox), l <= 256
            }
        } else {
            for (int k = tid; k < ll; k += NT) {
                const uint4 o = philox(make_uint4(t, (uint32_t)k, 0u, kTagDraw), key);
                const uint32_t v = (uint32_t)(((unsigned long long)o.x * (unsigned long long)ll) >> 32);
                sched[k] = (uint16_t)(((v / l) << 8) | (v % l));
            }
        }
        __syncthreads();

        for (int k = 0; k < ll; ++k) {
            if (cfg.schedule == 0 && k % KB == 0) {
                // ---- the proposals of sub-steps k .. k+KB-1, all threads
                for (int i = tid; i < KB * n; i += NT) {
                    const int kk = k + i / n, d = i % n;
                    if (kk >= ll) break;
                    const int vv = sched[kk];
                    const int q = ((vv >> 8) + l * (d / C)) * L + (vv & 0xFF) + l * (d % C);
                    float3 Sn, dS;
                    float thr, uacc, part;
                    proposal(q, kk, t, Sn, dS, thr, uacc, part);
                    pbS[i] = make_float4(Sn.x, Sn.y, Sn.z, thr);
                    pbX[i] = make_float4(dS.x, dS.y, dS.z, part);
                    pbU[i] = uacc;
                }
                __syncthreads();
            }
            const int v = sched[k];
            const int ox = v & 0xFF, oy = v >> 8;
            if (warp == 0) {
                // ---- control warp, while the field warps run: last sub-step's energy
                // bookkeeping, then every field-independent part of this sub-step's dE
                if (pending) {
                    bookkeeping();
                    pending = false;
                }
                if (lane < n) {
                    const RepParams &P = c_P;
                    const int qx = ox + l * (lane % C), qy = oy + l * (lane / C);
                    const int q = qy * L + qx;
                    float3 Sn, dS;
                    float thr, uacc, part;
                    if (cfg.schedule == 0) {
                        const int i = (k % KB) * n + lane;
                        const float4 a4 = pbS[i], b4 = pbX[i];
                        Sn = make_float3(a4.x, a4.y, a4.z);
                        thr = a4.w;
                        dS = make_float3(b4.x, b4.y, b4.z);
                        part = b4.w;
                        uacc = pbU[i];
                    } else {
                        proposal(q, k, t, Sn, dS, thr, uacc, part);
                    }
                    // exchange with the current neighbour spins
                    const int xp = (qx + 1 == L) ? q - qx : q + 1;
                    const int xm = (qx == 0) ? q + L - 1 : q - 1;
                    const int yp = (qy + 1 == L) ? qx : q + L;
                    const int ym = (qy == 0) ? q + N - L : q - L;
                    const float4 a = s4[xp], b = s4[xm], c = s4[yp], d = s4[ym];
                    const float n0 = (a.x + b.x) + (c.x + d.x);
                    const float n1 = (a.y + b.y) + (c.y + d.y);
                    const float n2 = (a.z + b.z) + (c.z + d.z);
                    const float dex = -P.J * (dS.x * n0 + dS.y * n1 + dS.z * n2);
                    c_S[0][lane] = Sn.x; c_S[1][lane] = Sn.y; c_S[2][lane] = Sn.z;
                    c_d[0][lane] = dS.x; c_d[1][lane] = dS.y; c_d[2][lane] = dS.z;
                    c_pre[lane] = dex + part;
                    c_thr[lane] = thr;
                    c_u[lane] = uacc;
                    c_q[lane] = q;
                }
            } else {
                // ---- field warps: partial fields at the n update sites (C = 2: their
                // 2 x 2 transform H(kappa) = sum_e T_e(kappa) S_e(kappa), inverted by the
                // control warp)
                float acc[n][3];
#pragma unroll
                for (int d = 0; d < n; ++d) acc[d][0] = acc[d][1] = acc[d][2] = 0.0f;
                if constexpr (C == 2) {
#pragma unroll
                    for (int j = 0; j < EPT; ++j) {
                        const int bx = ox + ex[j], by = oy + ey[j];
                        float3 sm[4];
#pragma unroll
                        for (int m = 0; m < 4; ++m) {
                            int xx = bx + l * (m & 1), yy = by + l * (m >> 1);
                            if (xx >= L) xx -= L;
                            if (yy >= L) yy -= L;
                            const float4 v = s4[yy * L + xx];
                            sm[m] = make_float3(v.x, v.y, v.z);
                        }
                        const float3 a = make_float3(sm[0].x + sm[1].x, sm[0].y + sm[1].y, sm[0].z + sm[1].z);
                        const float3 b = make_float3(sm[0].x - sm[1].x, sm[0].y - sm[1].y, sm[0].z - sm[1].z);
                        const float3 cc = make_float3(sm[2].x + sm[3].x, sm[2].y + sm[3].y, sm[2].z + sm[3].z);
                        const float3 dd = make_float3(sm[2].x - sm[3].x, sm[2].y - sm[3].y, sm[2].z - sm[3].z);
                        const float3 S[4] = {make_float3(a.x + cc.x, a.y + cc.y, a.z + cc.z),
                                             make_float3(b.x + dd.x, b.y + dd.y, b.z + dd.z),
                                             make_float3(a.x - cc.x, a.y - cc.y, a.z - cc.z),
                                             make_float3(b.x - dd.x, b.y - dd.y, b.z - dd.z)};
#pragma unroll
                        for (int kap = 0; kap < 4; ++kap) {
                            acc[kap][0] = fmaf(w[j][kap][0], S[kap].x, fmaf(w[j][kap][1], S[kap].y, acc[kap][0]));
                            acc[kap][1] = fmaf(w[j][kap][1], S[kap].x, fmaf(w[j][kap][2], S[kap].y, acc[kap][1]));
                            acc[kap][2] = fmaf(w[j][kap][3], S[kap].z, acc[kap][2]);
                        }
                    }
                } else {
#pragma unroll
                for (int j = 0; j < EPT; ++j) {
                    const int bx = ox + ex[j], by = oy + ey[j];
#pragma unroll
                    for (int my = 0; my < C; ++my) {
                        int yy = by + l * my;
                        if (yy >= L) yy -= L;
#pragma unroll
                        for (int mx = 0; mx < C; ++mx) {
                            int xx = bx + l * mx;
                            if (xx >= L) xx -= L;
                            const float4 sm = s4[yy * L + xx];
#pragma unroll
                            for (int dy = 0; dy < C; ++dy)
#pragma unroll
                                for (int dx = 0; dx < C; ++dx) {
                                    const int D = ((dx - mx + C) % C) + C * ((dy - my + C) % C);
                                    const int dq = dx + C * dy;
                                    acc[dq][0] = fmaf(w[j][D][0], sm.x, fmaf(w[j][D][1], sm.y, acc[dq][0]));
                                    acc[dq][1] = fmaf(w[j][D][1], sm.x, fmaf(w[j][D][2], sm.y, acc[dq][1]));
                                    acc[dq][2] = fmaf(w[j][D][3], sm.z, acc[dq][2]);
                                }
                        }
                    }
                }
                }
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    float vals[PV];
#pragma unroll
                    for (int i = 0; i < PV; ++i) {
                        const int vi = g * 32 + i;
                        vals[i] = (i < 32 && vi < V) ? acc[vi / 3][vi % 3] : 0.0f;
                    }
                    const float s = warp_reduce_scatter<PV>(vals, lane);
                    const int vi = g * 32 + reduce_scatter_index<PV>(lane);
                    if (reduce_scatter_writer<PV>(lane) && vi < V) red[(warp - 1) * V + vi] = s;
                }
            }
            __syncthreads();

            if (warp == 0) {
                // ---- critical path: field -> decide -> write
                float hsum[G];
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    const int vi = g * 32 + lane;
                    float s = 0.0f;
                    if (vi < V)
                        for (int ww = 0; ww < NWF; ++ww) s += red[ww * V + vi];
                    hsum[g] = s;
                }
                float h[3];
                if constexpr (C == 2) {
                    // cell d = lane: h = (1/4) sum_kappa (-1)^(kappa.d) H(kappa); H(kappa) sits at 3 kappa + c
                    const int d = lane & 3;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        float val = 0.0f;
#pragma unroll
                        for (int kap = 0; kap < 4; ++kap) {
                            const float Hk = __shfl_sync(0xffffffffu, hsum[0], 3 * kap + c);
                            val += (__popc(kap & d) & 1) ? -Hk : Hk;
                        }
                        h[c] = 0.25f * val;
                    }
                } else {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const int vi = 3 * (lane < n ? lane : 0) + c;
                    float val = 0.0f;
#pragma unroll
                    for (int g = 0; g < G; ++g) {
                        const float t2 = __shfl_sync(0xffffffffu, hsum[g], vi & 31);
                        if ((vi >> 5) == g) val = t2;
                    }
                    h[c] = val;
                }
                }
                int accept = 0;
                if (lane < n) {
                    const float dX = c_d[0][lane], dY = c_d[1][lane], dZ = c_d[2][lane];
                    const float dE = c_pre[lane] + c_P.CD * (dX * h[0] + dY * h[1] + dZ * h[2]);
                    accept = dE < c_thr[lane];
                    const int q = c_q[lane];
                    const float S0 = c_S[0][lane], S1 = c_S[1][lane], S2 = c_S[2][lane];
                    if (accept) s4[q] = make_float4(S0, S1, S2, 0.0f);
                    b_d[0][lane] = accept ? dX : 0.0f;
                    b_d[1][lane] = accept ? dY : 0.0f;
                    b_d[2][lane] = accept ? dZ : 0.0f;
                    b_E[lane] = accept ? dE : 0.0f;
                    if (buf.trace) {
                        float *tr = buf.trace + ((((size_t)r * cfg.nsweeps + it) * ll + k) * n + lane) * MC_TRACE_W;
                        tr[0] = (float)q;
                        tr[1] = h[0]; tr[2] = h[1]; tr[3] = h[2];
                        tr[4] = dE;
                        tr[5] = c_u[lane];
                        tr[6] = (float)accept;
                        tr[7] = S0; tr[8] = S1; tr[9] = S2;
                    }
                }
                const unsigned ball = __ballot_sync(0xffffffffu, accept);
                if (lane == 0) n_acc += __popc(ball);
                pending = true;
            }
            __syncthreads();
        }
        if (warp == 0) {
            if (pending) {
                bookkeeping();
                pending = false;
            }
            // fold the sweep's energy change into the tracked energy, so that the
            // sum does not depend on how the sweeps are split into launches
            double et = c_epart[lane];
            c_epart[lane] = 0.0;
            for (int off = 16; off; off >>= 1) et += __shfl_xor_sync(0xffffffffu, et, off);
            if (lane == 0) e_track_s += et;
        }

        // ---- observables of this sweep
        if (measuring && ((mphase + (uint32_t)it + 1u) % (uint32_t)cfg.measure_every) == 0) {
            float mv_[12] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            for (int i = tid; tid < NTO && i < N; i += NTO) {
                const float4 a = s4[i];
                const int iy = i / L, ix = i - iy * L;
                const float4 ax = s4[iy * L + (ix + 1 == L ? 0 : ix + 1)], ay = s4[(iy + 1 == L ? 0 : iy + 1) * L + ix];
                mv_[0] += a.x;
                mv_[1] += a.y;
                mv_[2] += a.z;
                mv_[3] += (iy & 1) ? -a.z : a.z;     // m1 + m2 - m3 - m4 (rows)
                mv_[4] += (ix & 1) ? -a.z : a.z;     // m1 + m4 - m3 - m2 (columns)
                mv_[5] += wall_term(a.x, ax.x);
                mv_[6] += wall_term(a.x, ay.x);
                mv_[7] += wall_term(a.y, ax.y);
                mv_[8] += wall_term(a.y, ay.y);
                mv_[9] += wall_term(a.z, ax.z);
                mv_[10] += wall_term(a.z, ay.z);
                const float th = acosf(fminf(1.0f, fmaxf(-1.0f, a.z))) - 0.5f * kPiF;
                mv_[11] += fabsf(th);
                if (gt) gt[i] += (double)(th * th);
            }
#pragma unroll
            for (int c = 0; c < 12; ++c)
                for (int off = 16; off; off >>= 1) mv_[c] += __shfl_xor_sync(0xffffffffu, mv_[c], off);
            if (lane == 0)
#pragma unroll
                for (int c = 0; c < 12; ++c) mred[warp * 12 + c] = mv_[c];
            __syncthreads();
            if (warp == 0) {
                if (lane == 0) {
                    double sm[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
                    for (int ww = 0; ww < NW; ++ww)
                        for (int c = 0; c < 12; ++c) sm[c] += mred[ww * 12 + c];
                    const double Mx = sm[0] / N, My = sm[1] / N, Mz = sm[2] / N, Mh = sm[3] / N, Mv = sm[4] / N;
                    const double nh[3] = {sm[5], sm[7], sm[9]}, nv[3] = {sm[6], sm[8], sm[10]};
                    double x[MC_NOBS];
                    x[MC_OBS_ABS_M] = sqrt(Mx * Mx + My * My + Mz * Mz);
                    x[MC_OBS_MZ] = Mz;
                    x[MC_OBS_ABS_MZ] = fabs(Mz);
                    x[MC_OBS_MPAR] = sqrt(Mx * Mx + My * My);
                    x[MC_OBS_E] = e_track_s / N;
                    x[MC_OBS_MST] = sqrt(Mh * Mh + Mv * Mv);
                    stripe_obs(x, nh, nv, sm[11], N);
                    if (obs_r) obs_push(acc_s, x);
                    if (!G0) hist_push(buf.hist, r, x[MC_OBS_E]);
                }
            }
            __syncthreads();
        }
    }

    // ---- write back
    float *gd = spins_r;
    for (int i = tid; i < N; i += NT) {
        const float4 a = s4[i];
        gd[i] = a.x;
        gd[N + i] = a.y;
        gd[2 * N + i] = a.z;
    }
    if (warp == 0) {
        if (lane == 0) {
            if (energy_r) *energy_r = e_track_s;
            if (obs_r) {
                acc_s.accepted += n_acc;
                acc_s.attempted += (long long)nsw * N;
                *obs_r = acc_s;
            }
        }
    }
}

struct Inst {
    int C, EPT, MAXT, MINB;
    cudaError_t (*launch)(const SweepConfig &, const SweepBuffers &, int, size_t, cudaStream_t);
    cudaError_t (*occupancy)(int, size_t, int *);
};

template <int C, int EPT, int MAXT, int MINB>
cudaError_t occupancy_inst(int threads, size_t smem, int *per_sm) {
    cudaError_t e = cudaFuncSetAttribute(k_sweep_direct<C, EPT, MAXT, MINB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_sweep_direct<C, EPT, MAXT, MINB>, threads, smem);
}

template <int C, int EPT, int MAXT, int MINB>
cudaError_t launch_inst(const SweepConfig &c, const SweepBuffers &b, int threads, size_t smem, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k_sweep_direct<C, EPT, MAXT, MINB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_sweep_direct<C, EPT, MAXT, MINB><<<c.R, threads, smem, st>>>(c, b);
    return cudaGetLastError();
}

// Threads = one control warp + ceil(l^2 / EPT) field threads (rounded to warps).
// The launch bound keeps C^2*4*EPT tensor values + 3*C^2 accumulators per
// thread in registers; MINB = 2 instances fit two CTAs per SM (8 warps each, so
// that each SM sub-partition holds 4 warps and 128 registers per thread).
#define INST(C, E, T, B) {C, E, T, B, launch_inst<C, E, T, B>, occupancy_inst<C, E, T, B>}
const Inst kInst[] = {
    INST(1, 1, 288, 2), INST(1, 2, 544, 1), INST(1, 4, 288, 2), INST(1, 8, 544, 1),
    INST(1, 19, 256, 2), INST(1, 18, 544, 1),
    INST(2, 1, 544, 1), INST(2, 2, 544, 1), INST(2, 5, 256, 2), INST(2, 5, 544, 1),
    INST(4, 1, 288, 1), INST(4, 2, 320, 1),
};
#undef INST

int threads_of(const Inst &in, int ll) {
    int th = (ll + in.EPT - 1) / in.EPT;
    return 32 + ((th + 31) / 32) * 32;
}

size_t smem_bytes(int L, int l, int threads) {
    const int N = L * L, C = L / l, n = C * C, NW = threads / 32;
    size_t b = sizeof(float4) * (size_t)N + sizeof(float) * (size_t)((NW - 1) * 3 * n + NW * 12 + 4 * n);
    b += sizeof(uint16_t) * (size_t)l * l;
    b = (b + 15) & ~(size_t)15;
    return b + (size_t)kPropBatch * (2 * sizeof(float4) + sizeof(float));
}

// Choose the instance.  Many replicas (more than one wave of SMs): prefer two
// CTAs per SM so that one CTA's serial update overlaps the other's field work;
// otherwise prefer the most threads per CTA (shortest sub-step).
const Inst *pick(int L, int l, int R, int nsm, int *threads) {
    if (l < 2 || L % l) return nullptr;
    const int C = L / l, ll = l * l;
    const bool many = R > nsm;
    const Inst *best = nullptr;
    int best_th = 0;
    for (const Inst &in : kInst) {
        if (in.C != C) continue;
        const int th = threads_of(in, ll);
        if (th > in.MAXT) continue;
        if (smem_bytes(L, l, th) * in.MINB > 220 * 1024) continue;
        bool better = false;
        if (!best) better = true;
        else if (many && in.MINB != best->MINB) better = in.MINB > best->MINB;
        else better = th > best_th;
        if (better) {
            best = &in;
            best_th = th;
        }
    }
    if (!best) return nullptr;
    *threads = best_th;
    return best;
}

}  // namespace

bool direct_lone_shape(int L, int l, int R, int *threads, int *ept) {
    int dev = 0, nsm = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const Inst *in = pick(L, l, R, nsm, threads);
    if (!in) return false;
    *ept = in->EPT;
    return true;
}

size_t direct_smem_bytes(int L, int l, int threads) { return smem_bytes(L, l, threads); }

// The instance of a grouped launch: the fewest cell offsets per thread that cover
// every slot's lone EPT and thread count (the extra offsets of a thread are empty).
const Inst *pick_grouped(int C, int max_ept, int threads) {
    const Inst *best = nullptr;
    for (const Inst &in : kInst) {
        if (in.C != C || in.EPT < max_ept || in.MAXT < threads) continue;
        if (!best || in.EPT < best->EPT || (in.EPT == best->EPT && in.MAXT > best->MAXT)) best = &in;
    }
    return best;
}

int direct_grouped_resident(int C, int max_ept, int threads, size_t smem) {
    const Inst *in = pick_grouped(C, max_ept, threads);
    if (!in || smem > 227 * 1024) return 0;
    int dev = 0, nsm = 148, per_sm = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (in->occupancy(threads, smem, &per_sm) != cudaSuccess) return 0;
    return per_sm * nsm;
}

cudaError_t launch_sweep_direct_grouped(int C, int max_ept, int threads, size_t smem, const SweepConfig &c,
                                        const SlotGeom *geom_dev, int count, cudaStream_t st) {
    const Inst *best = pick_grouped(C, max_ept, threads);
    if (!best || smem > 227 * 1024) return cudaErrorNotSupported;
    SweepConfig g = c;
    g.R = count;
    SweepBuffers b;
    b.geom = geom_dev;
    return best->launch(g, b, threads, smem, st);
}

bool direct_supported(int L, int l) {
    int th = 0;
    return pick(L, l, 1, 1, &th) != nullptr;
}

int direct_resident_ctas(int L, int l) {
    int dev = 0, nsm = 148, th = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const Inst *in = pick(L, l, 1, nsm, &th);
    if (!in) return 0;
    int per_sm = 0;
    if (in->occupancy(th, smem_bytes(L, l, th), &per_sm) != cudaSuccess || per_sm < 1) per_sm = 1;
    return per_sm * nsm;
}

cudaError_t launch_sweep_direct(const SweepConfig &c, const SweepBuffers &b, int threads_hint,
                                cudaStream_t st) {
    (void)threads_hint;
    int dev = 0, nsm = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int threads = 0;
    // a packed launch uses the instance a lone replica would, so that every
    // slot's arithmetic (and trajectory) is the one it has alone
    const Inst *in = pick(c.L, c.l, b.slots ? 1 : c.R, nsm, &threads);
    if (!in) return cudaErrorNotSupported;
    return in->launch(c, b, threads, smem_bytes(c.L, c.l, threads), st);
}

}  // namespace dipmc
