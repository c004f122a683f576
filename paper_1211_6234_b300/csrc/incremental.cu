// incremental.cu -- the sweep with the dipole field kept at every site and
// updated after each sub-step by the moves it accepted (a rank-n update):
//     h(m) += sum_{q accepted} W~(m - q) (S_q - s_q)   for all m.
// The field at the sub-step's sites is then always exact for the current state
// (Sec. 2.1, Eq. 2; Sec. 3.1/3.2 update), and the energy of any measured sweep
// is an O(N) sum over the kept field, -J sum_bonds s.s + sum E_A +
// (C_D/2) sum s.h, with no full-field evaluation.
//
// One CTA per replica; spins, field and W~ live in shared memory (48 B per site,
// so L <= 64).  Per sub-step the threads d < n decide the n sites from the kept
// field, then every thread updates the field of its sites with the accepted
// moves.  The field is evaluated afresh by the caller every few sweeps (each
// launch) so that the FP32 rank-n updates do not accumulate rounding.
#include "incremental.cuh"

namespace dipmc {

namespace {

constexpr int kIThreads = 512;
constexpr float kPiF = 3.14159265358979f;


__global__ void __launch_bounds__(kIThreads, 1) k_sweep_incremental(const IncrConfig cfg, const IncrBuffers b) {
    const int L = cfg.L, l = cfg.l, N = L * L, C = L / l, n = C * C, ll = l * l;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, NW = kIThreads / 32;
    const int r = blockIdx.x;
    extern __shared__ float4 sm4[];
    float4 *s4 = sm4;                                        // [N] spins
    float4 *h4 = s4 + N;                                     // [N] field
    float4 *w4 = h4 + N;                                     // [N] W~ (xx, xy, yy, zz)
    float4 *mv = w4 + N;                                     // [n] move of site d (delta, accepted)
    float4 *mS = mv + n;                                     // [n] proposed spin of site d
    uint16_t *sched = reinterpret_cast<uint16_t *>(mS + n);  // [ll]
    __shared__ double red[kIThreads / 32][15];
    __shared__ int s_acc;

    const RepParams P = b.params[r];
    const float *gs = b.spins + (size_t)r * 3 * N, *gh = b.field + (size_t)r * 3 * N;
    for (int i = tid; i < N; i += kIThreads) {
        s4[i] = make_float4(gs[i], gs[N + i], gs[2 * N + i], 0.f);
        h4[i] = make_float4(gh[i], gh[N + i], gh[2 * N + i], 0.f);
        w4[i] = make_float4(b.W32[i], b.W32[N + i], b.W32[2 * N + i], b.W32[3 * N + i]);
    }
    if (tid == 0) s_acc = 0;
    const float4 W0 = make_float4(b.W32[0], b.W32[N], b.W32[2 * N], b.W32[3 * N]);
    const int hbits = ceil_log2_u((uint32_t)l);
    __syncthreads();

    for (int it = 0; it < cfg.nsweeps; ++it) {
        const uint32_t t = cfg.t0 + (uint32_t)it;
        if (cfg.schedule == 0) {
            const uint4 rk = philox(make_uint4(t, 0u, 0u, kTagPerm), cfg.key);
            for (int k = tid; k < ll; k += kIThreads) {
                const uint32_t v = perm_offset(rk, hbits, (uint32_t)ll, (uint32_t)k);
                sched[k] = (uint16_t)(((v / l) << 8) | (v % l));
            }
        } else {
            for (int k = tid; k < ll; k += kIThreads) {
                const uint4 o = philox(make_uint4(t, (uint32_t)k, 0u, kTagDraw), cfg.key);
                const uint32_t v = (uint32_t)(((unsigned long long)o.x * (unsigned long long)ll) >> 32);
                sched[k] = (uint16_t)(((v / l) << 8) | (v % l));
            }
        }
        __syncthreads();
        for (int k = 0; k < ll; ++k) {
            const int ox = sched[k] & 0xFF, oy = sched[k] >> 8;
            // ---- decide the n sites from the kept field (state before the sub-step)
            int nacc = 0;
            for (int d = tid; d < n; d += kIThreads) {
                const int qx = ox + l * (d % C), qy = oy + l * (d / C), q = qy * L + qx;
                const uint4 wds = philox(make_uint4((uint32_t)q, (uint32_t)r, t, ((uint32_t)k & 0x00FFFFFFu) | kTagAttempt),
                                         cfg.key);
                const float u1 = u24f(wds.x), uacc = u24f(wds.z);
                float sps, cps;
                sincospif(2.0f * u24f(wds.y), &sps, &cps);
                const float4 sq = s4[q];
                float S0, S1, S2;
                {
                    const float3 Sv = propose_spin(cfg.proposal, cfg.cap_c1, sq.x, sq.y, sq.z, u1, cps, sps);   // Sec. 3.1 proposal
                    S0 = Sv.x;
                    S1 = Sv.y;
                    S2 = Sv.z;
                }
                const float dX = S0 - sq.x, dY = S1 - sq.y, dZ = S2 - sq.z;
                const int xp = (qx + 1 == L) ? q - qx : q + 1;
                const int xm = (qx == 0) ? q + L - 1 : q - 1;
                const int yp = (qy + 1 == L) ? qx : q + L;
                const int ym = (qy == 0) ? q + N - L : q - L;
                const float4 a = s4[xp], bb = s4[xm], c = s4[yp], dd = s4[ym];
                const float n0 = (a.x + bb.x) + (c.x + dd.x);
                const float n1 = (a.y + bb.y) + (c.y + dd.y);
                const float n2 = (a.z + bb.z) + (c.z + dd.z);
                const float dex = -P.J * (dX * n0 + dY * n1 + dZ * n2);
                const float z0 = sq.z * sq.z, z1 = S2 * S2;
                const float dan = (-P.K2 * z1 - P.K4 * z1 * z1) - (-P.K2 * z0 - P.K4 * z0 * z0);
                const float self = W0.x * dX * dX + 2.0f * W0.y * dX * dY + W0.z * dY * dY + W0.w * dZ * dZ;
                const float4 h = h4[q];
                const float dE = dex + dan + P.CD * ((dX * h.x + dY * h.y + dZ * h.z) + 0.5f * self);
                const float thr = (uacc > 0.0f) ? -P.T * logf(uacc) : INFINITY;
                const int accept = dE < thr;
                if (b.trace) {
                    float *tr = b.trace + ((((size_t)r * cfg.nsweeps_call + cfg.it0 + it) * ll + k) * n + d) * MC_TRACE_W;
                    tr[0] = (float)q;
                    tr[1] = h.x; tr[2] = h.y; tr[3] = h.z;
                    tr[4] = dE;
                    tr[5] = uacc;
                    tr[6] = (float)accept;
                    tr[7] = S0; tr[8] = S1; tr[9] = S2;
                }
                mv[d] = accept ? make_float4(dX, dY, dZ, 1.0f) : make_float4(0.f, 0.f, 0.f, 0.f);
                mS[d] = make_float4(S0, S1, S2, 0.f);
                nacc += accept;
            }
            if (nacc) atomicAdd(&s_acc, nacc);
            __syncthreads();
            // ---- write the accepted moves and update the field everywhere
            for (int d = tid; d < n; d += kIThreads) {
                if (mv[d].w != 0.f) s4[(oy + l * (d / C)) * L + ox + l * (d % C)] = mS[d];
            }
            for (int i = tid; i < N; i += kIThreads) {
                const int iy = i / L, ix = i - iy * L;
                float4 h = h4[i];
                for (int d = 0; d < n; ++d) {
                    const float4 m = mv[d];
                    if (m.w == 0.f) continue;
                    int dx = ix - (ox + l * (d % C)), dy = iy - (oy + l * (d / C));
                    dx += dx < 0 ? L : 0;
                    dy += dy < 0 ? L : 0;
                    const float4 w = w4[dy * L + dx];
                    h.x = fmaf(w.x, m.x, fmaf(w.y, m.y, h.x));
                    h.y = fmaf(w.y, m.x, fmaf(w.z, m.y, h.y));
                    h.z = fmaf(w.w, m.z, h.z);
                }
                h4[i] = h;
            }
            __syncthreads();
        }
        // ---- observables of this sweep, energy from the kept field
        if (cfg.measure_every > 0 && ((cfg.it0 + it + 1) % cfg.measure_every) == 0) {
            // mx, my, mz, mh, mv, exchange, anisotropy, s.h, wall counts n_h/n_v of x, y, z, sum |theta - pi/2|
            double v[15] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
            double *gt = b.theta2 ? b.theta2 + (size_t)r * N : nullptr;
            for (int i = tid; i < N; i += kIThreads) {
                const int iy = i / L, ix = i - iy * L;
                const float4 a = s4[i], h = h4[i];
                const float4 ax = s4[iy * L + (ix + 1 == L ? 0 : ix + 1)], ay = s4[(iy + 1 == L ? 0 : iy + 1) * L + ix];
                v[0] += a.x;
                v[1] += a.y;
                v[2] += a.z;
                v[3] += (iy & 1) ? -a.z : a.z;
                v[4] += (ix & 1) ? -a.z : a.z;
                v[5] += (double)a.x * ((double)ax.x + ay.x) + (double)a.y * ((double)ax.y + ay.y) +
                        (double)a.z * ((double)ax.z + ay.z);
                const double z2 = (double)a.z * a.z;
                v[6] += -(double)P.K2 * z2 - (double)P.K4 * z2 * z2;
                v[7] += (double)a.x * h.x + (double)a.y * h.y + (double)a.z * h.z;
                v[8] += wall_term(a.x, ax.x);
                v[9] += wall_term(a.x, ay.x);
                v[10] += wall_term(a.y, ax.y);
                v[11] += wall_term(a.y, ay.y);
                v[12] += wall_term(a.z, ax.z);
                v[13] += wall_term(a.z, ay.z);
                const float th = acosf(fminf(1.0f, fmaxf(-1.0f, a.z))) - 0.5f * kPiF;
                v[14] += fabsf(th);
                if (gt) gt[i] += (double)(th * th);
            }
#pragma unroll
            for (int c = 0; c < 15; ++c)
                for (int off = 16; off; off >>= 1) v[c] += __shfl_xor_sync(0xffffffffu, v[c], off);
            if (lane == 0)
                for (int c = 0; c < 15; ++c) red[warp][c] = v[c];
            __syncthreads();
            if (tid == 0) {
                double s[15] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
                for (int w = 0; w < NW; ++w)
                    for (int c = 0; c < 15; ++c) s[c] += red[w][c];
                const double Mx = s[0] / N, My = s[1] / N, Mz = s[2] / N;
                const double E = -(double)P.J * s[5] + s[6] + 0.5 * (double)P.CD * s[7];
                double x[MC_NOBS];
                x[MC_OBS_ABS_M] = sqrt(Mx * Mx + My * My + Mz * Mz);
                x[MC_OBS_MZ] = Mz;
                x[MC_OBS_ABS_MZ] = fabs(Mz);
                x[MC_OBS_MPAR] = sqrt(Mx * Mx + My * My);
                x[MC_OBS_E] = E / N;
                x[MC_OBS_MST] = sqrt(s[3] * s[3] + s[4] * s[4]) / N;
                const double nh[3] = {s[8], s[10], s[12]}, nv[3] = {s[9], s[11], s[13]};
                stripe_obs(x, nh, nv, s[14], N);
                if (b.obs) obs_push(b.obs[r], x);
                hist_push(b.hist, r, E / N);
                if (b.energy) b.energy[r] = E;
            }
            __syncthreads();
        }
    }
    // ---- write back the spins and the counters
    float *gd = b.spins + (size_t)r * 3 * N;
    for (int i = tid; i < N; i += kIThreads) {
        const float4 a = s4[i];
        gd[i] = a.x;
        gd[N + i] = a.y;
        gd[2 * N + i] = a.z;
    }
    if (tid == 0 && b.obs) {
        b.obs[r].accepted += s_acc;
        b.obs[r].attempted += (long long)cfg.nsweeps * N;
    }
}

size_t incr_smem(int L, int l) {
    const size_t N = (size_t)L * L, n = (size_t)(L / l) * (L / l), ll = (size_t)l * l;
    return sizeof(float4) * (3 * N + 2 * n) + sizeof(uint16_t) * ll;
}

}  // namespace

bool incremental_supported(int L, int l) {
    if (l < 2 || L % l || l > 256) return false;
    const int C = L / l;
    return C * C <= 64 && incr_smem(L, l) <= 220 * 1024;
}

cudaError_t launch_sweep_incremental(const IncrConfig &c, const IncrBuffers &b, cudaStream_t st) {
    const size_t smem = incr_smem(c.L, c.l);
    cudaError_t e = cudaFuncSetAttribute(k_sweep_incremental, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_sweep_incremental<<<c.R, kIThreads, smem, st>>>(c, b);
    return cudaGetLastError();
}

}  // namespace dipmc
