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

// Orthonormal pair perpendicular to a unit vector n (Duff et al., "Building an
// orthonormal basis, revisited", JCGT 2017).
__device__ __forceinline__ void perp_basis(float nx, float ny, float nz, float3 &b1, float3 &b2) {
    const float sign = copysignf(1.0f, nz);
    const float a = -1.0f / (sign + nz);
    const float b = nx * ny * a;
    b1 = make_float3(1.0f + sign * nx * nx * a, sign * b, -sign * nx);
    b2 = make_float3(b, sign + ny * ny * a, -ny);
}

// One measurement sample into the binning accumulators (FP64, one thread).
__device__ void obs_push(ObsAcc &A, const double x[MC_NOBS]) {
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

template <int C, int EPT, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) k_sweep_direct(const SweepConfig cfg, const SweepBuffers buf) {
    constexpr int n = C * C;
    constexpr int V = 3 * n;                    // partial-field values per thread
    constexpr int G = (V + 31) / 32;            // groups of <= 32 values
    constexpr int PV = pow2_at_least(V < 32 ? V : 32);
    const int L = cfg.L, l = cfg.l, N = L * L, ll = l * l;
    const int tid = threadIdx.x, NT = blockDim.x, lane = tid & 31, warp = tid >> 5, NW = NT >> 5;
    const int r = blockIdx.x;

    extern __shared__ float4 smem_f4[];
    float *sx = reinterpret_cast<float *>(smem_f4);
    float *sy = sx + N;
    float *sz = sy + N;
    float *th2 = sz + N;                 // [N] per-site (theta - pi/2)^2 this launch
    float *red = th2 + N;                // [NW][V]
    float *mred = red + NW * V;          // [NW][4] magnetisation reduction
    uint16_t *sched = reinterpret_cast<uint16_t *>(mred + NW * 4);  // [ll]
    __shared__ ObsAcc acc_s;
    __shared__ double e_track_s;

    // ---- load state
    const float *gs = buf.spins + (size_t)r * 3 * N;
    for (int i = tid; i < 3 * N; i += NT) sx[i] = gs[i];
    const bool measuring = cfg.measure_every > 0;
    if (measuring)
        for (int i = tid; i < N; i += NT) th2[i] = 0.0f;
    if (tid == 0) {
        if (buf.obs) acc_s = buf.obs[r];
        e_track_s = buf.energy ? buf.energy[r] : 0.0;
    }

    // ---- tensor slices for this thread's cell offsets e (registers, whole launch)
    float w[EPT][n][4];
    int ex[EPT], ey[EPT];
#pragma unroll
    for (int j = 0; j < EPT; ++j) {
        const int e = tid + j * NT;
        const bool valid = e < ll;
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
            for (int c = 0; c < 4; ++c) w[j][D][c] = valid ? buf.W32[c * N + idx] : 0.0f;
        }
    }

    const RepParams P = buf.params[r];
    const float W0xx = buf.W32[0], W0xy = buf.W32[N], W0yy = buf.W32[2 * N], W0zz = buf.W32[3 * N];
    const uint2 key = cfg.key;
    const int hbits = ceil_log2_u((uint32_t)l);
    double e_part = 0.0;        // lanes < n of warp 0: this lane's tracked energy change
    long long n_acc = 0;        // lane 0 of warp 0: accepted moves
    __syncthreads();

    for (int it = 0; it < cfg.nsweeps; ++it) {
        const uint32_t t = cfg.t0 + (uint32_t)it;
        // ---- the sweep's schedule
        if (cfg.schedule == 0) {
            const uint4 rk = philox(make_uint4(t, 0u, 0u, kTagPerm), key);
            for (int k = tid; k < ll; k += NT) sched[k] = (uint16_t)perm_offset(rk, hbits, (uint32_t)ll, (uint32_t)k);
        } else {
            for (int k = tid; k < ll; k += NT) {
                const uint4 o = philox(make_uint4(t, (uint32_t)k, 0u, kTagDraw), key);
                sched[k] = (uint16_t)(uint32_t)(((unsigned long long)o.x * (unsigned long long)ll) >> 32);
            }
        }
        __syncthreads();

        for (int k = 0; k < ll; ++k) {
            const int v = sched[k];
            const int ox = v % l, oy = v / l;

            // random numbers of this sub-step (independent of the state): lanes d < n of warp 0
            float u1 = 0.f, cps = 0.f, sps = 0.f, uacc = 1.f;
            int qx = 0, qy = 0, q = 0;
            if (warp == 0 && lane < n) {
                qx = ox + l * (lane % C);
                qy = oy + l * (lane / C);
                q = qy * L + qx;
                const uint4 wds = philox(make_uint4((uint32_t)q, (uint32_t)r, t, ((uint32_t)k & 0x00FFFFFFu) | kTagAttempt), key);
                u1 = u24f(wds.x);
                sincospif(2.0f * u24f(wds.y), &sps, &cps);
                uacc = u24f(wds.z);
            }

            // ---- partial fields at the n update sites
            float acc[n][3];
#pragma unroll
            for (int d = 0; d < n; ++d) acc[d][0] = acc[d][1] = acc[d][2] = 0.0f;
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
                        const int m = yy * L + xx;
                        const float a = sx[m], b = sy[m], c = sz[m];
#pragma unroll
                        for (int dy = 0; dy < C; ++dy)
#pragma unroll
                            for (int dx = 0; dx < C; ++dx) {
                                const int D = ((dx - mx + C) % C) + C * ((dy - my + C) % C);
                                const int dq = dx + C * dy;
                                acc[dq][0] = fmaf(w[j][D][0], a, fmaf(w[j][D][1], b, acc[dq][0]));
                                acc[dq][1] = fmaf(w[j][D][1], a, fmaf(w[j][D][2], b, acc[dq][1]));
                                acc[dq][2] = fmaf(w[j][D][3], c, acc[dq][2]);
                            }
                    }
                }
            }
            // ---- CTA reduction: warp reduce-scatter, then warp 0 sums across warps
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
                if (reduce_scatter_writer<PV>(lane) && vi < V) red[warp * V + vi] = s;
            }
            __syncthreads();

            if (warp == 0) {
                // cross-warp sum: lane j owns values j, j+32, ...
                float hsum[G];
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    const int vi = g * 32 + lane;
                    float s = 0.0f;
                    if (vi < V)
                        for (int ww = 0; ww < NW; ++ww) s += red[ww * V + vi];
                    hsum[g] = s;
                }
                float h[3];
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
                float dX = 0.f, dY = 0.f, dZ = 0.f, dE = 0.f;
                int accept = 0;
                if (lane < n) {
                    const float s0 = sx[q], s1 = sy[q], s2 = sz[q];
                    float S0, S1, S2;
                    if (cfg.proposal == 1) {
                        const float z = 2.0f * u1 - 1.0f;
                        const float rr = sqrtf(fmaxf(0.0f, (1.0f - z) * (1.0f + z)));
                        S0 = rr * cps;
                        S1 = rr * sps;
                        S2 = z;
                    } else {
                        const float ca = 1.0f - u1 * cfg.cap_c1;
                        const float sa = sqrtf(fmaxf(0.0f, (1.0f - ca) * (1.0f + ca)));
                        float3 b1, b2;
                        perp_basis(s0, s1, s2, b1, b2);
                        S0 = ca * s0 + sa * (cps * b1.x + sps * b2.x);
                        S1 = ca * s1 + sa * (cps * b1.y + sps * b2.y);
                        S2 = ca * s2 + sa * (cps * b1.z + sps * b2.z);
                        const float inv = 1.0f / sqrtf(S0 * S0 + S1 * S1 + S2 * S2);
                        S0 *= inv;
                        S1 *= inv;
                        S2 *= inv;
                    }
                    dX = S0 - s0;
                    dY = S1 - s1;
                    dZ = S2 - s2;
                    const int xp = (qx + 1 == L) ? q - qx : q + 1;
                    const int xm = (qx == 0) ? q + L - 1 : q - 1;
                    const int yp = (qy + 1 == L) ? qx : q + L;
                    const int ym = (qy == 0) ? q + N - L : q - L;
                    const float n0 = (sx[xp] + sx[xm]) + (sx[yp] + sx[ym]);
                    const float n1 = (sy[xp] + sy[xm]) + (sy[yp] + sy[ym]);
                    const float n2 = (sz[xp] + sz[xm]) + (sz[yp] + sz[ym]);
                    const float dex = -P.J * (dX * n0 + dY * n1 + dZ * n2);
                    const float z0 = s2 * s2, z1 = S2 * S2;
                    const float dan = (-P.K2 * z1 - P.K4 * z1 * z1) - (-P.K2 * z0 - P.K4 * z0 * z0);
                    const float self = W0xx * dX * dX + 2.0f * W0xy * dX * dY + W0yy * dY * dY + W0zz * dZ * dZ;
                    const float ddip = P.CD * ((dX * h[0] + dY * h[1] + dZ * h[2]) + 0.5f * self);
                    dE = dex + dan + ddip;
                    accept = uacc < expf(-dE / P.T);
                    if (buf.trace) {
                        float *tr = buf.trace + ((((size_t)r * cfg.nsweeps + it) * ll + k) * n + lane) * MC_TRACE_W;
                        tr[0] = (float)q;
                        tr[1] = h[0]; tr[2] = h[1]; tr[3] = h[2];
                        tr[4] = dE;
                        tr[5] = uacc;
                        tr[6] = (float)accept;
                        tr[7] = S0; tr[8] = S1; tr[9] = S2;
                    }
                    if (accept) {
                        sx[q] = S0;
                        sy[q] = S1;
                        sz[q] = S2;
                    } else {
                        dX = dY = dZ = 0.0f;
                        dE = 0.0f;
                    }
                }
                // ---- exact energy bookkeeping: accepted dE plus pair cross terms
                float cross = 0.0f;
#pragma unroll
                for (int dp = 0; dp < n - 1; ++dp) {
                    const float pX = __shfl_sync(0xffffffffu, dX, dp);
                    const float pY = __shfl_sync(0xffffffffu, dY, dp);
                    const float pZ = __shfl_sync(0xffffffffu, dZ, dp);
                    if (lane < n && dp < lane) {
                        // W~(q_lane - q_dp) = W~(l * (D_lane - D_dp) mod L)
                        int rx = l * ((lane % C) - (dp % C));
                        int ry = l * ((lane / C) - (dp / C));
                        if (rx < 0) rx += L;
                        if (ry < 0) ry += L;
                        const int idx = ry * L + rx;
                        const float xx = __ldg(buf.W32 + idx), xy = __ldg(buf.W32 + N + idx);
                        const float yy = __ldg(buf.W32 + 2 * N + idx), zz = __ldg(buf.W32 + 3 * N + idx);
                        cross += pX * (xx * dX + xy * dY) + pY * (xy * dX + yy * dY) + pZ * (zz * dZ);
                    }
                }
                if (lane < n) e_part += (double)dE + (double)(P.CD * cross);
                const unsigned ball = __ballot_sync(0xffffffffu, accept);
                if (lane == 0) n_acc += __popc(ball);
            }
            __syncthreads();
        }

        // ---- observables of this sweep
        if (measuring && ((it + 1) % cfg.measure_every) == 0) {
            float mx = 0.f, my = 0.f, mz = 0.f;
            for (int i = tid; i < N; i += NT) {
                const float a = sx[i], b = sy[i], c = sz[i];
                mx += a;
                my += b;
                mz += c;
                const float th = acosf(fminf(1.0f, fmaxf(-1.0f, c))) - 0.5f * kPiF;
                th2[i] += th * th;
            }
            for (int off = 16; off; off >>= 1) {
                mx += __shfl_xor_sync(0xffffffffu, mx, off);
                my += __shfl_xor_sync(0xffffffffu, my, off);
                mz += __shfl_xor_sync(0xffffffffu, mz, off);
            }
            if (lane == 0) {
                mred[warp * 4 + 0] = mx;
                mred[warp * 4 + 1] = my;
                mred[warp * 4 + 2] = mz;
            }
            __syncthreads();
            if (warp == 0) {
                double et = e_part;
                for (int off = 16; off; off >>= 1) et += __shfl_xor_sync(0xffffffffu, et, off);
                if (lane == 0) {
                    double Mx = 0, My = 0, Mz = 0;
                    for (int ww = 0; ww < NW; ++ww) {
                        Mx += mred[ww * 4 + 0];
                        My += mred[ww * 4 + 1];
                        Mz += mred[ww * 4 + 2];
                    }
                    Mx /= N; My /= N; Mz /= N;
                    double x[MC_NOBS];
                    x[MC_OBS_ABS_M] = sqrt(Mx * Mx + My * My + Mz * Mz);
                    x[MC_OBS_MZ] = Mz;
                    x[MC_OBS_ABS_MZ] = fabs(Mz);
                    x[MC_OBS_MPAR] = sqrt(Mx * Mx + My * My);
                    x[MC_OBS_E] = (e_track_s + et) / N;
                    if (buf.obs) obs_push(acc_s, x);
                }
            }
            __syncthreads();
        }
    }

    // ---- write back
    float *gd = buf.spins + (size_t)r * 3 * N;
    for (int i = tid; i < 3 * N; i += NT) gd[i] = sx[i];
    if (measuring && buf.theta2) {
        double *gt = buf.theta2 + (size_t)r * N;
        for (int i = tid; i < N; i += NT) gt[i] += (double)th2[i];
    }
    if (warp == 0) {
        double et = e_part;
        for (int off = 16; off; off >>= 1) et += __shfl_xor_sync(0xffffffffu, et, off);
        if (lane == 0) {
            if (buf.energy) buf.energy[r] = e_track_s + et;
            if (buf.obs) {
                acc_s.accepted += n_acc;
                acc_s.attempted += (long long)cfg.nsweeps * N;
                buf.obs[r] = acc_s;
            }
        }
    }
}

struct Inst {
    int C, EPT, MAXT;
    cudaError_t (*launch)(const SweepConfig &, const SweepBuffers &, int, size_t, cudaStream_t);
};

template <int C, int EPT, int MAXT>
cudaError_t launch_inst(const SweepConfig &c, const SweepBuffers &b, int threads, size_t smem, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k_sweep_direct<C, EPT, MAXT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_sweep_direct<C, EPT, MAXT><<<c.R, threads, smem, st>>>(c, b);
    return cudaGetLastError();
}

// Register budget: C^2*4*EPT tensor values + 3*C^2 accumulators per thread; the
// launch bound caps threads so that they fit without spilling.
const Inst kInst[] = {
    {1, 1, 1024, launch_inst<1, 1, 1024>}, {1, 2, 512, launch_inst<1, 2, 512>},
    {1, 4, 512, launch_inst<1, 4, 512>},   {1, 8, 512, launch_inst<1, 8, 512>},
    {1, 18, 512, launch_inst<1, 18, 512>},
    {2, 1, 1024, launch_inst<2, 1, 1024>}, {2, 2, 512, launch_inst<2, 2, 512>},
    {2, 3, 512, launch_inst<2, 3, 512>},   {2, 5, 512, launch_inst<2, 5, 512>},
    {4, 1, 256, launch_inst<4, 1, 256>},   {4, 2, 256, launch_inst<4, 2, 256>},
};

size_t smem_bytes(int L, int l, int threads) {
    const int N = L * L, C = L / l, n = C * C, NW = threads / 32;
    size_t b = sizeof(float) * (size_t)(4 * N + NW * 3 * n + NW * 4);
    b += sizeof(uint16_t) * (size_t)l * l;
    return (b + 15) & ~(size_t)15;
}

// Choose the instance: fewest cell offsets per thread with at most
// min(max_threads, instance bound) threads.
const Inst *pick(int L, int l, int max_threads, int *threads) {
    if (l < 2 || L % l) return nullptr;
    const int C = L / l, ll = l * l;
    const Inst *best = nullptr;
    for (const Inst &in : kInst) {
        if (in.C != C) continue;
        int th = (ll + in.EPT - 1) / in.EPT;
        th = ((th + 31) / 32) * 32;
        if (th > max_threads || th > in.MAXT) continue;
        if (!best || in.EPT < best->EPT) {
            best = &in;
            *threads = th;
        }
    }
    if (!best) return nullptr;
    if (smem_bytes(L, l, *threads) > 200 * 1024) return nullptr;
    return best;
}

}  // namespace

bool direct_supported(int L, int l) {
    int th = 0;
    return pick(L, l, 1024, &th) != nullptr;
}

cudaError_t launch_sweep_direct(const SweepConfig &c, const SweepBuffers &b, int threads_hint,
                                cudaStream_t st) {
    int threads = 0;
    const Inst *in = pick(c.L, c.l, threads_hint > 0 ? threads_hint : 1024, &threads);
    if (!in) in = pick(c.L, c.l, 1024, &threads);
    if (!in) return cudaErrorNotSupported;
    return in->launch(c, b, threads, smem_bytes(c.L, c.l, threads), st);
}

}  // namespace dipmc
