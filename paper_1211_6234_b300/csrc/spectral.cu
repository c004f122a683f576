// spectral.cu -- the dipole field at a sub-step's update sites by sub-lattice
// spectra, and the sweep path built on it (Sec. 3.1, 3.2 update; Eq. 2 field).
//
// With C = L/l, every site is m = e + l*D (cell offset e in [0, l)^2, coarse
// position D in [0, C)^2), and the update sites of offset o are q = o + l*Dq.
// Their field splits into l^2 circular convolutions on the C x C coarse grid:
//     h(o + l*Dq) = sum_e sum_Dm W~(o - e + l*(Dq - Dm)) s(e + l*Dm).
// With the C x C DFT (omega = exp(-2 pi i / C)), S_e(K) = DFT_D s(e + l*D) and
// T_d(K) = DFT_D W~(d + l*D) for d in [0, l)^2, the convolution theorem gives
//     H_o(K) = sum_e omega^(K . sigma) T_{(o - e) mod l}(K) S_e(K),
// sigma_x = 1 where o_x < e_x (and likewise y): the wrap of o - e into [0, l)
// shifts the coarse sequence by one cell.  h at the n sites is the inverse DFT
// of H_o.  Only S_o changes in a sub-step (the update sites are exactly the
// sub-lattice of offset o), so after the update S_o is recomputed from the new
// spins.  A sub-step therefore costs O(N) -- the contraction over e -- instead
// of the O(N n) of a direct sum or the O(N log N) of a full-lattice FFT.
//
// Windows of wmax sub-steps: k_spec_wfield contracts, once per window, the spectra
// at the window's start against T for all of the window's offsets (grid over
// (replica, K, window slot) and chunks of e, partial spectra summed in a fixed
// order), so that every S_e is read once per window instead of once per sub-step.
// k_spec_wupdate (one CTA per replica) then runs the window's sub-steps in order:
// since only S_o of the updated offset o changes in a sub-step, the spectra of a
// later sub-step are its window-start spectra plus the terms
// omega^(K.sigma) T_{(o' - o) mod l}(K) dS_o(K) of the window's earlier changes
// dS_o; then the inverse DFT, Metropolis decisions and the forward DFT of the
// updated sub-lattice.  DFTs are separable direct sums in shared memory (C <= 32).
// T is built once in FP64.
#include <algorithm>

#include "spectral.cuh"

namespace dipmc {

namespace {

constexpr int kSpecThreads = 256;
constexpr int kUpdMaxThreads = 1024;
constexpr int kSpecMaxC = 32;
constexpr int kSpecWinMax = 8;    // sub-steps of a window (k_spec_wfield: one warp each)

// x / d by a multiply-high with m = ceil(2^32 / d): exact while x * d < 2^32
// (here x < 3 n <= 3072, d <= 1024)
__device__ __forceinline__ int qdiv(int x, uint32_t m) { return (int)__umulhi((uint32_t)x, m); }

__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {  // a*b + c
    return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}
// omega^m = exp(-2 pi i m / C), m in [0, C)
__device__ __forceinline__ float2 omega(int m, int C) {
    float s, c;
    sincospif(2.0f * (float)m / (float)C, &s, &c);
    return make_float2(c, -s);
}

// Real spins and W~ make every spectrum Hermitian, X(-K) = conj X(K), so the window
// field computes only an independent half of the C x C wave vectors: the row Ky = 0
// with Kx <= C/2, the rows 0 < Ky < C/2 (all Kx) and, for even C, the row Ky = C/2
// with Kx <= C/2.  half_count(C) of them; half_wave(t) is the t-th.
__host__ __device__ __forceinline__ int half_count(int C) {
    return C / 2 + 1 + ((C - 1) / 2) * C + (C % 2 == 0 ? C / 2 + 1 : 0);
}
__device__ __forceinline__ int half_wave(int t, int C) {   // K = Ky * C + Kx
    const int h0 = C / 2 + 1, mid = (C - 1) / 2;
    if (t < h0) return t;
    t -= h0;
    if (t < mid * C) return (1 + t / C) * C + t % C;
    return (C / 2) * C + (t - mid * C);
}
// K itself if it is in the computed half, else its partner -K (conjugate on use)
__device__ __forceinline__ int half_source(int K, int C, bool &conj) {
    const int Ky = K / C, Kx = K - Ky * C;
    const bool in = (Ky == 0 || 2 * Ky == C) ? 2 * Kx <= C : 2 * Ky < C;
    conj = !in;
    if (in) return K;
    return ((C - Ky) % C) * C + (C - Kx) % C;
}

// Stream state of replica r: its key, its sweep counter at sweep `it` of the
// call and the replica index its counters use; false for an idle slot.
__device__ __forceinline__ bool stream_state(const SpecConfig &cfg, const SpecBuffers &b, int r, uint2 &key,
                                             uint32_t &t, uint32_t &rid) {
    key = cfg.key;
    t = cfg.t_dev ? *cfg.t_dev + (uint32_t)cfg.it : cfg.t;
    rid = (uint32_t)r;
    if (b.slots) {
        const SlotState sl = b.slots[r];
        if (cfg.it >= sl.nsweeps) return false;
        key = make_uint2(sl.key_lo, sl.key_hi);
        t = sl.t0 + (uint32_t)cfg.it;
        rid = sl.rid;
    }
    return true;
}

// Offset (ox, oy) of sub-step k of sweep t (the schedule of the other paths).
__device__ __forceinline__ void sub_offset(const SpecConfig &cfg, uint2 key, uint32_t t, int &ox, int &oy) {
    const int l = cfg.l, ll = l * l;
    const uint32_t k = (uint32_t)cfg.k;
    uint32_t v;
    if (cfg.schedule == 0) {
        const uint4 rk = philox(make_uint4(t, 0u, 0u, kTagPerm), key);
        v = perm_offset(rk, ceil_log2_u((uint32_t)l), (uint32_t)ll, k);
    } else {
        const uint4 o = philox(make_uint4(t, k, 0u, kTagDraw), key);
        v = (uint32_t)(((unsigned long long)o.x * (unsigned long long)ll) >> 32);
    }
    ox = (int)(v % l);
    oy = (int)(v / l);
}

// ---------------------------------------------------------------------------
// Offsets of every sub-step of sweep `it` for every replica: off[r][k] =
// (oy << 16) | ox, or -1 for a slot idle in this sweep.
// ---------------------------------------------------------------------------
__global__ void k_spec_offsets(const SpecConfig cfg, const SpecBuffers b) {
    const int ll = cfg.l * cfg.l;
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (long long)cfg.R * ll) return;
    const int r = (int)(g / ll), k = (int)(g % ll);
    uint2 key;
    uint32_t t, rid;
    int v = -1;
    if (stream_state(cfg, b, r, key, t, rid)) {
        SpecConfig c = cfg;
        c.k = k;
        int ox, oy;
        sub_offset(c, key, t, ox, oy);
        v = (oy << 16) | ox;
    }
    b.off[g] = v;
}

// ---------------------------------------------------------------------------
// T_d^c(K) = sum_D W~_c(d + l*D) omega^(K.D): one CTA per (d, c), FP64.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kSpecThreads) k_spec_table(int L, int l, const double *__restrict__ W64,
                                                             float2 *__restrict__ T) {
    const int C = L / l, n = C * C, N = L * L;
    const int d = blockIdx.x >> 2, c = blockIdx.x & 3;
    const int dx = d % l, dy = d / l;
    extern __shared__ double2 sm_d[];
    double2 *U = sm_d;           // [Dy][Kx]
    double2 *tw = sm_d + n;      // [C]
    for (int m = threadIdx.x; m < C; m += blockDim.x) {
        double s, co;
        sincospi(2.0 * (double)m / (double)C, &s, &co);
        tw[m] = make_double2(co, -s);
    }
    __syncthreads();
    const double *w = W64 + (size_t)c * N;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int Dy = i / C, Kx = i % C;
        const double *row = w + (size_t)(dy + l * Dy) * L + dx;
        double re = 0, im = 0;
        for (int Dx = 0; Dx < C; ++Dx) {
            const double v = row[l * Dx];
            const double2 o = tw[(Kx * Dx) % C];
            re += v * o.x;
            im += v * o.y;
        }
        U[i] = make_double2(re, im);
    }
    __syncthreads();
    // four copies with the wrap phase omega^(K.sigma) applied, sigma = (sx, sy), copy sx + 2 sy
    const size_t csz = (size_t)l * l * 4 * n;
    float2 *out = T + ((size_t)d * 4 + c) * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int Ky = i / C, Kx = i % C;
        double re = 0, im = 0;
        for (int Dy = 0; Dy < C; ++Dy) {
            const double2 u = U[Dy * C + Kx], o = tw[(Ky * Dy) % C];
            re += u.x * o.x - u.y * o.y;
            im += u.x * o.y + u.y * o.x;
        }
#pragma unroll
        for (int sg = 0; sg < 4; ++sg) {
            const double2 p = tw[((sg & 1) * Kx + (sg >> 1) * Ky) % C];
            out[sg * csz + i] = make_float2((float)(re * p.x - im * p.y), (float)(re * p.y + im * p.x));
        }
    }
}

// Forward DFT of three real C x C planes in shared memory (x[3][n]) into
// out[3][n] (global), through U[3][n]; tw = omega^m.
__device__ __forceinline__ void dft3_forward(const float *x, float2 *U, const float2 *tw, int C, float2 *out,
                                             size_t out_stride) {
    const int n = C * C;
    for (int i = threadIdx.x; i < 3 * n; i += blockDim.x) {
        const int b = i / n, j = i % n, Dy = j / C, Kx = j % C;
        const float *row = x + b * n + Dy * C;
        float2 acc = make_float2(0.f, 0.f);
        for (int Dx = 0, m = 0; Dx < C; ++Dx) {       // m = Kx * Dx mod C
            const float2 o = tw[m];
            acc.x = fmaf(row[Dx], o.x, acc.x);
            acc.y = fmaf(row[Dx], o.y, acc.y);
            m += Kx;
            if (m >= C) m -= C;
        }
        U[i] = acc;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * n; i += blockDim.x) {
        const int b = i / n, j = i % n, Ky = j / C, Kx = j % C;
        const float2 *col = U + b * n + Kx;
        float2 acc = make_float2(0.f, 0.f);
        for (int Dy = 0, m = 0; Dy < C; ++Dy) {       // m = Ky * Dy mod C
            acc = cfma(col[Dy * C], tw[m], acc);
            m += Ky;
            if (m >= C) m -= C;
        }
        out[(size_t)b * out_stride + j] = acc;
    }
}

// ---------------------------------------------------------------------------
// S_e for every (replica, cell offset): one CTA per (e, r).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kSpecThreads) k_spec_init(int L, int l, const float *__restrict__ spins,
                                                            float2 *__restrict__ S) {
    const int C = L / l, n = C * C, N = L * L, ll = l * l;
    const int e = blockIdx.x, r = blockIdx.y;
    const int ex = e % l, ey = e / l;
    extern __shared__ float2 sm_f2[];
    float2 *tw = sm_f2;                                         // [C]
    float2 *U = tw + kSpecMaxC;                                 // [3][n]
    float *x = reinterpret_cast<float *>(U + 3 * n);            // [3][n]
    for (int m = threadIdx.x; m < C; m += blockDim.x) tw[m] = omega(m, C);
    const float *s = spins + (size_t)r * 3 * N;
    for (int i = threadIdx.x; i < 3 * n; i += blockDim.x) {
        const int b = i / n, D = i % n;
        x[i] = s[(size_t)b * N + (size_t)(ey + l * (D / C)) * L + ex + l * (D % C)];
    }
    __syncthreads();
    dft3_forward(x, U, tw, C, S + ((size_t)r * ll + e) * 3 * n, (size_t)n);
}

// ---------------------------------------------------------------------------
// A window is wlen <= wmax consecutive sub-steps k .. k + wlen - 1.
//
// k_spec_wfield: the field spectra of the window's offsets o_w from the spectra at
// the window's start, H_w(K) = sum_e omega^(K.sigma) T_{(o_w - e) mod l}(K) S_e(K).
// Thread = (replica r, wave vector K, window slot w) over a chunk of the cell
// offsets e (grid z); warp w of a CTA is slot w for 2 replicas x 16 wave vectors
// (a warp's table and spectra loads are 128-byte runs), so the CTA's warps read the
// same S_e through L1.  Partial spectra per chunk,
// Hw[z][r][w][3][n], are summed by the update in chunk order.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kSpecThreads) k_spec_wfield(const SpecConfig cfg, const SpecBuffers b) {
    pdl_trigger();
    pdl_wait();   // the spectra and offsets written by the previous kernels
    const int L = cfg.L, l = cfg.l, C = L / l, n = C * C, ll = l * l, R = cfg.R;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int th = blockIdx.x * 16 + (lane & 15), r = blockIdx.y * 2 + (lane >> 4);
    const bool mine = th < half_count(C) && r < R && w < cfg.wlen;
    const int K = mine ? half_wave(th, C) : 0;
    const int ov = mine ? b.off[(size_t)r * ll + cfg.k + w] : -1;
    float2 hx = make_float2(0.f, 0.f), hy = hx, hz = hx;
    if (ov >= 0) {
        const int ox = ov & 0xFFFF, oy = ov >> 16;
        const int ec = (ll + gridDim.z - 1) / gridDim.z;
        const int e0 = blockIdx.z * ec, e1 = min(ll, e0 + ec);
        const float2 *Sr = b.S + (size_t)r * ll * 3 * n + K;
        int ex = e0 % l, ey = e0 / l;
        constexpr int kU = 4;   // cell offsets in flight
        for (int eb = e0; eb < e1; eb += kU) {
            float2 tv[kU][4], sv[kU][3];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                if (eb + u < e1) {
                    int dx = ox - ex, dy = oy - ey;
                    const int sx = dx < 0, sy = dy < 0;
                    dx += sx ? l : 0;
                    dy += sy ? l : 0;
                    // the table copy with the wrap phase omega^(K.sigma) applied
                    const float2 *Tp = b.T + ((size_t)((sx + 2 * sy) * ll + dy * l + dx) * 4) * n + K;
                    const float2 *Sp = Sr + (size_t)(eb + u) * 3 * n;
#pragma unroll
                    for (int c = 0; c < 4; ++c) tv[u][c] = __ldg(Tp + c * n);
#pragma unroll
                    for (int c = 0; c < 3; ++c) sv[u][c] = Sp[c * n];
                } else {
#pragma unroll
                    for (int c = 0; c < 4; ++c) tv[u][c] = make_float2(0.f, 0.f);
#pragma unroll
                    for (int c = 0; c < 3; ++c) sv[u][c] = make_float2(0.f, 0.f);
                }
                if (++ex == l) {
                    ex = 0;
                    ++ey;
                }
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                hx = cfma(tv[u][0], sv[u][0], cfma(tv[u][1], sv[u][1], hx));
                hy = cfma(tv[u][1], sv[u][0], cfma(tv[u][2], sv[u][1], hy));
                hz = cfma(tv[u][3], sv[u][2], hz);
            }
        }
    }
    if (mine) {
        float2 *o = b.Hw + ((((size_t)blockIdx.z * R + r) * cfg.wmax + w) * 3) * n + K;
        o[0] = hx;
        o[n] = hy;
        o[2 * n] = hz;
    }
}

// ---------------------------------------------------------------------------
// k_spec_wupdate: one CTA per replica runs the window's sub-steps in order.  The
// field spectra of sub-step w are its window-start spectra (the chunk sum of Hw)
// plus, for every earlier sub-step v of the window, the term of the change of
// S_{o_v}: omega^(K.sigma) T_{(o_w - o_v) mod l}(K) dS_v(K).  Then as a single
// sub-step: inverse DFT to the n sites, Metropolis decisions, DFT of the updated
// sub-lattice, whose change dS_w is kept for the later sub-steps.
// ---------------------------------------------------------------------------
template <int MAXT>
__global__ void __launch_bounds__(MAXT) k_spec_wupdate(const SpecConfig cfg, const SpecBuffers b) {
    pdl_trigger();
    pdl_wait();   // the window's partial field spectra
    const int L = cfg.L, l = cfg.l, C = L / l, n = C * C, ll = l * l, N = L * L, R = cfg.R;
    const int r = blockIdx.x, tid = threadIdx.x;
    uint2 key;
    uint32_t t, rid;
    if (!stream_state(cfg, b, r, key, t, rid)) return;  // whole block, before any barrier
    extern __shared__ float2 sm_f2[];
    float2 *tw = sm_f2;                                          // [C]
    float2 *H = tw + kSpecMaxC;                                  // [3][n] field spectra
    float2 *U = H + 3 * n;                                       // [3][n]
    float2 *dS = U + 3 * n;                                      // [wmax][3][n] changes of S in the window
    float *hs = reinterpret_cast<float *>(dS + (size_t)cfg.wmax * 3 * n);   // [3][n] field at the sites
    float *sn = hs + 3 * n;                                      // [3][n] spins after the update
    __shared__ int s_acc, s_off[kSpecWinMax];
    if (tid == 0) s_acc = 0;
    if (tid < cfg.wlen) s_off[tid] = b.off[(size_t)r * ll + cfg.k + tid];
    for (int m = tid; m < C; m += blockDim.x) tw[m] = omega(m, C);
    float *s = b.spins + (size_t)r * 3 * N;
    const RepParams P = b.params[r];
    const float W0xx = __ldg(b.W32), W0xy = __ldg(b.W32 + N), W0yy = __ldg(b.W32 + 2 * N), W0zz = __ldg(b.W32 + 3 * N);
    const int nchunks = cfg.esplit;
    const size_t zstride = (size_t)R * cfg.wmax * 3 * n;
    __syncthreads();

    // ---- a sub-step's loads and field-free work, issued one sub-step ahead (during the
    // previous sub-step's forward DFT, after its spins are written).  First: the thread's
    // first spectral output i0 -- up to 16 chunks of its window-start spectra, the table
    // entries of the window's earlier offsets and S_o(before) for its change (MAXT = 256:
    // registers for all of them).
    constexpr int kHC = MAXT <= 256 ? 16 : 1;
    constexpr int kHV = MAXT <= 256 ? kSpecWinMax : 1;
    const int i0 = tid;
    const bool first = MAXT <= 256 && i0 < 3 * n;
    const int a0 = first ? qdiv(i0, cfg.mn) : 0, K0 = first ? i0 - a0 * n : 0;
    bool cj0 = false;
    const int src0 = first ? a0 * n + half_source(K0, C, cj0) : 0;
    float2 hv[kHC], tv0[kHV], tv1[kHV], sold = make_float2(0.f, 0.f);
    auto issue_loads = [&](int w) {
        if (!first) return;
        const int ov = s_off[w], ox = ov & 0xFFFF, oy = ov >> 16;
        const float2 *hp0 = b.Hw + (((size_t)r * cfg.wmax + w) * 3) * n + src0;
#pragma unroll
        for (int j = 0; j < kHC; ++j) hv[j] = j < nchunks ? hp0[(size_t)j * zstride] : make_float2(0.f, 0.f);
#pragma unroll
        for (int v = 0; v < kHV; ++v) {
            tv0[v] = tv1[v] = make_float2(0.f, 0.f);
            if (v < w) {
                const int pv = s_off[v];
                int dx = ox - (pv & 0xFFFF), dy = oy - (pv >> 16);
                const int sx = dx < 0, sy = dy < 0;
                dx += sx ? l : 0;
                dy += sy ? l : 0;
                const float2 *Tp = b.T + ((size_t)((sx + 2 * sy) * ll + dy * l + dx) * 4) * n + K0;
                tv0[v] = __ldg(Tp + (a0 == 2 ? 3 : a0) * n);
                if (a0 < 2) tv1[v] = __ldg(Tp + (a0 + 1) * n);
            }
        }
        // S_o(before); an offset drawn twice in a row is re-read after its first update
        if (w == 0 || s_off[w - 1] != ov) sold = b.S[((size_t)r * ll + (oy * l + ox)) * 3 * n + i0];
    };
    // Thread d < n (blockDim >= n) owns site d: its spins, neighbours, proposal and the
    // field-free part of dE.
    const int d = tid;
    const bool site = d < n;
    int q = 0;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, S0 = 0.f, S1 = 0.f, S2 = 0.f, pre = 0.f, thr = 0.f, uacc = 0.f;
    float nb[3][4];   // neighbour spins (+x, -x, +y, -y) per component
    // the site's spin and neighbours: loads only, consumed by prep() a phase later
    auto prep_load = [&](int w) {
        if (!site) return;
        const int ov = s_off[w], ox = ov & 0xFFFF, oy = ov >> 16;
        const int dy_ = qdiv(d, cfg.mC);
        const int qx = ox + l * (d - dy_ * C), qy = oy + l * dy_;
        q = qy * L + qx;
        s0 = s[q];
        s1 = s[N + q];
        s2 = s[2 * N + q];
        const int xp = (qx + 1 == L) ? q - qx : q + 1;
        const int xm = (qx == 0) ? q + L - 1 : q - 1;
        const int yp = (qy + 1 == L) ? qx : q + L;
        const int ym = (qy == 0) ? q + N - L : q - L;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            nb[c][0] = s[c * N + xp];
            nb[c][1] = s[c * N + xm];
            nb[c][2] = s[c * N + yp];
            nb[c][3] = s[c * N + ym];
        }
    };
    auto prep = [&](int w) {
        if (!site) return;
        const int k = cfg.k + w;
        const uint4 wds = philox(make_uint4((uint32_t)q, rid, t, ((uint32_t)k & 0x00FFFFFFu) | kTagAttempt), key);
        const float u1 = u24f(wds.x);
        uacc = u24f(wds.z);
        float sps, cps;
        sincospif(2.0f * u24f(wds.y), &sps, &cps);
        const float n0 = (nb[0][0] + nb[0][1]) + (nb[0][2] + nb[0][3]);
        const float n1 = (nb[1][0] + nb[1][1]) + (nb[1][2] + nb[1][3]);
        const float n2 = (nb[2][0] + nb[2][1]) + (nb[2][2] + nb[2][3]);
        {
            const float3 Sv = propose_spin(cfg.proposal, cfg.cap_c1, s0, s1, s2, u1, cps, sps);   // Sec. 3.1 proposal
            S0 = Sv.x;
            S1 = Sv.y;
            S2 = Sv.z;
        }
        const float dX = S0 - s0, dY = S1 - s1, dZ = S2 - s2;
        const float dex = -P.J * (dX * n0 + dY * n1 + dZ * n2);
        const float z0 = s2 * s2, z1 = S2 * S2;
        const float dan = (-P.K2 * z1 - P.K4 * z1 * z1) - (-P.K2 * z0 - P.K4 * z0 * z0);
        const float self = W0xx * dX * dX + 2.0f * W0xy * dX * dY + W0yy * dY * dY + W0zz * dZ * dZ;
        pre = dex + dan + P.CD * 0.5f * self;
        thr = (uacc > 0.0f) ? -P.T * logf(uacc) : INFINITY;
    };
    if (cfg.wlen > 0) {
        issue_loads(0);
        prep_load(0);
    }
    for (int w = 0; w < cfg.wlen; ++w) {
        const int k = cfg.k + w;
        prep(w);
        const int ov = s_off[w];
        const int ox = ov & 0xFFFF, oy = ov >> 16;
        float2 *So = b.S + ((size_t)r * ll + (oy * l + ox)) * 3 * n;
        const float2 *hp0 = b.Hw + (((size_t)r * cfg.wmax + w) * 3) * n + src0;
        const bool sold_ok = w == 0 || s_off[w - 1] != ov;
        // ---- field spectra: the chunk sum in chunk order, then the window's earlier changes
        if (first) {
            float2 acc = hv[0];
#pragma unroll
            for (int j = 1; j < kHC; ++j)
                if (j < nchunks) {
                    acc.x += hv[j].x;
                    acc.y += hv[j].y;
                }
            for (int z0 = kHC; z0 < nchunks; ++z0) {
                const float2 v = hp0[(size_t)z0 * zstride];
                acc.x += v.x;
                acc.y += v.y;
            }
            if (cj0) acc.y = -acc.y;
#pragma unroll
            for (int v = 0; v < kHV; ++v)
                if (v < w) {
                    const float2 *dv = dS + (size_t)v * 3 * n + K0;
                    if (a0 == 2) acc = cfma(tv0[v], dv[2 * n], acc);
                    else acc = cfma(tv0[v], dv[0], cfma(tv1[v], dv[n], acc));
                }
            H[i0] = acc;
        }
        for (int i = tid + (first ? blockDim.x : 0); i < 3 * n; i += blockDim.x) {
            const int a = qdiv(i, cfg.mn), K = i - a * n;
            bool cj = false;
            const float2 *hp = b.Hw + (((size_t)r * cfg.wmax + w) * 3) * n + a * n + half_source(K, C, cj);
            float2 acc = hp[0];
            for (int z0 = 1; z0 < nchunks; z0 += 8) {
                float2 v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = z0 + j < nchunks ? hp[(size_t)(z0 + j) * zstride] : make_float2(0.f, 0.f);
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (z0 + j < nchunks) {
                        acc.x += v[j].x;
                        acc.y += v[j].y;
                    }
            }
            if (cj) acc.y = -acc.y;
            if (w > 0) {
                for (int v = 0; v < w; ++v) {
                    const int pv = s_off[v];
                    int dx = ox - (pv & 0xFFFF), dy = oy - (pv >> 16);
                    const int sx = dx < 0, sy = dy < 0;
                    dx += sx ? l : 0;
                    dy += sy ? l : 0;
                    const float2 *Tp = b.T + ((size_t)((sx + 2 * sy) * ll + dy * l + dx) * 4) * n + K;
                    const float2 *dv = dS + (size_t)v * 3 * n + K;
                    if (a == 2) {
                        acc = cfma(__ldg(Tp + 3 * n), dv[2 * n], acc);
                    } else {
                        acc = cfma(__ldg(Tp + a * n), dv[0], cfma(__ldg(Tp + (a + 1) * n), dv[n], acc));
                    }
                }
            }
            H[i] = acc;
        }
        __syncthreads();
        // inverse DFT: over Kx, then over Ky (conjugate twiddles), real part / n
        for (int i = tid; i < 3 * n; i += blockDim.x) {
            const int a = qdiv(i, cfg.mn), jj = i - a * n, Ky = qdiv(jj, cfg.mC), Dx = jj - Ky * C;
            const float2 *row = H + a * n + Ky * C;
            float2 acc = make_float2(0.f, 0.f);
            for (int Kx = 0, m = 0; Kx < C; ++Kx) {       // m = Kx * Dx mod C
                const float2 o = tw[m];
                acc = cfma(row[Kx], make_float2(o.x, -o.y), acc);
                m += Dx;
                if (m >= C) m -= C;
            }
            U[i] = acc;
        }
        __syncthreads();
        const float inv_n = 1.0f / (float)n;
        for (int i = tid; i < 3 * n; i += blockDim.x) {
            const int a = qdiv(i, cfg.mn), jj = i - a * n, Dy = qdiv(jj, cfg.mC), Dx = jj - Dy * C;
            const float2 *col = U + a * n + Dx;
            float re = 0.f;
            for (int Ky = 0, m = 0; Ky < C; ++Ky) {       // m = Ky * Dy mod C
                const float2 u = col[Ky * C], o = tw[m];
                re = fmaf(u.x, o.x, fmaf(u.y, o.y, re));   // Re(u * conj(o))
                m += Dy;
                if (m >= C) m -= C;
            }
            hs[i] = re * inv_n;
        }
        __syncthreads();
        // ---- decisions (sites are numbered as in the other paths: d -> (d % C, d / C))
        int accept = 0;
        if (site) {
            const float dX = S0 - s0, dY = S1 - s1, dZ = S2 - s2;
            const float h0 = hs[d], h1 = hs[n + d], h2 = hs[2 * n + d];
            const float dE = pre + P.CD * (dX * h0 + dY * h1 + dZ * h2);
            accept = dE < thr;
            if (b.trace) {
                float *tr = b.trace + ((((size_t)r * cfg.nsweeps_call + cfg.it) * ll + k) * n + d) * MC_TRACE_W;
                tr[0] = (float)q;
                tr[1] = h0; tr[2] = h1; tr[3] = h2;
                tr[4] = dE;
                tr[5] = uacc;
                tr[6] = (float)accept;
                tr[7] = S0; tr[8] = S1; tr[9] = S2;
            }
            sn[d] = accept ? S0 : s0;
            sn[n + d] = accept ? S1 : s1;
            sn[2 * n + d] = accept ? S2 : s2;
            if (accept) {
                s[q] = S0;
                s[N + q] = S1;
                s[2 * N + q] = S2;
            }
        }
        const unsigned ball = __ballot_sync(0xffffffffu, accept);
        if ((tid & 31) == 0 && ball) atomicAdd(&s_acc, __popc(ball));
        __syncthreads();
        // ---- the next sub-step's loads and field-free work (its sites' spins and the
        // neighbours this sub-step may have changed are in global memory by now)
        const float2 sold_w = sold;
        if (w + 1 < cfg.wlen) {
            issue_loads(w + 1);
            prep_load(w + 1);
        }
        // ---- new S of the updated offset and its change
        for (int i = tid; i < 3 * n; i += blockDim.x) {
            const int bb = qdiv(i, cfg.mn), j = i - bb * n, Dy = qdiv(j, cfg.mC), Kx = j - Dy * C;
            const float *row = sn + bb * n + Dy * C;
            float2 acc = make_float2(0.f, 0.f);
            for (int Dx = 0, m = 0; Dx < C; ++Dx) {       // m = Kx * Dx mod C
                const float2 o = tw[m];
                acc.x = fmaf(row[Dx], o.x, acc.x);
                acc.y = fmaf(row[Dx], o.y, acc.y);
                m += Kx;
                if (m >= C) m -= C;
            }
            U[i] = acc;
        }
        __syncthreads();
        for (int i = tid; i < 3 * n; i += blockDim.x) {
            const int bb = qdiv(i, cfg.mn), j = i - bb * n, Ky = qdiv(j, cfg.mC), Kx = j - Ky * C;
            const float2 *col = U + bb * n + Kx;
            float2 acc = make_float2(0.f, 0.f);
            for (int Dy = 0, m = 0; Dy < C; ++Dy) {       // m = Ky * Dy mod C
                acc = cfma(col[Dy * C], tw[m], acc);
                m += Ky;
                if (m >= C) m -= C;
            }
            const float2 old = (first && i == i0 && sold_ok) ? sold_w : So[i];
            So[i] = acc;
            dS[(size_t)w * 3 * n + i] = make_float2(acc.x - old.x, acc.y - old.y);
        }
        __syncthreads();
    }
    if (tid == 0 && s_acc && b.obs)
        atomicAdd((unsigned long long *)&b.obs[r].accepted, (unsigned long long)s_acc);
}

template <int MAXT>
cudaError_t launch_wupdate(const SpecConfig &c, const SpecBuffers &b, size_t smem, int th, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k_spec_wupdate<MAXT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return launch_pdl(k_spec_wupdate<MAXT>, dim3(c.R), th, smem, st, c, b);
}

size_t wupdate_smem(int C, int wmax) {
    const size_t n = (size_t)C * C;
    return sizeof(float2) * (kSpecMaxC + (6 + 3 * (size_t)wmax) * n) + sizeof(float) * 6 * n;
}

size_t init_smem(int C) {
    const size_t n = (size_t)C * C;
    return sizeof(float2) * (kSpecMaxC + 3 * n) + sizeof(float) * 3 * n;
}

}  // namespace

bool spectral_supported(int L, int l) {
    if (l < 2 || L % l) return false;
    const int C = L / l;
    return C >= 2 && C <= kSpecMaxC && L <= 4096;
}

int spectral_window(int L, int l) {
    // the window's changes dS ([wmax][3][n] complex) stay in shared memory
    const long long n = (long long)(L / l) * (L / l);
    int w = kSpecWinMax;
    while (w > 1 && (long long)w * 24 * n > 96 * 1024) w >>= 1;
    return w;
}

int spectral_esplit(int L, int l, int R, int nsm) {
    // chunks of the cell offsets: about three CTAs of the window field per SM
    const long long ll = (long long)l * l;
    const long long tiles = ((half_count(L / l) + 15) / 16) * ((R + 1) / 2);
    long long z = (3LL * nsm + tiles - 1) / tiles;
    z = std::min(z, std::max(1LL, ll / 8));   // at least 8 cell offsets a chunk
    z = std::min(z, 16LL);                    // the update loads all chunks of a spectrum at once
    return (int)std::max(1LL, z);
}

size_t spectral_S_elems(int L, int R) { return (size_t)3 * L * L * R; }

size_t spectral_part_elems(int L, int l, int R, int esplit) {
    return (size_t)esplit * R * spectral_window(L, l) * 3 * (L / l) * (L / l);
}

cudaError_t launch_spec_table(int L, int l, const double *W64, float2 *T, cudaStream_t st) {
    const int C = L / l;
    const size_t smem = sizeof(double2) * ((size_t)C * C + C);
    cudaError_t e = cudaFuncSetAttribute(k_spec_table, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_spec_table<<<l * l * 4, kSpecThreads, smem, st>>>(L, l, W64, T);
    return cudaGetLastError();
}

cudaError_t launch_spec_init(int L, int l, int R, const float *spins, float2 *S, cudaStream_t st) {
    const size_t smem = init_smem(L / l);
    cudaError_t e = cudaFuncSetAttribute(k_spec_init, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_spec_init<<<dim3(l * l, R), kSpecThreads, smem, st>>>(L, l, spins, S);
    return cudaGetLastError();
}

cudaError_t launch_spec_offsets(const SpecConfig &c, const SpecBuffers &b, cudaStream_t st) {
    const long long tot = (long long)c.R * c.l * c.l;
    k_spec_offsets<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(c, b);
    return cudaGetLastError();
}

cudaError_t launch_spec_wfield(const SpecConfig &c, const SpecBuffers &b, cudaStream_t st) {
    const int C = c.L / c.l;
    return launch_pdl(k_spec_wfield, dim3((half_count(C) + 15) / 16, (c.R + 1) / 2, c.esplit), kSpecThreads, 0, st, c,
                      b);
}

cudaError_t launch_spec_wupdate(const SpecConfig &c, const SpecBuffers &b, cudaStream_t st) {
    const size_t smem = wupdate_smem(c.L / c.l, c.wmax);
    // one thread per output of a DFT stage (3 n), so that no warp idles at the
    // stage barriers; up to 256 threads the kernel holds a sub-step's loads in registers
    const int C = c.L / c.l, th = std::max(64, std::min(kUpdMaxThreads, ((3 * C * C + 31) / 32) * 32));
    return th <= 256 ? launch_wupdate<256>(c, b, smem, th, st) : launch_wupdate<kUpdMaxThreads>(c, b, smem, th, st);
}

}  // namespace dipmc
