// fft_field.cu -- the full dipole field h = W~ * s of every replica by 2D FFT
// convolution (Sec. 2.1, Eq. 2 as a circular convolution over the periodic cell),
// and the FFT sweep path: per sub-step the full field, then the simultaneous
// update of the sub-step's n sites (Sec. 3.1, 3.2).
//
// The tensor W~ is even, so its transform is real: W^_ab(k) (xx, xy, yy, zz).
// Per replica two complex transforms carry the three real spin planes:
//     C = FFT(s_x + i s_y),  Z = FFT(s_z),
// S_x(k) = (C(k) + conj C(-k))/2, S_y(k) = (C(k) - conj C(-k))/(2i),
// H_x + i H_y = (W^xx S_x + W^xy S_y) + i (W^xy S_x + W^yy S_y),  H_z = W^zz Z,
// and two inverse transforms give h_x + i h_y and h_z.
//
// A 2D transform is a row pass (radix-2 Stockham in shared memory), a tiled
// transpose and a second row pass; spectra stay in the transposed layout
// [k_x][k_y] (W^ is stored the same way), so the inverse is row pass,
// transpose, row pass back to [y][x].  L must be a power of two, 8 <= L <= 1024.
#include <cuda_bf16.h>

#include "fft_field.cuh"
#include "internal.cuh"

namespace dipmc {

namespace {

constexpr float kPiF = 3.14159265358979f;

// Radix-2 Stockham auto-sort FFT of nrows rows of length L (in place in global
// memory through shared memory).  Stage with half-span Ns: output
// y[(t/Ns)*2Ns + t%Ns] = a + w b, y[... + Ns] = a - w b with a = x[t],
// b = x[t + L/2], w = exp(-+ 2 pi i (t%Ns) / (2 Ns)) = tw[(t%Ns) * L/(2Ns)],
// tw[m] = exp(-+ 2 pi i m / L) tabulated once per CTA (the same sincospif values
// as per-butterfly evaluation: the fractions k/Ns and 2m/L are equal and exact).
template <bool INV>
__global__ void k_fft_rows(float2 *data, int L, int logL, long long nrows) {
    extern __shared__ float2 fbuf[];
    const int half = L >> 1;
    const int rpc = blockDim.x / half;                  // rows per CTA
    const int rr = threadIdx.x / half, t = threadIdx.x % half;
    const long long row = (long long)blockIdx.x * rpc + rr;
    if (rpc == 0) return;
    float2 *tw = fbuf + (size_t)rpc * 2 * L;             // [L/2]
    for (int m = threadIdx.x; m < half; m += blockDim.x) {
        float sw, cw;
        sincospif((INV ? 1.0f : -1.0f) * (float)(2 * m) / (float)L, &sw, &cw);
        tw[m] = make_float2(cw, sw);
    }
    float2 *x = fbuf + (size_t)rr * 2 * L, *y = x + L;
    const bool valid = row < nrows;
    float2 *g = data + (valid ? row : 0) * L;
    if (valid) {
        x[t] = g[t];
        x[t + half] = g[t + half];
    }
    __syncthreads();
    for (int s = 0; s < logL; ++s) {
        const int Ns = 1 << s;
        const int k = t & (Ns - 1);
        const float2 wv = tw[k << (logL - 1 - s)];
        const float sw = wv.y, cw = wv.x;
        const float2 a = x[t], b0 = x[t + half];
        const float2 b = make_float2(b0.x * cw - b0.y * sw, b0.x * sw + b0.y * cw);
        const int j = ((t >> s) << (s + 1)) + k;
        y[j] = make_float2(a.x + b.x, a.y + b.y);
        y[j + Ns] = make_float2(a.x - b.x, a.y - b.y);
        __syncthreads();
        float2 *tmp = x;
        x = y;
        y = tmp;
    }
    if (valid) {
        g[t] = x[t];
        g[t + half] = x[t + half];
    }
}

// out[b][c][r] = in[b][r][c] for L x L matrices (32 x 32 tiles).
__global__ void k_transpose(const float2 *__restrict__ in, float2 *__restrict__ out, int L) {
    __shared__ float2 tile[32][33];
    const size_t base = (size_t)blockIdx.z * L * L;
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = by + i, c = bx + threadIdx.x;
        if (r < L && c < L) tile[i][threadIdx.x] = in[base + (size_t)r * L + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = bx + i, c = by + threadIdx.x;
        if (r < L && c < L) out[base + (size_t)r * L + c] = tile[threadIdx.x][i];
    }
}

__global__ void k_pack(const float *__restrict__ spins, int N, int R, float2 *C, float2 *Z) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)N * R) return;
    const size_t r = i / N, p = i % N;
    const float *s = spins + r * 3 * N;
    C[i] = make_float2(s[p], s[N + p]);
    Z[i] = make_float2(s[2 * N + p], 0.0f);
}

// Spectral product in the transposed layout i = kx*L + ky.
__global__ void k_spectral(const float2 *__restrict__ C, float2 *__restrict__ Hxy, float2 *Z,
                           const float *__restrict__ What, int L, int R) {
    const int N = L * L;
    const size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (size_t)N * R) return;
    const size_t r = g / N;
    const int i = (int)(g % N);
    const int kx = i / L, ky = i % L;
    const int ni = ((L - kx) & (L - 1)) * L + ((L - ky) & (L - 1));
    const float2 c = C[r * N + i], cm = C[r * N + ni];
    // S_x = (c + conj cm)/2, S_y = (c - conj cm)/(2i)
    const float2 sx = make_float2(0.5f * (c.x + cm.x), 0.5f * (c.y - cm.y));
    const float2 sy = make_float2(0.5f * (c.y + cm.y), -0.5f * (c.x - cm.x));
    const float wxx = What[i], wxy = What[N + i], wyy = What[2 * N + i], wzz = What[3 * N + i];
    const float2 hx = make_float2(wxx * sx.x + wxy * sy.x, wxx * sx.y + wxy * sy.y);
    const float2 hy = make_float2(wxy * sx.x + wyy * sy.x, wxy * sx.y + wyy * sy.y);
    Hxy[r * N + i] = make_float2(hx.x - hy.y, hx.y + hy.x);      // H_x + i H_y
    const float2 z = Z[r * N + i];
    Z[r * N + i] = make_float2(wzz * z.x, wzz * z.y);
}

__global__ void k_unpack(const float2 *__restrict__ Hxy, const float2 *__restrict__ Hz, int N, int R, float scale,
                         float *field) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)N * R) return;
    const size_t r = i / N, p = i % N;
    float *f = field + r * 3 * N;
    const float2 a = Hxy[i];
    f[p] = a.x * scale;
    f[N + p] = a.y * scale;
    f[2 * N + p] = Hz[i].x * scale;
}

// W^(kx, ky) = sum_{x,y} W~(x, y) exp(-2 pi i (kx x + ky y)/L), real for the even
// tensor, in FP64 by two separable DFT passes with a twiddle table
// tw[j] = exp(-2 pi i j / L) in shared memory.  Pass 1: T[c][y][kx] (complex).
__global__ void k_what_pass1(const double *__restrict__ W64, int L, double2 *T) {
    extern __shared__ double2 tw[];
    for (int j = threadIdx.x; j < L; j += blockDim.x) {
        double sn, cs;
        sincospi(-2.0 * (double)j / (double)L, &sn, &cs);
        tw[j] = make_double2(cs, sn);
    }
    __syncthreads();
    const int N = L * L;
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= 4LL * N) return;
    const int c = (int)(g / N), i = (int)(g % N);
    const int y = i / L, kx = i % L;
    double re = 0.0, im = 0.0;
    int ph = 0;                                   // kx * x mod L
    for (int x = 0; x < L; ++x) {
        const double w = W64[(size_t)c * N + (size_t)y * L + x];
        re += w * tw[ph].x;
        im += w * tw[ph].y;
        ph += kx;
        if (ph >= L) ph -= L;
    }
    T[g] = make_double2(re, im);
}

// Pass 2: What[c][kx][ky] = Re sum_y T[c][y][kx] exp(-2 pi i ky y / L).
__global__ void k_what_pass2(const double2 *__restrict__ T, int L, float *What) {
    extern __shared__ double2 tw[];
    for (int j = threadIdx.x; j < L; j += blockDim.x) {
        double sn, cs;
        sincospi(-2.0 * (double)j / (double)L, &sn, &cs);
        tw[j] = make_double2(cs, sn);
    }
    __syncthreads();
    const int N = L * L;
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= 4LL * N) return;
    const int c = (int)(g / N), i = (int)(g % N);
    const int kx = i / L, ky = i % L;
    double re = 0.0;
    int ph = 0;                                   // ky * y mod L
    for (int y = 0; y < L; ++y) {
        const double2 v = T[(size_t)c * N + (size_t)y * L + kx];
        re += v.x * tw[ph].x - v.y * tw[ph].y;
        ph += ky;
        if (ph >= L) ph -= L;
    }
    What[(size_t)c * N + i] = (float)re;
}

// ---------------------------------------------------------------------------
// FFT sweep: the update of one sub-step at all n sites of all replicas, from the
// full field of the state before the sub-step (in place: update sites are never
// nearest neighbours for l >= 2).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void perp_basis_f(float nx, float ny, float nz, float3 &b1, float3 &b2) {
    const float sign = copysignf(1.0f, nz);
    const float a = -1.0f / (sign + nz);
    const float b = nx * ny * a;
    b1 = make_float3(1.0f + sign * nx * nx * a, sign * b, -sign * nx);
    b2 = make_float3(b, sign + ny * ny * a, -ny);
}

__global__ void k_fft_update(const FftStepConfig cfg, const FftStepBuffers buf) {
    const int L = cfg.L, l = cfg.l, N = L * L, C = L / l, n = C * C, ll = l * l;
    const int r = blockIdx.y;
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    uint2 key = cfg.key;
    uint32_t t = cfg.t_dev ? *cfg.t_dev + (uint32_t)cfg.it : cfg.t, rid = (uint32_t)r;
    if (buf.slots) {
        const SlotState sl = buf.slots[r];
        if (cfg.it >= sl.nsweeps) return;   // idle or finished slot: whole block, before any barrier
        key = make_uint2(sl.key_lo, sl.key_hi);
        t = sl.t0 + (uint32_t)cfg.it;
        rid = sl.rid;
    }
    __shared__ int s_acc;
    if (threadIdx.x == 0) s_acc = 0;
    __syncthreads();
    int accept = 0;
    if (d < n) {
        const uint32_t k = (uint32_t)cfg.k;
        uint32_t v;
        if (cfg.schedule == 0) {
            const uint4 rk = philox(make_uint4(t, 0u, 0u, kTagPerm), key);
            v = perm_offset(rk, ceil_log2_u((uint32_t)l), (uint32_t)ll, k);
        } else {
            const uint4 o = philox(make_uint4(t, k, 0u, kTagDraw), key);
            v = (uint32_t)(((unsigned long long)o.x * (unsigned long long)ll) >> 32);
        }
        const int qx = (int)(v % l) + l * (d % C), qy = (int)(v / l) + l * (d / C);
        const int q = qy * L + qx;
        const RepParams P = buf.params[r];
        float *s = buf.spins + (size_t)r * 3 * N;
        const float *h = buf.field + (size_t)r * 3 * N;
        const uint4 wds = philox(make_uint4((uint32_t)q, rid, t, (k & 0x00FFFFFFu) | kTagAttempt), key);
        const float u1 = u24f(wds.x), uacc = u24f(wds.z);
        float sps, cps;
        sincospif(2.0f * u24f(wds.y), &sps, &cps);
        const float s0 = s[q], s1 = s[N + q], s2 = s[2 * N + q];
        float S0, S1, S2;
        if (cfg.proposal == kPropFlip) {            // Appendix B reversal
            S0 = -s0;
            S1 = -s1;
            S2 = -s2;
        } else if (cfg.proposal == kPropSphere) {
            const float z = 2.0f * u1 - 1.0f;
            const float rr = sqrtf(fmaxf(0.0f, (1.0f - z) * (1.0f + z)));
            S0 = rr * cps;
            S1 = rr * sps;
            S2 = z;
        } else {
            const float omc = u1 * cfg.cap_c1;             // 1 - cos(alpha), no cancellation
            const float ca = 1.0f - omc;
            const float sa = sqrtf(fmaxf(0.0f, omc * (2.0f - omc)));
            float3 b1, b2;
            perp_basis_f(s0, s1, s2, b1, b2);
            S0 = ca * s0 + sa * (cps * b1.x + sps * b2.x);
            S1 = ca * s1 + sa * (cps * b1.y + sps * b2.y);
            S2 = ca * s2 + sa * (cps * b1.z + sps * b2.z);
            const float inv = 1.0f / sqrtf(S0 * S0 + S1 * S1 + S2 * S2);
            S0 *= inv;
            S1 *= inv;
            S2 *= inv;
        }
        const float dX = S0 - s0, dY = S1 - s1, dZ = S2 - s2;
        const int xp = (qx + 1 == L) ? q - qx : q + 1;
        const int xm = (qx == 0) ? q + L - 1 : q - 1;
        const int yp = (qy + 1 == L) ? qx : q + L;
        const int ym = (qy == 0) ? q + N - L : q - L;
        const float n0 = (s[xp] + s[xm]) + (s[yp] + s[ym]);
        const float n1 = (s[N + xp] + s[N + xm]) + (s[N + yp] + s[N + ym]);
        const float n2 = (s[2 * N + xp] + s[2 * N + xm]) + (s[2 * N + yp] + s[2 * N + ym]);
        const float dex = -P.J * (dX * n0 + dY * n1 + dZ * n2);
        const float z0 = s2 * s2, z1 = S2 * S2;
        const float dan = (-P.K2 * z1 - P.K4 * z1 * z1) - (-P.K2 * z0 - P.K4 * z0 * z0);
        const float W0xx = __ldg(buf.W32), W0xy = __ldg(buf.W32 + N), W0yy = __ldg(buf.W32 + 2 * N), W0zz = __ldg(buf.W32 + 3 * N);
        const float self = W0xx * dX * dX + 2.0f * W0xy * dX * dY + W0yy * dY * dY + W0zz * dZ * dZ;
        const float h0 = h[q], h1 = h[N + q], h2 = h[2 * N + q];
        const float dE = dex + dan + P.CD * ((dX * h0 + dY * h1 + dZ * h2) + 0.5f * self);
        const float thr = (uacc > 0.0f) ? -P.T * logf(uacc) : INFINITY;
        accept = dE < thr;
        if (buf.trace) {
            float *tr = buf.trace + ((((size_t)r * cfg.nsweeps_call + cfg.it) * ll + cfg.k) * n + d) * MC_TRACE_W;
            tr[0] = (float)q;
            tr[1] = h0; tr[2] = h1; tr[3] = h2;
            tr[4] = dE;
            tr[5] = uacc;
            tr[6] = (float)accept;
            tr[7] = S0; tr[8] = S1; tr[9] = S2;
        }
        if (accept) {
            s[q] = S0;
            s[N + q] = S1;
            s[2 * N + q] = S2;
        }
    }
    const unsigned ball = __ballot_sync(0xffffffffu, accept);
    if ((threadIdx.x & 31) == 0 && ball) atomicAdd(&s_acc, __popc(ball));
    __syncthreads();
    if (threadIdx.x == 0 && s_acc && buf.obs) atomicAdd((unsigned long long *)&buf.obs[r].accepted, (unsigned long long)s_acc);
}

// Observables of the current state from the full field of the same state: M,
// per-site (theta - pi/2)^2, total energy (stored as the replica's energy), and
// the log-binning push (thread k < kNB updates level k).
__global__ void __launch_bounds__(256) k_fft_observe(int L, const float *__restrict__ spins,
                                                     const float *__restrict__ field, const RepParams *__restrict__ P,
                                                     double *energy, ObsAcc *obs, double *theta2,
                                                     const SlotState *slots, int it, int measure_every,
                                                     const EnergyHist hist) {
    const int N = L * L, r = blockIdx.x, tid = threadIdx.x;
    if (slots) {
        const SlotState sl = slots[r];
        if (it >= sl.nsweeps || measure_every <= 0 || (sl.t0 + (uint32_t)it + 1u) % (uint32_t)measure_every) return;
    }
    const float *s = spins + (size_t)r * 3 * N;
    const float *f = field + (size_t)r * 3 * N;
    const RepParams p = P[r];
    double mx = 0, my = 0, mz = 0, ex = 0, an = 0, dp = 0, mh = 0, mv = 0;
    double wc[7] = {0, 0, 0, 0, 0, 0, 0};   // n_h^x, n_v^x, n_h^y, n_v^y, n_h^z, n_v^z, sum |theta - pi/2|
    for (int i = tid; i < N; i += blockDim.x) {
        const int x = i % L, y = i / L;
        const int ixp = y * L + (x + 1 == L ? 0 : x + 1);
        const int iyp = (y + 1 == L ? 0 : y + 1) * L + x;
        const double a = s[i], b = s[N + i], c = s[2 * N + i];
        mx += a;
        my += b;
        mz += c;
        mh += (y & 1) ? -c : c;     // m1 + m2 - m3 - m4 (rows)
        mv += (x & 1) ? -c : c;     // m1 + m4 - m3 - m2 (columns)
        wc[0] += wall_term(s[i], s[ixp]);
        wc[1] += wall_term(s[i], s[iyp]);
        wc[2] += wall_term(s[N + i], s[N + ixp]);
        wc[3] += wall_term(s[N + i], s[N + iyp]);
        wc[4] += wall_term(s[2 * N + i], s[2 * N + ixp]);
        wc[5] += wall_term(s[2 * N + i], s[2 * N + iyp]);
        wc[6] += fabsf(acosf(fminf(1.0f, fmaxf(-1.0f, (float)c))) - 0.5f * kPiF);
        ex += a * ((double)s[ixp] + (double)s[iyp]) + b * ((double)s[N + ixp] + (double)s[N + iyp]) +
              c * ((double)s[2 * N + ixp] + (double)s[2 * N + iyp]);
        const double z2 = c * c;
        an += -(double)p.K2 * z2 - (double)p.K4 * z2 * z2;
        dp += a * (double)f[i] + b * (double)f[N + i] + c * (double)f[2 * N + i];
        if (theta2) {
            const float th = acosf(fminf(1.0f, fmaxf(-1.0f, (float)c))) - 0.5f * kPiF;
            theta2[(size_t)r * N + i] += (double)(th * th);
        }
    }
    __shared__ double red[15][8];
    double v[15] = {mx, my, mz, ex, an, dp, mh, mv, wc[0], wc[1], wc[2], wc[3], wc[4], wc[5], wc[6]};
    for (int k = 0; k < 15; ++k)
        for (int off = 16; off; off >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
    if ((tid & 31) == 0)
        for (int k = 0; k < 15; ++k) red[k][tid >> 5] = v[k];
    __syncthreads();
    __shared__ double x_s[MC_NOBS];
    if (tid == 0) {
        double t[15] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            for (int k = 0; k < 15; ++k) t[k] += red[k][w];
        const double Mx = t[0] / N, My = t[1] / N, Mz = t[2] / N;
        const double E = -(double)p.J * t[3] + t[4] + 0.5 * (double)p.CD * t[5];
        energy[r] = E;
        x_s[MC_OBS_ABS_M] = sqrt(Mx * Mx + My * My + Mz * Mz);
        x_s[MC_OBS_MZ] = Mz;
        x_s[MC_OBS_ABS_MZ] = fabs(Mz);
        x_s[MC_OBS_MPAR] = sqrt(Mx * Mx + My * My);
        x_s[MC_OBS_E] = E / N;
        x_s[MC_OBS_MST] = sqrt(t[6] * t[6] + t[7] * t[7]) / N;
        const double nh[3] = {t[8], t[10], t[12]}, nv[3] = {t[9], t[11], t[13]};
        stripe_obs(x_s, nh, nv, t[14], N);
        hist_push(hist, r, E / N);
    }
    __syncthreads();
    if (obs && tid < kNB) {
        ObsAcc &A = obs[r];
        const int k = tid;
        const long long pc = A.pcnt[k] + 1;
        const bool done = pc == (1LL << k);
        const double inv = 1.0 / (double)(1LL << k);
        for (int o = 0; o < MC_NOBS; ++o) {
            const double pv = A.psum[o][k] + x_s[o];
            if (done) {
                const double mean = pv * inv;
                A.bsum[o][k] += mean;
                A.bsq[o][k] += mean * mean;
                A.psum[o][k] = 0.0;
            } else {
                A.psum[o][k] = pv;
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
}

__global__ void k_add_attempted(ObsAcc *obs, int R, long long add, const SlotState *slots, int nsweeps_call,
                                long long N) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    if (slots) add = (long long)min(nsweeps_call, (int)slots[r].nsweeps) * N;
    obs[r].attempted += add;
}

int ilog2(int v) {
    int b = 0;
    while ((1 << b) < v) ++b;
    return b;
}

cudaError_t rows(float2 *data, int L, long long nrows, bool inv, cudaStream_t st) {
    const int half = L / 2;
    const int threads = half >= 256 ? half : 256;
    const int rpc = threads / half;
    const unsigned blocks = (unsigned)((nrows + rpc - 1) / rpc);
    const size_t smem = sizeof(float2) * (2 * L * rpc + half);
    if (inv) {
        cudaFuncSetAttribute(k_fft_rows<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_fft_rows<true><<<blocks, threads, smem, st>>>(data, L, ilog2(L), nrows);
    } else {
        cudaFuncSetAttribute(k_fft_rows<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_fft_rows<false><<<blocks, threads, smem, st>>>(data, L, ilog2(L), nrows);
    }
    return cudaGetLastError();
}

cudaError_t transpose(const float2 *in, float2 *out, int L, int R, cudaStream_t st) {
    dim3 grid((L + 31) / 32, (L + 31) / 32, R), block(32, 8);
    k_transpose<<<grid, block, 0, st>>>(in, out, L);
    return cudaGetLastError();
}

}  // namespace

bool fft_supported(int L) { return L >= 8 && L <= 1024 && (L & (L - 1)) == 0; }

size_t fft_scratch_bytes(int L, int R) { return sizeof(float2) * (size_t)L * L * R * 3; }

cudaError_t launch_build_what(int L, const double *W64, float *What, cudaStream_t st) {
    const int N = L * L;
    double2 *T = nullptr;
    cudaError_t e = cudaMallocAsync(&T, sizeof(double2) * 4 * (size_t)N, st);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)((4LL * N + 255) / 256);
    const size_t smem = sizeof(double2) * (size_t)L;
    k_what_pass1<<<blocks, 256, smem, st>>>(W64, L, T);
    k_what_pass2<<<blocks, 256, smem, st>>>(T, L, What);
    e = cudaGetLastError();
    cudaFreeAsync(T, st);
    return e;
}

cudaError_t launch_fft_field(int L, int R, const float *spins, const float *What, float2 *scratch, float *field,
                             cudaStream_t st) {
    const int N = L * L;
    const size_t tot = (size_t)N * R;
    float2 *C = scratch, *Z = scratch + tot, *T = scratch + 2 * tot;
    const unsigned nb = (unsigned)((tot + 255) / 256);
    cudaError_t e;
    k_pack<<<nb, 256, 0, st>>>(spins, N, R, C, Z);
    // forward: rows over x, transpose to [x][y], rows over y -> spectra [kx][ky]
    if ((e = rows(C, L, (long long)L * R, false, st)) != cudaSuccess) return e;
    if ((e = rows(Z, L, (long long)L * R, false, st)) != cudaSuccess) return e;
    if ((e = transpose(C, T, L, R, st)) != cudaSuccess) return e;
    if ((e = rows(T, L, (long long)L * R, false, st)) != cudaSuccess) return e;
    if ((e = transpose(Z, C, L, R, st)) != cudaSuccess) return e;
    if ((e = rows(C, L, (long long)L * R, false, st)) != cudaSuccess) return e;
    // now T = C^ and C = Z^ (both [kx][ky]); spectral product: T -> Z (H_xy), C (H_z) in place
    k_spectral<<<nb, 256, 0, st>>>(T, Z, C, What, L, R);
    // inverse: rows over ky, transpose back to [y][kx], rows over kx
    if ((e = rows(Z, L, (long long)L * R, true, st)) != cudaSuccess) return e;
    if ((e = rows(C, L, (long long)L * R, true, st)) != cudaSuccess) return e;
    if ((e = transpose(Z, T, L, R, st)) != cudaSuccess) return e;
    if ((e = rows(T, L, (long long)L * R, true, st)) != cudaSuccess) return e;
    if ((e = transpose(C, Z, L, R, st)) != cudaSuccess) return e;
    if ((e = rows(Z, L, (long long)L * R, true, st)) != cudaSuccess) return e;
    k_unpack<<<nb, 256, 0, st>>>(T, Z, N, R, 1.0f / (float)N, field);
    return cudaGetLastError();
}

cudaError_t launch_fft_update(const FftStepConfig &c, const FftStepBuffers &b, cudaStream_t st) {
    const int n = (c.L / c.l) * (c.L / c.l);
    const int threads = n >= 256 ? 256 : ((n + 31) / 32) * 32;
    dim3 grid((n + threads - 1) / threads, c.R);
    k_fft_update<<<grid, threads, 0, st>>>(c, b);
    return cudaGetLastError();
}

cudaError_t launch_fft_observe(int L, int R, const float *spins, const float *field, const RepParams *P,
                               double *energy, ObsAcc *obs, double *theta2, const SlotState *slots, int it,
                               int measure_every, const EnergyHist &hist, cudaStream_t st) {
    k_fft_observe<<<R, 256, 0, st>>>(L, spins, field, P, energy, obs, theta2, slots, it, measure_every, hist);
    return cudaGetLastError();
}

cudaError_t launch_add_attempted(ObsAcc *obs, int R, long long add, const SlotState *slots, int nsweeps_call,
                                 long long N, cudaStream_t st) {
    k_add_attempted<<<(R + 127) / 128, 128, 0, st>>>(obs, R, add, slots, nsweeps_call, N);
    return cudaGetLastError();
}

}  // namespace dipmc
