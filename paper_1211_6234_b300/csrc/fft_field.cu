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
// One full field is three kernels, with no transposes: k_fft_fwd_rows transforms
// the rows of C and Z from the spins (over x, giving [y][kx]); k_fft_cols_conv takes
// tiles of columns kx together with their mirrors -kx (the split of C into S_x and
// S_y needs C(-k)), transforms them over y, multiplies by W^ and transforms back
// over ky, in shared memory, writing H_x + i H_y and H_z in place; k_fft_inv_rows
// transforms the rows back over kx and writes the field.  The transforms are
// Stockham passes in shared memory (radix 16, after one pass of radix 2, 4 or 8
// when log2 L is not a multiple of 4), each thread taking one DFT of the pass in
// registers, one barrier per pass.  L must be a power of two, 8 <= L <= 1024.
#include <algorithm>

#include <cuda_bf16.h>

#include "fft_field.cuh"
#include "internal.cuh"

namespace dipmc {

namespace {

constexpr float kPiF = 3.14159265358979f;

// Transforms of length L = 2^logL along rows of shared memory, by Stockham
// auto-sort passes: a first pass of radix 2^(logL mod 4) when logL is not a
// multiple of 4, then radix-16 passes.  A radix-R pass of span Ns takes, for t in
// [0, L/R) and k = t mod Ns, the inputs v_r = x[t + r L/R] w^(r k),
// w = exp(-+ 2 pi i / (R Ns)), their R-point DFT b_m (in registers), and writes
// y[(t - k) R + k + m Ns] = b_m; the span grows by R per pass.
//
// Element i of a row sits at pad16(i) = i + i/16: with one slot of padding after
// every 16 elements, the stride-R stores of a pass with a small span and the
// strided loads land in distinct banks.  The twiddles w^(r k) of each pass with
// Ns > 1 are a table [r - 1][k] in shared memory, read with consecutive k by
// consecutive threads.  All threads of a CTA take (row, t) tasks, one barrier per
// pass.
__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }

// Row pitch in float2 of a padded row (odd, so that the same element of
// neighbouring rows falls in different banks).
__host__ __device__ constexpr int fft_pitch(int L) { return L + L / 16 + 1; }

// Asynchronous global -> shared copies of 4 and 8 bytes (all of a thread's copies
// in flight at once), completed by cp_async_wait_all and a barrier.
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ float2 cmulw(float2 a, float2 w, bool inv) {   // a * w (or * conj w)
    const float ws = inv ? -w.y : w.y;
    return make_float2(a.x * w.x - a.y * ws, a.x * ws + a.y * w.x);
}

// cos and sin of pi E / 8, E in [0, 8)
__device__ __forceinline__ float cos_pi8(int E) {
    constexpr float c1 = 0.92387953251128674f, h = 0.70710678118654752f, s1 = 0.38268343236508977f;
    return E == 0 ? 1.0f : E == 1 ? c1 : E == 2 ? h : E == 3 ? s1 : E == 4 ? 0.0f : E == 5 ? -s1 : E == 6 ? -h : -c1;
}
__device__ __forceinline__ float sin_pi8(int E) {
    constexpr float c1 = 0.92387953251128674f, h = 0.70710678118654752f, s1 = 0.38268343236508977f;
    return E == 0 ? 0.0f : E == 1 ? s1 : E == 2 ? h : E == 3 ? c1 : E == 4 ? 1.0f : E == 5 ? c1 : E == 6 ? h : s1;
}

// a * exp(-+ 2 pi i E / 16) (forward: minus), E in [0, 8); E = 0 and 4 exact
__device__ __forceinline__ float2 rot16(float2 a, int E, bool inv) {
    if (E == 0) return a;
    if (E == 4) return inv ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
    const float c = cos_pi8(E), s = inv ? sin_pi8(E) : -sin_pi8(E);
    return make_float2(a.x * c - a.y * s, a.x * s + a.y * c);
}

__device__ __forceinline__ int bitrev_bits(int m, int bits) {
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((m >> b) & 1) << (bits - 1 - b);
    return r;
}

// R-point DFT in registers (R = 2, 4, 8, 16): radix-2 decimation in frequency,
// natural input order, output in bit-reversed order (v[j] = X[bitrev(j)]).  The
// butterfly of span h multiplies the difference by w_(2h)^k = w_16^(8k/h).
template <int R, bool INV>
__device__ __forceinline__ void dft_reg(float2 (&v)[R]) {
#pragma unroll
    for (int h = R / 2; h >= 1; h >>= 1) {
#pragma unroll
        for (int j = 0; j < R; ++j) {
            if (j & h) continue;
            const int k = j & (h - 1);
            const float2 a = v[j], b = v[j + h];
            v[j] = make_float2(a.x + b.x, a.y + b.y);
            v[j + h] = rot16(make_float2(a.x - b.x, a.y - b.y), (8 * k) / h, INV);
        }
    }
}

// One pass in place: thread u < nu = nrow L / 16 takes the 16 / R tasks u + j nu,
// loads their inputs, applies the twiddles and the DFTs in registers, waits at a
// barrier (every load of the pass done) and stores.  Needs blockDim.x >= nu.
template <int R, int LGR, bool INV>
__device__ __forceinline__ void fft_pass(float2 *x, const float2 *tw, int logL, int lgNs, int nrow, int ld) {
    constexpr int TPT = 16 / R;
    const int lgq = logL - LGR, q = 1 << lgq, Ns = 1 << lgNs, nu = (nrow << logL) >> 4;
    const int u = threadIdx.x;
    float2 v[TPT][R];
    if (u < nu) {
#pragma unroll
        for (int j = 0; j < TPT; ++j) {
            const int task = u + j * nu, tt = task & (q - 1), base = (task >> lgq) * ld, k = tt & (Ns - 1);
#pragma unroll
            for (int r = 0; r < R; ++r) v[j][r] = x[base + pad16(tt + r * q)];
            if (Ns > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) v[j][r] = cmulw(v[j][r], tw[(r - 1) * Ns + k], INV);
            }
            dft_reg<R, INV>(v[j]);
        }
    }
    __syncthreads();
    if (u < nu) {
#pragma unroll
        for (int j = 0; j < TPT; ++j) {
            const int task = u + j * nu, tt = task & (q - 1), base = (task >> lgq) * ld, k = tt & (Ns - 1);
            const int o = (tt - k) * R + k;
#pragma unroll
            for (int m = 0; m < R; ++m) x[base + pad16(o + m * Ns)] = v[j][bitrev_bits(m, LGR)];
        }
    }
    __syncthreads();
}

// The twiddle tables of the radix-16 passes with span Ns > 1, one after another:
// tw[(r - 1) Ns + k] = exp(-2 pi i r k / (16 Ns)) (the argument r k / (8 Ns) of
// sincospif is exact: 8 Ns is a power of two).  At most L - 1 entries.
__device__ __forceinline__ void fft_twiddles(float2 *tw, int logL) {
    int off = 0;
    for (int lg = logL & 3; lg < logL; lg += 4) {
        if (lg == 0) continue;
        const int Ns = 1 << lg, cnt = 15 * Ns;
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            const int r = (i >> lg) + 1, k = i & (Ns - 1);
            float sw, cw;
            sincospif(-(float)(r * k) / (float)(8 * Ns), &sw, &cw);
            tw[off + i] = make_float2(cw, sw);
        }
        off += cnt;
    }
}

// Transform of nrow padded rows of pitch ld in x, in place (nrow L / 16 <= blockDim.x).
// Starts and ends with a barrier inside each pass.
template <bool INV>
__device__ void fft_rows_smem(float2 *x, const float2 *tw, int logL, int nrow, int ld) {
    const int r0 = logL & 3;
    int lg = 0;
    if (r0) {
        if (r0 == 1) fft_pass<2, 1, INV>(x, tw, logL, 0, nrow, ld);
        else if (r0 == 2) fft_pass<4, 2, INV>(x, tw, logL, 0, nrow, ld);
        else fft_pass<8, 3, INV>(x, tw, logL, 0, nrow, ld);
        lg = r0;
    }
    int off = 0;
    for (; lg < logL; lg += 4) {
        fft_pass<16, 4, INV>(x, tw + off, logL, lg, nrow, ld);
        if (lg) off += 15 << lg;
    }
}

// Forward row transforms from the spins: C[r][y][kx] = FFT_x(s_x + i s_y),
// Z[r][y][kx] = FFT_x(s_z); a CTA takes Y rows of one replica.
__global__ void __launch_bounds__(1024) k_fft_fwd_rows(const float *__restrict__ spins, int L, int logL, int Y, float2 *C, float2 *Z) {
    extern __shared__ float2 fbuf[];
    const int N = L * L, r = blockIdx.y, y0 = blockIdx.x * Y, ld = fft_pitch(L);
    float2 *tw = fbuf, *x = tw + L;   // x: [2Y][ld] (C rows, then Z rows)
    pdl_trigger();
    fft_twiddles(tw, logL);
    pdl_wait();   // the spins of the previous update, and no reader of C, Z left
    const float *s = spins + (size_t)r * 3 * N;
    for (int i = threadIdx.x; i < Y * L; i += blockDim.x) {
        const int row = i >> logL, col = i & (L - 1), q = (y0 + row) * L + col;
        float2 *cx = x + row * ld + pad16(col), *zx = x + (Y + row) * ld + pad16(col);
        cp_async4(&cx->x, s + q);
        cp_async4(&cx->y, s + N + q);
        cp_async4(&zx->x, s + 2 * N + q);
        zx->y = 0.0f;
    }
    cp_async_wait_all();
    __syncthreads();
    fft_rows_smem<false>(x, tw, logL, 2 * Y, ld);
    float2 *Cr = C + (size_t)r * N + (size_t)y0 * L, *Zr = Z + (size_t)r * N + (size_t)y0 * L;
    for (int i = threadIdx.x; i < Y * L; i += blockDim.x) {
        const int row = i >> logL, col = pad16(i & (L - 1));
        Cr[i] = x[row * ld + col];
        Zr[i] = x[(Y + row) * ld + col];
    }
}

// Columns kx in [tb*CT, tb*CT + CT) of [0, L/2] and their mirrors (L - kx) mod L, of C
// and Z: transform over y, spectral product (S_x = (C + conj C(-k))/2,
// S_y = (C - conj C(-k))/(2i), H_x + i H_y = (W^xx S_x + W^xy S_y) + i (W^xy S_x + W^yy S_y),
// H_z = W^zz Z, W^ real and stored [kx][ky]), inverse transform over ky; the result
// replaces the columns of C (H_x + i H_y) and Z (H_z).
__global__ void __launch_bounds__(1024) k_fft_cols_conv(float2 *C, float2 *Z, const float *__restrict__ What, int L, int logL, int CT) {
    extern __shared__ float2 fbuf[];
    __shared__ int s_col[32], s_mir[32];
    const int N = L * L, r = blockIdx.y, k0 = blockIdx.x * CT, hl = L >> 1;
    // the tile's distinct columns: kx, then its mirror when different
    if (threadIdx.x == 0) {
        int nc = 0;
        for (int kx = k0; kx < k0 + CT && kx <= hl; ++kx) {
            s_col[nc++] = kx;
            const int m = (L - kx) & (L - 1);
            if (m != kx) s_col[nc++] = m;
        }
        for (int c = nc; c < 32; ++c) s_col[c] = -1;
        for (int c = 0; c < nc; ++c) {
            const int m = (L - s_col[c]) & (L - 1);
            int cm = c;
            for (int d = 0; d < nc; ++d)
                if (s_col[d] == m) cm = d;
            s_mir[c] = cm;
        }
    }
    __syncthreads();
    int nc = 0;
    while (nc < 32 && s_col[nc] >= 0) ++nc;
    const int ld = fft_pitch(L);   // odd pitch: a row of the tile's columns lands in distinct banks
    float2 *tw = fbuf, *x = tw + L;   // x: [2nc][ld] (C columns, then Z columns)
    pdl_trigger();
    fft_twiddles(tw, logL);
    pdl_wait();   // the row transforms
    float2 *Cr = C + (size_t)r * N, *Zr = Z + (size_t)r * N;
    for (int i = threadIdx.x; i < nc * L; i += blockDim.x) {
        const int yy = i / nc, c = i % nc;                // consecutive threads: neighbouring columns of a row
        const size_t g = (size_t)yy * L + s_col[c];
        cp_async8(x + c * ld + pad16(yy), Cr + g);
        cp_async8(x + (nc + c) * ld + pad16(yy), Zr + g);
    }
    cp_async_wait_all();
    __syncthreads();
    fft_rows_smem<false>(x, tw, logL, 2 * nc, ld);
    // In place: the item (c, ky) and its partner (mirror of c, -ky) read the same two
    // values of C, so one thread takes both (the one with c < mirror, or c = mirror
    // and ky <= -ky mod L).
    for (int i = threadIdx.x; i < nc * L; i += blockDim.x) {
        const int c = i >> logL, ky = i & (L - 1), cmi = s_mir[c];
        const int kym = (L - ky) & (L - 1), p = pad16(ky), pm = pad16(kym);
        const float2 z = x[(nc + c) * ld + p];
        const float wzz = What[3 * N + (size_t)s_col[c] * L + ky];
        x[(nc + c) * ld + p] = make_float2(wzz * z.x, wzz * z.y);
        if (c > cmi || (c == cmi && ky > kym)) continue;
        const float2 cv = x[c * ld + p], cm = x[cmi * ld + pm];
#pragma unroll
        for (int side = 0; side < 2; ++side) {    // the item (c, ky), then its partner
            const float2 a = side ? cm : cv, b = side ? cv : cm;
            const size_t wi = (size_t)s_col[side ? cmi : c] * L + (side ? kym : ky);
            const float2 sx = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
            const float2 sy = make_float2(0.5f * (a.y + b.y), -0.5f * (a.x - b.x));
            const float wxx = What[wi], wxy = What[N + wi], wyy = What[2 * N + wi];
            const float2 hx = make_float2(wxx * sx.x + wxy * sy.x, wxx * sx.y + wxy * sy.y);
            const float2 hy = make_float2(wxy * sx.x + wyy * sy.x, wxy * sx.y + wyy * sy.y);
            x[(side ? cmi : c) * ld + (side ? pm : p)] = make_float2(hx.x - hy.y, hx.y + hy.x);
            if (cmi == c && kym == ky) break;    // its own partner
        }
    }
    __syncthreads();
    fft_rows_smem<true>(x, tw, logL, 2 * nc, ld);
    for (int i = threadIdx.x; i < nc * L; i += blockDim.x) {
        const int yy = i / nc, c = i % nc;
        const size_t g = (size_t)yy * L + s_col[c];
        Cr[g] = x[c * ld + pad16(yy)];
        Zr[g] = x[(nc + c) * ld + pad16(yy)];
    }
}

// Inverse row transforms over kx and the field: h_x + i h_y = IFFT(H_x + i H_y),
// h_z = Re IFFT(H_z), scaled by 1/N.
__global__ void __launch_bounds__(1024) k_fft_inv_rows(const float2 *__restrict__ C, const float2 *__restrict__ Z, int L, int logL, int Y,
                               float scale, float *field) {
    extern __shared__ float2 fbuf[];
    const int N = L * L, r = blockIdx.y, y0 = blockIdx.x * Y, ld = fft_pitch(L);
    float2 *tw = fbuf, *x = tw + L;
    pdl_trigger();
    fft_twiddles(tw, logL);
    pdl_wait();   // the column pass
    const float2 *Cr = C + (size_t)r * N + (size_t)y0 * L, *Zr = Z + (size_t)r * N + (size_t)y0 * L;
    for (int i = threadIdx.x; i < Y * L; i += blockDim.x) {
        const int row = i >> logL, col = pad16(i & (L - 1));
        cp_async8(x + row * ld + col, Cr + i);
        cp_async8(x + (Y + row) * ld + col, Zr + i);
    }
    cp_async_wait_all();
    __syncthreads();
    fft_rows_smem<true>(x, tw, logL, 2 * Y, ld);
    float *f = field + (size_t)r * 3 * N + (size_t)y0 * L;
    for (int i = threadIdx.x; i < Y * L; i += blockDim.x) {
        const int row = i >> logL, col = pad16(i & (L - 1));
        const float2 a = x[row * ld + col];
        f[i] = a.x * scale;
        f[N + i] = a.y * scale;
        f[2 * N + i] = x[(Y + row) * ld + col].x * scale;
    }
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

__global__ void k_fft_update(const FftStepConfig cfg, const FftStepBuffers buf) {
    pdl_trigger();
    pdl_wait();   // the field of the state before the sub-step
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
        {
            const float3 Sv = propose_spin(cfg.proposal, cfg.cap_c1, s0, s1, s2, u1, cps, sps);   // Sec. 3.1 proposal
            S0 = Sv.x;
            S1 = Sv.y;
            S2 = Sv.z;
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
    if (obs && tid < kNB) obs_push_level(obs[r], x_s, tid);
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

// rows Y of a row-pass CTA: 2Y rows of L/4 radix-4 butterflies, at least 256 a stage
// Rows of a row-pass CTA: at least 64 tasks in a radix-16 pass (2Y rows x L/16),
// then doubled while the grid keeps four CTAs per SM and a CTA at most 256 tasks.
int fft_rows_per_cta(int L, int R, int nsm) {
    int Y = std::min(L, std::max(1, 512 / L));
    while (2 * Y <= L && 4 * Y * L / 16 <= 256 && (long long)(L / (2 * Y)) * R >= 4LL * nsm) Y *= 2;
    return Y;
}

int fft_cols_per_tile(int L) {      // columns kx (plus mirrors) of a column-pass CTA
    const int ct = 1024 / L;
    return ct < 1 ? 1 : (ct > 8 ? 8 : ct);
}

int fft_threads(int tasks) { return std::min(1024, std::max(64, (tasks + 31) / 32 * 32)); }


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
    const int N = L * L, logL = ilog2(L);
    const size_t tot = (size_t)N * R;
    float2 *C = scratch, *Z = scratch + tot;
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int Y = fft_rows_per_cta(L, R, nsm), CT = fft_cols_per_tile(L), ld = fft_pitch(L);
    // threads: the tasks of a radix-16 pass (16 points a task); a grid smaller than
    // the SM count gets wider CTAs, for more loads in flight in the gather, the
    // spectral product and the scatter
    const int rblocks = L / Y * R, cblocks = (L / 2 + 1 + CT - 1) / CT * R;
    const int rthreads = rblocks < nsm ? fft_threads(std::max(2 * Y * L / 16, Y * L / 2)) : fft_threads(2 * Y * L / 16);
    const int cthreads = cblocks < nsm ? 1024 : fft_threads(2 * 2 * CT * L / 16);
    const size_t rsmem = sizeof(float2) * ((size_t)L + (size_t)2 * Y * ld);
    const size_t csmem = sizeof(float2) * ((size_t)L + (size_t)2 * 2 * CT * ld);
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_fft_fwd_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsmem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_fft_inv_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsmem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_fft_cols_conv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csmem)) != cudaSuccess) return e;
    if ((e = launch_pdl(k_fft_fwd_rows, dim3(L / Y, R), rthreads, rsmem, st, spins, L, logL, Y, C, Z)) != cudaSuccess)
        return e;
    if ((e = launch_pdl(k_fft_cols_conv, dim3((L / 2 + 1 + CT - 1) / CT, R), cthreads, csmem, st, C, Z, What, L, logL,
                        CT)) != cudaSuccess)
        return e;
    return launch_pdl(k_fft_inv_rows, dim3(L / Y, R), rthreads, rsmem, st, (const float2 *)C, (const float2 *)Z, L, logL,
                      Y, 1.0f / (float)N, field);
}

cudaError_t launch_fft_update(const FftStepConfig &c, const FftStepBuffers &b, cudaStream_t st) {
    const int n = (c.L / c.l) * (c.L / c.l);
    const int threads = n >= 256 ? 256 : ((n + 31) / 32) * 32;
    dim3 grid((n + threads - 1) / threads, c.R);
    return launch_pdl(k_fft_update, grid, threads, 0, st, c, b);
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
