// aux_kernels.cu -- W~ precompute (FP64), spin initialisation, full field and
// total energy.  None of these is in the per-sub-step loop; they run once per
// lattice (W~), per init, or once per mc_sweep call (energy anchor).
#include "internal.cuh"

namespace dipmc {

// ---------------------------------------------------------------------------
// W~(rho) (Sec. 2.1, Eq. 2): image sum over |a|, |b| <= A of the planar dipole
// tensor W(r) = (delta_ab - 3 r^_a r^_b)/r^3 (a, b in x, y), W_zz = 1/r^3, for the
// minimum-image representative of rho (both +-L/2 averaged on the half-way
// line), plus the continuum tail beyond the square of half-width (A + 1/2) L.
// One CTA per rho; threads stride over the (2A+1)^2 images; FP64 throughout.
// ---------------------------------------------------------------------------
constexpr int kWThreads = 256;

__device__ __forceinline__ int reps_of(int v, int L, double out[2]) {
    if (2 * v < L) { out[0] = v; return 1; }
    if (2 * v > L) { out[0] = v - L; return 1; }
    out[0] = 0.5 * L;
    out[1] = -0.5 * L;
    return 2;
}

__global__ void __launch_bounds__(kWThreads) k_wtilde(int L, int A, int tail, double *W64, float *W32) {
    const int N = L * L;
    const int rho = blockIdx.x;
    const int x = rho % L, y = rho / L;
    double xr[2], yr[2];
    const int nx = reps_of(x, L, xr), ny = reps_of(y, L, yr);
    const int side = 2 * A + 1;
    const long long nimg = (long long)side * side;
    double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
            for (long long g = threadIdx.x; g < nimg; g += kWThreads) {
                const int ga = (int)(g % side) - A, gb = (int)(g / side) - A;
                const double rx = xr[i] + (double)ga * L;
                const double ry = yr[j] + (double)gb * L;
                const double r2 = rx * rx + ry * ry;
                if (r2 == 0.0) continue;  // the site itself
                const double inv_r2 = 1.0 / r2;
                const double inv_r3 = inv_r2 / sqrt(r2);
                const double k = 3.0 * inv_r3 * inv_r2;
                a0 += inv_r3 - k * rx * rx;
                a1 -= k * rx * ry;
                a2 += inv_r3 - k * ry * ry;
                a3 += inv_r3;
            }
    __shared__ double red[4][kWThreads / 32];
    for (int off = 16; off; off >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, off);
        a1 += __shfl_xor_sync(0xffffffffu, a1, off);
        a2 += __shfl_xor_sync(0xffffffffu, a2, off);
        a3 += __shfl_xor_sync(0xffffffffu, a3, off);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        red[0][warp] = a0; red[1][warp] = a1; red[2][warp] = a2; red[3][warp] = a3;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s[4] = {0, 0, 0, 0};
        for (int w = 0; w < kWThreads / 32; ++w)
            for (int c = 0; c < 4; ++c) s[c] += red[c][w];
        const double inv = 1.0 / (double)(nx * ny);
        for (int c = 0; c < 4; ++c) s[c] *= inv;
        if (tail) {
            const double Rw = ((double)A + 0.5) * (double)L;
            const double tz = 4.0 * sqrt(2.0) / (Rw * (double)L * (double)L);
            s[3] += tz;
            s[0] -= 0.5 * tz;
            s[2] -= 0.5 * tz;
        }
        for (int c = 0; c < 4; ++c) {
            W64[c * N + rho] = s[c];
            W32[c * N + rho] = (float)s[c];
        }
    }
}

// ---------------------------------------------------------------------------
// W~ by the Ewald/Harris split (Sec. 2.1) for two layers a height z apart
// (z = 0: the lattice itself), all six components xx, xy, yy, zz, xz, yz.
// With W_ab = -d_a d_b (1/r) and 1/r = erfc(r/a)/r + erf(r/a)/r, a = 2 eta:
// the erfc part is summed in real space over the images, the erf part as the
// in-plane Fourier series over the reciprocal lattice k = 2 pi (m, n) / L of
//   g^(k, z) = (pi/k)[e^{kz} erfc(k eta + z/a) + e^{-kz} erfc(k eta - z/a)]
// (d_z g^ = pi[e^{kz} erfc(..) - e^{-kz} erfc(..)], d_z^2 g^ = k^2 g^ -
// (2 sqrt(pi)/eta) exp(-k^2 eta^2 - z^2/a^2); k = 0 reaches zz only).  At z = 0
// the site itself is left out and the R -> 0 limit of the erf part,
// -4/(3 a^3 sqrt(pi)) on the diagonal, is taken back out.  One CTA per rho,
// threads over the real and reciprocal terms, FP64.
// ---------------------------------------------------------------------------
constexpr double kPiD = 3.141592653589793238462643383279502884;

__global__ void __launch_bounds__(kWThreads) k_wtilde_ewald(int L, double z, double eta, int nreal, int nrec,
                                                            double *W6) {
    const int N = L * L, rho = blockIdx.x, x = rho % L, y = rho / L;
    const double a = 2.0 * eta, area = (double)L * L, spi = sqrt(kPiD);
    const int sr = 2 * nreal + 1, sk = 2 * nrec + 1;
    const long long nr = (long long)sr * sr, nt = nr + (long long)sk * sk;
    double w[6] = {0, 0, 0, 0, 0, 0};
    for (long long g = threadIdx.x; g < nt; g += kWThreads) {
        if (g < nr) {
            const int i = (int)(g % sr) - nreal, j = (int)(g / sr) - nreal;
            const double d0 = x + (double)i * L, d1 = y + (double)j * L, d2 = z;
            const double R2 = d0 * d0 + d1 * d1 + d2 * d2;
            if (R2 == 0.0) continue;
            const double R = sqrt(R2), ga = exp(-R2 / (a * a)), ec = erfc(R / a);
            const double g1 = -(2.0 / (a * spi)) * ga / R - ec / R2;
            const double g2 = (4.0 / (a * a * a * spi)) * ga + (4.0 / (a * spi)) * ga / R2 + 2.0 * ec / (R2 * R);
            const double d[3] = {d0, d1, d2};
            const int ia[6] = {0, 0, 1, 2, 0, 1}, ib[6] = {0, 1, 1, 2, 2, 2};
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                const double dd = d[ia[c]] * d[ib[c]] / R2;
                w[c] -= g2 * dd + g1 * ((ia[c] == ib[c] ? 1.0 : 0.0) - dd) / R;
            }
        } else {
            const long long h = g - nr;
            const int m = (int)(h % sk) - nrec, n = (int)(h / sk) - nrec;
            if (m == 0 && n == 0) continue;
            const double kx = 2.0 * kPiD * m / L, ky = 2.0 * kPiD * n / L;
            const double k = sqrt(kx * kx + ky * ky);
            const double ep = exp(k * z) * erfc(k * eta + z / a), em = exp(-k * z) * erfc(k * eta - z / a);
            const double gh = kPiD / k * (ep + em), dgh = kPiD * (ep - em);
            const double d2gh = k * k * gh - (2.0 * spi / eta) * exp(-k * k * eta * eta - z * z / (a * a));
            double sn, cs;
            sincos(kx * x + ky * y, &sn, &cs);
            w[0] += kx * kx * gh * cs / area;
            w[1] += kx * ky * gh * cs / area;
            w[2] += ky * ky * gh * cs / area;
            w[3] -= d2gh * cs / area;
            w[4] += kx * dgh * sn / area;
            w[5] += ky * dgh * sn / area;
        }
    }
    __shared__ double red[6][kWThreads / 32];
#pragma unroll
    for (int c = 0; c < 6; ++c)
        for (int off = 16; off; off >>= 1) w[c] += __shfl_xor_sync(0xffffffffu, w[c], off);
    if ((threadIdx.x & 31) == 0)
        for (int c = 0; c < 6; ++c) red[c][threadIdx.x >> 5] = w[c];
    __syncthreads();
    if (threadIdx.x == 0) {
        double s[6] = {0, 0, 0, 0, 0, 0};
        for (int v = 0; v < kWThreads / 32; ++v)
            for (int c = 0; c < 6; ++c) s[c] += red[c][v];
        s[3] += (2.0 * spi / eta) * exp(-z * z / (a * a)) / area;
        if (z == 0.0 && rho == 0) {
            const double self = -4.0 / (3.0 * a * a * a * spi);
            s[0] += self;
            s[2] += self;
            s[3] += self;
        }
        for (int c = 0; c < 6; ++c) W6[(size_t)c * N + rho] = s[c];
    }
}

cudaError_t launch_wtilde_ewald(int L, double z, double eta, double *W6, cudaStream_t st) {
    const int nreal = (int)ceil(6.0 * 2.0 * eta / L) + 1;
    const int nrec = (int)ceil(6.5 / eta * L / (2.0 * kPiD)) + 1;
    k_wtilde_ewald<<<L * L, kWThreads, 0, st>>>(L, z, eta, nreal, nrec, W6);
    return cudaGetLastError();
}

// The in-plane components of a six-component tensor as W~ (FP64 and FP32).
__global__ void k_take_plane(size_t N, const double *__restrict__ W6, double *W64, float *W32) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 4 * N) return;
    W64[i] = W6[i];
    W32[i] = (float)W6[i];
}

cudaError_t launch_take_plane(int L, const double *W6, double *W64, float *W32, cudaStream_t st) {
    const size_t N = (size_t)L * L;
    k_take_plane<<<(unsigned)((4 * N + 255) / 256), 256, 0, st>>>(N, W6, W64, W32);
    return cudaGetLastError();
}

__global__ void k_cast_W(size_t n, const double *__restrict__ W64, float *W32) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) W32[i] = (float)W64[i];
}

cudaError_t launch_cast_W(int L, const double *W64, float *W32, cudaStream_t st) {
    const size_t n = (size_t)4 * L * L;
    k_cast_W<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, W64, W32);
    return cudaGetLastError();
}

cudaError_t launch_wtilde(int L, int A, int tail, double *W64, float *W32, cudaStream_t st) {
    k_wtilde<<<L * L, kWThreads, 0, st>>>(L, A, tail, W64, W32);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Initial spins: mode 0 uniform on S^2 from Philox {site, r, 0, tag}; 1 = +z;
// 3 = Ising +-z from the same counter.
// ---------------------------------------------------------------------------
__global__ void k_init_spins(int L, int R, uint2 key, int mode, float *spins) {
    const int N = L * L;
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (long long)N * R) return;
    const int r = (int)(gid / N), i = (int)(gid % N);
    float sx = 0.f, sy = 0.f, sz = 1.f;
    if (mode == 3) {
        // Ising spin (Appendix B): +z where the first uniform is below 1/2
        const uint4 w = philox(make_uint4((uint32_t)i, (uint32_t)r, 0u, kTagInit), key);
        sz = u24f(w.x) < 0.5f ? 1.0f : -1.0f;
    } else if (mode == 0) {
        const uint4 w = philox(make_uint4((uint32_t)i, (uint32_t)r, 0u, kTagInit), key);
        sz = 2.0f * u24f(w.x) - 1.0f;
        const float rr = sqrtf(fmaxf(0.0f, (1.0f - sz) * (1.0f + sz)));
        float sp, cp;
        sincospif(2.0f * u24f(w.y), &sp, &cp);
        sx = rr * cp;
        sy = rr * sp;
    }
    float *s = spins + (size_t)r * 3 * N;
    s[i] = sx;
    s[N + i] = sy;
    s[2 * N + i] = sz;
}

cudaError_t launch_init_spins(int L, int R, uint2 key, int mode, float *spins, cudaStream_t st) {
    const long long tot = (long long)L * L * R;
    k_init_spins<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(L, R, key, mode, spins);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Full field h_p = sum_d W~(d) s_{p-d} at every site (FP32, direct O(N^2) per
// replica).  Thread = site p; W~(d) is the same address across the warp
// (broadcast); s_{p-d} is coalesced across consecutive p.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_full_field(int L, const float *__restrict__ W32,
                                                    const float *__restrict__ spins,
                                                    float *__restrict__ h) {
    const int N = L * L;
    const int r = blockIdx.y;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    const int px = p % L, py = p / L;
    const float *s = spins + (size_t)r * 3 * N;
    float h0 = 0.f, h1 = 0.f, h2 = 0.f;
    for (int dy = 0; dy < L; ++dy) {
        int y = py - dy;
        if (y < 0) y += L;
        const float *s0 = s + y * L, *s1 = s0 + N, *s2 = s1 + N;
        const float *w0 = W32 + dy * L, *w1 = w0 + N, *w2 = w1 + N, *w3 = w2 + N;
        for (int dx = 0; dx < L; ++dx) {
            int x = px - dx;
            if (x < 0) x += L;
            const float a = __ldg(s0 + x), b = __ldg(s1 + x), c = __ldg(s2 + x);
            const float xx = __ldg(w0 + dx), xy = __ldg(w1 + dx), yy = __ldg(w2 + dx), zz = __ldg(w3 + dx);
            h0 = fmaf(xx, a, fmaf(xy, b, h0));
            h1 = fmaf(xy, a, fmaf(yy, b, h1));
            h2 = fmaf(zz, c, h2);
        }
    }
    float *o = h + (size_t)r * 3 * N;
    o[p] = h0;
    o[N + p] = h1;
    o[2 * N + p] = h2;
}

cudaError_t launch_full_field(int L, int R, const float *W32, const float *spins, float *h,
                              cudaStream_t st) {
    const int N = L * L;
    dim3 grid((N + 255) / 256, R);
    k_full_field<<<grid, 256, 0, st>>>(L, W32, spins, h);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Total energy per replica (Sec. 4 energy, with the ferromagnetic-exchange and
// E_A = -K2 z^2 - K4 z^4 readings), FP64 sums.  One CTA per replica.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_energy(int L, const float *__restrict__ spins,
                                                const float *__restrict__ h,
                                                const RepParams *__restrict__ P, double *E) {
    const int N = L * L, r = blockIdx.x;
    const RepParams p = P[r];
    const double e = cta_replica_energy(L, spins + (size_t)r * 3 * N, h + (size_t)r * 3 * N, p.J, p.CD, p.K2, p.K4);
    if (threadIdx.x == 0) E[r] = e;
}

cudaError_t launch_energy(int L, int R, const float *spins, const float *h, const RepParams *p,
                          double *E, cudaStream_t st) {
    k_energy<<<R, 256, 0, st>>>(L, spins, h, p, E);
    return cudaGetLastError();
}

// Cone-angle order parameter of Sec. 4.1 per replica:
//     eta = (1/N) sum_i sqrt((2/pi)^2 <(theta_i - pi/2)^2>),
// the per-site mean over the n measured sweeps (theta2 holds the per-site sums).
// One CTA per replica; a fixed-order reduction (deterministic).
__global__ void k_eta(int N, const double *__restrict__ theta2, const ObsAcc *__restrict__ obs, double *eta) {
    const int r = blockIdx.x;
    const long long n = obs[r].bcnt[0];
    const double pi = 3.14159265358979323846;
    const double c = n > 0 ? (2.0 / pi) * (2.0 / pi) / (double)n : 0.0;
    double acc = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) acc += sqrt(c * theta2[(size_t)r * N + i]);
    for (int off = 16; off; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        eta[r] = n > 0 ? s / N : (double)NAN;
    }
}

cudaError_t launch_eta(int N, int count, const double *theta2, const ObsAcc *obs, double *eta, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    k_eta<<<count, 256, 0, st>>>(N, theta2, obs, eta);
    return cudaGetLastError();
}

}  // namespace dipmc
