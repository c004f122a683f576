/*
 * oracle.c -- plain CPU FP64 oracle for the dipolar Heisenberg Monte Carlo sweep
 * of Stamps & Ambrose, "Monte Carlo simulation of the effects of higher order
 * anisotropy on the spin reorientation transition in the two dimensional
 * Heisenberg model with long range interactions" (arXiv:1211.6234).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this file.  The CUDA library shares no
 * code, header, table or constant generator with it; both implement the same
 * definitions independently.
 *
 * Everything here is deliberately slow and literal: direct sums, FP64, no
 * blocking, no reordering beyond what the definitions state.
 *
 * Readings of the paper used here (each is discussed in the design notes):
 *   - Exchange is ferromagnetic: E_ex = -J sum_bonds s_i.s_j, each nearest
 *     neighbour bond counted once (Sec. 4 total energy; the printed +J/2 sign is
 *     read against the paper's own statement that exchange is minimised in the
 *     ferromagnetic state).
 *   - Anisotropy: E_A(s) = -K2 s_z^2 - K4 s_z^4 (Sec. 4, anisotropy equation,
 *     with K<0 folded into positive K2, K4 = |K|(1-a), |K| a).
 *   - Dipole tensor of one image (Sec. 2.1, first equation, lattice in the x-y
 *     plane): W(r) = (delta_ab - 3 r^_a r^_b)/|r|^3 for a,b in {x,y}, W_zz = 1/|r|^3.
 *   - Replica-summed tensor (Sec. 2.1, Eq. 2): W~(rho) = sum_{|a|,|b|<=A} W(rho+G),
 *     G = (aL, bL), excluding rho+G = 0 (that G != 0 part at rho = 0 is the
 *     self-image term), plus the continuum tail of all images outside the square
 *     of half-width (A+1/2)L:  zz += 4 sqrt(2)/((A+1/2) L^3),  xx, yy -= half of it.
 *   - Field h_n = sum_m W~(n-m) s_m, including m = n through W~(0);
 *     E_D = (C_D/2) sum_n s_n.h_n;  single-site change s -> S, d = S - s:
 *     dE_D = C_D [ d.h_n + 1/2 d.W~(0).d ].
 *   - Metropolis (Sec. 2.2, Eq. Metro): accept iff u < exp(-dE/T), k_B = 1.
 *   - Simultaneous flipping (Sec. 3.1, 3.2): update sites o + l(a,b), all of
 *     them decided from the state before the step, accepted moves applied
 *     together; l = L leaves one site per step, i.e. exact sequential Metropolis.
 *   - Site schedule: per sweep a random permutation of the l^2 offsets (every site
 *     attempted once per sweep); the paper's draw-with-replacement (Sec. 3.1,
 *     host part of Appendix A) is kind 1.
 *   - Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), counter
 *     layout below.  u = (word >> 8) * 2^-24.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846
#define ORC_NOBS 11  /* |m|, m_z, |m_z|, M_par, E/N, m_st, wall density, O_x, O_y, O_z, cone */

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, written from its published definition (Salmon et al.,     */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds of a    */
/* multiply-hi/lo S-box on words 0 and 2, a word permutation, and a Weyl     */
/* key schedule.                                                              */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static double u24(uint32_t w) { return (double)(w >> 8) * (1.0 / 16777216.0); }

/* Stream tags in the top byte of counter word 3. */
#define TAG_ATTEMPT 0x01u
#define TAG_PERM 0x02u
#define TAG_DRAW 0x03u
#define TAG_INIT 0x04u

/* ------------------------------------------------------------------------ */
/* Replica-summed dipole tensor W~ (Sec. 2.1, Eq. 2).                         */
/* Layout: W[c*L*L + y*L + x], c = 0 xx, 1 xy, 2 yy, 3 zz; (x, y) = rho.       */
/*                                                                          */
/* The window of images is centred on the minimum-image representative of   */
/* each component of rho (x if 2x < L, x - L if 2x > L); a component equal to */
/* L/2 has two representatives, +-L/2, and the windows of both are averaged. */
/* This keeps every symmetry of the infinite sum exact: W~(-rho) = W~(rho),   */
/* the reflections x -> -x, y -> -y and the swap x <-> y.                     */
/* ------------------------------------------------------------------------ */
static void window_sum(double x0, double y0, int L, int A, double acc[4])
{
    for (int b = -A; b <= A; ++b) {
        for (int a = -A; a <= A; ++a) {
            double rx = x0 + (double)a * L;
            double ry = y0 + (double)b * L;
            double r2 = rx * rx + ry * ry;
            if (r2 == 0.0) continue; /* the site itself, not an image */
            double r = sqrt(r2);
            double ir3 = 1.0 / (r2 * r);
            double ux = rx / r, uy = ry / r;
            acc[0] += ir3 * (1.0 - 3.0 * ux * ux);
            acc[1] += ir3 * (-3.0 * ux * uy);
            acc[2] += ir3 * (1.0 - 3.0 * uy * uy);
            acc[3] += ir3;
        }
    }
}

/* Representatives of one component v in [0, L): returns their count (1 or 2). */
static int reps(int v, int L, double out[2])
{
    if (2 * v < L) { out[0] = v; return 1; }
    if (2 * v > L) { out[0] = v - L; return 1; }
    out[0] = 0.5 * L;
    out[1] = -0.5 * L;
    return 2;
}

int orc_wtilde(int L, int A, int tail, double *W)
{
    if (L < 1 || A < 0 || !W) return -1;
    const int N = L * L;
    for (int y = 0; y < L; ++y) {
        for (int x = 0; x < L; ++x) {
            double xr[2], yr[2];
            int nx = reps(x, L, xr), ny = reps(y, L, yr);
            double acc[4] = {0, 0, 0, 0};
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) window_sum(xr[i], yr[j], L, A, acc);
            double w = 1.0 / (double)(nx * ny);
            double xx = acc[0] * w, xy = acc[1] * w, yy = acc[2] * w, zz = acc[3] * w;
            if (tail) {
                double R = ((double)A + 0.5) * (double)L;
                double tz = 4.0 * sqrt(2.0) / (R * (double)L * (double)L);
                zz += tz;
                xx -= 0.5 * tz;
                yy -= 0.5 * tz;
            }
            W[0 * N + y * L + x] = xx;
            W[1 * N + y * L + x] = xy;
            W[2 * N + y * L + x] = yy;
            W[3 * N + y * L + x] = zz;
        }
    }
    return 0;
}

/*
 * W~ by the Ewald/Harris split of Sec. 2.1 (real-space erfc part plus a Fourier
 * part over the reciprocal lattice of the L x L cell), for two layers a height
 * z apart (z = 0: the lattice itself).  With F(R) = sum_G 1/|R + G| over the
 * in-plane lattice vectors G and the tensor W_ab = -d_a d_b (1/r) =
 * (delta_ab - 3 r^_a r^_b)/r^3 of Sec. 2.1, 1/r = erfc(r/a)/r + erf(r/a)/r,
 * a = 2 eta:
 *   short range: -d_a d_b of g(R) = erfc(R/a)/R summed over G, using
 *     d_a d_b g(|d|) = g'' d_a d_b / R^2 + g' (delta_ab - d_a d_b / R^2) / R;
 *   long range: the in-plane Fourier series (1/A) sum_k g^(k, z) e^{i k.rho}
 *     (A = L^2, k = 2 pi (m, n) / L) of the erf part, with
 *     g^(k, z) = (pi/k) [e^{kz} erfc(k eta + z/a) + e^{-kz} erfc(k eta - z/a)],
 *     d_z g^ = pi [e^{kz} erfc(k eta + z/a) - e^{-kz} erfc(k eta - z/a)],
 *     d_z^2 g^ = k^2 g^ - (2 sqrt(pi)/eta) exp(-k^2 eta^2 - z^2/a^2);
 *     the k = 0 term only reaches zz: -(1/A)(-(2 sqrt(pi)/eta) exp(-z^2/a^2));
 *   self term (z = 0, rho = 0): the site itself is excluded, G = 0 is dropped
 *     from the real-space sum and d_a d_b [erf(R/a)/R] at R = 0,
 *     -4 delta_ab / (3 a^3 sqrt(pi)), is added back.
 * Output W6[c][L][L], c = xx, xy, yy, zz, xz, yz.  The sums run until the
 * neglected terms are below 1e-16 relative (erfc(6) ~ 2e-17; exp(-42) ~ 6e-19).
 */
int orc_wtilde_ewald(int L, double z, double eta, double *W6)
{
    if (L < 1 || !(eta > 0.0) || !W6) return -1;
    const int N = L * L;
    const double a = 2.0 * eta, area = (double)L * L, spi = sqrt(ORC_PI);
    const int nreal = (int)ceil(6.0 * a / L) + 1;
    const int nrec = (int)ceil(6.5 / eta * L / (2.0 * ORC_PI)) + 1;
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x) {
            double w[6] = {0, 0, 0, 0, 0, 0};
            /* short range */
            for (int j = -nreal; j <= nreal; ++j)
                for (int i = -nreal; i <= nreal; ++i) {
                    const double d[3] = {x + (double)i * L, y + (double)j * L, z};
                    const double R2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                    if (R2 == 0.0) continue;
                    const double R = sqrt(R2), ga = exp(-R2 / (a * a)), ec = erfc(R / a);
                    const double g1 = -(2.0 / (a * spi)) * ga / R - ec / R2;
                    const double g2 = (4.0 / (a * a * a * spi)) * ga + (4.0 / (a * spi)) * ga / R2 + 2.0 * ec / (R2 * R);
                    const int ia[6] = {0, 0, 1, 2, 0, 1}, ib[6] = {0, 1, 1, 2, 2, 2};
                    for (int c = 0; c < 6; ++c) {
                        const double dd = d[ia[c]] * d[ib[c]] / R2;
                        w[c] -= g2 * dd + g1 * ((ia[c] == ib[c] ? 1.0 : 0.0) - dd) / R;
                    }
                }
            /* long range */
            for (int n = -nrec; n <= nrec; ++n)
                for (int m = -nrec; m <= nrec; ++m) {
                    if (m == 0 && n == 0) continue;
                    const double kx = 2.0 * ORC_PI * m / L, ky = 2.0 * ORC_PI * n / L;
                    const double k = sqrt(kx * kx + ky * ky);
                    const double ep = exp(k * z) * erfc(k * eta + z / a), em = exp(-k * z) * erfc(k * eta - z / a);
                    const double gh = ORC_PI / k * (ep + em), dgh = ORC_PI * (ep - em);
                    const double d2gh = k * k * gh - (2.0 * spi / eta) * exp(-k * k * eta * eta - z * z / (a * a));
                    const double ph = kx * x + ky * y, cs = cos(ph), sn = sin(ph);
                    w[0] += kx * kx * gh * cs / area;
                    w[1] += kx * ky * gh * cs / area;
                    w[2] += ky * ky * gh * cs / area;
                    w[3] -= d2gh * cs / area;
                    w[4] += kx * dgh * sn / area;
                    w[5] += ky * dgh * sn / area;
                }
            w[3] += (2.0 * spi / eta) * exp(-z * z / (a * a)) / area;
            if (z == 0.0 && x == 0 && y == 0) {
                const double self = -4.0 / (3.0 * a * a * a * spi);
                w[0] += self;
                w[2] += self;
                w[3] += self;
            }
            for (int c = 0; c < 6; ++c) W6[c * N + y * L + x] = w[c];
        }
    return 0;
}

static inline int wrap(int v, int L) { v %= L; return v < 0 ? v + L : v; }

/* W~(p - m) applied to a vector s: out = W~(d) s, d = (dx, dy) taken mod L. */
static void wapply(const double *W, int L, int dx, int dy, const double s[3], double out[3])
{
    const int N = L * L;
    int i = wrap(dy, L) * L + wrap(dx, L);
    double xx = W[i], xy = W[N + i], yy = W[2 * N + i], zz = W[3 * N + i];
    out[0] = xx * s[0] + xy * s[1];
    out[1] = xy * s[0] + yy * s[1];
    out[2] = zz * s[2];
}

/* Field at one site q: h_q = sum_m W~(q - m) s_m (all m, including m = q). */
static void field_at(const double *W, int L, const double *s, int qx, int qy, double h[3])
{
    const int N = L * L;
    h[0] = h[1] = h[2] = 0.0;
    for (int my = 0; my < L; ++my) {
        for (int mx = 0; mx < L; ++mx) {
            int m = my * L + mx;
            double sm[3] = {s[m], s[N + m], s[2 * N + m]};
            double t[3];
            wapply(W, L, qx - mx, qy - my, sm, t);
            h[0] += t[0];
            h[1] += t[1];
            h[2] += t[2];
        }
    }
}

/* Field at every site; s and h are [3][L][L]. */
void orc_field(int L, const double *W, const double *s, double *h)
{
    const int N = L * L;
    for (int qy = 0; qy < L; ++qy)
        for (int qx = 0; qx < L; ++qx) {
            double t[3];
            field_at(W, L, s, qx, qy, t);
            int q = qy * L + qx;
            h[q] = t[0];
            h[N + q] = t[1];
            h[2 * N + q] = t[2];
        }
}

/* Total energy (Sec. 4 total energy, with the readings above).
 * out[0] exchange, out[1] anisotropy, out[2] dipole, out[3] total. */
void orc_energy(int L, const double *W, const double *s, double J, double CD, double K2,
                double K4, double *out)
{
    const int N = L * L;
    double *h = (double *)malloc(sizeof(double) * 3 * N);
    orc_field(L, W, s, h);
    double ex = 0, an = 0, dp = 0;
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x) {
            int i = y * L + x;
            int ixp = y * L + wrap(x + 1, L);
            int iyp = wrap(y + 1, L) * L + x;
            for (int c = 0; c < 3; ++c)
                ex += s[c * N + i] * (s[c * N + ixp] + s[c * N + iyp]);
            double z = s[2 * N + i];
            an += -K2 * z * z - K4 * z * z * z * z;
            dp += s[i] * h[i] + s[N + i] * h[N + i] + s[2 * N + i] * h[2 * N + i];
        }
    free(h);
    out[0] = -J * ex;
    out[1] = an;
    out[2] = 0.5 * CD * dp;
    out[3] = out[0] + out[1] + out[2];
}

/* Dipole energy by explicit pairs and images, without W~ (Sec. 2.1, first
 * equation summed over the periodic tiling): (C_D/2) sum_{n,m in cell}
 * sum_{|a|,|b|<=A} [s_n.s_m - 3 (s_n.r^)(s_m.r^)]/r^3 over r = rho + G != 0, with
 * rho the minimum-image representative(s) of n - m (the pair term is even in r;
 * this is the window of images W~ uses), plus the same continuum tail applied
 * pairwise when tail != 0. */
double orc_dipole_energy_pairs(int L, int A, int tail, const double *s, double CD)
{
    const int N = L * L;
    double tz = 0.0;
    if (tail) {
        double R = ((double)A + 0.5) * (double)L;
        tz = 4.0 * sqrt(2.0) / (R * (double)L * (double)L);
    }
    double E = 0.0;
    for (int n = 0; n < N; ++n) {
        int nx = n % L, ny = n / L;
        double sn[3] = {s[n], s[N + n], s[2 * N + n]};
        for (int m = 0; m < N; ++m) {
            int mx = m % L, my = m / L;
            double sm[3] = {s[m], s[N + m], s[2 * N + m]};
            double dot = sn[0] * sm[0] + sn[1] * sm[1] + sn[2] * sm[2];
            double xr[2], yr[2];
            int cx = reps(wrap(nx - mx, L), L, xr), cy = reps(wrap(ny - my, L), L, yr);
            double pair = 0.0;
            for (int j = 0; j < cy; ++j)
                for (int i = 0; i < cx; ++i)
                    for (int b = -A; b <= A; ++b)
                        for (int a = -A; a <= A; ++a) {
                            double rx = xr[i] + (double)a * L;
                            double ry = yr[j] + (double)b * L;
                            double r2 = rx * rx + ry * ry;
                            if (r2 == 0.0) continue;
                            double r = sqrt(r2);
                            double ux = rx / r, uy = ry / r;
                            double sn_r = sn[0] * ux + sn[1] * uy;
                            double sm_r = sm[0] * ux + sm[1] * uy;
                            pair += (dot - 3.0 * sn_r * sm_r) / (r2 * r);
                        }
            E += pair / (double)(cx * cy);
            if (tail)
                E += tz * (sn[2] * sm[2] - 0.5 * sn[0] * sm[0] - 0.5 * sn[1] * sm[1]);
        }
    }
    return 0.5 * CD * E;
}

/* ------------------------------------------------------------------------ */
/* Parameters of one replica.                                                */
/* ------------------------------------------------------------------------ */
typedef struct {
    int L, l;
    double J, CD, K2, K4, T;
    int proposal;   /* 0: uniform on the cap of half-angle `cone` around s; 1: uniform on S^2;
                       2: reversal S = -s (Appendix B: Ising spins s = (0, 0, +-1)) */
    double cone;    /* radians */
    int schedule;   /* 0: permutation of the l^2 offsets per sweep; 1: draw with replacement */
    uint64_t seed;  /* Philox key */
    uint32_t replica;
} orc_params;

static void keyof(uint64_t seed, uint32_t k[2])
{
    k[0] = (uint32_t)(seed & 0xFFFFFFFFu);
    k[1] = (uint32_t)(seed >> 32);
}

/* Number of bits b with 2^b >= v. */
static int ceil_log2(uint32_t v)
{
    int b = 0;
    while ((1u << b) < v) ++b;
    return b;
}

/* Feistel round function: any function gives a bijection; this one mixes with
 * a golden-ratio multiply and a shift. */
static uint32_t feistel_f(uint32_t x, uint32_t rk)
{
    uint32_t y = (x ^ rk) * 0x9E3779B1u;
    y ^= y >> 15;
    return y;
}

/* Offset index v in [0, l^2) for sub-step k of sweep t (v = oy*l + ox).
 * kind 0: a per-sweep pseudo-random permutation of [0, l^2): a 4-round
 *         balanced Feistel network on 2h bits (2^h >= l) keyed by one Philox
 *         draw, with cycle walking back into [0, l^2).
 * kind 1: independent uniform draw per sub-step (the paper's host loop). */
uint32_t orc_offset(uint64_t seed, int l, int kind, uint32_t t, uint32_t k)
{
    uint32_t key[2];
    keyof(seed, key);
    const uint32_t D = (uint32_t)l * (uint32_t)l;
    if (kind == 1) {
        uint32_t c[4] = {t, k, 0u, TAG_DRAW << 24}, o[4];
        orc_philox4x32_10(c, key, o);
        return (uint32_t)(((uint64_t)o[0] * (uint64_t)D) >> 32);
    }
    uint32_t c[4] = {t, 0u, 0u, TAG_PERM << 24}, rk[4];
    orc_philox4x32_10(c, key, rk);
    const int h = ceil_log2((uint32_t)l);
    const uint32_t mask = (h == 0) ? 0u : ((1u << h) - 1u);
    uint32_t v = k;
    /* The walk stays inside the cycle of k, whose length is at most 4^h. */
    for (uint32_t guard = 0; guard <= (1u << (2 * h)); ++guard) {
        uint32_t lo = v & mask, hi = (v >> h) & mask;
        for (int r = 0; r < 4; ++r) {
            uint32_t nlo = hi ^ (feistel_f(lo, rk[r]) & mask);
            hi = lo;
            lo = nlo;
        }
        v = (hi << h) | lo;
        if (v < D) return v;
    }
    return 0xFFFFFFFFu; /* unreachable for a bijection */
}

/* Duff, Burgess, Christensen, Hery, Kensler, Liani, Villemin, "Building an
 * orthonormal basis, revisited" (JCGT 2017): two unit vectors orthogonal to a
 * unit vector n, continuous except across n_z = 0. */
static void perp_basis(const double n[3], double b1[3], double b2[3])
{
    double sign = copysign(1.0, n[2]);
    double a = -1.0 / (sign + n[2]);
    double b = n[0] * n[1] * a;
    b1[0] = 1.0 + sign * n[0] * n[0] * a;
    b1[1] = sign * b;
    b1[2] = -sign * n[0];
    b2[0] = b;
    b2[1] = sign + n[1] * n[1] * a;
    b2[2] = -n[1];
}

/* Proposal S for current spin s from uniforms u1, u2 (Sec. 3.1 proposal; cap
 * of half-angle `cone` when kind 0, whole sphere when kind 1, the complete
 * reversal of Appendix B when kind 2). */
static void propose(int kind, double cone, const double s[3], double u1, double u2, double S[3])
{
    if (kind == 2) {
        for (int c = 0; c < 3; ++c) S[c] = -s[c];
        return;
    }
    double psi = 2.0 * ORC_PI * u2;
    if (kind == 1) {
        double z = 2.0 * u1 - 1.0;
        double r = sqrt(fmax(0.0, 1.0 - z * z));
        S[0] = r * cos(psi);
        S[1] = r * sin(psi);
        S[2] = z;
        return;
    }
    double ca = 1.0 - u1 * (1.0 - cos(cone));
    double sa = sqrt(fmax(0.0, (1.0 - ca) * (1.0 + ca)));
    double b1[3], b2[3];
    perp_basis(s, b1, b2);
    double cp = cos(psi), sp = sin(psi);
    for (int c = 0; c < 3; ++c) S[c] = ca * s[c] + sa * (cp * b1[c] + sp * b2[c]);
    double nrm = sqrt(S[0] * S[0] + S[1] * S[1] + S[2] * S[2]);
    for (int c = 0; c < 3; ++c) S[c] /= nrm;
}

/* Energy change of the single move s_q -> S at site q with field h
 * (Sec. 4 energy; dipole part from Sec. 2.1 Eq. 2 with the self-image term). */
static double delta_e(const orc_params *p, const double *W, const double *s, int qx, int qy,
                      const double h[3], const double S[3])
{
    const int L = p->L, N = L * L;
    int q = qy * L + qx;
    double sq[3] = {s[q], s[N + q], s[2 * N + q]};
    double d[3] = {S[0] - sq[0], S[1] - sq[1], S[2] - sq[2]};
    int nb[4] = {qy * L + wrap(qx + 1, L), qy * L + wrap(qx - 1, L), wrap(qy + 1, L) * L + qx,
                 wrap(qy - 1, L) * L + qx};
    double ns[3] = {0, 0, 0};
    for (int j = 0; j < 4; ++j)
        for (int c = 0; c < 3; ++c) ns[c] += s[c * N + nb[j]];
    double dex = -p->J * (d[0] * ns[0] + d[1] * ns[1] + d[2] * ns[2]);
    double z0 = sq[2], z1 = S[2];
    double dan = (-p->K2 * z1 * z1 - p->K4 * z1 * z1 * z1 * z1) -
                 (-p->K2 * z0 * z0 - p->K4 * z0 * z0 * z0 * z0);
    double w0[3];
    wapply(W, L, 0, 0, d, w0);
    double ddip = p->CD * ((d[0] * h[0] + d[1] * h[1] + d[2] * h[2]) +
                           0.5 * (d[0] * w0[0] + d[1] * w0[1] + d[2] * w0[2]));
    return dex + dan + ddip;
}

/* Observables of one state: out = {|m|, m_z, |m_z|, M_par, E/N, m_st}.
 * m_st (Appendix B): with the four sub-lattices of the 2 x 2 cell, 1 = (x even,
 * y even), 2 = (x odd, y even), 3 = (x odd, y odd), 4 = (x even, y odd), and
 * m_lambda = (1/N) sum_{i in lambda} s_i^z, m_h = m1 + m2 - m3 - m4 (horizontal
 * stripes), m_v = m1 + m4 - m3 - m2 (vertical stripes), m_st = sqrt(m_h^2 + m_v^2). */
static void observe(const orc_params *p, const double *W, const double *s, double *out)
{
    const int L = p->L, N = L * L;
    double mx = 0, my = 0, mz = 0;
    double m[4] = {0, 0, 0, 0};
    for (int i = 0; i < N; ++i) {
        mx += s[i];
        my += s[N + i];
        mz += s[2 * N + i];
        const int x = i % L, y = i / L;
        const int lam = (y & 1) ? ((x & 1) ? 2 : 3) : ((x & 1) ? 1 : 0);   /* 0-based: 1, 2, 3, 4 */
        m[lam] += s[2 * N + i];
    }
    for (int k = 0; k < 4; ++k) m[k] /= N;
    const double mh = m[0] + m[1] - m[2] - m[3], mv = m[0] + m[3] - m[2] - m[1];
    mx /= N;
    my /= N;
    mz /= N;
    double e[4];
    orc_energy(L, W, s, p->J, p->CD, p->K2, p->K4, e);
    out[0] = sqrt(mx * mx + my * my + mz * mz);
    out[1] = mz;
    out[2] = fabs(mz);
    out[3] = sqrt(mx * mx + my * my);
    out[4] = e[3] / N;
    out[5] = sqrt(mh * mh + mv * mv);
    /* Sec. 4.1 domain walls: n_v^a = sum_i 1 - sgn(s_i^a s_{i+y}^a), n_h^a with i+x;
     * wall density (n_v^z + n_h^z)/(4N); orientational order of one state
     * |n_h^a - n_v^a| / (n_h^a + n_v^a) (0 when there is no wall); and the cone
     * angle of one state (2/pi)(1/N) sum_i |theta_i - pi/2|, theta_i = acos s_i^z. */
    double nh[3] = {0, 0, 0}, nv[3] = {0, 0, 0}, cone = 0.0;
    for (int i = 0; i < N; ++i) {
        const int x = i % L, y = i / L;
        const int ix = y * L + (x + 1) % L, iy = ((y + 1) % L) * L + x;
        for (int c = 0; c < 3; ++c) {
            const double a = s[c * N + i];
            const double ph = a * s[c * N + ix], pv = a * s[c * N + iy];
            nh[c] += 1.0 - (ph > 0 ? 1.0 : (ph < 0 ? -1.0 : 0.0));
            nv[c] += 1.0 - (pv > 0 ? 1.0 : (pv < 0 ? -1.0 : 0.0));
        }
        const double zc = fmax(-1.0, fmin(1.0, s[2 * N + i]));
        cone += fabs(acos(zc) - 0.5 * ORC_PI);
    }
    out[6] = (nv[2] + nh[2]) / (4.0 * N);
    for (int c = 0; c < 3; ++c) out[7 + c] = (nh[c] + nv[c] > 0) ? fabs(nh[c] - nv[c]) / (nh[c] + nv[c]) : 0.0;
    out[10] = (2.0 / ORC_PI) * cone / N;
}

/*
 * Decisions of one sub-step (Sec. 3.1 algorithm, Sec. 3.2 approximation): sub-step
 * k of sweep t uses offset o = schedule(t, k); each of the n = (L/l)^2 update sites
 * q = o + l(a, b), in the order d = b*C + a (C = L/l), gets its field, a proposal,
 * dE and the Metropolis decision, all from the state s as given (s is not
 * changed).  Per site d: q[d], h[3d..3d+2], dE[d], u[d], acc[d], S[3d..3d+2].
 */
void orc_substep(const orc_params *p, const double *W, const double *s, uint32_t t, uint32_t k,
                 int32_t *q, double *h, double *dE, double *u, int32_t *acc, double *S)
{
    const int L = p->L, l = p->l;
    const int N = L * L, C = L / l, n = C * C;
    uint32_t key[2];
    keyof(p->seed, key);
    uint32_t v = orc_offset(p->seed, l, p->schedule, t, k);
    int ox = (int)(v % (uint32_t)l), oy = (int)(v / (uint32_t)l);
    for (int d = 0; d < n; ++d) {
        int qx = ox + l * (d % C), qy = oy + l * (d / C);
        int qq = qy * L + qx;
        q[d] = qq;
        field_at(W, L, s, qx, qy, h + 3 * d);
        uint32_t c[4] = {(uint32_t)qq, p->replica, t, (k & 0x00FFFFFFu) | (TAG_ATTEMPT << 24)};
        uint32_t w[4];
        orc_philox4x32_10(c, key, w);
        double sq[3] = {s[qq], s[N + qq], s[2 * N + qq]};
        propose(p->proposal, p->cone, sq, u24(w[0]), u24(w[1]), S + 3 * d);
        dE[d] = delta_e(p, W, s, qx, qy, h + 3 * d, S + 3 * d);
        u[d] = u24(w[2]);
        acc[d] = (u[d] < exp(-dE[d] / p->T)) ? 1 : 0;
    }
}

/* Per-sweep observables and cone-angle sums of the state after sweep `it`. */
static void observe_sweep(const orc_params *p, const double *W, const double *s, int it, double *obs,
                          double *theta2)
{
    const int N = p->L * p->L;
    if (obs) observe(p, W, s, obs + ORC_NOBS * it);
    if (theta2)
        for (int i = 0; i < N; ++i) {
            double zc = fmax(-1.0, fmin(1.0, s[2 * N + i]));
            double dt = acos(zc) - 0.5 * ORC_PI;
            theta2[i] += dt * dt;
        }
}

/*
 * Approximated parallel sweeps (Sec. 3.1 algorithm, Sec. 3.2 approximation).
 * s is [3][L][L], updated in place.  Sweeps t0 .. t0+nsweeps-1; each has l^2
 * sub-steps, decided by orc_substep from the state before the step, after which
 * all accepted moves are applied together.  Trace arrays (may be NULL) hold one
 * record per attempt, in order (sweep, sub-step, site d = Dy*C + Dx with
 * C = L/l):  q (site index), h[3], dE, u, accept, S[3].  obs (may be NULL) gets
 * ORC_NOBS values per sweep; theta2 (may be NULL) accumulates
 * (acos s_z - pi/2)^2 per site per sweep.
 */
int orc_sweeps(const orc_params *p, const double *W, double *s, uint32_t t0, int nsweeps,
               int32_t *tr_q, double *tr_h, double *tr_dE, double *tr_u, int32_t *tr_acc,
               double *tr_S, double *obs, double *theta2)
{
    const int L = p->L, l = p->l;
    if (l < 1 || L % l != 0) return -1;
    const int N = L * L, C = L / l, n = C * C;
    double *hq = (double *)malloc(sizeof(double) * 3 * n);
    double *Sq = (double *)malloc(sizeof(double) * 3 * n);
    double *dE = (double *)malloc(sizeof(double) * n);
    double *u = (double *)malloc(sizeof(double) * n);
    int32_t *acc = (int32_t *)malloc(sizeof(int32_t) * n);
    int32_t *qs = (int32_t *)malloc(sizeof(int32_t) * n);
    size_t rec = 0;
    for (int it = 0; it < nsweeps; ++it) {
        uint32_t t = t0 + (uint32_t)it;
        for (uint32_t k = 0; k < (uint32_t)(l * l); ++k) {
            /* decide every site from the state before the step */
            orc_substep(p, W, s, t, k, qs, hq, dE, u, acc, Sq);
            for (int d = 0; d < n; ++d, ++rec) {
                if (tr_q) tr_q[rec] = qs[d];
                if (tr_h) for (int c3 = 0; c3 < 3; ++c3) tr_h[3 * rec + c3] = hq[3 * d + c3];
                if (tr_dE) tr_dE[rec] = dE[d];
                if (tr_u) tr_u[rec] = u[d];
                if (tr_acc) tr_acc[rec] = acc[d];
                if (tr_S) for (int c3 = 0; c3 < 3; ++c3) tr_S[3 * rec + c3] = Sq[3 * d + c3];
            }
            /* then apply all accepted moves together */
            for (int d = 0; d < n; ++d)
                if (acc[d])
                    for (int c3 = 0; c3 < 3; ++c3) s[c3 * N + qs[d]] = Sq[3 * d + c3];
        }
        observe_sweep(p, W, s, it, obs, theta2);
    }
    free(hq);
    free(Sq);
    free(dE);
    free(u);
    free(acc);
    free(qs);
    return 0;
}

/*
 * Decisions re-synchronised to another trajectory (the decision parity of the
 * simultaneous update, Sec. 3.1, judged per sub-step): the sub-steps of sweeps
 * t0 .. t0+nsweeps-1 are decided in order by orc_substep from the state s, and
 * s then takes the moves that the other trajectory made at that sub-step's sites
 * (ext_acc[rec] = 1: the site becomes ext_S[3 rec .. 3 rec + 2]), whatever the
 * oracle decided.  So every sub-step is decided from the other trajectory's
 * pre-step state (up to the FP32 rounding of ext_S), and one differing decision
 * does not separate the two for the rest of the run.  Records as orc_sweeps.
 */
int orc_replay(const orc_params *p, const double *W, double *s, uint32_t t0, int nsweeps,
               const int32_t *ext_acc, const double *ext_S, int32_t *tr_q, double *tr_h, double *tr_dE,
               double *tr_u, int32_t *tr_acc, double *tr_S)
{
    const int L = p->L, l = p->l;
    if (l < 1 || L % l != 0) return -1;
    const int N = L * L, C = L / l, n = C * C;
    size_t rec = 0;
    for (int it = 0; it < nsweeps; ++it) {
        uint32_t t = t0 + (uint32_t)it;
        for (uint32_t k = 0; k < (uint32_t)(l * l); ++k, rec += (size_t)n) {
            orc_substep(p, W, s, t, k, tr_q + rec, tr_h + 3 * rec, tr_dE + rec, tr_u + rec, tr_acc + rec,
                        tr_S + 3 * rec);
            for (int d = 0; d < n; ++d)
                if (ext_acc[rec + d])
                    for (int c3 = 0; c3 < 3; ++c3) s[c3 * N + tr_q[rec + d]] = ext_S[3 * (rec + d) + c3];
        }
    }
    return 0;
}

/* orc_replay for R independent replicas over all host threads: s is [R][3][L][L],
 * ext and trace arrays are replica-major with nsweeps * L^2 records each. */
int orc_replay_batch(int R, const orc_params *ps, const double *W, double *s, uint32_t t0, int nsweeps,
                     const int32_t *ext_acc, const double *ext_S, int32_t *tr_q, double *tr_h,
                     double *tr_dE, double *tr_u, int32_t *tr_acc, double *tr_S)
{
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int r = 0; r < R; ++r) {
        const size_t N = (size_t)ps[r].L * ps[r].L, m = (size_t)nsweeps * N, o = (size_t)r * m;
        bad |= orc_replay(&ps[r], W, s + (size_t)r * 3 * N, t0, nsweeps, ext_acc + o, ext_S + 3 * o, tr_q + o,
                          tr_h + 3 * o, tr_dE + o, tr_u + o, tr_acc + o, tr_S + 3 * o) != 0;
    }
    return bad ? -1 : 0;
}

/* Several independent replicas (one params struct and one [3][L][L] state
 * each), over all host threads.  obs is [R][nsweeps][5], theta2 [R][N]. */
int orc_sweeps_batch(int R, const orc_params *ps, const double *W, double *s, uint32_t t0,
                     int nsweeps, double *obs, double *theta2)
{
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int r = 0; r < R; ++r) {
        const int N = ps[r].L * ps[r].L;
        bad |= orc_sweeps(&ps[r], W, s + (size_t)r * 3 * N, t0, nsweeps, NULL, NULL, NULL, NULL,
                          NULL, NULL, obs ? obs + (size_t)r * nsweeps * ORC_NOBS : NULL,
                          theta2 ? theta2 + (size_t)r * N : NULL) != 0;
    }
    return bad ? -1 : 0;
}

/*
 * Exact sequential single-spin Metropolis written independently of the
 * simultaneous update: sites are visited one at a time in the order the
 * permutation schedule with l = L gives, and dE is the difference of two
 * full-energy evaluations (O(N^2) per attempt; meant for L <= 8).
 * Trace: dE and accept per attempt.
 */
int orc_sweeps_exact(const orc_params *p, const double *W, double *s, uint32_t t0, int nsweeps,
                     double *tr_dE, int32_t *tr_acc)
{
    const int L = p->L, N = L * L;
    uint32_t key[2];
    keyof(p->seed, key);
    double *trial = (double *)malloc(sizeof(double) * 3 * N);
    size_t rec = 0;
    for (int it = 0; it < nsweeps; ++it) {
        uint32_t t = t0 + (uint32_t)it;
        for (uint32_t k = 0; k < (uint32_t)N; ++k) {
            uint32_t q = orc_offset(p->seed, L, p->schedule, t, k);
            uint32_t c[4] = {q, p->replica, t, (k & 0x00FFFFFFu) | (TAG_ATTEMPT << 24)};
            uint32_t w[4];
            orc_philox4x32_10(c, key, w);
            double sq[3] = {s[q], s[N + q], s[2 * N + q]};
            double S[3];
            propose(p->proposal, p->cone, sq, u24(w[0]), u24(w[1]), S);
            memcpy(trial, s, sizeof(double) * 3 * N);
            for (int c3 = 0; c3 < 3; ++c3) trial[c3 * N + q] = S[c3];
            double e0[4], e1[4];
            orc_energy(L, W, s, p->J, p->CD, p->K2, p->K4, e0);
            orc_energy(L, W, trial, p->J, p->CD, p->K2, p->K4, e1);
            double dE = e1[3] - e0[3];
            int a = (u24(w[2]) < exp(-dE / p->T)) ? 1 : 0;
            if (a) memcpy(s, trial, sizeof(double) * 3 * N);
            if (tr_dE) tr_dE[rec] = dE;
            if (tr_acc) tr_acc[rec] = a;
            ++rec;
        }
    }
    free(trial);
    return 0;
}

/* Random Ising initial spins (Appendix B): s = (0, 0, +1) if u0 < 1/2 else
 * (0, 0, -1), u0 from the counter (site, replica, 0, TAG_INIT). */
void orc_init_ising(int L, uint64_t seed, uint32_t replica, double *s)
{
    const int N = L * L;
    uint32_t key[2];
    keyof(seed, key);
    for (int i = 0; i < N; ++i) {
        uint32_t c[4] = {(uint32_t)i, replica, 0u, TAG_INIT << 24}, w[4];
        orc_philox4x32_10(c, key, w);
        s[i] = 0.0;
        s[N + i] = 0.0;
        s[2 * N + i] = u24(w[0]) < 0.5 ? 1.0 : -1.0;
    }
}

/* Random-uniform initial spins on S^2 from the seed (counter = site, replica,
 * 0, TAG_INIT): z = 2 u0 - 1, azimuth 2 pi u1. */
void orc_init_random(int L, uint64_t seed, uint32_t replica, double *s)
{
    const int N = L * L;
    uint32_t key[2];
    keyof(seed, key);
    for (int i = 0; i < N; ++i) {
        uint32_t c[4] = {(uint32_t)i, replica, 0u, TAG_INIT << 24}, w[4];
        orc_philox4x32_10(c, key, w);
        double z = 2.0 * u24(w[0]) - 1.0;
        double r = sqrt(fmax(0.0, 1.0 - z * z));
        double ph = 2.0 * ORC_PI * u24(w[1]);
        s[i] = r * cos(ph);
        s[N + i] = r * sin(ph);
        s[2 * N + i] = z;
    }
}

/* Cone angle eta (Sec. 4.1, cone-angle equation) from per-site accumulated
 * (theta - pi/2)^2 over `count` samples. */
double orc_eta(int N, const double *theta2, double count)
{
    double acc = 0.0;
    for (int i = 0; i < N; ++i) acc += sqrt((2.0 / ORC_PI) * (2.0 / ORC_PI) * theta2[i] / count);
    return acc / N;
}

/* Pair error of two simultaneous flips (Sec. 3.2, epsilon_12 equation):
 * D = |d1.d2 - 3 (d1.r^)(d2.r^)| with r^ the unit vector between the sites;
 * returns C_D D / r^3. */
double orc_eps12(const double d1[3], const double d2[3], const double rvec[3], double CD)
{
    double r = sqrt(rvec[0] * rvec[0] + rvec[1] * rvec[1] + rvec[2] * rvec[2]);
    double u[3] = {rvec[0] / r, rvec[1] / r, rvec[2] / r};
    double d12 = d1[0] * d2[0] + d1[1] * d2[1] + d1[2] * d2[2];
    double a = d1[0] * u[0] + d1[1] * u[1] + d1[2] * u[2];
    double b = d2[0] * u[0] + d2[1] * u[1] + d2[2] * u[2];
    return CD * fabs(d12 - 3.0 * a * b) / (r * r * r);
}

/* Error of the flip probability (Sec. 3.2, epsilon_Total equation, divided by
 * k_B T), with D = 2.
 * mode 0: the other update sites of one cell only (no images) -- the reading
 *         that reproduces the worked example at the end of Sec. 3.2;
 * mode 1: every other site of the update sublattice l Z^2 over all images,
 *         truncated at |lv| <= A L (A image cells each way). */
double orc_eps_total(int L, int l, double CD, double T, int mode, int A)
{
    const int C = L / l;
    double acc = 0.0;
    if (mode == 0) {
        for (int b = 0; b < C; ++b)
            for (int a = 0; a < C; ++a) {
                if (a == 0 && b == 0) continue;
                /* nearest periodic image of the displacement within the cell */
                double dx = (double)(a * l), dy = (double)(b * l);
                if (dx > 0.5 * L) dx -= L;
                if (dy > 0.5 * L) dy -= L;
                double r = sqrt(dx * dx + dy * dy);
                acc += 2.0 * CD / (r * r * r);
            }
    } else {
        const int M = A * C;
        for (int b = -M; b <= M; ++b)
            for (int a = -M; a <= M; ++a) {
                if (a == 0 && b == 0) continue;
                double r = (double)l * sqrt((double)a * a + (double)b * b);
                acc += 2.0 * CD / (r * r * r);
            }
    }
    return acc / T;
}

/* Exported proposal, for checking its distribution. */
void orc_propose(int kind, double cone, const double s[3], double u1, double u2, double S[3])
{
    propose(kind, cone, s, u1, u2, S);
}
