// Ewald correction table (Secs. 2.2.3-2.2.5, App. A), generated in FP64 on the device.
//
// For a unit mass and all its periodic images, phi is the Ewald sum of eq. ewpotential (3P),
// eq. potential2p1i (2P1I, Fourier factor I~ of eq. intijscaled and I(0,0) of eq. int00) or
// eq. potential1p2i (1P2I, Fourier integrals K of eq. int00p1 and M of eq. e4fceM by Gauss-Legendre
// quadrature), with alpha = 2/Lx, real-space images i1^2 + (b i2)^2 + (c i3)^2 <= 15 and Fourier
// terms l1^2 + (l2/b)^2 + (l3/c)^2 <= 10.  The table stores the smooth remainder
//   C = phi - 1/|d|,  A_c = A - d/|d|^3,  A = -grad phi,
// on the folded grid d = (i ex, j ey, k ez)/(n-1); the singular part of the i = 0 image is removed
// analytically (series in alpha r near the origin).
//
// 3P includes the neutralising-background constant -pi/(alpha^2 V) so that the potential of a
// uniform box averages to zero.  For 1P2I the divergent constant of K(0, eta) is dropped, as the
// paper does for I(0,0) of 2P1I.
//
// Cost: one thread per table point, ~400 (3P) to ~10^4 (1P2I quadrature) FP64 terms; run once.
#include <math.h>

#include <vector>

#include "ts_internal.cuh"

#define EW_GL_PTS 16
#define EW_GL_PANELS 96

__constant__ double c_gl_x[EW_GL_PTS];
__constant__ double c_gl_w[EW_GL_PTS];

struct EwGen {
    int kind, n;
    double Lx, b, c, alpha, zeta;
    double ext[3];
    double rcut2, kcut2;
};

// i = 0 image with its 1/r (and d/r^3) removed: returns f_phi and f_A such that the image adds
// f_phi to C and f_A * d to A_c.
__device__ void self_image(double alpha, double u, double& fp, double& fa) {
    const double r = sqrt(u), x = alpha * r;
    const double two_over_sqrtpi = 1.1283791670955126;
    if (x < 0.05) {
        // -erf(x)/r = -(2 alpha/sqrt(pi)) sum_m (-1)^m x^{2m} / (m! (2m+1))
        // [2a/sqrt(pi) e^{-x^2}/u - erf(x)/r^3] = (2 a^3/sqrt(pi)) sum_m (-1)^{m+1} 2 x^{2m} / (m! (2m+3))
        const double x2 = x * x;
        double term = 1.0, sp = 0, sa = 0;
        for (int m = 0; m < 8; ++m) {
            if (m) term *= -x2 / m;
            sp += term / (2 * m + 1);
            sa -= 2.0 * term / (2 * m + 3);
        }
        fp = -alpha * two_over_sqrtpi * sp;
        fa = alpha * alpha * alpha * two_over_sqrtpi * sa;
    } else {
        const double ef = erf(x);
        fp = -ef / r;
        fa = alpha * two_over_sqrtpi * exp(-x * x) / u - ef / (u * r);
    }
}

__device__ void image(double alpha, double u, double& fp, double& fa) {
    const double r = sqrt(u), x = alpha * r;
    const double ec = erfc(x);
    fp = ec / r;
    fa = alpha * 1.1283791670955126 * exp(-x * x) / u + ec / (u * r);
}

__device__ void corr_3p(const EwGen& g, const double d[3], double out[4]) {
    double C = 0, A0 = 0, A1 = 0, A2 = 0;
    const double Lx = g.Lx, Ly = g.b * g.Lx, Lz = g.c * g.Lx;
    const int m1 = (int)floor(sqrt(g.rcut2)), m2 = (int)floor(sqrt(g.rcut2) / g.b), m3 = (int)floor(sqrt(g.rcut2) / g.c);
    for (int i3 = -m3; i3 <= m3; ++i3)
        for (int i2 = -m2; i2 <= m2; ++i2)
            for (int i1 = -m1; i1 <= m1; ++i1) {
                const double q = (double)i1 * i1 + g.b * g.b * i2 * i2 + g.c * g.c * i3 * i3;
                if (q > g.rcut2) continue;
                const double v0 = d[0] - i1 * Lx, v1 = d[1] - i2 * Ly, v2 = d[2] - i3 * Lz;
                const double u = v0 * v0 + v1 * v1 + v2 * v2;
                double fp, fa;
                if (i1 == 0 && i2 == 0 && i3 == 0) self_image(g.alpha, u, fp, fa);
                else image(g.alpha, u, fp, fa);
                C += fp; A0 += fa * v0; A1 += fa * v1; A2 += fa * v2;
            }
    const double V = Lx * Ly * Lz;
    const int l1m = (int)floor(sqrt(g.kcut2)), l2m = (int)floor(sqrt(g.kcut2) * g.b), l3m = (int)floor(sqrt(g.kcut2) * g.c);
    for (int l3 = -l3m; l3 <= l3m; ++l3)
        for (int l2 = -l2m; l2 <= l2m; ++l2)
            for (int l1 = -l1m; l1 <= l1m; ++l1) {
                const double s2 = (double)l1 * l1 + (l2 / g.b) * (l2 / g.b) + (l3 / g.c) * (l3 / g.c);
                if (s2 == 0 || s2 > g.kcut2) continue;
                const double k0 = 2 * M_PI * l1 / Lx, k1 = 2 * M_PI * l2 / Ly, k2 = 2 * M_PI * l3 / Lz;
                const double kk = k0 * k0 + k1 * k1 + k2 * k2;
                const double amp = 4 * M_PI / (V * kk) * exp(-kk / (4 * g.alpha * g.alpha));
                double sn, cs;
                sincos(k0 * d[0] + k1 * d[1] + k2 * d[2], &sn, &cs);
                C += amp * cs;
                A0 += amp * k0 * sn; A1 += amp * k1 * sn; A2 += amp * k2 * sn;
            }
    C -= M_PI / (g.alpha * g.alpha * V);
    out[0] = C; out[1] = A0; out[2] = A1; out[3] = A2;
}

__device__ void corr_2p1i(const EwGen& g, const double d[3], double out[4]) {
    double C = 0, A0 = 0, A1 = 0, A2 = 0;
    const double Lx = g.Lx, Ly = g.b * g.Lx;
    const int m1 = (int)floor(sqrt(g.rcut2)), m2 = (int)floor(sqrt(g.rcut2) / g.b);
    for (int i2 = -m2; i2 <= m2; ++i2)
        for (int i1 = -m1; i1 <= m1; ++i1) {
            if ((double)i1 * i1 + g.b * g.b * i2 * i2 > g.rcut2) continue;
            const double v0 = d[0] - i1 * Lx, v1 = d[1] - i2 * Ly, v2 = d[2];
            const double u = v0 * v0 + v1 * v1 + v2 * v2;
            double fp, fa;
            if (i1 == 0 && i2 == 0) self_image(g.alpha, u, fp, fa);
            else image(g.alpha, u, fp, fa);
            C += fp; A0 += fa * v0; A1 += fa * v1; A2 += fa * v2;
        }
    const double zeta = g.zeta, sz = sqrt(zeta);
    const double gam = 2 * M_PI * d[2] / Lx, ag = fabs(gam);
    const double sgn = gam < 0 ? -1.0 : 1.0;
    const int l1m = (int)floor(sqrt(g.kcut2)), l2m = (int)floor(sqrt(g.kcut2) * g.b);
    for (int l2 = -l2m; l2 <= l2m; ++l2)
        for (int l1 = -l1m; l1 <= l1m; ++l1) {
            const double s2 = (double)l1 * l1 + (l2 / g.b) * (l2 / g.b);
            if (s2 > g.kcut2) continue;
            double It, Ip;
            if (s2 == 0) {
                It = -M_PI * (ag * erf(ag / (2 * sz)) + 2 * sqrt(zeta / M_PI) * exp(-ag * ag / (4 * zeta))) +
                     2 * sqrt(M_PI * zeta);
                Ip = -M_PI * erf(ag / (2 * sz));
            } else {
                const double s = sqrt(s2);
                const double p = exp(-ag * ag / (4 * zeta) - zeta * s2) * erfcx((zeta * s + ag / 2) / sz);
                const double m = exp(-ag * s) * erfc((zeta * s - ag / 2) / sz);
                It = M_PI / (2 * s) * (p + m);
                Ip = M_PI / 2 * (p - m);
            }
            double sn, cs;
            sincos(2 * M_PI * l1 * d[0] / Lx + 2 * M_PI * l2 * d[1] / Ly, &sn, &cs);
            C += cs * It / (M_PI * Lx * g.b);
            A0 += 2.0 * l1 * sn * It / (g.b * Lx * Lx);
            A1 += 2.0 * l2 * sn * It / (g.b * g.b * Lx * Lx);
            A2 -= 2.0 * cs * sgn * Ip / (g.b * Lx * Lx);
        }
    out[0] = C; out[1] = A0; out[2] = A1; out[3] = A2;
}

// K(l1, eta) and M(l1, eta) of the 1P2I Fourier term by composite Gauss-Legendre on [0, Q],
// exp(-zeta Q^2) = e^-46.
__device__ void km_quad(int l1, double eta, double zeta, double& K, double& M) {
    const double Q = sqrt(46.0 / zeta), h = Q / EW_GL_PANELS, l2 = (double)l1 * l1;
    double sk = 0, sm = 0;
    for (int p = 0; p < EW_GL_PANELS; ++p)
        for (int i = 0; i < EW_GL_PTS; ++i) {
            const double q = h * (p + 0.5 * (c_gl_x[i] + 1.0)), w = 0.5 * h * c_gl_w[i];
            const double gq = exp(-zeta * q * q);
            const double b0 = j0(eta * q), b1 = j1(eta * q);
            sk += l1 ? w * b0 * gq * q / (l2 + q * q) : w * (b0 - 1.0) * gq / q;
            sm += w * b1 * gq * q * q / (l2 + q * q);
        }
    K = sk;
    M = sm;
}

__device__ void corr_1p2i(const EwGen& g, const double d[3], double out[4]) {
    double C = 0, A0 = 0, A1 = 0, A2 = 0;
    const double Lx = g.Lx;
    const int m1 = (int)floor(sqrt(g.rcut2));
    for (int i1 = -m1; i1 <= m1; ++i1) {
        const double v0 = d[0] - i1 * Lx;
        const double u = v0 * v0 + d[1] * d[1] + d[2] * d[2];
        double fp, fa;
        if (i1 == 0) self_image(g.alpha, u, fp, fa);
        else image(g.alpha, u, fp, fa);
        C += fp; A0 += fa * v0; A1 += fa * d[1]; A2 += fa * d[2];
    }
    const double R = sqrt(d[1] * d[1] + d[2] * d[2]), eta = 2 * M_PI * R / Lx;
    const int l1m = (int)floor(sqrt(g.kcut2));
    double sumM = 0;
    for (int l1 = -l1m; l1 <= l1m; ++l1) {
        double K, M;
        km_quad(l1 < 0 ? -l1 : l1, eta, g.zeta, K, M);
        const double e = exp(-g.zeta * l1 * l1);
        double sn, cs;
        sincos(2 * M_PI * l1 * d[0] / Lx, &sn, &cs);
        C += 2.0 / Lx * e * cs * K;
        A0 += 4 * M_PI / (Lx * Lx) * l1 * e * sn * K;
        sumM += e * cs * M;
    }
    if (R > 0) {
        A1 += 4 * M_PI / (Lx * Lx) * d[1] / R * sumM;
        A2 += 4 * M_PI / (Lx * Lx) * d[2] / R * sumM;
    }
    out[0] = C; out[1] = A0; out[2] = A1; out[3] = A2;
}

__global__ void k_ewald_table(EwGen g, double* __restrict__ out) {
    const int64_t npts = (int64_t)g.n * g.n * g.n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < npts; t += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(t % g.n), j = (int)((t / g.n) % g.n), i = (int)(t / ((int64_t)g.n * g.n));
        const double d[3] = {g.ext[0] * i / (g.n - 1), g.ext[1] * j / (g.n - 1), g.ext[2] * k / (g.n - 1)};
        double r[4];
        if (g.kind == TS_EW_3P) corr_3p(g, d, r);
        else if (g.kind == TS_EW_2P1I) corr_2p1i(g, d, r);
        else corr_1p2i(g, d, r);
        out[4 * t] = r[0]; out[4 * t + 1] = r[1]; out[4 * t + 2] = r[2]; out[4 * t + 3] = r[3];
    }
}

// First-order Taylor table (Sec. 2.2.5, approach 2): at every grid point the correction and the
// Jacobian J_ij = dA_c,i/dd_j of its acceleration part by central differences of the series with
// step eps (A_c is a gradient field, so J is symmetrised).  Records of 4 dbl4 per point:
// (C, A_cx, A_cy, A_cz), (Jxx, Jyy, Jzz, Jxy), (Jxz, Jyz, 0, 0), 0.
__device__ void corr_any(const EwGen& g, const double d[3], double out[4]) {
    if (g.kind == TS_EW_3P) corr_3p(g, d, out);
    else if (g.kind == TS_EW_2P1I) corr_2p1i(g, d, out);
    else corr_1p2i(g, d, out);
}

__global__ void k_ewald_taylor(EwGen g, double eps, dbl4* __restrict__ out) {
    const int64_t npts = (int64_t)g.n * g.n * g.n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < npts; t += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(t % g.n), j = (int)((t / g.n) % g.n), i = (int)(t / ((int64_t)g.n * g.n));
        const double d[3] = {g.ext[0] * i / (g.n - 1), g.ext[1] * j / (g.n - 1), g.ext[2] * k / (g.n - 1)};
        double v[4], J[3][3];
        corr_any(g, d, v);
        for (int c = 0; c < 3; ++c) {
            double dp[3] = {d[0], d[1], d[2]}, dm[3] = {d[0], d[1], d[2]}, vp[4], vm[4];
            dp[c] += eps;
            dm[c] -= eps;
            corr_any(g, dp, vp);
            corr_any(g, dm, vm);
            for (int r = 0; r < 3; ++r) J[r][c] = (vp[1 + r] - vm[1 + r]) / (2 * eps);
        }
        dbl4* o = out + 4 * t;
        o[0] = dbl4{v[0], v[1], v[2], v[3]};
        o[1] = dbl4{J[0][0], J[1][1], J[2][2], 0.5 * (J[0][1] + J[1][0])};
        o[2] = dbl4{0.5 * (J[0][2] + J[2][0]), 0.5 * (J[1][2] + J[2][1]), 0.0, 0.0};
        o[3] = dbl4{0.0, 0.0, 0.0, 0.0};
    }
}

// Gauss-Legendre nodes and weights on [-1, 1]: roots of P_n by Newton's method on the three-term
// recurrence, w = 2 / ((1 - x^2) P_n'(x)^2).
static void legendre_rule(int n, double* x, double* w) {
    for (int i = 0; i < n; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1;
        for (int it = 0; it < 200; ++it) {
            double p0 = 1, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1);
            const double step = p1 / dp;
            z -= step;
            if (fabs(step) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1 - z * z) * dp * dp);
    }
}

static cudaError_t ewald_setup(ts_ctx* c, int n, EwGen& g);

static int ewald_grid(ts_ctx* c, int n) {
    int nsm = 152;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
    const int64_t npts = (int64_t)n * n * n;
    return (int)std::min<int64_t>((npts + 127) / 128, (int64_t)nsm * 16);
}

cudaError_t launch_ewald_table(ts_ctx* c, int n, double* d_out) {
    EwGen g;
    cudaError_t e = ewald_setup(c, n, g);
    if (e != cudaSuccess) return e;
    k_ewald_table<<<ewald_grid(c, n), 128, 0, c->stream>>>(g, d_out);
    return cudaGetLastError();
}

cudaError_t launch_ewald_taylor(ts_ctx* c, int n, double eps, dbl4* d_out) {
    EwGen g;
    cudaError_t e = ewald_setup(c, n, g);
    if (e != cudaSuccess) return e;
    k_ewald_taylor<<<ewald_grid(c, n), 128, 0, c->stream>>>(g, eps, d_out);
    return cudaGetLastError();
}

// series parameters of the context's BCs and box; uploads the quadrature rule for 1P2I
static cudaError_t ewald_setup(ts_ctx* c, int n, EwGen& g) {
    g.kind = c->ew.kind;
    g.n = n;
    g.Lx = c->L[0];
    g.b = c->L[1] / c->L[0];
    g.c = c->L[2] / c->L[0];
    g.alpha = 2.0 / c->L[0];
    g.zeta = M_PI * M_PI / (g.alpha * g.Lx * g.alpha * g.Lx);
    for (int a = 0; a < 3; ++a) g.ext[a] = c->ew.ext[a];
    g.rcut2 = 15.0;
    g.kcut2 = 10.0;
    if (g.kind == TS_EW_1P2I) {
        double x[EW_GL_PTS], w[EW_GL_PTS];
        legendre_rule(EW_GL_PTS, x, w);
        cudaError_t e = cudaMemcpyToSymbolAsync(c_gl_x, x, sizeof(x), 0, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_gl_w, w, sizeof(w), 0, cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) return e;
        // host arrays must outlive the async copies
        e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// ------------------------------------------------------------------------------ training samples
// Random separations of the 2P1I surrogate's domain, one per thread: features (u, v, w, beta)
// uniform in [0,1]^4 from a counter-based hash of (seed, sample, component); box Lx = 1,
// Ly = b = b_min + beta (b_max - b_min); d = (u/2, b v/2, F w) with F = 2 max(1, b); targets are the
// FP64 correction (C, A_c) of the series above.  Stored features are 2 t - 1 for
// t = u, v, |dz|/F_net (F_net = 2 max(1, b_max)), beta.
__device__ __forceinline__ double hash_uniform(uint64_t seed, uint64_t i, uint64_t k) {
    uint64_t x = seed + 0x9E3779B97F4A7C15ull * (i + 1) + 0xBF58476D1CE4E5B9ull * (k + 1);
    x ^= x >> 30; x *= 0xBF58476D1CE4E5B9ull;
    x ^= x >> 27; x *= 0x94D049BB133111EBull;
    x ^= x >> 31;
    return (double)(x >> 11) * (1.0 / 9007199254740992.0);
}

__global__ void k_ewald_samples_2p1i(int64_t n, double bmin, double bmax, uint64_t seed, double zpow,
                                     float* __restrict__ feat, double* __restrict__ targ) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const double u = hash_uniform(seed, s, 0), v = hash_uniform(seed, s, 1),
                     w = pow(hash_uniform(seed, s, 2), zpow), be = hash_uniform(seed, s, 3);
        EwGen g;
        g.kind = TS_EW_2P1I;
        g.n = 2;
        g.Lx = 1.0;
        g.b = bmin + be * (bmax - bmin);
        g.c = 1.0;
        g.alpha = 2.0;
        g.zeta = M_PI * M_PI / 4.0;
        g.rcut2 = 15.0;
        g.kcut2 = 10.0;
        const double F = 2.0 * fmax(1.0, g.b);
        g.ext[0] = 0.5; g.ext[1] = 0.5 * g.b; g.ext[2] = F;
        const double d[3] = {0.5 * u, 0.5 * g.b * v, F * w};
        double r[4];
        corr_2p1i(g, d, r);
        feat[4 * s] = (float)(2 * u - 1); feat[4 * s + 1] = (float)(2 * v - 1);
        // |dz| in units of the far distance of the widest box covered (b_max), constant over b
        const double Fnet = 2.0 * fmax(1.0, bmax);
        feat[4 * s + 2] = (float)(2 * (F * w / Fnet) - 1); feat[4 * s + 3] = (float)(2 * be - 1);
        for (int c = 0; c < 4; ++c) targ[4 * s + c] = r[c];
    }
}

cudaError_t launch_ewald_samples_2p1i(cudaStream_t st, int64_t n, double bmin, double bmax, uint64_t seed,
                                      double zpow, float* feat, double* targ) {
    const int grid = (int)std::min<int64_t>((n + 127) / 128, 152 * 16);
    k_ewald_samples_2p1i<<<grid, 128, 0, st>>>(n, bmin, bmax, seed, zpow > 0 ? zpow : 1.0, feat, targ);
    return cudaGetLastError();
}
