/*
 * FP64 CPU oracle for the tree-based gravity and optical-depth solver of Wünsch et al. (2018),
 * "Tree-based solvers for adaptive mesh refinement code FLASH - I: gravity and optical depths".
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the tests, the smoke
 * check and the CPU-baseline leg of the benchmark compare the CUDA library against.  It shares no
 * code, header, table or constant generator with the CUDA library, and the library never calls
 * it.  Everything is double precision; loops follow the paper's definitions in its order, with
 * OpenMP only over independent target cells.
 *
 * Units: G is a parameter (default 1).  Mesh layout: see the comment at the top of inputs.py
 * (level, child[8], lo[3], size[3] per block; block 0 = root; rho[leaf][k][j][i]).
 *
 * Parity status per function (what pins it lives in tests/test_oracle_*.py):
 *   or_tree_build        pinned (total mass, analytic centre of mass, brute-force moments)
 *   or_gravity_walk      pinned (theta->0 equals or_direct_sum; uniform-sphere closed form; the
 *                        MPE walk's error is below the sum of its per-node bounds)
 *   or_tree_bmoments     pinned (numpy sums over cells; uniform-node closed form)
 *   or_direct_sum        pinned (uniform sphere, Plummer, Jeans sine wave, uniform periodic box)
 *   or_ewald             pinned (alpha invariance, Madelung constant, sheet and line asymptotes,
 *                                isothermal layer / Gauss's law for the cylinder)
 *   or_ewald_table       pinned through or_ewald (the table is or_ewald's correction on a grid)
 *   or_ewald_taylor_table pinned (trace of J = -4 pi / V for 3P and 0 for 2P1I / 1P2I, J against
 *                        differences of the table values, second-order convergence of the lookup)
 *   or_healpix_*         pinned (pix2ang/ang2pix round trip, equal-area histogram, ring latitudes)
 *   or_noderay_table     parity unpinned against the paper (the paper gives only the table axes);
 *                        pinned to its own definition: weights sum to one, point limit, and the
 *                        symmetries that the cube shares with the HEALPix grid.
 *   or_column_walk       pinned (uniform-sphere centre column rho*R, slab, conservation)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NB 8                 /* cells per block edge, 2^l_bt with l_bt = 3 (Sec. 2) */
#define NCB (NB * NB * NB)   /* cells per block */

/* ======================================================================================
 * Tree build (Sec. 2.1): masses summed bottom-up; each node stores total mass and centre of
 * mass.  Block-tree levels inside a leaf-block: 8 nodes (level l_lb+1), 64 nodes (l_lb+2),
 * 512 cells (l_lb+3).  Index conventions inside a leaf-block:
 *   level-1 node q = qx + 2 qy + 4 qz (qx in 0..1), level-2 node p = px + 4 py + 16 pz
 *   (px in 0..3), cell c = i + 8 j + 64 k.
 * ====================================================================================== */
typedef struct {
    int nb, nleaf;
    const int *level, *child;
    const double *lo, *size;
    int *leaf_of;        /* [nb] leaf index or -1 */
    int *block_of;       /* [nleaf] block index */
    double *bM, *bC;     /* [nb], [nb][3] */
    double *n1M, *n1C;   /* [nleaf][8], [nleaf][8][3] */
    double *n2M, *n2C;   /* [nleaf][64], [nleaf][64][3] */
    double *cm;          /* [nleaf][512] cell masses */
    double *bB, *n1B, *n2B;   /* MPE moments (B2, B3) per node, [nb][2], [nleaf][8][2], [nleaf][64][2] */
    double L[3];         /* domain edge lengths */
    int bc[3];
} otree;

static void cell_centre(const otree* T, int b, int i, int j, int k, double r[3]) {
    r[0] = T->lo[3 * b + 0] + (i + 0.5) * T->size[3 * b + 0] / NB;
    r[1] = T->lo[3 * b + 1] + (j + 0.5) * T->size[3 * b + 1] / NB;
    r[2] = T->lo[3 * b + 2] + (k + 0.5) * T->size[3 * b + 2] / NB;
}

/* Moments of a non-leaf block: sum over its 8 child blocks in child order (post-order). */
static void build_block(otree* T, int b) {
    if (T->child[8 * b] < 0) return;
    double M = 0, S[3] = {0, 0, 0};
    for (int c = 0; c < 8; ++c) {
        int cb = T->child[8 * b + c];
        build_block(T, cb);
        M += T->bM[cb];
        for (int a = 0; a < 3; ++a) S[a] += T->bM[cb] * T->bC[3 * cb + a];
    }
    T->bM[b] = M;
    for (int a = 0; a < 3; ++a)
        T->bC[3 * b + a] = M > 0 ? S[a] / M : T->lo[3 * b + a] + 0.5 * T->size[3 * b + a];
}

static void otree_free(otree* T) {
    free(T->leaf_of); free(T->block_of); free(T->bM); free(T->bC);
    free(T->n1M); free(T->n1C); free(T->n2M); free(T->n2C); free(T->cm);
    free(T->bB); free(T->n1B); free(T->n2B);
}

/* ---- multipole moments of the MPE MAC (Sec. 2.2.1, eq. mpe): B_p = sum_i |m_i| |r_i - r_a|^p
 * over the grid cells i of a node, r_a the node's centre of mass; p = 2 and 3 for monopoles. */
static void cells_bmom(const otree* T, int b, int i0, int i1, int j0, int j1, int k0, int k1,
                       const double ra[3], double* B2, double* B3) {
    int n = T->leaf_of[b];
    for (int k = k0; k < k1; ++k)
        for (int j = j0; j < j1; ++j)
            for (int i = i0; i < i1; ++i) {
                double r[3];
                cell_centre(T, b, i, j, k, r);
                double m = fabs(T->cm[(size_t)n * NCB + i + NB * j + NB * NB * k]);
                double u = (r[0] - ra[0]) * (r[0] - ra[0]) + (r[1] - ra[1]) * (r[1] - ra[1]) +
                           (r[2] - ra[2]) * (r[2] - ra[2]);
                *B2 += m * u;
                *B3 += m * u * sqrt(u);
            }
}

static void block_bmom(const otree* T, int b, const double ra[3], double* B2, double* B3) {
    if (T->child[8 * b] >= 0) {
        for (int c = 0; c < 8; ++c) block_bmom(T, T->child[8 * b + c], ra, B2, B3);
        return;
    }
    cells_bmom(T, b, 0, NB, 0, NB, 0, NB, ra, B2, B3);
}

static int otree_bmoments(otree* T) {
    if (T->bB) return 0;
    T->bB = (double*)calloc(2 * (size_t)T->nb, sizeof(double));
    T->n1B = (double*)calloc(16 * (size_t)T->nleaf, sizeof(double));
    T->n2B = (double*)calloc(128 * (size_t)T->nleaf, sizeof(double));
    if (!T->bB || !T->n1B || !T->n2B) return -1;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int b = 0; b < T->nb; ++b) block_bmom(T, b, &T->bC[3 * b], &T->bB[2 * b], &T->bB[2 * b + 1]);
    #pragma omp parallel for schedule(static)
    for (int n = 0; n < T->nleaf; ++n) {
        int b = T->block_of[n];
        for (int q = 0; q < 8; ++q) {
            int qx = q & 1, qy = (q >> 1) & 1, qz = q >> 2;
            double* o = &T->n1B[(n * 8 + q) * 2];
            cells_bmom(T, b, 4 * qx, 4 * qx + 4, 4 * qy, 4 * qy + 4, 4 * qz, 4 * qz + 4,
                       &T->n1C[(n * 8 + q) * 3], o, o + 1);
        }
        for (int p = 0; p < 64; ++p) {
            int px = p & 3, py = (p >> 2) & 3, pz = p >> 4;
            double* o = &T->n2B[(n * 64 + p) * 2];
            cells_bmom(T, b, 2 * px, 2 * px + 2, 2 * py, 2 * py + 2, 2 * pz, 2 * pz + 2,
                       &T->n2C[(n * 64 + p) * 3], o, o + 1);
        }
    }
    return 0;
}

static int otree_build(otree* T, int nb, const int* level, const int* child, const double* lo,
                       const double* size, const double* rho, const int* bc) {
    memset(T, 0, sizeof(*T));
    T->nb = nb; T->level = level; T->child = child; T->lo = lo; T->size = size;
    for (int a = 0; a < 3; ++a) { T->L[a] = size[a]; T->bc[a] = bc ? bc[a] : 0; }
    T->leaf_of = (int*)malloc(sizeof(int) * nb);
    int nleaf = 0;
    for (int b = 0; b < nb; ++b) T->leaf_of[b] = child[8 * b] < 0 ? nleaf++ : -1;
    T->nleaf = nleaf;
    T->block_of = (int*)malloc(sizeof(int) * (nleaf ? nleaf : 1));
    for (int b = 0; b < nb; ++b) if (T->leaf_of[b] >= 0) T->block_of[T->leaf_of[b]] = b;
    T->bM = (double*)calloc(nb, sizeof(double));
    T->bC = (double*)calloc(3 * nb, sizeof(double));
    T->n1M = (double*)calloc((size_t)nleaf * 8, sizeof(double));
    T->n1C = (double*)calloc((size_t)nleaf * 24, sizeof(double));
    T->n2M = (double*)calloc((size_t)nleaf * 64, sizeof(double));
    T->n2C = (double*)calloc((size_t)nleaf * 192, sizeof(double));
    T->cm = (double*)calloc((size_t)nleaf * NCB, sizeof(double));
    if (!T->bM || !T->bC || !T->n1M || !T->n1C || !T->n2M || !T->n2C || !T->cm) return -1;

    #pragma omp parallel for schedule(static)
    for (int n = 0; n < nleaf; ++n) {
        int b = T->block_of[n];
        double dV = (size[3 * b] / NB) * (size[3 * b + 1] / NB) * (size[3 * b + 2] / NB);
        for (int c = 0; c < NCB; ++c) T->cm[(size_t)n * NCB + c] = rho[(size_t)n * NCB + c] * dV;
        /* level-2 nodes: 8 cells each, children in octant order */
        for (int p = 0; p < 64; ++p) {
            int px = p & 3, py = (p >> 2) & 3, pz = p >> 4;
            double M = 0, S[3] = {0, 0, 0};
            for (int o = 0; o < 8; ++o) {
                int i = 2 * px + (o & 1), j = 2 * py + ((o >> 1) & 1), k = 2 * pz + (o >> 2);
                double m = T->cm[(size_t)n * NCB + i + NB * j + NB * NB * k], r[3];
                cell_centre(T, b, i, j, k, r);
                M += m;
                for (int a = 0; a < 3; ++a) S[a] += m * r[a];
            }
            T->n2M[n * 64 + p] = M;
            for (int a = 0; a < 3; ++a) {
                double cen = lo[3 * b + a] + ((a == 0 ? px : a == 1 ? py : pz) + 0.5) * size[3 * b + a] / 4;
                T->n2C[(n * 64 + p) * 3 + a] = M > 0 ? S[a] / M : cen;
            }
        }
        /* level-1 nodes: 8 level-2 nodes each */
        for (int q = 0; q < 8; ++q) {
            int qx = q & 1, qy = (q >> 1) & 1, qz = q >> 2;
            double M = 0, S[3] = {0, 0, 0};
            for (int o = 0; o < 8; ++o) {
                int p = (2 * qx + (o & 1)) + 4 * (2 * qy + ((o >> 1) & 1)) + 16 * (2 * qz + (o >> 2));
                double m = T->n2M[n * 64 + p];
                M += m;
                for (int a = 0; a < 3; ++a) S[a] += m * T->n2C[(n * 64 + p) * 3 + a];
            }
            T->n1M[n * 8 + q] = M;
            for (int a = 0; a < 3; ++a) {
                double cen = lo[3 * b + a] + ((a == 0 ? qx : a == 1 ? qy : qz) + 0.5) * size[3 * b + a] / 2;
                T->n1C[(n * 8 + q) * 3 + a] = M > 0 ? S[a] / M : cen;
            }
        }
        /* leaf-block node: 8 level-1 nodes */
        double M = 0, S[3] = {0, 0, 0};
        for (int q = 0; q < 8; ++q) {
            M += T->n1M[n * 8 + q];
            for (int a = 0; a < 3; ++a) S[a] += T->n1M[n * 8 + q] * T->n1C[(n * 8 + q) * 3 + a];
        }
        T->bM[b] = M;
        for (int a = 0; a < 3; ++a)
            T->bC[3 * b + a] = M > 0 ? S[a] / M : lo[3 * b + a] + 0.5 * size[3 * b + a];
    }
    build_block(T, 0);
    return 0;
}

/* Exported: per-block mass and centre of mass, and the block-tree nodes of every leaf-block. */
int or_tree_build(int nb, const int* level, const int* child, const double* lo, const double* size,
                  const double* rho, double* blk_mass, double* blk_com, double* n1_mass,
                  double* n1_com, double* n2_mass, double* n2_com) {
    otree T;
    if (otree_build(&T, nb, level, child, lo, size, rho, NULL)) { otree_free(&T); return -1; }
    memcpy(blk_mass, T.bM, sizeof(double) * nb);
    memcpy(blk_com, T.bC, sizeof(double) * 3 * nb);
    if (n1_mass) memcpy(n1_mass, T.n1M, sizeof(double) * 8 * T.nleaf);
    if (n1_com) memcpy(n1_com, T.n1C, sizeof(double) * 24 * T.nleaf);
    if (n2_mass) memcpy(n2_mass, T.n2M, sizeof(double) * 64 * T.nleaf);
    if (n2_com) memcpy(n2_com, T.n2C, sizeof(double) * 192 * T.nleaf);
    otree_free(&T);
    return 0;
}

/* Exported: MPE moments (B2, B3) of every block, level-1 and level-2 node. */
int or_tree_bmoments(int nb, const int* level, const int* child, const double* lo, const double* size,
                     const double* rho, double* blk_B, double* n1_B, double* n2_B) {
    otree T;
    if (otree_build(&T, nb, level, child, lo, size, rho, NULL) || otree_bmoments(&T)) { otree_free(&T); return -1; }
    memcpy(blk_B, T.bB, sizeof(double) * 2 * nb);
    if (n1_B) memcpy(n1_B, T.n1B, sizeof(double) * 16 * T.nleaf);
    if (n2_B) memcpy(n2_B, T.n2B, sizeof(double) * 128 * T.nleaf);
    otree_free(&T);
    return 0;
}

/* ======================================================================================
 * Ewald sums (Sec. 2.2.3 fully periodic, Sec. 2.2.4 mixed, App. A accelerations).
 * phi(d) is the Green's function of one unit mass and all its periodic images:
 *   Phi(r) = -G sum_a M_a phi(r - r_a),   a(r) = -G sum_a M_a A(r - r_a),   A = -grad phi.
 * Box: Lx, Ly = b Lx, Lz = c Lx.  zeta = pi^2 / (alpha Lx)^2.
 * Real-space images: i1^2 + (b i2)^2 + (c i3)^2 <= rcut2 (15 in Sec. 2.2.3);
 * Fourier terms: l1^2 + (l2/b)^2 + (l3/c)^2 <= kcut2 (10).
 * ====================================================================================== */
enum { EW_NONE = 0, EW_3P = 1, EW_2P1I = 2, EW_1P2I = 3 };

typedef struct {
    int kind;
    double Lx, b, c, alpha, zeta, rcut2, kcut2;
} ewcfg;

static int ew_kind_from_bc(const int bc[3]) {
    if (!bc[0] && !bc[1] && !bc[2]) return EW_NONE;
    if (bc[0] && bc[1] && bc[2]) return EW_3P;
    if (bc[0] && bc[1] && !bc[2]) return EW_2P1I;
    if (bc[0] && !bc[1] && !bc[2]) return EW_1P2I;
    return -1; /* other axis choices: the paper fixes the periodic axes to x (and y) */
}

static void ew_setup(ewcfg* E, int kind, const double L[3], double alpha_lx, double rcut2, double kcut2) {
    E->kind = kind;
    E->Lx = L[0]; E->b = L[1] / L[0]; E->c = L[2] / L[0];
    E->alpha = alpha_lx / L[0];
    E->zeta = M_PI * M_PI / (E->alpha * E->Lx * E->alpha * E->Lx);
    E->rcut2 = rcut2; E->kcut2 = kcut2;
}

/* erfcx(x) = exp(x^2) erfc(x), x >= 0; continued fraction for large x (Abramowitz & Stegun 7.1.14). */
static double or_erfcx(double x) {
    if (x < 25.0) return exp(x * x) * erfc(x);
    double t = 0.0;
    for (int n = 60; n >= 1; --n) t = (n / 2.0) / (x + t);
    return 1.0 / (sqrt(M_PI) * (x + t));
}

/* Real-space image term of phi: erfc(alpha r)/r, and of A: [2a/sqrt(pi) e^{-a^2 u}/u + erfc(a sqrt u)/u^{3/2}] v */
static double real_pot(double alpha, double r) { return erfc(alpha * r) / r; }
static double real_acc_factor(double alpha, double u) {
    double r = sqrt(u);
    return 2.0 * alpha / sqrt(M_PI) * exp(-alpha * alpha * u) / u + erfc(alpha * r) / (u * r);
}

/* Gauss-Legendre nodes/weights on [-1,1] (Newton on P_n). */
static void gauss_legendre(int n, double* x, double* w) {
    for (int i = 0; i < n; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5)), pp = 0;
        for (int it = 0; it < 100; ++it) {
            double p1 = 1, p2 = 0;
            for (int j = 1; j <= n; ++j) { double p3 = p2; p2 = p1; p1 = ((2 * j - 1) * z * p2 - (j - 1) * p3) / j; }
            pp = n * (z * p1 - p2) / (z * z - 1);
            double dz = p1 / pp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = z; w[i] = 2.0 / ((1 - z * z) * pp * pp);
    }
}

#define GL_N 16
#define GL_PANELS 96
static double gl_x[GL_N], gl_w[GL_N];
static int gl_ready = 0;
static void gl_init(void) {
    if (!gl_ready) {
        #pragma omp critical(or_gl)
        { if (!gl_ready) { gauss_legendre(GL_N, gl_x, gl_w); gl_ready = 1; } }
    }
}

/* 1P2I Fourier integrals (eq. int00p1 and App. A eq. e4fceM):
 *   K(l1, eta) = int_0^inf J0(eta q) exp(-zeta q^2) q / (l1^2 + q^2) dq,     l1 != 0
 *   K(0, eta)  = int_0^inf (J0(eta q) - 1) exp(-zeta q^2) / q dq    (divergent constant dropped,
 *                as the paper does for I(0,0) in 2P1I)
 *   M(l1, eta) = int_0^inf J1(eta q) exp(-zeta q^2) q^2 / (l1^2 + q^2) dq
 * by composite Gauss-Legendre on [0, Q] with exp(-zeta Q^2) < 1e-20. */
static void k_m_1p2i(double l1, double eta, double zeta, double* K, double* Mv) {
    gl_init();
    double Q = sqrt(46.0 / zeta), h = Q / GL_PANELS, sk = 0, sm = 0, l2 = l1 * l1;
    for (int p = 0; p < GL_PANELS; ++p)
        for (int i = 0; i < GL_N; ++i) {
            double q = h * (p + 0.5 * (gl_x[i] + 1.0)), w = 0.5 * h * gl_w[i];
            double g = exp(-zeta * q * q), j0v = j0(eta * q), j1v = j1(eta * q);
            if (l1 != 0.0) sk += w * j0v * g * q / (l2 + q * q);
            else sk += w * (j0v - 1.0) * g / q;
            sm += w * j1v * g * q * q / (l2 + q * q);
        }
    *K = sk; *Mv = sm;
}

/* 2P1I Fourier integral scaled by exp(-zeta s^2) (App. A eq. intijscaled), gam >= 0:
 *   It = pi/(2s) { exp(-gam^2/4zeta - zeta s^2) erfcx((zeta s + gam/2)/sqrt zeta)
 *                  + exp(-gam s) erfc((zeta s - gam/2)/sqrt zeta) }
 *   Ip = dIt/dgam = pi/2 { same first term - same second term }
 * and for l1 = l2 = 0 (eq. int00): It = -pi {gam erf(gam/2 sqrt zeta) + 2 sqrt(zeta/pi) e^{-gam^2/4zeta}} + 2 sqrt(pi zeta),
 *   Ip = -pi erf(gam / 2 sqrt zeta). */
static void itilde_2p1i(double s, double gam, double zeta, double* It, double* Ip) {
    double sz = sqrt(zeta);
    if (s == 0.0) {
        *It = -M_PI * (gam * erf(gam / (2 * sz)) + 2 * sqrt(zeta / M_PI) * exp(-gam * gam / (4 * zeta)))
              + 2 * sqrt(M_PI * zeta);
        *Ip = -M_PI * erf(gam / (2 * sz));
        return;
    }
    double t1 = exp(-gam * gam / (4 * zeta) - zeta * s * s) * or_erfcx((zeta * s + gam / 2) / sz);
    double t2 = exp(-gam * s) * erfc((zeta * s - gam / 2) / sz);
    *It = M_PI / (2 * s) * (t1 + t2);
    *Ip = M_PI / 2 * (t1 - t2);
}

/* Exported for the pins of the two Fourier integrals against independent quadrature. */
void or_itilde_2p1i(double s, double gam, double zeta, double* It, double* Ip) { itilde_2p1i(s, gam, zeta, It, Ip); }
void or_km_1p2i(double l1, double eta, double zeta, double* K, double* M) { k_m_1p2i(l1, eta, zeta, K, M); }

/* phi and A of eqs. ewpotential / potential2p1i / potential1p2i and App. A.
 * If corr != 0 the singular term 1/|d| (and d/|d|^3) is removed analytically from the i=0 image,
 * giving the smooth correction C = phi - 1/|d|, A_c = A - d/|d|^3 (Sec. 2.2.5, approach 2). */
static void ewald_eval(const ewcfg* E, const double d[3], int corr, double* phi_out, double A[3]) {
    const double Lx = E->Lx, b = E->b, c = E->c, al = E->alpha, zeta = E->zeta;
    double phi = 0, Ax = 0, Ay = 0, Az = 0;
    int n1 = (int)floor(sqrt(E->rcut2));
    int n2 = E->kind == EW_1P2I ? 0 : (int)floor(sqrt(E->rcut2) / b);
    int n3 = E->kind == EW_3P ? (int)floor(sqrt(E->rcut2) / c) : 0;
    /* real-space images */
    for (int i1 = -n1; i1 <= n1; ++i1)
        for (int i2 = -n2; i2 <= n2; ++i2)
            for (int i3 = -n3; i3 <= n3; ++i3) {
                if (i1 * i1 + b * b * i2 * i2 + c * c * i3 * i3 > E->rcut2) continue;
                double v[3] = {d[0] - i1 * Lx, d[1] - i2 * b * Lx, d[2] - i3 * c * Lx};
                double u = v[0] * v[0] + v[1] * v[1] + v[2] * v[2], r = sqrt(u);
                double fp, fa;
                if (corr && i1 == 0 && i2 == 0 && i3 == 0) {
                    /* erfc(ar)/r - 1/r = -erf(ar)/r; the A factor minus 1/r^3 */
                    double x = al * r;
                    if (x < 0.05) {
                        double x2 = x * x, sp = 0, sa = 0, tp = 1, fact = 1;
                        for (int m = 0; m <= 7; ++m) {
                            if (m > 0) { tp *= x2; fact *= m; }
                            sp += (m & 1 ? -1.0 : 1.0) * tp / (fact * (2 * m + 1));
                            sa += (m & 1 ? 2.0 : -2.0) * tp / (fact * (2 * m + 3));
                        }
                        fp = -2 * al / sqrt(M_PI) * sp;
                        fa = 2 * al * al * al / sqrt(M_PI) * sa;
                    } else {
                        fp = -erf(x) / r;
                        fa = 2 * al / sqrt(M_PI) * exp(-x * x) / u - erf(x) / (u * r);
                    }
                } else {
                    fp = real_pot(al, r);
                    fa = real_acc_factor(al, u);
                }
                phi += fp; Ax += fa * v[0]; Ay += fa * v[1]; Az += fa * v[2];
            }
    /* Fourier-space terms */
    if (E->kind == EW_3P) {
        double V = b * c * Lx * Lx * Lx;
        int m1 = (int)floor(sqrt(E->kcut2)), m2 = (int)floor(sqrt(E->kcut2) * b), m3 = (int)floor(sqrt(E->kcut2) * c);
        for (int l1 = -m1; l1 <= m1; ++l1)
            for (int l2 = -m2; l2 <= m2; ++l2)
                for (int l3 = -m3; l3 <= m3; ++l3) {
                    double ll = l1 * l1 + (l2 / b) * (l2 / b) + (l3 / c) * (l3 / c);
                    if (ll == 0 || ll > E->kcut2) continue;
                    double k[3] = {2 * M_PI * l1 / Lx, 2 * M_PI * l2 / (b * Lx), 2 * M_PI * l3 / (c * Lx)};
                    double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
                    double kd = k[0] * d[0] + k[1] * d[1] + k[2] * d[2];
                    double f = 4 * M_PI / k2 * exp(-k2 / (4 * al * al)) / V;
                    phi += f * cos(kd);
                    Ax += f * k[0] * sin(kd); Ay += f * k[1] * sin(kd); Az += f * k[2] * sin(kd);
                }
        /* uniform neutralising background: makes the cell average of phi zero */
        phi -= M_PI / (al * al * V);
    } else if (E->kind == EW_2P1I) {
        double gam = 2 * M_PI * d[2] / Lx, ag = fabs(gam), sg = gam < 0 ? -1.0 : 1.0;
        int m1 = (int)floor(sqrt(E->kcut2)), m2 = (int)floor(sqrt(E->kcut2) * b);
        for (int l1 = -m1; l1 <= m1; ++l1)
            for (int l2 = -m2; l2 <= m2; ++l2) {
                double ss = l1 * l1 + (l2 / b) * (l2 / b);
                if (ss > E->kcut2) continue;
                double It, Ip;
                itilde_2p1i(sqrt(ss), ag, zeta, &It, &Ip);
                double v = 2 * M_PI * l1 * d[0] / Lx + 2 * M_PI * l2 * d[1] / (b * Lx);
                phi += cos(v) * It / (M_PI * Lx * b);
                Ax += 2.0 / (b * Lx * Lx) * l1 * sin(v) * It;
                Ay += 2.0 / (b * b * Lx * Lx) * l2 * sin(v) * It;
                Az -= 2.0 / (b * Lx * Lx) * cos(v) * sg * Ip;
            }
    } else if (E->kind == EW_1P2I) {
        double R = sqrt(d[1] * d[1] + d[2] * d[2]), eta = 2 * M_PI * R / Lx;
        int m1 = (int)floor(sqrt(E->kcut2));
        double sumM = 0;
        for (int l1 = -m1; l1 <= m1; ++l1) {
            double K, Mv, e = exp(-zeta * l1 * l1), v = 2 * M_PI * l1 * d[0] / Lx;
            k_m_1p2i((double)l1, eta, zeta, &K, &Mv);
            phi += 2.0 / Lx * e * cos(v) * K;
            Ax += 4 * M_PI / (Lx * Lx) * l1 * e * sin(v) * K;
            sumM += e * cos(v) * Mv;
        }
        if (R > 0) {
            Ay += 4 * M_PI / (Lx * Lx) * d[1] / R * sumM;
            Az += 4 * M_PI / (Lx * Lx) * d[2] / R * sumM;
        }
    }
    *phi_out = phi; A[0] = Ax; A[1] = Ay; A[2] = Az;
}

/* Exported: phi and A (corr = 0) or the smooth correction C, A_c (corr = 1) at n points d[n][3].
 * bc: per axis 0/1; L: box edge lengths; alpha_lx = alpha * Lx (paper: 2). Returns -1 on an
 * unsupported BC combination. */
int or_ewald(const int* bc, const double* L, double alpha_lx, double rcut2, double kcut2, int corr,
             int64_t n, const double* d, double* phi, double* A) {
    ewcfg E;
    int kind = ew_kind_from_bc(bc);
    if (kind <= 0) return -1;
    ew_setup(&E, kind, L, alpha_lx, rcut2, kcut2);
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) ewald_eval(&E, d + 3 * i, corr, phi + i, A + 3 * i);
    return 0;
}

/* Far-field forms used beyond the far distance (Sec. 2.2.5, approach 2).  2P1I: the l1=l2=0 term alone,
 *   phi -> -2 pi |dz| / (b Lx^2) + 2 sqrt(pi zeta) / (pi b Lx),  A = (0, 0, 2 pi sgn(dz) / (b Lx^2)).
 * 1P2I: the l1=0 term alone with K(0, eta) = -1/2 [gamma_E + ln(eta^2/4zeta) + E1(eta^2/4zeta)]
 * and E1 dropped, phi -> -(1/Lx) [gamma_E + 2 ln eta - ln 4zeta],  A = (0, 2 dy/(Lx R^2), 2 dz/(Lx R^2)). */
static void ewald_far(const ewcfg* E, const double d[3], double* phi, double A[3]) {
    const double Lx = E->Lx, b = E->b;
    if (E->kind == EW_2P1I) {
        double az = fabs(d[2]);
        *phi = -2 * M_PI * az / (b * Lx * Lx) + 2 * sqrt(M_PI * E->zeta) / (M_PI * b * Lx);
        A[0] = 0; A[1] = 0; A[2] = (d[2] < 0 ? -1.0 : 1.0) * 2 * M_PI / (b * Lx * Lx);
    } else {
        double R2 = d[1] * d[1] + d[2] * d[2], eta = 2 * M_PI * sqrt(R2) / Lx;
        const double euler_gamma = 0.57721566490153286061;
        *phi = -(euler_gamma + 2 * log(eta) - log(4 * E->zeta)) / Lx;
        A[0] = 0; A[1] = 2 * d[1] / (Lx * R2); A[2] = 2 * d[2] / (Lx * R2);
    }
}

int or_ewald_far(const int* bc, const double* L, double alpha_lx, int64_t n, const double* d,
                 double* phi, double* A) {
    ewcfg E;
    int kind = ew_kind_from_bc(bc);
    if (kind != EW_2P1I && kind != EW_1P2I) return -1;
    ew_setup(&E, kind, L, alpha_lx, 15, 10);
    for (int64_t i = 0; i < n; ++i) ewald_far(&E, d + 3 * i, phi + i, A + 3 * i);
    return 0;
}

/* Extent of the correction table per axis (Sec. 2.2.5): half the box on periodic axes
 * (minimum image), the box edge on isolated axes, capped at 2 Lx for the isolated axes of
 * mixed BCs where the far-field form takes over. */
/* Distance beyond which the far-field form is used.  The paper quotes 2 Lx; the slowest
 * neglected Fourier mode decays as exp(-2 pi |dz| / max(Lx, Ly)) in 2P1I, so for Ly > Lx the
 * threshold is taken as 2 max(Lx, Ly) (equal to the paper's for b <= 1). */
static double far_distance(const ewcfg* E) {
    return E->kind == EW_2P1I ? 2 * E->Lx * fmax(1.0, E->b) : 2 * E->Lx;
}

static void table_extent(const ewcfg* E, const int bc[3], const double L[3], double ext[3]) {
    for (int a = 0; a < 3; ++a) {
        ext[a] = bc[a] ? 0.5 * L[a] : L[a];
        if (!bc[a] && ext[a] > far_distance(E)) ext[a] = far_distance(E);
    }
}

/* Exported: correction table tab[i][j][k][4] = (C, A_cx, A_cy, A_cz) at
 * d = (i ex/(n-1), j ey/(n-1), k ez/(n-1)) with x the slowest index, i.e. [ix][iy][iz]. */
int or_ewald_table(const int* bc, const double* L, double alpha_lx, int n, double* tab, double* ext_out) {
    ewcfg E;
    int kind = ew_kind_from_bc(bc);
    if (kind <= 0 || n < 2) return -1;
    ew_setup(&E, kind, L, alpha_lx, 15, 10);
    double ext[3];
    table_extent(&E, bc, L, ext);
    for (int a = 0; a < 3; ++a) ext_out[a] = ext[a];
    #pragma omp parallel for collapse(2) schedule(dynamic, 4)
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            for (int k = 0; k < n; ++k) {
                double d[3] = {ext[0] * i / (n - 1), ext[1] * j / (n - 1), ext[2] * k / (n - 1)}, phi, A[3];
                ewald_eval(&E, d, 1, &phi, A);
                double* o = tab + 4 * (((size_t)i * n + j) * n + k);
                o[0] = phi; o[1] = A[0]; o[2] = A[1]; o[3] = A[2];
            }
    return 0;
}

/* Exported: the table of Sec. 2.2.5, approach 2, for first-order Taylor expansion: at every grid
 * point of or_ewald_table, the correction (C, A_c) and the gradient of each component of A_c,
 * J[i][j] = dA_c,i / dd_j, by central differences of the series with step eps:
 *   J[i][j] = (A_c,i(d + eps e_j) - A_c,i(d - eps e_j)) / (2 eps),  then (J + J^T) / 2
 * (A_c is a gradient field, so J is symmetric).  The gradient of C needs no storage: it is -A_c.
 * tab[i][j][k][10] = (C, A_cx, A_cy, A_cz, Jxx, Jxy, Jxz, Jyy, Jyz, Jzz). */
int or_ewald_taylor_table(const int* bc, const double* L, double alpha_lx, int n, double eps, double* tab,
                          double* ext_out) {
    ewcfg E;
    int kind = ew_kind_from_bc(bc);
    if (kind <= 0 || n < 2 || !(eps > 0)) return -1;
    ew_setup(&E, kind, L, alpha_lx, 15, 10);
    double ext[3];
    table_extent(&E, bc, L, ext);
    for (int a = 0; a < 3; ++a) ext_out[a] = ext[a];
    #pragma omp parallel for collapse(2) schedule(dynamic, 4)
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            for (int k = 0; k < n; ++k) {
                double d[3] = {ext[0] * i / (n - 1), ext[1] * j / (n - 1), ext[2] * k / (n - 1)}, phi, A[3];
                ewald_eval(&E, d, 1, &phi, A);
                double J[3][3];
                for (int c = 0; c < 3; ++c) {
                    double dp[3] = {d[0], d[1], d[2]}, dm[3] = {d[0], d[1], d[2]}, pp, pm, Ap[3], Am[3];
                    dp[c] += eps;
                    dm[c] -= eps;
                    ewald_eval(&E, dp, 1, &pp, Ap);
                    ewald_eval(&E, dm, 1, &pm, Am);
                    for (int r = 0; r < 3; ++r) J[r][c] = (Ap[r] - Am[r]) / (2 * eps);
                }
                double* o = tab + 10 * (((size_t)i * n + j) * n + k);
                o[0] = phi; o[1] = A[0]; o[2] = A[1]; o[3] = A[2];
                o[4] = J[0][0];
                o[5] = 0.5 * (J[0][1] + J[1][0]);
                o[6] = 0.5 * (J[0][2] + J[2][0]);
                o[7] = J[1][1];
                o[8] = 0.5 * (J[1][2] + J[2][1]);
                o[9] = J[2][2];
            }
    return 0;
}

/* Trilinear interpolation of the folded correction table, signs restored per axis. */
typedef struct { const double* tab; int n; double ext[3]; int taylor; } etable;

/* First-order Taylor expansion (Sec. 2.2.5, approach 2) about the nearest grid point g of the
 * folded separation u = |d|: C(u) = C(g) - A_c(g) . (u - g), A_c,i(u) = A_c,i(g) + sum_j J_ij (u_j - g_j),
 * then the sign of d restored on each A_c component (A_c,i is odd in d_i, even in the others). */
static void taylor_lookup(const etable* T, const double d[3], double* C, double Ac[3]) {
    double du[3], sgn[3];
    int g[3];
    for (int a = 0; a < 3; ++a) {
        double x = fabs(d[a]), h = T->ext[a] / (T->n - 1);
        sgn[a] = d[a] < 0 ? -1.0 : 1.0;
        int i = (int)floor(x / h + 0.5);
        if (i > T->n - 1) i = T->n - 1;
        g[a] = i;
        du[a] = x - i * h;
    }
    const double* v = T->tab + 10 * (((size_t)g[0] * T->n + g[1]) * T->n + g[2]);
    const double J[3][3] = {{v[4], v[5], v[6]}, {v[5], v[7], v[8]}, {v[6], v[8], v[9]}};
    *C = v[0] - (v[1] * du[0] + v[2] * du[1] + v[3] * du[2]);
    for (int r = 0; r < 3; ++r) Ac[r] = sgn[r] * (v[1 + r] + J[r][0] * du[0] + J[r][1] * du[1] + J[r][2] * du[2]);
}

static void table_lookup(const etable* T, const double d[3], double* C, double Ac[3]) {
    double f[3], sgn[3], out[4] = {0, 0, 0, 0};
    int i0[3];
    for (int a = 0; a < 3; ++a) {
        double x = fabs(d[a]);
        sgn[a] = d[a] < 0 ? -1.0 : 1.0;
        double u = x / T->ext[a] * (T->n - 1);
        if (u > T->n - 1) u = T->n - 1;
        int i = (int)floor(u);
        if (i > T->n - 2) i = T->n - 2;
        i0[a] = i; f[a] = u - i;
    }
    for (int o = 0; o < 8; ++o) {
        int dx = o & 1, dy = (o >> 1) & 1, dz = o >> 2;
        double w = (dx ? f[0] : 1 - f[0]) * (dy ? f[1] : 1 - f[1]) * (dz ? f[2] : 1 - f[2]);
        const double* v = T->tab + 4 * (((size_t)(i0[0] + dx) * T->n + (i0[1] + dy)) * T->n + (i0[2] + dz));
        for (int c = 0; c < 4; ++c) out[c] += w * v[c];
    }
    *C = out[0];
    for (int a = 0; a < 3; ++a) Ac[a] = out[1 + a] * sgn[a];
}

/* ======================================================================================
 * Tree walk for gravity (Sec. 2.1 walk and BH MAC eq. bhmac with the safe box eta_SB;
 * Sec. 2.2.1 APE MAC eq. ape with p = 1 and the absolute limit eq. abs_err; Sec. 2.2.2
 * eqs. pot/accel; Secs. 2.2.3-2.2.5 Ewald).
 * ====================================================================================== */
typedef struct {
    int mac;             /* 0 BH, 1 APE, 2 MPE */
    double theta, safe_box, a_lim, G;
    int ewald;           /* 0 exact series per interaction, 1 correction table (trilinear), 2 Taylor table */
    ewcfg E;
    etable tab;
} wparams;

typedef struct { double phi, a[3]; int64_t n_int, n_mac; } wacc;

/* node kinds: 0 amr block, 1 level-1 block-tree node, 2 level-2 node, 3 cell */
typedef struct { int kind, b, n, idx; } onode;

static void node_geom(const otree* T, onode nd, double cen[3], double half[3]) {
    int div = nd.kind == 0 ? 1 : nd.kind == 1 ? 2 : nd.kind == 2 ? 4 : 8;
    int ix = 0, iy = 0, iz = 0;
    if (nd.kind == 1) { ix = nd.idx & 1; iy = (nd.idx >> 1) & 1; iz = nd.idx >> 2; }
    if (nd.kind == 2) { ix = nd.idx & 3; iy = (nd.idx >> 2) & 3; iz = nd.idx >> 4; }
    if (nd.kind == 3) { ix = nd.idx & 7; iy = (nd.idx >> 3) & 7; iz = nd.idx >> 6; }
    int id[3] = {ix, iy, iz};
    for (int a = 0; a < 3; ++a) {
        double s = T->size[3 * nd.b + a] / div;
        half[a] = 0.5 * s;
        cen[a] = T->lo[3 * nd.b + a] + (id[a] + 0.5) * s;
    }
}

static void node_moments(const otree* T, onode nd, double* M, double com[3]) {
    double cen[3], half[3];
    switch (nd.kind) {
    case 0: *M = T->bM[nd.b]; for (int a = 0; a < 3; ++a) com[a] = T->bC[3 * nd.b + a]; break;
    case 1: *M = T->n1M[nd.n * 8 + nd.idx]; for (int a = 0; a < 3; ++a) com[a] = T->n1C[(nd.n * 8 + nd.idx) * 3 + a]; break;
    case 2: *M = T->n2M[nd.n * 64 + nd.idx]; for (int a = 0; a < 3; ++a) com[a] = T->n2C[(nd.n * 64 + nd.idx) * 3 + a]; break;
    default:
        *M = T->cm[(size_t)nd.n * NCB + nd.idx];
        node_geom(T, nd, cen, half);
        for (int a = 0; a < 3; ++a) com[a] = cen[a];
    }
}

static void node_bmom(const otree* T, onode nd, double* B2, double* B3) {
    const double* v = nd.kind == 0 ? &T->bB[2 * nd.b] : nd.kind == 1 ? &T->n1B[(nd.n * 8 + nd.idx) * 2]
                                                                      : &T->n2B[(nd.n * 64 + nd.idx) * 2];
    *B2 = v[0];
    *B3 = v[1];
}

/* children of a node, in octant order */
static int node_children(const otree* T, onode nd, onode out[8]) {
    if (nd.kind == 3) return 0;
    for (int o = 0; o < 8; ++o) {
        int ox = o & 1, oy = (o >> 1) & 1, oz = o >> 2;
        onode c = nd;
        if (nd.kind == 0) {
            int cb = T->child[8 * nd.b + o];
            if (cb >= 0) { c.b = cb; c.kind = 0; c.n = -1; c.idx = 0; }
            else { c.kind = 1; c.n = T->leaf_of[nd.b]; c.idx = o; }
        } else if (nd.kind == 1) {
            int qx = nd.idx & 1, qy = (nd.idx >> 1) & 1, qz = nd.idx >> 2;
            c.kind = 2; c.idx = (2 * qx + ox) + 4 * (2 * qy + oy) + 16 * (2 * qz + oz);
        } else {
            int px = nd.idx & 3, py = (nd.idx >> 2) & 3, pz = nd.idx >> 4;
            c.kind = 3; c.idx = (2 * px + ox) + 8 * (2 * py + oy) + 64 * (2 * pz + oz);
        }
        out[o] = c;
    }
    /* an amr block whose children are block-tree nodes: all 8 share the "leaf" flag */
    return 8;
}

static void min_image(const otree* T, double v[3]) {
    for (int a = 0; a < 3; ++a)
        if (T->bc[a]) v[a] -= T->L[a] * nearbyint(v[a] / T->L[a]);
}

static void interact(const wparams* P, const otree* T, double M, const double dv[3], wacc* acc) {
    double u = dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2], r = sqrt(u);
    acc->n_int++;
    if (P->E.kind == EW_NONE) {                         /* eqs. pot, accel */
        acc->phi -= P->G * M / r;
        for (int a = 0; a < 3; ++a) acc->a[a] -= P->G * M * dv[a] / (u * r);
        return;
    }
    double phi, A[3];
    int far = (P->E.kind == EW_2P1I && fabs(dv[2]) > far_distance(&P->E)) ||
              (P->E.kind == EW_1P2I && sqrt(dv[1] * dv[1] + dv[2] * dv[2]) > far_distance(&P->E));
    if (P->ewald == 0) {
        ewald_eval(&P->E, dv, 0, &phi, A);
    } else if (far) {
        ewald_far(&P->E, dv, &phi, A);
    } else {
        double C, Ac[3];
        if (P->tab.taylor) taylor_lookup(&P->tab, dv, &C, Ac);
        else table_lookup(&P->tab, dv, &C, Ac);
        phi = 1.0 / r + C;
        for (int a = 0; a < 3; ++a) A[a] = dv[a] / (u * r) + Ac[a];
    }
    (void)T;
    acc->phi -= P->G * M * phi;
    for (int a = 0; a < 3; ++a) acc->a[a] -= P->G * M * A[a];
}

static void walk(const otree* T, const wparams* P, const double r[3], int tn, int tc, onode nd, wacc* acc) {
    double M, com[3], dv[3];
    node_moments(T, nd, &M, com);
    for (int a = 0; a < 3; ++a) dv[a] = r[a] - com[a];
    min_image(T, dv);
    if (nd.kind == 3) {                                  /* leaf-node: always accepted */
        if (nd.n == tn && nd.idx == tc) return;          /* no self-interaction */
        interact(P, T, M, dv, acc);
        return;
    }
    acc->n_mac++;
    double cen[3], half[3], rc[3];
    node_geom(T, nd, cen, half);
    for (int a = 0; a < 3; ++a) rc[a] = r[a] - cen[a];
    min_image(T, rc);
    /* safe box: target outside the cuboid eta_SB times the node (Sec. 2.1) */
    int outside = 0;
    for (int a = 0; a < 3; ++a) if (fabs(rc[a]) > P->safe_box * half[a]) outside = 1;
    double h = 2 * fmax(half[0], fmax(half[1], half[2]));   /* node size: longest edge */
    double d2 = dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2];
    int ok;
    if (P->mac == 0) {
        ok = h * h < P->theta * P->theta * d2;                           /* eq. bhmac */
    } else if (P->mac == 1) {
        ok = P->G * M * h * h < P->a_lim * d2 * d2;                      /* eq. ape, p = 1 */
    } else {
        /* eq. mpe, p = 1: b_max is the distance from the centre of mass to the furthest point of
         * the node (a corner); the bound needs d > b_max, otherwise the node is opened */
        double B2, B3, bmax2 = 0, d = sqrt(d2);
        node_bmom(T, nd, &B2, &B3);
        for (int a = 0; a < 3; ++a) {
            double t = half[a] + fabs(com[a] - cen[a]);
            bmax2 += t * t;
        }
        double bmax = sqrt(bmax2);
        ok = 0;
        if (d > bmax) {
            double q = 1 - bmax / d;
            double da = P->G / d2 / (q * q) * (3 * B2 / d2 - 2 * B3 / (d2 * d));
            ok = da < P->a_lim;
        }
    }
    if (outside && ok) { interact(P, T, M, dv, acc); return; }
    onode ch[8];
    int nc = node_children(T, nd, ch);
    for (int o = 0; o < nc; ++o) walk(T, P, r, tn, tc, ch[o], acc);
}

static int setup_walk(wparams* P, const otree* T, const int* bc, int mac, double theta, double safe_box,
                      double a_lim, double G, int ewald_mode, const double* tab, int tab_n,
                      const double* tab_ext) {
    memset(P, 0, sizeof(*P));
    P->mac = mac; P->theta = theta; P->safe_box = safe_box; P->a_lim = a_lim; P->G = G;
    int kind = ew_kind_from_bc(bc);
    if (kind < 0) return -1;
    ew_setup(&P->E, kind, T->L, 2.0, 15, 10);
    P->ewald = ewald_mode;
    if (kind != EW_NONE && (ewald_mode == 1 || ewald_mode == 2)) {
        if (!tab) return -1;
        P->tab.tab = tab; P->tab.n = tab_n; P->tab.taylor = ewald_mode == 2;
        for (int a = 0; a < 3; ++a) P->tab.ext[a] = tab_ext[a];
    }
    return 0;
}

/* Exported: potential and acceleration at target cells (flat index leaf*512 + k*64 + j*8 + i).
 * ewald_mode 0: exact series per interaction; 1: correction table tab[n][n][n][4] (as built by
 * or_ewald_table), trilinear; 2: Taylor table tab[n][n][n][10] (as built by or_ewald_taylor_table),
 * first order about the nearest grid point; table modes use the far-field forms beyond the far
 * distance.  counts[0] = interactions, counts[1] = MAC
 * tests (summed over targets). */
int or_gravity_walk(int nb, const int* level, const int* child, const double* lo, const double* size,
                    const double* rho, const int* bc, int mac, double theta, double safe_box,
                    double a_lim, double G, int ewald_mode, const double* tab, int tab_n,
                    const double* tab_ext, int64_t nt, const int64_t* targets, double* pot,
                    double* acc, int64_t* counts) {
    otree T;
    if (otree_build(&T, nb, level, child, lo, size, rho, bc)) { otree_free(&T); return -1; }
    if (mac == 2 && otree_bmoments(&T)) { otree_free(&T); return -1; }
    wparams P;
    if (setup_walk(&P, &T, bc, mac, theta, safe_box, a_lim, G, ewald_mode, tab, tab_n, tab_ext)) {
        otree_free(&T); return -2;
    }
    int64_t ni = 0, nm = 0;
    #pragma omp parallel for schedule(dynamic, 8) reduction(+ : ni, nm)
    for (int64_t t = 0; t < nt; ++t) {
        int n = (int)(targets[t] / NCB), c = (int)(targets[t] % NCB), b = T.block_of[n];
        double r[3];
        cell_centre(&T, b, c & 7, (c >> 3) & 7, c >> 6, r);
        wacc A = {0, {0, 0, 0}, 0, 0};
        onode root = {0, 0, -1, 0};
        walk(&T, &P, r, n, c, root, &A);
        pot[t] = A.phi;
        for (int a = 0; a < 3; ++a) acc[3 * t + a] = A.a[a];
        ni += A.n_int; nm += A.n_mac;
    }
    if (counts) { counts[0] = ni; counts[1] = nm; }
    otree_free(&T);
    return 0;
}

/* ---- SumSquare MAC (Sec. 2.2.1, the variant of SW94 that limits the error of the total
 * acceleration): the frontier of nodes waiting for evaluation is a priority queue ordered by the
 * node's estimated error, the MPE bound of eq. mpe with p = 1.  Starting from the root, the node with
 * the largest bound is replaced by its children until the sum of the squared bounds over the
 * frontier is at most a_lim^2; then every frontier node is accepted.  Bounds are infinite where they
 * do not apply (target within b_max of the centre of mass) and where the target lies inside the
 * node's safe box, so such nodes are always opened; cells are exact (bound 0) and accepted when
 * reached, the target's own cell excluded.  Equal bounds are ordered by the node's depth, then its
 * integer position (x, y, z).  The summed squares are kept exactly in integer units of
 * 2^-20 a_lim^2 (sq_units).  Refinement stops, with the frontier accepted, when opening the next
 * node would hold more than queue_max nodes (counted in counts[2]).  The bound and the queue
 * operations below are the steps a parity implementation must repeat in this order.
 * (The paper gives no more detail of its experimental implementation: these are readings.) */
typedef struct { double e2; int64_t key; onode nd; } sq_item;

static int64_t sq_key(const otree* T, onode nd) {
    int dep = T->level[nd.b] - 1 + nd.kind;
    double cen[3], half[3];
    node_geom(T, nd, cen, half);
    int64_t k = (int64_t)dep << 57;
    for (int a = 0; a < 3; ++a) {
        int64_t i = llrint((cen[a] - T->lo[a]) / T->L[a] * ldexp(1.0, dep) - 0.5);
        k |= i << (38 - 19 * a);
    }
    return k;
}

static int sq_before(const sq_item* a, const sq_item* b) {   /* a leaves the queue before b */
    return a->e2 > b->e2 || (a->e2 == b->e2 && a->key < b->key);
}

static void sq_push(sq_item* h, int* n, sq_item it) {
    int i = (*n)++;
    while (i > 0) {
        int p = (i - 1) / 2;
        if (!sq_before(&it, &h[p])) break;
        h[i] = h[p];
        i = p;
    }
    h[i] = it;
}

static sq_item sq_pop(sq_item* h, int* n) {
    sq_item top = h[0], last = h[--*n];
    int i = 0;
    for (;;) {
        int c = 2 * i + 1;
        if (c >= *n) break;
        if (c + 1 < *n && sq_before(&h[c + 1], &h[c])) ++c;
        if (!sq_before(&h[c], &last)) break;
        h[i] = h[c];
        i = c;
    }
    if (*n > 0) h[i] = last;
    return top;
}

/* squared MPE bound of an internal node (INFINITY if it must be opened) */
static double sq_bound2(const otree* T, const wparams* P, const double r[3], onode nd) {
    double M, com[3], dv[3], cen[3], half[3], rc[3];
    node_moments(T, nd, &M, com);
    for (int a = 0; a < 3; ++a) dv[a] = r[a] - com[a];
    min_image(T, dv);
    node_geom(T, nd, cen, half);
    for (int a = 0; a < 3; ++a) rc[a] = r[a] - cen[a];
    min_image(T, rc);
    int outside = 0;
    for (int a = 0; a < 3; ++a) if (fabs(rc[a]) > P->safe_box * half[a]) outside = 1;
    double d2 = dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2];
    double B2, B3, bmax2 = 0, d = sqrt(d2);
    node_bmom(T, nd, &B2, &B3);
    for (int a = 0; a < 3; ++a) {
        double t = half[a] + fabs(com[a] - cen[a]);
        bmax2 += t * t;
    }
    double bmax = sqrt(bmax2);
    if (!outside || !(d > bmax)) return INFINITY;
    double q = 1 - bmax / d;
    double da = P->G / d2 / (q * q) * (3 * B2 / d2 - 2 * B3 / (d2 * d));
    return da * da;
}

static void sq_accept(const otree* T, const wparams* P, const double r[3], onode nd, wacc* acc) {
    double M, com[3], dv[3];
    node_moments(T, nd, &M, com);
    for (int a = 0; a < 3; ++a) dv[a] = r[a] - com[a];
    min_image(T, dv);
    interact(P, T, M, dv, acc);
}

/* The frontier's summed squares, kept exactly: each bound counts as ceil(2^20 e2 / a_lim^2) in an
 * integer sum (adding and removing terms in any order gives the same sum, so terms of very
 * different size cannot absorb one another), bounds of 2^30 a_lim^2 or more are counted apart as
 * "large" (a frontier holding one cannot meet the limit); the limit holds when nothing is large and
 * the sum is at most 2^20.  (The rounding up overstates the sum by at most n 2^-20 a_lim^2.) */
#define SQ_ONE 1048576.0                 /* 2^20 */
#define SQ_LARGE 1073741824.0            /* 2^30 */
static int64_t sq_units(double e2, double lim2, int* large) {
    double t = e2 / lim2;
    if (!(t < SQ_LARGE)) { *large = 1; return 0; }
    *large = 0;
    return (int64_t)ceil(t * SQ_ONE);
}

static int64_t sumsq_walk(const otree* T, const wparams* P, const double r[3], int tn, int tc, int qmax, sq_item* h,
                          wacc* acc) {
    int n = 0, n_large = 0, lg;
    int64_t E = 0, u;
    const double lim2 = P->a_lim * P->a_lim;
    onode root = {0, 0, -1, 0};
    sq_item it = {sq_bound2(T, P, r, root), sq_key(T, root), root};
    acc->n_mac++;
    u = sq_units(it.e2, lim2, &lg);
    n_large += lg; E += u;
    sq_push(h, &n, it);
    int64_t overflow = 0;
    while (n > 0 && (n_large > 0 || E > (int64_t)SQ_ONE)) {
        if (n - 1 + 8 > qmax) { overflow = 1; break; }
        sq_item top = sq_pop(h, &n);
        u = sq_units(top.e2, lim2, &lg);
        n_large -= lg; E -= u;
        onode ch[8];
        int nc = node_children(T, top.nd, ch);
        for (int o = 0; o < nc; ++o) {
            if (ch[o].kind == 3) {
                if (ch[o].n == tn && ch[o].idx == tc) continue;
                sq_accept(T, P, r, ch[o], acc);
                continue;
            }
            sq_item c = {sq_bound2(T, P, r, ch[o]), sq_key(T, ch[o]), ch[o]};
            acc->n_mac++;
            u = sq_units(c.e2, lim2, &lg);
            n_large += lg; E += u;
            sq_push(h, &n, c);
        }
    }
    for (int i = 0; i < n; ++i) sq_accept(T, P, r, h[i].nd, acc);
    return overflow;
}

/* Exported: the SumSquare walk at target cells; a_lim is the limit on the root of the summed
 * squared bounds; counts[0] interactions, [1] bounds evaluated, [2] targets whose queue filled. */
int or_gravity_walk_sumsq(int nb, const int* level, const int* child, const double* lo, const double* size,
                          const double* rho, const int* bc, double safe_box, double a_lim, double G, int queue_max,
                          int64_t nt, const int64_t* targets, double* pot, double* acc, int64_t* counts) {
    otree T;
    if (queue_max < 9) return -3;
    if (otree_build(&T, nb, level, child, lo, size, rho, bc)) { otree_free(&T); return -1; }
    if (otree_bmoments(&T)) { otree_free(&T); return -1; }
    wparams P;
    if (setup_walk(&P, &T, bc, 2, 0.0, safe_box, a_lim, G, 0, NULL, 0, NULL)) { otree_free(&T); return -2; }
    int64_t ni = 0, nm = 0, no = 0;
    #pragma omp parallel reduction(+ : ni, nm, no)
    {
        sq_item* h = (sq_item*)malloc(sizeof(sq_item) * (size_t)queue_max);
        #pragma omp for schedule(dynamic, 4)
        for (int64_t t = 0; t < nt; ++t) {
            int n = (int)(targets[t] / NCB), c = (int)(targets[t] % NCB), b = T.block_of[n];
            double r[3];
            cell_centre(&T, b, c & 7, (c >> 3) & 7, c >> 6, r);
            wacc A = {0, {0, 0, 0}, 0, 0};
            no += h ? sumsq_walk(&T, &P, r, n, c, queue_max, h, &A) : 0;
            pot[t] = A.phi;
            for (int a = 0; a < 3; ++a) acc[3 * t + a] = A.a[a];
            ni += A.n_int; nm += A.n_mac;
        }
        free(h);
    }
    if (counts) { counts[0] = ni; counts[1] = nm; counts[2] = no; }
    otree_free(&T);
    return 0;
}

/* Exported: the reference "N^2" solution (Sec. 3): every target cell against every other cell,
 * as point masses at cell centres; 1/|d| for isolated BCs, the Ewald series phi/A otherwise. */
int or_direct_sum(int nb, const int* level, const int* child, const double* lo, const double* size,
                  const double* rho, const int* bc, double G, int64_t nt, const int64_t* targets,
                  double* pot, double* acc) {
    otree T;
    if (otree_build(&T, nb, level, child, lo, size, rho, bc)) { otree_free(&T); return -1; }
    ewcfg E;
    int kind = ew_kind_from_bc(bc);
    if (kind < 0) { otree_free(&T); return -2; }
    ew_setup(&E, kind, T.L, 2.0, 15, 10);
    int64_t ncell = (int64_t)T.nleaf * NCB;
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < nt; ++t) {
        int n = (int)(targets[t] / NCB), c = (int)(targets[t] % NCB);
        double r[3];
        cell_centre(&T, T.block_of[n], c & 7, (c >> 3) & 7, c >> 6, r);
        double phi = 0, a3[3] = {0, 0, 0};
        for (int64_t s = 0; s < ncell; ++s) {
            if (s == targets[t]) continue;
            int sn = (int)(s / NCB), sc = (int)(s % NCB);
            double rs[3], dv[3];
            cell_centre(&T, T.block_of[sn], sc & 7, (sc >> 3) & 7, sc >> 6, rs);
            for (int a = 0; a < 3; ++a) dv[a] = r[a] - rs[a];
            min_image(&T, dv);
            double m = T.cm[s];
            if (kind == EW_NONE) {
                double u = dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2], rr = sqrt(u);
                phi -= G * m / rr;
                for (int a = 0; a < 3; ++a) a3[a] -= G * m * dv[a] / (u * rr);
            } else {
                double p, A[3];
                ewald_eval(&E, dv, 0, &p, A);
                phi -= G * m * p;
                for (int a = 0; a < 3; ++a) a3[a] -= G * m * A[a];
            }
        }
        pot[t] = phi;
        for (int a = 0; a < 3; ++a) acc[3 * t + a] = a3[a];
    }
    otree_free(&T);
    return 0;
}

/* ======================================================================================
 * HEALPix, RING scheme (Gorski et al. 2005): 12 nside^2 equal-area pixels on 4 nside - 1
 * iso-latitude rings.  Polar caps: ring i (1 <= i < nside from the pole) has 4 i pixels at
 * z = +-(1 - i^2/(3 nside^2)); equatorial rings i = nside..3 nside have 4 nside pixels at
 * z = 4/3 - 2 i/(3 nside).
 * ====================================================================================== */
static int64_t ang2pix_ring(int64_t ns, double z, double phi) {
    z = fmin(1.0, fmax(-1.0, z));
    double za = fabs(z);
    double tt = fmod(phi, 2 * M_PI);
    if (tt < 0) tt += 2 * M_PI;
    tt /= 0.5 * M_PI;                                     /* in [0, 4) */
    if (za <= 2.0 / 3.0) {
        /* equatorial belt: pixel edges are the lines ns(t + 1/2) -+ (3/4) ns z = integer */
        double a = ns * (0.5 + tt), bq = 0.75 * ns * z;
        int64_t jp = (int64_t)floor(a - bq), jm = (int64_t)floor(a + bq);
        int64_t ir = ns + 1 + jp - jm;                   /* 1 .. 2 ns + 1, counted from z = 2/3 */
        int64_t kshift = 1 - (ir & 1);
        int64_t ip = (jp + jm - ns + kshift + 1) / 2;
        ip %= 4 * ns;
        if (ip < 0) ip += 4 * ns;
        return 2 * ns * (ns - 1) + (ir - 1) * 4 * ns + ip;
    }
    double tp = tt - floor(tt);
    double tmp = ns * sqrt(3.0 * (1.0 - za));
    int64_t jp = (int64_t)floor(tp * tmp), jm = (int64_t)floor((1.0 - tp) * tmp);
    int64_t ir = jp + jm + 1;                            /* ring counted from the pole */
    int64_t ip = (int64_t)floor(tt * ir);
    ip %= 4 * ir;
    if (z > 0) return 2 * ir * (ir - 1) + ip;
    return 12 * ns * ns - 2 * ir * (ir + 1) + ip;
}

static void pix2ang_ring(int64_t ns, int64_t pix, double* z, double* phi) {
    int64_t npix = 12 * ns * ns, ncap = 2 * ns * (ns - 1);
    if (pix < ncap) {
        int64_t p = pix + 1;
        int64_t ir = (int64_t)floor(0.5 * (1.0 + sqrt(2.0 * p - 1.0)));
        int64_t ip = p - 2 * ir * (ir - 1);
        *z = 1.0 - (double)(ir * ir) / (3.0 * ns * ns);
        *phi = (ip - 0.5) * M_PI / (2.0 * ir);
    } else if (pix < npix - ncap) {
        int64_t p = pix - ncap;
        int64_t ir = p / (4 * ns) + ns;
        int64_t ip = p % (4 * ns) + 1;
        double fodd = ((ir + ns) & 1) ? 1.0 : 0.5;
        *z = (2.0 * ns - ir) * 2.0 / (3.0 * ns);
        *phi = (ip - fodd) * M_PI / (2.0 * ns);
    } else {
        int64_t p = npix - pix;
        int64_t ir = (int64_t)floor(0.5 * (1.0 + sqrt(2.0 * p - 1.0)));
        int64_t ip = 4 * ir + 1 - (p - 2 * ir * (ir - 1));
        *z = -1.0 + (double)(ir * ir) / (3.0 * ns * ns);
        *phi = (ip - 0.5) * M_PI / (2.0 * ir);
    }
}

void or_healpix_vec2pix(int nside, int64_t n, const double* v, int64_t* pix) {
    for (int64_t i = 0; i < n; ++i) {
        const double* u = v + 3 * i;
        double r = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        pix[i] = ang2pix_ring(nside, u[2] / r, atan2(u[1], u[0]));
    }
}

void or_healpix_pix2ang(int nside, int64_t n, const int64_t* pix, double* z, double* phi) {
    for (int64_t i = 0; i < n; ++i) pix2ang_ring(nside, pix[i], z + i, phi + i);
}

/* ======================================================================================
 * Node-ray weight table (Sec. 2.3): for a node at polar angle theta, azimuth phi and angular
 * size psi = h/d as seen from the target, the fraction w_i of the node that lies in HEALPix
 * pixel i.  Reading: the node is an axis-aligned uniform cube of edge psi at unit distance,
 * split into nsub^3 equal sub-cubes, each assigned to the pixel of its centre's direction.
 * Bins: theta uniform in [0, pi] (ntheta), phi uniform in [0, 2 pi) (nphi), psi log-uniform in
 * [psi_min, psi_max] (npsi); entries are evaluated at bin centres.  w[it][ip][is][npix].
 * ====================================================================================== */
static void bin_centre(int it, int ip, int is, int nt, int nph, int nps, double pmin, double pmax,
                       double* th, double* ph, double* ps) {
    *th = (it + 0.5) * M_PI / nt;
    *ph = (ip + 0.5) * 2 * M_PI / nph;
    *ps = pmin * pow(pmax / pmin, (is + 0.5) / nps);
}

static void cube_weights(int ns, double th, double ph, double ps, int nsub, double* w) {
    int npix = 12 * ns * ns;
    double c[3] = {sin(th) * cos(ph), sin(th) * sin(ph), cos(th)};
    for (int i = 0; i < npix; ++i) w[i] = 0;
    double inv = 1.0 / ((double)nsub * nsub * nsub);
    for (int a = 0; a < nsub; ++a)
        for (int bq = 0; bq < nsub; ++bq)
            for (int cq = 0; cq < nsub; ++cq) {
                double p[3] = {c[0] + ps * ((a + 0.5) / nsub - 0.5), c[1] + ps * ((bq + 0.5) / nsub - 0.5),
                               c[2] + ps * ((cq + 0.5) / nsub - 0.5)};
                double r = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
                w[ang2pix_ring(ns, p[2] / r, atan2(p[1], p[0]))] += inv;
            }
}

int or_noderay_table(int nside, int ntheta, int nphi, int npsi, double psi_min, double psi_max,
                     int nsub, double* w) {
    int npix = 12 * nside * nside;
    #pragma omp parallel for collapse(2) schedule(dynamic, 4)
    for (int it = 0; it < ntheta; ++it)
        for (int ip = 0; ip < nphi; ++ip)
            for (int is = 0; is < npsi; ++is) {
                double th, ph, ps;
                bin_centre(it, ip, is, ntheta, nphi, npsi, psi_min, psi_max, &th, &ph, &ps);
                cube_weights(nside, th, ph, ps, nsub,
                             w + (((size_t)it * nphi + ip) * npsi + is) * npix);
            }
    return 0;
}

/* ======================================================================================
 * Column-density walk (Sec. 2.3, the OpticalDepth module): the same depth-first walk with the
 * BH MAC and safe box; each accepted node of mass M at distance d adds M w_i / (Omega_pix d^2)
 * to pixel i of the target's map, Omega_pix = 4 pi / N_PIX (eq. for Omega_PIX).  The target's
 * own cell adds rho dx/2 to every pixel.  Periodic axes use the minimum image; nodes farther than
 * max_dist are skipped.
 * ====================================================================================== */
typedef struct {
    double theta, safe_box, max_dist;
    int nside, ntheta, nphi, npsi, nsub;
    double psi_min, psi_max;
    const double* w;      /* table, or NULL: weights by direct sub-cube quadrature per node */
} cparams;

static void column_node(const cparams* P, double M, const double dv[3], double h, double* col) {
    /* dv = r - r_a; the node lies in direction -dv from the target */
    double u[3] = {-dv[0], -dv[1], -dv[2]};
    double d = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    if (d > P->max_dist) return;
    int npix = 12 * P->nside * P->nside;
    double omega = 4 * M_PI / npix, f = M / (omega * d * d);
    double th = acos(fmax(-1.0, fmin(1.0, u[2] / d))), ph = atan2(u[1], u[0]);
    if (ph < 0) ph += 2 * M_PI;
    double ps = h / d;
    if (P->w) {
        int it = (int)floor(th / M_PI * P->ntheta), ip = (int)floor(ph / (2 * M_PI) * P->nphi);
        int is = (int)floor(P->npsi * log(ps / P->psi_min) / log(P->psi_max / P->psi_min));
        if (it < 0) it = 0; if (it >= P->ntheta) it = P->ntheta - 1;
        if (ip < 0) ip = 0; if (ip >= P->nphi) ip = P->nphi - 1;
        if (is < 0) is = 0; if (is >= P->npsi) is = P->npsi - 1;
        const double* w = P->w + (((size_t)it * P->nphi + ip) * P->npsi + is) * npix;
        for (int i = 0; i < npix; ++i) col[i] += f * w[i];
    } else {
        double w[12 * 16 * 16];
        cube_weights(P->nside, th, ph, ps, P->nsub, w);
        for (int i = 0; i < npix; ++i) col[i] += f * w[i];
    }
}

/* The walk decides with the total mass (its centre of mass, its MAC); an accepted node adds its
 * total mass to map 0 and the mass of each extra quantity k (the same node of the tree TQ[k] built
 * from that quantity's density) to map 1 + k, with the same node-ray weights (Sec. 2.3: l_q maps
 * filled by the same walk). */
static void column_walk_rec(const otree* T, const otree* TQ, int nq, const cparams* P, const double r[3], int tn,
                            int tc, onode nd, double* col, int64_t* ni) {
    double M, com[3], dv[3], cen[3], half[3];
    node_moments(T, nd, &M, com);
    node_geom(T, nd, cen, half);
    for (int a = 0; a < 3; ++a) dv[a] = r[a] - com[a];
    min_image(T, dv);
    double h = 2 * fmax(half[0], fmax(half[1], half[2]));
    const int npix = 12 * P->nside * P->nside;
    int accept;
    if (nd.kind == 3) {
        if (nd.n == tn && nd.idx == tc) return;
        accept = 1;
    } else {
        double rc[3];
        for (int a = 0; a < 3; ++a) rc[a] = r[a] - cen[a];
        min_image(T, rc);
        int outside = 0;
        for (int a = 0; a < 3; ++a) if (fabs(rc[a]) > P->safe_box * half[a]) outside = 1;
        double d2 = dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2];
        accept = outside && h * h < P->theta * P->theta * d2;
    }
    if (accept) {
        column_node(P, M, dv, h, col);
        for (int k = 0; k < nq; ++k) {
            double Mq, comq[3];
            node_moments(&TQ[k], nd, &Mq, comq);
            column_node(P, Mq, dv, h, col + (size_t)(1 + k) * npix);
        }
        ++*ni;
        return;
    }
    onode ch[8];
    int nc = node_children(T, nd, ch);
    for (int o = 0; o < nc; ++o) column_walk_rec(T, TQ, nq, P, r, tn, tc, ch[o], col, ni);
}

/* Column maps of the total mass and of nq (0..2) extra quantities with densities q [nq][ncell]:
 * cols [nt][1 + nq][npix]. */
int or_column_walk_q(int nb, const int* level, const int* child, const double* lo, const double* size,
                     const double* rho, int nq, const double* q, const int* bc, double theta, double safe_box,
                     double max_dist, int nside, int ntheta, int nphi, int npsi, double psi_min, double psi_max,
                     int nsub, const double* table, int64_t nt, const int64_t* targets, double* cols,
                     int64_t* counts) {
    otree T, TQ[2];
    if (nside < 1 || nside > 16 || nq < 0 || nq > 2) return -3;
    if (otree_build(&T, nb, level, child, lo, size, rho, bc)) { otree_free(&T); return -1; }
    int64_t ncell = (int64_t)T.nleaf * NCB;
    for (int k = 0; k < nq; ++k)
        if (otree_build(&TQ[k], nb, level, child, lo, size, q + (size_t)k * ncell, bc)) {
            for (int j = 0; j <= k; ++j) otree_free(&TQ[j]);
            otree_free(&T);
            return -1;
        }
    cparams P = {theta, safe_box, max_dist, nside, ntheta, nphi, npsi, nsub, psi_min, psi_max, table};
    int npix = 12 * nside * nside, lq = 1 + nq;
    int64_t ni = 0;
    #pragma omp parallel for schedule(dynamic, 8) reduction(+ : ni)
    for (int64_t t = 0; t < nt; ++t) {
        int n = (int)(targets[t] / NCB), c = (int)(targets[t] % NCB), b = T.block_of[n];
        double r[3], *col = cols + t * lq * npix;
        cell_centre(&T, b, c & 7, (c >> 3) & 7, c >> 6, r);
        for (int i = 0; i < lq * npix; ++i) col[i] = 0;
        onode root = {0, 0, -1, 0};
        int64_t cnt = 0;
        column_walk_rec(&T, TQ, nq, &P, r, n, c, root, col, &cnt);
        for (int k = 0; k < lq; ++k) {
            const double* dens = k == 0 ? rho : q + (size_t)(k - 1) * ncell;
            double own = dens[targets[t]] * 0.5 * T.size[3 * b] / NB;   /* own cell: rho dx / 2 */
            for (int i = 0; i < npix; ++i) col[k * npix + i] += own;
        }
        ni += cnt;
    }
    if (counts) counts[0] = ni;
    for (int k = 0; k < nq; ++k) otree_free(&TQ[k]);
    otree_free(&T);
    return 0;
}

int or_column_walk(int nb, const int* level, const int* child, const double* lo, const double* size,
                   const double* rho, const int* bc, double theta, double safe_box, double max_dist,
                   int nside, int ntheta, int nphi, int npsi, double psi_min, double psi_max, int nsub,
                   const double* table, int64_t nt, const int64_t* targets, double* cols, int64_t* counts) {
    return or_column_walk_q(nb, level, child, lo, size, rho, 0, NULL, bc, theta, safe_box, max_dist, nside, ntheta,
                            nphi, npsi, psi_min, psi_max, nsub, table, nt, targets, cols, counts);
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
