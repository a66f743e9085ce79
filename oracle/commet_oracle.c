/*
 * FP64 CPU oracle for the neural-constitutive hot path of COMMET
 * (Alheit, Peirlinck & Kumar, "COMMET: orders-of-magnitude speed-up in finite
 * element method via batch-vectorized neural constitutive updates").
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may call, link or load
 * this file: only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark use it. It shares no code, header, table or constant with the CUDA
 * library; the two meet only through seeded inputs.
 *
 * Everything is plain double precision, one quadrature point (qp) or one
 * element at a time, with fourth-order tensors written out as 81 entries.
 * Index conventions:
 *   F_iJ  -> F[3*i + J]                 (row = spatial i, column = material J)
 *   A_iJkL = d2Psi/dF_iJ dF_kL -> A[(3*i+J)*9 + 3*k+L]      (App. A.1)
 *   hex8 nodes lexicographic in (xi, eta, zeta), x fastest; 2x2x2 Gauss points
 *   at +-1/sqrt(3), weight 1, same order; element dof 3*I + i (Sec. 2.1).
 * Per-qp arrays are qp-major here (AoS: F[q][9], P[q][9], A[q][81]); element
 * arrays are element-major (f_e[e][24], K_e[e][24][24]).
 *
 * Functions and the passages they follow:
 *   kinematic layer K(F, A^i) and dK/dF, d2K/dF2 .... Eq. 454, App. A.2 (isochoric
 *                                                     invariants), material form
 *   MICNN value, gradient, Hessian (one pass) ........ Eq. icnn, Algorithm 4
 *   closed-form inner functions (Gent-Thomas, HGO) ... Eq. gt (App. C); target model
 *   P and A by the CGO chain rule .................... Eq. nncm-chain, App. A.1 (P, C^P)
 *   F at a qp ........................................ Algorithm 1 (trial F)
 *   f_int and K_e per element ........................ Eq. r-quad, k-quad (material form)
 *   Kirchhoff stress, spatial stiffness (Voigt) ...... App. A.1 (push-forward of P, A)
 *   f_int and K_e from tau, c ........................ Eq. r-quad, k-quad (spatial form)
 *   backward dL/dF, dL/dtheta (MICNN, CANN) .......... chain rule on G : P(F; theta)
 *   adjoints of r-quad and of the trial F ............. transposes for a residual loss (eq. loss)
 *
 * Parity status: every function here is pinned by the CPU tests (closed forms,
 * hyper-dual exact derivatives, finite differences, invariance, patch tests);
 * none is "parity unpinned".
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ model */

enum { OR_KIN_ISO_SHIFTED = 0, OR_KIN_RAW = 1, OR_KIN_POLYCONVEX = 2 };
enum { OR_INNER_MICNN = 0, OR_INNER_GENT_THOMAS = 1, OR_INNER_HGO = 2, OR_INNER_CANN = 3, OR_INNER_ICKAN = 4 };
enum { OR_F0_ID = 0, OR_F0_MACAULAY = 1, OR_F0_ABS = 2 };
enum { OR_F2_LINEAR = 0, OR_F2_EXP = 1, OR_F2_LOG = 2 };

/*
 * Strain-energy model Psi(F) = N(K(F)) + kappa (J-1)^2 [- n0 . (K - K0)].
 * Kinematic layer (kin):
 *   OR_KIN_ISO_SHIFTED: K = (Ibar1 - 3, Ibar2 - 3, J - 1),                  d = 3
 *   OR_KIN_RAW:         K = (Ibar1, Ibar2, J, I4_11..I4_nn, I5_11..I5_nn),   d = 3 + 2 n_fib
 *   OR_KIN_POLYCONVEX:  K = (Ibar1 - 3, Ibar2^{3/2} - 3^{3/2}, (J - 1)^2),     d = 3
 *                       (the kinematic layer of the paper's trained NCMs, App. C)
 * Inner function (inner):
 *   OR_INNER_MICNN: eq. icnn with n-1 = L hidden layers. Layer 1 carries one
 *     matrix W1 (A^(1) acting on z^(0) = K and B^(1) acting on K act on the
 *     same vector, so they are one matrix); layers k = 2..L carry A_k (W x W),
 *     B_k (W x d), c_k; the output is a . z^(L) + b . K (no output bias).
 *   OR_INNER_GENT_THOMAS: N = 0.5 (K0 - 3) + log(K1 / 3) + (K2 - 1)^2 on raw
 *     (Ibar1, Ibar2, J)  (eq. gt).
 *   OR_INNER_HGO: N = mu/2 (K0 - 3) + sum_f k1/(2 k2) (exp(k2 (K_{3+f} - 1)^2) - 1)
 *     on raw kinematics (Neo-Hookean plus exponential fibre terms).
 *   OR_INNER_ICKAN: the KAN of App. B, z^(r)_i = sum_j phi_rij(z^(r-1)_j), N = z^(R),
 *     phi = w_s psi, psi = sum_l c_l B_l,k (B-splines by the recursion of App. B).
 *   OR_INNER_CANN: eq. cann-def, N = sum_m sum_k w2_mk f2_k(f1_k(f0_k(K_m)); w1_mk) with
 *     term k's functions from the menus of eq. cann-fs: f0 in {x, <x>, |x|}, f1 = x^p
 *     (p = 1, 2, 3), f2 in {w1 y, exp(w1 y) - 1, -ln(1 - w1 y)}.
 * stress_free: subtract n0 . (K - K0), n0 = dN/dK at K0 = K(I), so that P(I) = 0.
 */
typedef struct {
    int d, W, L;
    int kin;
    int n_fib;
    const double *fib; /* [n_fib][3] reference structural vectors A^i */
    int inner;
    const double *W1; /* [W][d] */
    const double *Ak; /* [L-1][W][W] */
    const double *Bk; /* [L-1][W][d] */
    const double *c;  /* [L][W] or NULL (= 0) */
    const double *a;  /* [W] */
    const double *b;  /* [d] */
    double kappa;
    int stress_free;
    double mu, k1, k2;
    int cann_n;             /* CANN: terms per input */
    const int *cann_kind;   /* CANN: [n][3] (f0, p, f2) */
    const double *cann_w;   /* CANN: [d][n][2] (w1, w2) */
    /* ICKAN: R spline layers of widths kw[0] = d, kw[1..R-1], kw[R] = 1; B-splines of degree
     * kdeg on G uniform intervals of [lo_r, hi_r] per layer (knots extended by kdeg on each
     * side, nb = G + kdeg basis functions); per spline (layer r, output i, input j, in that
     * order) the weight w_s then the nb control points. */
    int kan_R, kan_deg, kan_G;
    const int *kan_w;
    const double *kan_lo, *kan_hi, *kan_par;
} oracle_model;

#define OR_MAXD 16
#define OR_MAXW 128

/* ------------------------------------------------------- small tensor help */

static int levi(int i, int j, int k) {
    /* Levi-Civita symbol eps_ijk for i,j,k in {0,1,2}. */
    if (i == j || j == k || i == k) return 0;
    if ((i == 0 && j == 1 && k == 2) || (i == 1 && j == 2 && k == 0) || (i == 2 && j == 0 && k == 1)) return 1;
    return -1;
}

static double kd(int i, int j) { return i == j ? 1.0 : 0.0; }

/* cof F_iJ = 1/2 eps_ikl eps_JKL F_kK F_lL ; det F = 1/3 F_iJ cof F_iJ */
static void cofactor(const double *F, double *cof, double *detF) {
    for (int i = 0; i < 3; ++i)
        for (int J = 0; J < 3; ++J) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l)
                    for (int K = 0; K < 3; ++K)
                        for (int L = 0; L < 3; ++L) {
                            int e = levi(i, k, l) * levi(J, K, L);
                            if (e) s += 0.5 * e * F[3 * k + K] * F[3 * l + L];
                        }
            cof[3 * i + J] = s;
        }
    double d = 0.0;
    for (int i = 0; i < 9; ++i) d += F[i] * cof[i];
    *detF = d / 3.0;
}

/* ------------------------------------------------------- kinematic layer */

/*
 * One invariant with its first (9) and second (81) derivatives w.r.t. F.
 * Standard invariants (eq. 454): I1 = tr C, I2 = 1/2 (tr C^2... ), J = det F,
 * I4 = A.CA, I5 = A.C^2 A, differentiated by hand in material form:
 *   dI1/dF_iJ = 2 F_iJ ;            d2I1 = 2 d_ik d_JL
 *   dI2/dF    = 2 (I1 F - F C) ;    d2I2 = 4 F_iJ F_kL + 2 I1 d_ik d_JL - 2 d_ik C_JL
 *                                          - 2 F_iL F_kJ - 2 B_ik d_JL
 *   dJ/dF     = cof F ;             d2J  = eps_ikm eps_JLM F_mM
 *   dI4/dF_kL = 2 a_k A_L ;         d2I4 = 2 d_ik A_J A_L           (a = F A)
 *   dI5/dF_kL = 2 (a_k v_L + (F v)_k A_L)                           (v = C A)
 *   d2I5 = 2 [d_JL a_i a_k + F_iL A_J a_k + d_ik A_J v_L + d_ik v_J A_L
 *             + F_kJ a_i A_L + B_ik A_J A_L]
 */
static void inv_I1(const double *F, double *v, double *g, double *h) {
    double s = 0.0;
    for (int i = 0; i < 9; ++i) s += F[i] * F[i];
    *v = s;
    for (int i = 0; i < 9; ++i) g[i] = 2.0 * F[i];
    for (int i = 0; i < 3; ++i)
        for (int J = 0; J < 3; ++J)
            for (int k = 0; k < 3; ++k)
                for (int L = 0; L < 3; ++L) h[(3 * i + J) * 9 + 3 * k + L] = 2.0 * kd(i, k) * kd(J, L);
}

static void right_cg(const double *F, double *C) {
    for (int I = 0; I < 3; ++I)
        for (int J = 0; J < 3; ++J) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += F[3 * k + I] * F[3 * k + J];
            C[3 * I + J] = s;
        }
}

static void left_cg(const double *F, double *B) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int K = 0; K < 3; ++K) s += F[3 * i + K] * F[3 * j + K];
            B[3 * i + j] = s;
        }
}

static void inv_I2(const double *F, double *v, double *g, double *h) {
    double C[9], B[9], I1 = 0.0, trC2 = 0.0;
    right_cg(F, C);
    left_cg(F, B);
    for (int I = 0; I < 3; ++I) I1 += C[4 * I];
    for (int I = 0; I < 3; ++I)
        for (int J = 0; J < 3; ++J) trC2 += C[3 * I + J] * C[3 * J + I];
    *v = 0.5 * (I1 * I1 - trC2);
    for (int i = 0; i < 3; ++i)
        for (int J = 0; J < 3; ++J) {
            double FC = 0.0;
            for (int K = 0; K < 3; ++K) FC += F[3 * i + K] * C[3 * K + J];
            g[3 * i + J] = 2.0 * (I1 * F[3 * i + J] - FC);
        }
    for (int i = 0; i < 3; ++i)
        for (int J = 0; J < 3; ++J)
            for (int k = 0; k < 3; ++k)
                for (int L = 0; L < 3; ++L)
                    h[(3 * i + J) * 9 + 3 * k + L] = 4.0 * F[3 * i + J] * F[3 * k + L] + 2.0 * I1 * kd(i, k) * kd(J, L) -
                                                     2.0 * kd(i, k) * C[3 * J + L] - 2.0 * F[3 * i + L] * F[3 * k + J] -
                                                     2.0 * B[3 * i + k] * kd(J, L);
}

static void inv_J(const double *F, double *v, double *g, double *h) {
    double cof[9], J;
    cofactor(F, cof, &J);
    *v = J;
    for (int i = 0; i < 9; ++i) g[i] = cof[i];
    for (int i = 0; i < 3; ++i)
        for (int J_ = 0; J_ < 3; ++J_)
            for (int k = 0; k < 3; ++k)
                for (int L = 0; L < 3; ++L) {
                    double s = 0.0;
                    for (int m = 0; m < 3; ++m)
                        for (int M = 0; M < 3; ++M) s += levi(i, k, m) * levi(J_, L, M) * F[3 * m + M];
                    h[(3 * i + J_) * 9 + 3 * k + L] = s;
                }
}

static void inv_I4(const double *F, const double *A0, double *v, double *g, double *h) {
    double a[3];
    for (int i = 0; i < 3; ++i) a[i] = F[3 * i] * A0[0] + F[3 * i + 1] * A0[1] + F[3 * i + 2] * A0[2];
    *v = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
    for (int k = 0; k < 3; ++k)
        for (int L = 0; L < 3; ++L) g[3 * k + L] = 2.0 * a[k] * A0[L];
    for (int i = 0; i < 3; ++i)
        for (int J = 0; J < 3; ++J)
            for (int k = 0; k < 3; ++k)
                for (int L = 0; L < 3; ++L) h[(3 * i + J) * 9 + 3 * k + L] = 2.0 * kd(i, k) * A0[J] * A0[L];
}

static void inv_I5(const double *F, const double *A0, double *v, double *g, double *h) {
    double C[9], B[9], a[3], vv[3], Fv[3];
    right_cg(F, C);
    left_cg(F, B);
    for (int i = 0; i < 3; ++i) a[i] = F[3 * i] * A0[0] + F[3 * i + 1] * A0[1] + F[3 * i + 2] * A0[2];
    for (int I = 0; I < 3; ++I) vv[I] = C[3 * I] * A0[0] + C[3 * I + 1] * A0[1] + C[3 * I + 2] * A0[2];
    for (int i = 0; i < 3; ++i) Fv[i] = F[3 * i] * vv[0] + F[3 * i + 1] * vv[1] + F[3 * i + 2] * vv[2];
    *v = vv[0] * vv[0] + vv[1] * vv[1] + vv[2] * vv[2];
    for (int k = 0; k < 3; ++k)
        for (int L = 0; L < 3; ++L) g[3 * k + L] = 2.0 * (a[k] * vv[L] + Fv[k] * A0[L]);
    for (int i = 0; i < 3; ++i)
        for (int J = 0; J < 3; ++J)
            for (int k = 0; k < 3; ++k)
                for (int L = 0; L < 3; ++L)
                    h[(3 * i + J) * 9 + 3 * k + L] =
                        2.0 * (kd(J, L) * a[i] * a[k] + F[3 * i + L] * A0[J] * a[k] + kd(i, k) * A0[J] * vv[L] +
                               kd(i, k) * vv[J] * A0[L] + F[3 * k + J] * a[i] * A0[L] + B[3 * i + k] * A0[J] * A0[L]);
}

/*
 * Isochoric invariant Ibar = I * I3^alpha = J^q I with q = 2 alpha
 * (alpha = -1/3 for I1, -2/3 for I2; App. A.2). With H = F^{-T} = dlnJ/dF and
 * dH_iJ/dF_kL = -H_iL H_kJ:
 *   dIbar   = J^q (dI + q I H)
 *   d2Ibar  = J^q [d2I + q (dI (x) H + H (x) dI) + q^2 I H (x) H - q I H_iL H_kJ]
 */
static void isochoric(double q, const double *F, double I, const double *gI, const double *hI, double *v, double *g,
                      double *h) {
    double cof[9], J, H[9];
    cofactor(F, cof, &J);
    for (int i = 0; i < 9; ++i) H[i] = cof[i] / J;
    double Jq = pow(J, q);
    *v = Jq * I;
    for (int i = 0; i < 9; ++i) g[i] = Jq * (gI[i] + q * I * H[i]);
    for (int i = 0; i < 3; ++i)
        for (int J_ = 0; J_ < 3; ++J_)
            for (int k = 0; k < 3; ++k)
                for (int L = 0; L < 3; ++L) {
                    int a = 3 * i + J_, b = 3 * k + L;
                    h[a * 9 + b] = Jq * (hI[a * 9 + b] + q * (gI[a] * H[b] + H[a] * gI[b]) + q * q * I * H[a] * H[b] -
                                         q * I * H[3 * i + L] * H[3 * k + J_]);
                }
}

/* K(F) with dK/dF [d][9] and d2K/dF2 [d][81]. Returns d. */
static int oracle_kinematics(const oracle_model *m, const double *F, double *K, double *dK, double *d2K) {
    double v, g[9], h[81];
    double I1, g1[9], h1[81], I2, g2[9], h2[81];
    inv_I1(F, &I1, g1, h1);
    isochoric(-2.0 / 3.0, F, I1, g1, h1, &K[0], &dK[0], &d2K[0]);
    inv_I2(F, &I2, g2, h2);
    isochoric(-4.0 / 3.0, F, I2, g2, h2, &K[1], &dK[9], &d2K[81]);
    inv_J(F, &v, g, h);
    K[2] = v;
    memcpy(&dK[18], g, sizeof g);
    memcpy(&d2K[162], h, sizeof h);
    if (m->kin == OR_KIN_ISO_SHIFTED) {
        K[0] -= 3.0;
        K[1] -= 3.0;
        K[2] -= 1.0;
        return 3;
    }
    if (m->kin == OR_KIN_POLYCONVEX) {
        /* K_m = phi_m(I_m) of an invariant: dK = phi' dI, d2K = phi'' dI (x) dI + phi' d2I */
        const double Ib2 = K[1], Jv = K[2];
        const double d1[3] = {1.0, 1.5 * sqrt(Ib2), 2.0 * (Jv - 1.0)};
        const double d2[3] = {0.0, 0.75 / sqrt(Ib2), 2.0};
        for (int m2 = 0; m2 < 3; ++m2) {
            for (int a = 0; a < 9; ++a)
                for (int b = 0; b < 9; ++b)
                    d2K[81 * m2 + a * 9 + b] = d2[m2] * dK[9 * m2 + a] * dK[9 * m2 + b] + d1[m2] * d2K[81 * m2 + a * 9 + b];
            for (int a = 0; a < 9; ++a) dK[9 * m2 + a] *= d1[m2];
        }
        K[0] -= 3.0;
        K[1] = Ib2 * sqrt(Ib2) - 3.0 * sqrt(3.0);
        K[2] = (Jv - 1.0) * (Jv - 1.0);
        return 3;
    }
    int nf = m->n_fib;
    for (int f = 0; f < nf; ++f) {
        inv_I4(F, &m->fib[3 * f], &K[3 + f], &dK[9 * (3 + f)], &d2K[81 * (3 + f)]);
        inv_I5(F, &m->fib[3 * f], &K[3 + nf + f], &dK[9 * (3 + nf + f)], &d2K[81 * (3 + nf + f)]);
    }
    return 3 + 2 * nf;
}

/* ------------------------------------------------------- inner functions */

/* softplus (beta = 1) and its first two derivatives, in a form that does not overflow */
static double softplus(double y) { return (y > 0.0 ? y : 0.0) + log1p(exp(-fabs(y))); }
static double logistic(double y) {
    if (y >= 0.0) return 1.0 / (1.0 + exp(-y));
    double e = exp(y);
    return e / (1.0 + e);
}
/* F''(y) = logistic(y) (1 - logistic(y)), written as e / (1 + e)^2 with e = exp(-|y|): the
 * same function without the cancellation of 1 - logistic(y) once logistic(y) -> 1 (large y),
 * where the product form keeps only a few correct digits of a tiny value */
static double softplus_dd(double y) {
    double e = exp(-fabs(y)), u = 1.0 + e;
    return e / (u * u);
}

/*
 * MICNN value, gradient and Hessian in one pass, following Algorithm 4:
 *   z <- K, dz <- I, d2z <- 0
 *   per hidden layer k: y = A z + B K + c ; dy = A dz + B ; d2y = A d2z ;
 *     d2z = F'(y) * d2y + F''(y) * dy (x) dy ; dz = F'(y) * dy ; z = F(y)
 *   N = A^(n) z + B^(n) K ; dN = A^(n) dz + B^(n) ; d2N = A^(n) d2z
 * Layer 1 uses A = W1 (acting on z = K) and no B; the output layer uses a, b.
 */
static void micnn_alg4(const oracle_model *m, const double *K, double *N, double *dN, double *d2N) {
    const int d = m->d, W = m->W, L = m->L;
    int nin = d; /* current width of z */
    double *z = (double *)calloc(OR_MAXW, sizeof(double));
    double *dz = (double *)calloc((size_t)OR_MAXW * OR_MAXD, sizeof(double));
    double *d2z = (double *)calloc((size_t)OR_MAXW * OR_MAXD * OR_MAXD, sizeof(double));
    double *y = (double *)calloc(OR_MAXW, sizeof(double));
    double *dy = (double *)calloc((size_t)OR_MAXW * OR_MAXD, sizeof(double));
    double *d2y = (double *)calloc((size_t)OR_MAXW * OR_MAXD * OR_MAXD, sizeof(double));
    for (int i = 0; i < d; ++i) {
        z[i] = K[i];
        for (int p = 0; p < d; ++p) dz[i * OR_MAXD + p] = kd(i, p);
    }
    for (int k = 1; k <= L; ++k) {
        const double *A = (k == 1) ? m->W1 : &m->Ak[(size_t)(k - 2) * W * W];
        const double *B = (k == 1) ? NULL : &m->Bk[(size_t)(k - 2) * W * d];
        const double *c = m->c ? &m->c[(size_t)(k - 1) * W] : NULL;
        for (int j = 0; j < W; ++j) {
            double s = c ? c[j] : 0.0;
            for (int i = 0; i < nin; ++i) s += A[j * nin + i] * z[i];
            if (B)
                for (int i = 0; i < d; ++i) s += B[j * d + i] * K[i];
            y[j] = s;
            for (int p = 0; p < d; ++p) {
                double t = B ? B[j * d + p] : 0.0;
                for (int i = 0; i < nin; ++i) t += A[j * nin + i] * dz[i * OR_MAXD + p];
                dy[j * OR_MAXD + p] = t;
                for (int q = 0; q < d; ++q) {
                    double u = 0.0;
                    for (int i = 0; i < nin; ++i) u += A[j * nin + i] * d2z[(i * OR_MAXD + p) * OR_MAXD + q];
                    d2y[(j * OR_MAXD + p) * OR_MAXD + q] = u;
                }
            }
        }
        for (int j = 0; j < W; ++j) {
            double s1 = logistic(y[j]);
            double s2 = softplus_dd(y[j]);
            for (int p = 0; p < d; ++p)
                for (int q = 0; q < d; ++q)
                    d2z[(j * OR_MAXD + p) * OR_MAXD + q] =
                        s1 * d2y[(j * OR_MAXD + p) * OR_MAXD + q] + s2 * dy[j * OR_MAXD + p] * dy[j * OR_MAXD + q];
            for (int p = 0; p < d; ++p) dz[j * OR_MAXD + p] = s1 * dy[j * OR_MAXD + p];
            z[j] = softplus(y[j]);
        }
        nin = W;
    }
    double s = 0.0;
    for (int i = 0; i < W; ++i) s += m->a[i] * z[i];
    for (int i = 0; i < d; ++i) s += m->b[i] * K[i];
    *N = s;
    for (int p = 0; p < d; ++p) {
        double t = m->b[p];
        for (int i = 0; i < W; ++i) t += m->a[i] * dz[i * OR_MAXD + p];
        dN[p] = t;
        for (int q = 0; q < d; ++q) {
            double u = 0.0;
            for (int i = 0; i < W; ++i) u += m->a[i] * d2z[(i * OR_MAXD + p) * OR_MAXD + q];
            d2N[p * d + q] = u;
        }
    }
    free(z);
    free(dz);
    free(d2z);
    free(y);
    free(dy);
    free(d2y);
}

/* Gent-Thomas, eq. gt, on raw (Ibar1, Ibar2, J). */
static void gent_thomas(const double *K, double *N, double *dN, double *d2N) {
    *N = 0.5 * (K[0] - 3.0) + log(K[1] / 3.0) + (K[2] - 1.0) * (K[2] - 1.0);
    dN[0] = 0.5;
    dN[1] = 1.0 / K[1];
    dN[2] = 2.0 * (K[2] - 1.0);
    for (int i = 0; i < 9; ++i) d2N[i] = 0.0;
    d2N[1 * 3 + 1] = -1.0 / (K[1] * K[1]);
    d2N[2 * 3 + 2] = 2.0;
}

/* Neo-Hookean plus exponential fibre terms (HGO type, smooth) on raw kinematics. */
static void hgo(const oracle_model *m, const double *K, double *N, double *dN, double *d2N) {
    const int d = m->d, nf = m->n_fib;
    for (int i = 0; i < d * d; ++i) d2N[i] = 0.0;
    for (int i = 0; i < d; ++i) dN[i] = 0.0;
    double s = 0.5 * m->mu * (K[0] - 3.0);
    dN[0] = 0.5 * m->mu;
    for (int f = 0; f < nf; ++f) {
        double x = K[3 + f] - 1.0, e = exp(m->k2 * x * x);
        s += m->k1 / (2.0 * m->k2) * (e - 1.0);
        dN[3 + f] = m->k1 * x * e;
        d2N[(3 + f) * d + 3 + f] = m->k1 * e * (1.0 + 2.0 * m->k2 * x * x);
    }
    *N = s;
}

/*
 * CANN (eq. cann-def) and its derivatives by the chain rule of eq. cann-chain-rule:
 *   dN/dK_m   = sum_k w2 f2' f1' f0'
 *   d2N/dK_m2 = sum_k w2 [(f2'' f1'^2 + f2' f1'') f0'^2 + f2' f1' f0'']
 * and d2N/dK_m dK_n = 0 for m != n. The menus' derivatives are written from their
 * definitions: d/dy (-ln(1 - w1 y)) = w1 / (1 - w1 y), second derivative
 * + w1^2 / (1 - w1 y)^2 (the printed table has a minus sign here); <x>' = (1 + sign x)/2,
 * |x|' = sign x, both with zero second derivative away from 0.
 */
static void cann(const oracle_model *m, const double *K, double *N, double *dN, double *d2N) {
    const int d = m->d, n = m->cann_n;
    for (int i = 0; i < d * d; ++i) d2N[i] = 0.0;
    double s = 0.0;
    for (int mm = 0; mm < d; ++mm) {
        double g = 0.0, h = 0.0;
        for (int k = 0; k < n; ++k) {
            const int *kind = &m->cann_kind[3 * k];
            const double w1 = m->cann_w[(mm * n + k) * 2], w2 = m->cann_w[(mm * n + k) * 2 + 1];
            const double x = K[mm];
            double f0, f0d, f0dd = 0.0;
            if (kind[0] == OR_F0_MACAULAY) {
                f0 = x > 0.0 ? x : 0.0;
                f0d = 0.5 * (1.0 + (x > 0.0 ? 1.0 : (x < 0.0 ? -1.0 : 0.0)));
            } else if (kind[0] == OR_F0_ABS) {
                f0 = fabs(x);
                f0d = x > 0.0 ? 1.0 : (x < 0.0 ? -1.0 : 0.0);
            } else {
                f0 = x;
                f0d = 1.0;
            }
            const int p = kind[1];
            const double f1 = pow(f0, p), f1d = p * pow(f0, p - 1), f1dd = p * (p - 1) * (p >= 2 ? pow(f0, p - 2) : 0.0);
            double f2, f2d, f2dd;
            if (kind[2] == OR_F2_EXP) {
                const double e = exp(w1 * f1);
                f2 = e - 1.0;
                f2d = w1 * e;
                f2dd = w1 * w1 * e;
            } else if (kind[2] == OR_F2_LOG) {
                const double q = 1.0 - w1 * f1;
                f2 = -log(q);
                f2d = w1 / q;
                f2dd = w1 * w1 / (q * q);
            } else {
                f2 = w1 * f1;
                f2d = w1;
                f2dd = 0.0;
            }
            s += w2 * f2;
            g += w2 * f2d * f1d * f0d;
            h += w2 * ((f2dd * f1d * f1d + f2d * f1dd) * f0d * f0d + f2d * f1d * f0dd);
        }
        dN[mm] = g;
        d2N[mm * d + mm] = h;
    }
    *N = s;
}

/*
 * B-spline basis of degree k on the knots t[0..nk-1] at x by the recursion of App. B: the
 * zero-degree indicators of [t_l, t_l+1), then
 *   B_l,q(x) = (x - t_l) / (t_l+q - t_l) B_l,q-1(x) + (t_l+q+1 - x) / (t_l+q+1 - t_l+1) B_l+1,q-1(x),
 * with the first and second x-derivatives of the same recursion by the product rule:
 *   B'_l,q  = [B_l,q-1 + (x - t_l) B'_l,q-1] / (t_l+q - t_l) + [-B_l+1,q-1 + (t_l+q+1 - x) B'_l+1,q-1] / (t_l+q+1 - t_l+1)
 *   B''_l,q = [2 B'_l,q-1 + (x - t_l) B''_l,q-1] / (.)     + [-2 B'_l+1,q-1 + (t_l+q+1 - x) B''_l+1,q-1] / (.)
 * B, dB, d2B receive the nk - 1 - k basis functions of degree k.
 */
#define OR_MAXKNOTS 160
static void bspline_basis(int k, const double *t, int nk, double x, double *B, double *dB, double *d2B) {
    double b[OR_MAXKNOTS], db[OR_MAXKNOTS], d2b[OR_MAXKNOTS];
    for (int l = 0; l + 1 < nk; ++l) {
        b[l] = (t[l] <= x && x < t[l + 1]) ? 1.0 : 0.0;
        db[l] = 0.0;
        d2b[l] = 0.0;
    }
    for (int q = 1; q <= k; ++q)
        for (int l = 0; l + q + 1 < nk; ++l) {
            const double a1 = 1.0 / (t[l + q] - t[l]), a2 = 1.0 / (t[l + q + 1] - t[l + 1]);
            const double u1 = (x - t[l]) * a1, u2 = (t[l + q + 1] - x) * a2;
            const double nb = u1 * b[l] + u2 * b[l + 1];
            const double ndb = a1 * b[l] + u1 * db[l] - a2 * b[l + 1] + u2 * db[l + 1];
            const double nd2b = 2.0 * a1 * db[l] + u1 * d2b[l] - 2.0 * a2 * db[l + 1] + u2 * d2b[l + 1];
            b[l] = nb;
            db[l] = ndb;
            d2b[l] = nd2b;
        }
    for (int l = 0; l + 1 + k < nk; ++l) {
        B[l] = b[l];
        dB[l] = db[l];
        d2B[l] = d2b[l];
    }
}

/* Knots of ICKAN layer r: t_m = lo + (m - k) h, h = (hi - lo) / G, m = 0 .. G + 2k. */
static int kan_knots(const oracle_model *m, int r, double *t) {
    const int k = m->kan_deg, G = m->kan_G;
    const double h = (m->kan_hi[r] - m->kan_lo[r]) / G;
    for (int q = 0; q <= G + 2 * k; ++q) t[q] = m->kan_lo[r] + (q - k) * h;
    return G + 2 * k + 1;
}

/* ICKAN value, gradient and Hessian by forward propagation of (z, dz/dK, d2z/dK2) through the
 * spline layers (App. B): z_i = sum_j phi_ij(z_j), dz_i = sum_j phi'_ij dz_j,
 * d2z_i = sum_j [phi''_ij dz_j (x) dz_j + phi'_ij d2z_j]. */
static void ickan(const oracle_model *m, const double *K, double *N, double *dN, double *d2N) {
    const int d = m->d, R = m->kan_R, k = m->kan_deg, nb = m->kan_G + k;
    int wmax = d;
    for (int r = 0; r <= R; ++r) wmax = m->kan_w[r] > wmax ? m->kan_w[r] : wmax;
    double *z = calloc((size_t)wmax, sizeof(double)), *dz = calloc((size_t)wmax * d, sizeof(double));
    double *d2z = calloc((size_t)wmax * d * d, sizeof(double));
    double *zn = calloc((size_t)wmax, sizeof(double)), *dzn = calloc((size_t)wmax * d, sizeof(double));
    double *d2zn = calloc((size_t)wmax * d * d, sizeof(double));
    double t[OR_MAXKNOTS], B[OR_MAXKNOTS], dB[OR_MAXKNOTS], d2B[OR_MAXKNOTS];
    for (int j = 0; j < d; ++j) {
        z[j] = K[j];
        dz[j * d + j] = 1.0;
    }
    const double *par = m->kan_par;
    for (int r = 0; r < R; ++r) {
        const int nin = m->kan_w[r], nout = m->kan_w[r + 1];
        const int nk = kan_knots(m, r, t);
        for (int i = 0; i < nout; ++i) {
            zn[i] = 0.0;
            for (int a = 0; a < d; ++a) dzn[i * d + a] = 0.0;
            for (int a = 0; a < d * d; ++a) d2zn[i * d * d + a] = 0.0;
            for (int j = 0; j < nin; ++j) {
                const double ws = par[0], *c = par + 1;
                par += 1 + nb;
                bspline_basis(k, t, nk, z[j], B, dB, d2B);
                double f = 0.0, f1 = 0.0, f2 = 0.0;
                for (int l = 0; l < nb; ++l) {
                    f += c[l] * B[l];
                    f1 += c[l] * dB[l];
                    f2 += c[l] * d2B[l];
                }
                f *= ws;
                f1 *= ws;
                f2 *= ws;
                zn[i] += f;
                for (int a = 0; a < d; ++a) dzn[i * d + a] += f1 * dz[j * d + a];
                for (int a = 0; a < d; ++a)
                    for (int b = 0; b < d; ++b)
                        d2zn[i * d * d + a * d + b] += f2 * dz[j * d + a] * dz[j * d + b] + f1 * d2z[j * d * d + a * d + b];
            }
        }
        for (int i = 0; i < nout; ++i) {
            z[i] = zn[i];
            for (int a = 0; a < d; ++a) dz[i * d + a] = dzn[i * d + a];
            for (int a = 0; a < d * d; ++a) d2z[i * d * d + a] = d2zn[i * d * d + a];
        }
    }
    *N = z[0];
    for (int a = 0; a < d; ++a) dN[a] = dz[a];
    for (int a = 0; a < d * d; ++a) d2N[a] = d2z[a];
    free(z);
    free(dz);
    free(d2z);
    free(zn);
    free(dzn);
    free(d2zn);
}

/* Exported for the spline pins: basis functions of ICKAN layer r at x. */
int oracle_kan_basis(const oracle_model *m, int r, double x, double *B, double *dB, double *d2B) {
    double t[OR_MAXKNOTS];
    const int nk = kan_knots(m, r, t);
    bspline_basis(m->kan_deg, t, nk, x, B, dB, d2B);
    return nk - 1 - m->kan_deg;
}

static void inner_eval(const oracle_model *m, const double *K, double *N, double *dN, double *d2N) {
    if (m->inner == OR_INNER_ICKAN)
        ickan(m, K, N, dN, d2N);
    else if (m->inner == OR_INNER_CANN)
        cann(m, K, N, dN, d2N);
    else if (m->inner == OR_INNER_GENT_THOMAS)
        gent_thomas(K, N, dN, d2N);
    else if (m->inner == OR_INNER_HGO)
        hgo(m, K, N, dN, d2N);
    else
        micnn_alg4(m, K, N, dN, d2N);
}

/* Network value/gradient/Hessian at a given K (exported for the Algorithm 4 pins). */
void oracle_inner(const oracle_model *m, const double *K, double *N, double *dN, double *d2N) {
    inner_eval(m, K, N, dN, d2N);
}

/* ---------------------------------------------------- constitutive update */

/*
 * One qp: Psi, P = dPsi/dF (9) and A = d2Psi/dF dF (81) by the chain rule of
 * eq. nncm-chain plus the volumetric penalty kappa (J-1)^2:
 *   P_iJ    = N_m dK_m/dF_iJ + 2 kappa (J-1) dJ/dF_iJ
 *   A_iJkL  = N_mn dK_m/dF_iJ dK_n/dF_kL + N_m d2K_m/dF_iJ dF_kL
 *             + 2 kappa dJ/dF_iJ dJ/dF_kL + 2 kappa (J-1) d2J/dF_iJ dF_kL
 * n0 (or NULL) is dN/dK at K(I) for the stress-free shift.
 */
static void qp_update(const oracle_model *m, const double *n0, const double *F, double *psi, double *P, double *A) {
    double K[OR_MAXD], dK[OR_MAXD * 9], d2K[OR_MAXD * 81];
    double N, dN[OR_MAXD], d2N[OR_MAXD * OR_MAXD];
    int d = oracle_kinematics(m, F, K, dK, d2K);
    inner_eval(m, K, &N, dN, d2N);
    double J, gJ[9], hJ[81];
    inv_J(F, &J, gJ, hJ);
    double Psi = N + m->kappa * (J - 1.0) * (J - 1.0);
    if (n0) {
        double K0[OR_MAXD], dK0[OR_MAXD * 9], d2K0[OR_MAXD * 81], I9[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
        oracle_kinematics(m, I9, K0, dK0, d2K0);
        for (int i = 0; i < d; ++i) {
            Psi -= n0[i] * (K[i] - K0[i]);
            dN[i] -= n0[i];
        }
    }
    if (psi) *psi = Psi;
    for (int a = 0; a < 9; ++a) {
        double s = 2.0 * m->kappa * (J - 1.0) * gJ[a];
        for (int i = 0; i < d; ++i) s += dN[i] * dK[9 * i + a];
        P[a] = s;
    }
    if (!A) return;
    for (int a = 0; a < 9; ++a)
        for (int b = 0; b < 9; ++b) {
            double s = 2.0 * m->kappa * (gJ[a] * gJ[b] + (J - 1.0) * hJ[a * 9 + b]);
            for (int i = 0; i < d; ++i) {
                s += dN[i] * d2K[81 * i + a * 9 + b];
                for (int j = 0; j < d; ++j) s += d2N[i * d + j] * dK[9 * i + a] * dK[9 * j + b];
            }
            A[a * 9 + b] = s;
        }
}

static void stress_free_shift(const oracle_model *m, double *n0) {
    double K0[OR_MAXD], dK0[OR_MAXD * 9], d2K0[OR_MAXD * 81], I9[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    double N, d2N[OR_MAXD * OR_MAXD];
    oracle_kinematics(m, I9, K0, dK0, d2K0);
    inner_eval(m, K0, &N, n0, d2N);
}

/* {Psi}, {P}, {A} <- model({F}) over n_qp points (Algorithm 2's constitutive call). psi, A may be NULL. */
int oracle_const_update(const oracle_model *m, int64_t n_qp, const double *F, double *psi, double *P, double *A) {
    double n0[OR_MAXD];
    if (m->d > OR_MAXD || m->W > OR_MAXW) return -1;
    if (m->stress_free) stress_free_shift(m, n0);
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < n_qp; ++q)
        qp_update(m, m->stress_free ? n0 : NULL, &F[9 * q], psi ? &psi[q] : NULL, &P[9 * q], A ? &A[81 * q] : NULL);
    return 0;
}

/* Kinematic scalars and their derivatives at one F (exported for the kinematics pins). */
int oracle_kinematics_at(const oracle_model *m, const double *F, double *K, double *dK, double *d2K) {
    return oracle_kinematics(m, F, K, dK, d2K);
}

/* ------------------------------------------------------------- hex8 element */

static const double GP = 0.57735026918962576451; /* 1/sqrt(3) */

/* Reference coordinates of node I (lexicographic, x fastest). */
static double node_xi(int I, int a) { return ((I >> a) & 1) ? 1.0 : -1.0; }
/* Gauss point q coordinates (lexicographic, x fastest). */
static double gauss_xi(int q, int a) { return ((q >> a) & 1) ? GP : -GP; }

/*
 * Shape-function gradients of one element at its 8 Gauss points:
 *   phi_I(xi) = 1/8 prod_a (1 + xi_I,a xi_a)
 *   Je_ab = dX_a/dxi_b = sum_I X_I,a dphi_I/dxi_b ; grad_X phi = Je^{-T} grad_xi phi
 *   w_q = det Je (Gauss weight 1): the "volume" of the qp (Sec. 2.1)
 * dphi[q][I][a], w[q].
 */
void oracle_hex8_gradients(const double *Xe, double *dphi, double *w) {
    for (int q = 0; q < 8; ++q) {
        double gxi[8][3];
        for (int I = 0; I < 8; ++I)
            for (int b = 0; b < 3; ++b) {
                double p = 0.125 * node_xi(I, b);
                for (int c = 0; c < 3; ++c)
                    if (c != b) p *= 1.0 + node_xi(I, c) * gauss_xi(q, c);
                gxi[I][b] = p;
            }
        double Je[9] = {0}, cof[9], det;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                for (int I = 0; I < 8; ++I) Je[3 * a + b] += Xe[3 * I + a] * gxi[I][b];
        cofactor(Je, cof, &det);
        /* Je^{-T} = cof(Je) / det */
        for (int I = 0; I < 8; ++I)
            for (int a = 0; a < 3; ++a) {
                double s = 0.0;
                for (int b = 0; b < 3; ++b) s += cof[3 * a + b] / det * gxi[I][b];
                dphi[(q * 8 + I) * 3 + a] = s;
            }
        w[q] = det;
    }
}

static void gather_X(const double *X, const int32_t *conn, int64_t e, double *Xe) {
    for (int I = 0; I < 8; ++I)
        for (int a = 0; a < 3; ++a) Xe[3 * I + a] = X[3 * (int64_t)conn[8 * e + I] + a];
}

/* F = I + sum_I u^I (x) grad_X phi^I at every qp (Algorithm 1, trial F). u[n_nodes][3], F[n_el*8][9]. */
void oracle_compute_F(int64_t n_el, const int32_t *conn, const double *X, const double *u, double *F) {
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < n_el; ++e) {
        double Xe[24], dphi[192], w[8];
        gather_X(X, conn, e, Xe);
        oracle_hex8_gradients(Xe, dphi, w);
        for (int q = 0; q < 8; ++q) {
            double *Fq = &F[9 * (8 * e + q)];
            for (int i = 0; i < 3; ++i)
                for (int J = 0; J < 3; ++J) {
                    double s = kd(i, J);
                    for (int I = 0; I < 8; ++I) s += u[3 * (int64_t)conn[8 * e + I] + i] * dphi[(q * 8 + I) * 3 + J];
                    Fq[3 * i + J] = s;
                }
        }
    }
}

/*
 * Element residual and stiffness from qp tables (Algorithm 2, second loop), in
 * material form (App. A.1 relates it to the spatial eq. r-quad / k-quad):
 *   f_e[3I+i]         = sum_q w_q P_iJ dphi_I/dX_J
 *   K_e[3I+i][3K+k]   = sum_q w_q dphi_I/dX_J A_iJkL dphi_K/dX_L
 * Element e owns qp 8e..8e+7. f_e or K_e may be NULL.
 */
void oracle_elem_assemble(int64_t n_el, const int32_t *conn, const double *X, const double *P, const double *A,
                          double *f_e, double *K_e) {
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < n_el; ++e) {
        double Xe[24], dphi[192], w[8];
        gather_X(X, conn, e, Xe);
        oracle_hex8_gradients(Xe, dphi, w);
        if (f_e)
            for (int r = 0; r < 24; ++r) f_e[24 * e + r] = 0.0;
        if (K_e)
            for (int r = 0; r < 576; ++r) K_e[576 * e + r] = 0.0;
        for (int q = 0; q < 8; ++q) {
            const double *Pq = &P[9 * (8 * e + q)];
            const double *Aq = A ? &A[81 * (8 * e + q)] : NULL;
            const double *g = &dphi[q * 24];
            for (int I = 0; I < 8; ++I)
                for (int i = 0; i < 3; ++i) {
                    if (f_e) {
                        double s = 0.0;
                        for (int J = 0; J < 3; ++J) s += Pq[3 * i + J] * g[3 * I + J];
                        f_e[24 * e + 3 * I + i] += w[q] * s;
                    }
                    if (K_e && Aq)
                        for (int K = 0; K < 8; ++K)
                            for (int k = 0; k < 3; ++k) {
                                double s = 0.0;
                                for (int J = 0; J < 3; ++J)
                                    for (int L = 0; L < 3; ++L)
                                        s += g[3 * I + J] * Aq[(3 * i + J) * 9 + 3 * k + L] * g[3 * K + L];
                                K_e[576 * e + (3 * I + i) * 24 + 3 * K + k] += w[q] * s;
                            }
                }
        }
    }
}

/* ------------------------------------------------------------ spatial form */

/* Voigt pairs in the order (11, 22, 33, 23, 13, 12). */
static const int VOIGT_I[6] = {0, 1, 2, 1, 0, 0};
static const int VOIGT_J[6] = {0, 1, 2, 2, 2, 1};

/*
 * Kirchhoff stress and spatial stiffness from P and A by the push-forward of App. A.1:
 *   tau_ij    = P_iJ F_jJ
 *   c_ijkl    = F_jJ A_iJkL F_lL - delta_ik tau_jl
 * tau[6] in Voigt order; c[21] the upper triangle (row-major, I <= J) of the 6 x 6
 * Voigt matrix C_IJ = c_{ij kl}, (i, j) the pair of I and (k, l) the pair of J.
 * F, P, A are one point's; c may be NULL.
 */
void oracle_push_forward(const double *F, const double *P, const double *A, double *tau, double *c) {
    double t[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int J = 0; J < 3; ++J) s += P[3 * i + J] * F[3 * j + J];
            t[3 * i + j] = s;
        }
    for (int v = 0; v < 6; ++v) tau[v] = t[3 * VOIGT_I[v] + VOIGT_J[v]];
    if (!c) return;
    int e = 0;
    for (int I = 0; I < 6; ++I)
        for (int Jv = I; Jv < 6; ++Jv) {
            const int i = VOIGT_I[I], j = VOIGT_J[I], k = VOIGT_I[Jv], l = VOIGT_J[Jv];
            double s = 0.0;
            for (int J = 0; J < 3; ++J)
                for (int L = 0; L < 3; ++L) s += F[3 * j + J] * A[(3 * i + J) * 9 + 3 * k + L] * F[3 * l + L];
            c[e++] = s - kd(i, k) * t[3 * j + l];
        }
}

/* Voigt slot of the symmetric pair (i, j). */
static int voigt_of(int i, int j) {
    if (i == j) return i;
    if (i > j) { int x = i; i = j; j = x; }
    return (i == 1) ? 3 : (j == 2 ? 4 : 5);
}

/* c_{ijkl} from the 21 stored values. */
static double voigt_c(const double *c, int i, int j, int k, int l) {
    int I = voigt_of(i, j), J = voigt_of(k, l);
    if (I > J) { int x = I; I = J; J = x; }
    /* row I of the upper triangle starts at I*6 - I(I-1)/2 */
    return c[I * 6 - I * (I - 1) / 2 + (J - I)];
}

/*
 * Element residual and stiffness in the spatial form of eq. r-quad and k-quad:
 *   f_e[3I+i]       = sum_q w_q tau_ij grad phi_I,j
 *   K_e[3I+i][3K+k] = sum_q w_q grad phi_I,m (delta_ik tau_ml + c_imkl) grad phi_K,l
 * with the spatial gradients grad phi_I,m = dphi_I/dX_M (F^{-1})_Mm and w_q the qp's
 * reference volume. F[q][9], tau[q][6], c[q][21] (c may be NULL).
 */
void oracle_elem_assemble_spatial(int64_t n_el, const int32_t *conn, const double *X, const double *F,
                                  const double *tau, const double *c, double *f_e, double *K_e) {
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < n_el; ++e) {
        double Xe[24], dphi[192], w[8];
        gather_X(X, conn, e, Xe);
        oracle_hex8_gradients(Xe, dphi, w);
        if (f_e)
            for (int r = 0; r < 24; ++r) f_e[24 * e + r] = 0.0;
        if (K_e)
            for (int r = 0; r < 576; ++r) K_e[576 * e + r] = 0.0;
        for (int q = 0; q < 8; ++q) {
            const int64_t qq = 8 * e + q;
            const double *Fq = &F[9 * qq], *tq = &tau[6 * qq];
            const double *cq = c ? &c[21 * qq] : NULL;
            double cof[9], det, Finv[9];
            cofactor(Fq, cof, &det);
            /* F^{-1}_Mm = cof(F)_mM / det F */
            for (int M = 0; M < 3; ++M)
                for (int m = 0; m < 3; ++m) Finv[3 * M + m] = cof[3 * m + M] / det;
            double g[8][3];
            for (int I = 0; I < 8; ++I)
                for (int m = 0; m < 3; ++m) {
                    double s = 0.0;
                    for (int M = 0; M < 3; ++M) s += dphi[(q * 8 + I) * 3 + M] * Finv[3 * M + m];
                    g[I][m] = s;
                }
            for (int I = 0; I < 8; ++I)
                for (int i = 0; i < 3; ++i) {
                    if (f_e) {
                        double s = 0.0;
                        for (int j = 0; j < 3; ++j) s += tq[voigt_of(i, j)] * g[I][j];
                        f_e[24 * e + 3 * I + i] += w[q] * s;
                    }
                    if (K_e && cq)
                        for (int K = 0; K < 8; ++K)
                            for (int k = 0; k < 3; ++k) {
                                double s = 0.0;
                                for (int m = 0; m < 3; ++m)
                                    for (int l = 0; l < 3; ++l)
                                        s += g[I][m] * (kd(i, k) * tq[voigt_of(m, l)] + voigt_c(cq, i, m, k, l)) *
                                             g[K][l];
                                K_e[576 * e + (3 * I + i) * 24 + 3 * K + k] += w[q] * s;
                            }
                }
        }
    }
}

/*
 * Adjoints of the assembly chain for a residual-based loss (eq. loss of App. C, the NN-EUCLID
 * objective, is a function of the global residual r):
 *   r = sum_e sum_q w_q P_q grad phi  (eq. r-quad)  =>  dL/dP_q,iJ = w_q sum_I lam_I,i dphi_I/dX_J
 *   F_q = I + sum_I u_I (x) grad phi  (Algorithm 1) =>  dL/du_I,i = sum_{e,q} dL/dF_q,iJ dphi_I/dX_J
 * with lam = dL/dr. lam[n_nodes][3] -> G[n_qp][9]; dF[n_qp][9] -> du[n_nodes][3] (summed over
 * elements in order).
 */
void oracle_residual_adjoint(int64_t n_el, const int32_t *conn, const double *X, const double *lam, double *G) {
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < n_el; ++e) {
        double Xe[24], dphi[192], w[8];
        gather_X(X, conn, e, Xe);
        oracle_hex8_gradients(Xe, dphi, w);
        for (int q = 0; q < 8; ++q)
            for (int i = 0; i < 3; ++i)
                for (int J = 0; J < 3; ++J) {
                    double s = 0.0;
                    for (int I = 0; I < 8; ++I) s += lam[3 * (int64_t)conn[8 * e + I] + i] * dphi[(q * 8 + I) * 3 + J];
                    G[9 * (8 * e + q) + 3 * i + J] = w[q] * s;
                }
    }
}

void oracle_compute_F_adjoint(int64_t n_el, const int32_t *conn, const double *X, const double *dF, int64_t n_nodes,
                              double *du) {
    for (int64_t i = 0; i < 3 * n_nodes; ++i) du[i] = 0.0;
    for (int64_t e = 0; e < n_el; ++e) {
        double Xe[24], dphi[192], w[8];
        gather_X(X, conn, e, Xe);
        oracle_hex8_gradients(Xe, dphi, w);
        for (int q = 0; q < 8; ++q)
            for (int I = 0; I < 8; ++I)
                for (int i = 0; i < 3; ++i) {
                    double s = 0.0;
                    for (int J = 0; J < 3; ++J) s += dF[9 * (8 * e + q) + 3 * i + J] * dphi[(q * 8 + I) * 3 + J];
                    du[3 * (int64_t)conn[8 * e + I] + i] += s;
                }
    }
}

/* Global residual r[3*n_nodes] = sum_e f_e scattered to dofs 3*node + i, elements in order. */
void oracle_scatter_residual(int64_t n_el, const int32_t *conn, const double *f_e, int64_t n_nodes, double *r) {
    for (int64_t i = 0; i < 3 * n_nodes; ++i) r[i] = 0.0;
    for (int64_t e = 0; e < n_el; ++e)
        for (int I = 0; I < 8; ++I)
            for (int i = 0; i < 3; ++i) r[3 * (int64_t)conn[8 * e + I] + i] += f_e[24 * e + 3 * I + i];
}

/*
 * Global K in CSR form (caller's pattern rowptr/col, columns sorted within a
 * row): vals[p] = sum_e K_e entries landing on (row, col), elements in order.
 * Returns the number of element entries that found no slot in the pattern.
 */
int64_t oracle_scatter_csr(int64_t n_el, const int32_t *conn, const double *K_e, int64_t n_rows, const int64_t *rowptr,
                           const int32_t *col, double *vals) {
    int64_t missing = 0;
    for (int64_t p = 0; p < rowptr[n_rows]; ++p) vals[p] = 0.0;
    for (int64_t e = 0; e < n_el; ++e)
        for (int a = 0; a < 24; ++a)
            for (int b = 0; b < 24; ++b) {
                int64_t row = 3 * (int64_t)conn[8 * e + a / 3] + a % 3;
                int32_t c = 3 * conn[8 * e + b / 3] + b % 3;
                int64_t lo = rowptr[row], hi = rowptr[row + 1], found = -1;
                for (int64_t p = lo; p < hi; ++p)
                    if (col[p] == c) {
                        found = p;
                        break;
                    }
                if (found < 0)
                    ++missing;
                else
                    vals[found] += K_e[576 * e + a * 24 + b];
            }
    return missing;
}

/* ---------------------------------------------------------------- backward */

/*
 * Parameter vector theta, in this order:
 *   W1 [W][d], c1 [W], then for k = 2..L: A_k [W][W], B_k [W][d], c_k [W], then a [W], b [d].
 */
int64_t oracle_n_params(int d, int W, int L) {
    return (int64_t)W * d + W + (int64_t)(L - 1) * ((int64_t)W * W + (int64_t)W * d + W) + W + d;
}

/*
 * Backward of G : P(F; theta) summed over qp, for G = dL/dP given per qp:
 *   dL/dF_kL   = sum_iJ G_iJ A_iJkL                        (A from qp_update)
 *   dL/dtheta  = sum_q d/dtheta [ sum_m r_m dN/dK_m ],  r_m = G : dK_m/dF
 * The inner term s = grad_K N . r is propagated forward as a tangent
 * (zdot = F'(y) ydot, ydot = A zdot + B r) and then differentiated in reverse
 * with respect to every weight. Every entry of theta receives exactly one term
 * t_q per point. The points are split into contiguous blocks, one per OpenMP
 * thread in thread order; each block sums its t_q in index order and the block
 * sums are then added in thread order (with one thread: index order).
 * dLdtheta_abs (nullable) receives sum_q |t_q| per entry, the magnitude a
 * floating-point sum of the t_q is rounded against.
 * The volumetric penalty does not depend on theta. MICNN and CANN inner functions
 * (any other returns -1); the stress-free shift is not supported here (returns -2).
 */
static void backward_point(const oracle_model *m, const double *Fq, const double *Gq, double *dLdF_q, double *t,
                           double *y, double *z, double *yd, double *zd, double *zb, double *zdb, double *yb,
                           double *ydb) {
    const int d = m->d, W = m->W, L = m->L;
    int64_t off_W1 = 0, off_c1 = (int64_t)W * d;
    int64_t off_layer = off_c1 + W; /* start of layer 2 block */
    int64_t layer_sz = (int64_t)W * W + (int64_t)W * d + W;
    int64_t off_a = off_layer + (int64_t)(L - 1) * layer_sz, off_b = off_a + W;
    double psi, P[9], A[81];
    qp_update(m, NULL, Fq, &psi, P, A);
    if (dLdF_q)
        for (int b = 0; b < 9; ++b) {
            double s = 0.0;
            for (int a = 0; a < 9; ++a) s += Gq[a] * A[a * 9 + b];
            dLdF_q[b] = s;
        }
    double K[OR_MAXD], dK[OR_MAXD * 9], d2K[OR_MAXD * 81], r[OR_MAXD];
    oracle_kinematics(m, Fq, K, dK, d2K);
    for (int i = 0; i < d; ++i) {
        double s = 0.0;
        for (int a = 0; a < 9; ++a) s += Gq[a] * dK[9 * i + a];
        r[i] = s;
    }
    /* forward: values and tangents along r; z[0] = K, zd[0] = r */
    for (int i = 0; i < d; ++i) {
        z[i] = K[i];
        zd[i] = r[i];
    }
    for (int k = 1; k <= L; ++k) {
        int nin = (k == 1) ? d : W;
        const double *A_ = (k == 1) ? m->W1 : &m->Ak[(size_t)(k - 2) * W * W];
        const double *B_ = (k == 1) ? NULL : &m->Bk[(size_t)(k - 2) * W * d];
        const double *c_ = m->c ? &m->c[(size_t)(k - 1) * W] : NULL;
        const double *zin = &z[(k - 1) * OR_MAXW], *zdin = &zd[(k - 1) * OR_MAXW];
        for (int j = 0; j < W; ++j) {
            double s = c_ ? c_[j] : 0.0, tt = 0.0;
            for (int i = 0; i < nin; ++i) {
                s += A_[j * nin + i] * zin[i];
                tt += A_[j * nin + i] * zdin[i];
            }
            if (B_)
                for (int i = 0; i < d; ++i) {
                    s += B_[j * d + i] * K[i];
                    tt += B_[j * d + i] * r[i];
                }
            y[(k - 1) * W + j] = s;
            yd[(k - 1) * W + j] = tt;
            z[k * OR_MAXW + j] = softplus(s);
            zd[k * OR_MAXW + j] = logistic(s) * tt;
        }
    }
    /* s = a . zd[L] + b . r ; reverse. Every entry of t is assigned once. */
    for (int j = 0; j < W; ++j) {
        t[off_a + j] = zd[L * OR_MAXW + j];
        zb[j] = 0.0;
        zdb[j] = m->a[j];
    }
    for (int i = 0; i < d; ++i) t[off_b + i] = r[i];
    for (int k = L; k >= 1; --k) {
        int nin = (k == 1) ? d : W;
        const double *A_ = (k == 1) ? m->W1 : &m->Ak[(size_t)(k - 2) * W * W];
        const double *zin = &z[(k - 1) * OR_MAXW], *zdin = &zd[(k - 1) * OR_MAXW];
        for (int j = 0; j < W; ++j) {
            double yy = y[(k - 1) * W + j], s1 = logistic(yy), s2 = softplus_dd(yy);
            ydb[j] = s1 * zdb[j];
            yb[j] = s1 * zb[j] + s2 * yd[(k - 1) * W + j] * zdb[j];
        }
        int64_t oA = (k == 1) ? off_W1 : off_layer + (int64_t)(k - 2) * layer_sz;
        int64_t oB = oA + (int64_t)W * W, oc = (k == 1) ? off_c1 : oB + (int64_t)W * d;
        for (int j = 0; j < W; ++j) {
            for (int i = 0; i < nin; ++i) t[oA + (int64_t)j * nin + i] = yb[j] * zin[i] + ydb[j] * zdin[i];
            if (k > 1)
                for (int i = 0; i < d; ++i) t[oB + (int64_t)j * d + i] = yb[j] * K[i] + ydb[j] * r[i];
            t[oc + j] = yb[j];
        }
        if (k > 1)
            for (int i = 0; i < nin; ++i) {
                double s = 0.0, tt = 0.0;
                for (int j = 0; j < W; ++j) {
                    s += A_[j * nin + i] * yb[j];
                    tt += A_[j * nin + i] * ydb[j];
                }
                zb[i] = s;
                zdb[i] = tt;
            }
    }
}

/*
 * The same backward for the CANN inner function (eq. cann-def), theta = the weights
 * w[d][n][2] = (w1, w2) per input m and term k. With r_m = G : dK_m/dF, the inner term
 * s = sum_m r_m dN/dK_m and dN/dK_m = sum_k w2 f2'(f1(f0(K_m)); w1) f1'(f0(K_m)) f0'(K_m):
 *   ds/dw2_mk = r_m f2' f1' f0',   ds/dw1_mk = r_m w2 (d f2'/d w1) f1' f0',
 * with f2' and d f2'/d w1 of the menu of eq. cann-fs written out:
 *   w1 y:           f2' = w1,              d f2'/d w1 = 1
 *   exp(w1 y) - 1:  f2' = w1 exp(w1 y),    d f2'/d w1 = exp(w1 y) (1 + w1 y)
 *   -ln(1 - w1 y):  f2' = w1 / (1 - w1 y), d f2'/d w1 = 1 / (1 - w1 y)^2
 */
static void cann_backward_point(const oracle_model *m, const double *Fq, const double *Gq, double *dLdF_q,
                                double *t) {
    const int d = m->d, n = m->cann_n;
    double psi, P[9], A[81];
    qp_update(m, NULL, Fq, &psi, P, A);
    if (dLdF_q)
        for (int b = 0; b < 9; ++b) {
            double s = 0.0;
            for (int a = 0; a < 9; ++a) s += Gq[a] * A[a * 9 + b];
            dLdF_q[b] = s;
        }
    double K[OR_MAXD], dK[OR_MAXD * 9], d2K[OR_MAXD * 81];
    oracle_kinematics(m, Fq, K, dK, d2K);
    for (int mm = 0; mm < d; ++mm) {
        double r = 0.0;
        for (int a = 0; a < 9; ++a) r += Gq[a] * dK[9 * mm + a];
        const double x = K[mm];
        for (int k = 0; k < n; ++k) {
            const int *kind = &m->cann_kind[3 * k];
            const double w1 = m->cann_w[(mm * n + k) * 2], w2 = m->cann_w[(mm * n + k) * 2 + 1];
            double f0, f0d;
            if (kind[0] == OR_F0_MACAULAY) {
                f0 = x > 0.0 ? x : 0.0;
                f0d = 0.5 * (1.0 + (x > 0.0 ? 1.0 : (x < 0.0 ? -1.0 : 0.0)));
            } else if (kind[0] == OR_F0_ABS) {
                f0 = fabs(x);
                f0d = x > 0.0 ? 1.0 : (x < 0.0 ? -1.0 : 0.0);
            } else {
                f0 = x;
                f0d = 1.0;
            }
            const int p = kind[1];
            const double f1 = pow(f0, p), f1d = p * pow(f0, p - 1);
            double f2d, f2d_w1;
            if (kind[2] == OR_F2_EXP) {
                const double e = exp(w1 * f1);
                f2d = w1 * e;
                f2d_w1 = e * (1.0 + w1 * f1);
            } else if (kind[2] == OR_F2_LOG) {
                const double q = 1.0 - w1 * f1;
                f2d = w1 / q;
                f2d_w1 = 1.0 / (q * q);
            } else {
                f2d = w1;
                f2d_w1 = 1.0;
            }
            t[(mm * n + k) * 2] = r * w2 * f2d_w1 * f1d * f0d;
            t[(mm * n + k) * 2 + 1] = r * f2d * f1d * f0d;
        }
    }
}

int oracle_const_backward(const oracle_model *m, int64_t n_qp, const double *F, const double *G, double *dLdF,
                          double *dLdtheta, double *dLdtheta_abs) {
    const int d = m->d, W = m->W, L = m->L;
    const int cann = m->inner == OR_INNER_CANN;
    if (m->inner != OR_INNER_MICNN && !cann) return -1;
    if (m->stress_free) return -2;
    const int64_t np = cann ? (int64_t)2 * d * m->cann_n : oracle_n_params(d, W, L);
    int nthr = 1;
#ifdef _OPENMP
    nthr = omp_get_max_threads();
#endif
    /* per-thread block sums (and magnitude sums), zero for threads that get no points */
    double *part = (double *)calloc((size_t)nthr * np * 2, sizeof(double));
    if (!part) return -3;
    int fail = 0;
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *y = (double *)malloc(sizeof(double) * L * W);
        double *z = (double *)malloc(sizeof(double) * (L + 1) * OR_MAXW);
        double *yd = (double *)malloc(sizeof(double) * L * W);
        double *zd = (double *)malloc(sizeof(double) * (L + 1) * OR_MAXW);
        double *zb = (double *)malloc(sizeof(double) * OR_MAXW), *zdb = (double *)malloc(sizeof(double) * OR_MAXW);
        double *yb = (double *)malloc(sizeof(double) * OR_MAXW), *ydb = (double *)malloc(sizeof(double) * OR_MAXW);
        double *t = (double *)malloc(sizeof(double) * np);
        int ok = y && z && yd && zd && zb && zdb && yb && ydb && t;
        if (!ok) {
#pragma omp atomic write
            fail = 1;
        }
        double *sum = &part[(size_t)tid * np * 2], *mag = sum + np;
        /* static schedule: thread tid gets one contiguous block of points, blocks in thread order */
#pragma omp for schedule(static)
        for (int64_t q = 0; q < n_qp; ++q) {
            if (!ok) continue;
            if (cann)
                cann_backward_point(m, &F[9 * q], &G[9 * q], dLdF ? &dLdF[9 * q] : NULL, t);
            else
                backward_point(m, &F[9 * q], &G[9 * q], dLdF ? &dLdF[9 * q] : NULL, t, y, z, yd, zd, zb, zdb, yb,
                               ydb);
            for (int64_t i = 0; i < np; ++i) {
                sum[i] += t[i];
                mag[i] += fabs(t[i]);
            }
        }
        free(y);
        free(z);
        free(yd);
        free(zd);
        free(zb);
        free(zdb);
        free(yb);
        free(ydb);
        free(t);
    }
    for (int64_t i = 0; i < np; ++i) {
        double s = 0.0, a = 0.0;
        for (int th = 0; th < nthr; ++th) {
            s += part[(size_t)th * np * 2 + i];
            a += part[(size_t)th * np * 2 + np + i];
        }
        dLdtheta[i] = s;
        if (dLdtheta_abs) dLdtheta_abs[i] = a;
    }
    free(part);
    return fail ? -3 : 0;
}
