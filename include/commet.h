/*
 * commet.h -- C ABI of the GB300 (sm_103a) neural-constitutive hot path.
 *
 * The operation is the constitutive call of COMMET's batch-vectorised assembly
 * (Algorithm 2/3: {Psi},{tau},{c} <- vectorized_constitutive_model({F})), written
 * in material form (App. A.1: P = dPsi/dF, A = C^P = d2Psi/dF dF), followed by the
 * element integrals of eq. r-quad / k-quad and their sum into the global residual
 * and stiffness (Sec. 2.1, Algorithm 1).
 *
 * Conventions (all entry points):
 *  - F_iJ at component 3*i + J; A_iJkL = dP_iJ/dF_kL at component (3*i+J)*9 + 3*k+L.
 *  - Per-qp tables are structure-of-arrays, component-major: X[c * n_qp + q].
 *    Per-element tables likewise: f_e[r * n_el + e], K_e[(24*r + s) * n_el + e].
 *  - Element e owns quadrature points 8e..8e+7 (2x2x2 Gauss, lexicographic, x fastest);
 *    hex8 nodes are lexicographic in the reference cube; element dof 3*I + i;
 *    global dof 3*node + i (the node-major block layout of Sec. 2.1).
 *  - Every pointer passed to a compute call is a DEVICE pointer owned by the caller,
 *    except where a comment says "host". The library never frees caller memory and
 *    allocates nothing in compute calls; model/mesh creation allocates device memory
 *    owned by the returned handle.
 *  - Compute calls are asynchronous on `stream` (a cudaStream_t, NULL = legacy default
 *    stream). Arguments are checked on the host before any launch; a failed check
 *    returns an error code and launches nothing.
 *  - Element type of P/A/F/u/r/K buffers: double for COMMET_F64 handles, float for
 *    COMMET_F32 and COMMET_BF16_MLP handles.
 *  - Data errors (J <= 0 or a non-finite result at a qp) do not abort: the affected
 *    outputs are set to NaN and, when `status` (device int32[2]) is given, status[0]
 *    receives the number of such qp and status[1] the smallest such qp index
 *    (INT32_MAX when none). The call resets `status` itself, in stream order.
 */
#ifndef COMMET_H
#define COMMET_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---- */
#define COMMET_OK 0
#define COMMET_ERR_INVALID_ARG 1 /* NULL where required, bad size, bad enum, misaligned pointer */
#define COMMET_ERR_UNSUPPORTED 2 /* shape, precision or kinematics not built into this library */
#define COMMET_ERR_CUDA 3        /* a CUDA runtime call or kernel launch failed */
#define COMMET_ERR_NO_CSR 4      /* the mesh was created without the CSR pattern */

/* ---- precisions ---- */
#define COMMET_F64 0      /* everything in double */
#define COMMET_F32 1      /* everything in float */
#define COMMET_BF16_MLP 2 /* hidden W x W layers as tcgen05 MMAs on the fifth-generation tensor cores
                             (bf16 operands, fp32 accumulators in tensor memory, 128 points per MMA
                             tile), the rest in fp32; needs (d + L) W <= 512 tensor-memory columns,
                             else UNSUPPORTED at the compute call */

/* ---- kinematic layers (Sec. 2.2 eq. comp-se; App. A.2) ---- */
#define COMMET_KIN_ISO_SHIFTED 0 /* K = (Ibar1 - 3, Ibar2 - 3, J - 1), d = 3, no fibres */
#define COMMET_KIN_RAW 1         /* K = (Ibar1, Ibar2, J, I4_11..I4_nn, I5_11..I5_nn), d = 3 + 2n */
#define COMMET_KIN_POLYCONVEX 2  /* K = (Ibar1 - 3, Ibar2^{3/2} - 3^{3/2}, (J - 1)^2), d = 3, no fibres:
                                    the polyconvex inputs of the paper's trained NCMs (App. C);
                                    every input has zero F-gradient at F = I, so P(I) = 0 */

#define COMMET_ACT_SOFTPLUS 0 /* F(y) = log(1 + exp(y)), the only activation built */

/* ---- inner functions N(K) (App. B; eq. gt) ---- */
#define COMMET_INNER_MICNN 0        /* eq. icnn (default; the fields W .. activation) */
#define COMMET_INNER_CANN 1         /* eq. cann-def (the cann_* fields) */
#define COMMET_INNER_GENT_THOMAS 2  /* eq. gt, 0.5 (K0 - 3) + log(K1 / 3) + (K2 - 1)^2 on COMMET_KIN_RAW
                                       without fibres; no parameters */
#define COMMET_INNER_ICKAN 3        /* the input-convex KAN of App. B (the kan_* fields), d = 3 */
#define COMMET_KAN_MAX_LAYERS 8
#define COMMET_KAN_MAX_WIDTH 8
/* CANN term menus of eq. cann-fs: f0 (applied to K_m), f1 = x^p, f2 (with weight w1) */
#define COMMET_CANN_F0_ID 0       /* x */
#define COMMET_CANN_F0_MACAULAY 1 /* <x> = max(x, 0) */
#define COMMET_CANN_F0_ABS 2      /* |x| */
#define COMMET_CANN_F2_LINEAR 0   /* w1 y */
#define COMMET_CANN_F2_EXP 1      /* exp(w1 y) - 1 */
#define COMMET_CANN_F2_LOG 2      /* -ln(1 - w1 y); points with w1 y >= 1 are reported */
#define COMMET_CANN_MAX_TERMS 8

typedef struct commet_model commet_model;
typedef struct commet_mesh commet_mesh;

/*
 * Strain energy Psi(F) = N(K(F, {A^i})) + kappa (J - 1)^2  [- n0 . (K - K(I)) if stress_free]
 * with N the monotone input-convex network of App. B, eq. icnn:
 *   y1 = W1 K + c1 ; z_k = softplus(y_k) ;
 *   y_k = A_k z_{k-1} + B_k K + c_k (k = 2..L) ; N = a_out . z_L + b_out . K.
 * (Layer 1's A^(1) z^(0) and B^(1) K act on the same vector K and are one matrix W1.)
 * stress_free subtracts the linear term n0 = dN/dK at K(I) so that P(I) = 0.
 * All arrays are HOST row-major double; they are copied at creation.
 */
typedef struct commet_model_desc {
    int32_t kinematics;   /* COMMET_KIN_* */
    int32_t n_fibres;     /* structural vectors, 0..2 (must be 0 for ISO_SHIFTED) */
    const double *fibres; /* [n_fibres][3] reference vectors A^i */
    int32_t d;            /* network inputs; must equal the kinematic layer's count */
    int32_t W;            /* hidden width 1..64; the kernels are built for 16, 32, 64, and 4, 8 without
                             fibres (BF16: 32, 64); other widths run as the next built one with zero
                             rows and columns (exact), and theta stays the caller's */
    int32_t L;            /* hidden layers, >= 1 */
    const double *W1;     /* [W][d] */
    const double *A;      /* [L-1][W][W] (may be NULL when L == 1) */
    const double *B;      /* [L-1][W][d] (may be NULL when L == 1) */
    const double *c;      /* [L][W] biases, or NULL for zero biases */
    const double *a_out;  /* [W] */
    const double *b_out;  /* [d] */
    int32_t activation;   /* COMMET_ACT_SOFTPLUS */
    double kappa;         /* volumetric penalty; 0 = none */
    int32_t stress_free;  /* 0 or 1 */
    /* inner function; a zero-initialised tail selects the MICNN above */
    int32_t inner;            /* COMMET_INNER_* */
    int32_t cann_terms;       /* CANN: terms n per input, 1..COMMET_CANN_MAX_TERMS */
    const int32_t *cann_kind; /* CANN: [n][3] per term (f0, p in 1..3, f2), shared by the inputs */
    const double *cann_w;     /* CANN: [d][n][2] per input m and term k: (w1, w2) of
                                 N = sum_m sum_k w2 f2(f1(f0(K_m)); w1)  (eq. cann-def) */
    /* ICKAN (App. B): z^(r)_i = sum_j w_s,rij sum_l c_rij,l B_l,k(z^(r-1)_j), z^(0) = K, N = z^(R);
       B-splines of degree k (the recursion of App. B) on G uniform intervals of [lo_r, hi_r],
       knots extended by k on each side: G + k control points per spline */
    int32_t kan_layers;        /* R, 1..COMMET_KAN_MAX_LAYERS */
    const int32_t *kan_widths; /* [R + 1]: widths[0] = d, widths[R] = 1, each <= COMMET_KAN_MAX_WIDTH */
    int32_t kan_degree;        /* k, 2..4 */
    int32_t kan_grid;          /* G, 1..128 */
    const double *kan_lo;      /* [R] */
    const double *kan_hi;      /* [R], > lo */
    const double *kan_params;  /* per spline (layer r, output i, input j, in that order): w_s, then c[G + k] */
} commet_model_desc;

/*
 * Create a model handle for one precision. Copies the weights to the current CUDA
 * device in the layouts the kernels use. Synchronous. *out is set on success only.
 * Errors: INVALID_ARG (NULL, d inconsistent with the kinematics, negative sizes,
 * bad CANN kinds), UNSUPPORTED (W or n_fibres not built, activation unknown, a CANN or
 * Gent-Thomas model in COMMET_BF16_MLP), CUDA. CANN and Gent-Thomas models serve the
 * constitutive updates (both forms) and the element integrals; the backward and the
 * fused Newton assembly return UNSUPPORTED for them.
 */
int commet_model_create(const commet_model_desc *desc, int32_t precision, commet_model **out);
int commet_model_destroy(commet_model *m);
/* Number of parameters theta = [W1, c1, (A_k, B_k, c_k) for k = 2..L, a_out, b_out]. */
int64_t commet_model_n_params(const commet_model *m);

/*
 * Constitutive update (Algorithm 2, "vectorized_constitutive_model", material form,
 * chain rule of eq. nncm-chain): for every qp q < n_qp,
 *   psi[q] = Psi(F_q), P[:, q] = dPsi/dF (9), A[:, q] = d2Psi/dF dF (81).
 * F   [9][n_qp]  in.
 * psi [n_qp]     out, or NULL.
 * P   [9][n_qp]  out (required).
 * A   [81][n_qp] out, or NULL (stress only).
 * status: device int32[2] or NULL (see top of file).
 * n_qp == 0 is a no-op returning COMMET_OK. Pointers must be 16-byte aligned.
 * With A == NULL the tangent pass is skipped (stress only); P agrees with the full
 * call's to rounding.
 */
int commet_const_update(const commet_model *m, int64_t n_qp, const void *F, void *psi, void *P, void *A,
                        int32_t *status, void *stream);

/*
 * Host-buffer form of commet_const_update and, with a mesh, of commet_elem_assemble
 * (Algorithm 2 with its tables in host memory): the points, or the mesh's elements with
 * their 8 points each, in chunks of `chunk` (points without a mesh, elements with one).
 * Chunk c is copied to the device while chunk c - 1 is computed on `stream` and chunk
 * c - 2 is copied back, so copies and kernels overlap; the results are those of the
 * device calls on the same inputs, bit for bit.
 * F, psi, P, A, f_e, K_e are HOST pointers in the layouts of the device calls
 * (F [9][n_qp], psi [n_qp], P [9][n_qp], A [81][n_qp], f_e [24][n_el], K_e [576][n_el]),
 * page-locked for the copies to overlap; psi, A, f_e, K_e may be NULL (K_e only with A).
 * Element type: double for a COMMET_F64 model, float otherwise.
 * mesh: NULL (update only; f_e and K_e must be NULL) or a mesh with 8 n_el = n_qp. The
 * element integrals are those of commet_elem_assemble_symmetric: A is the update's own
 * tangent, the Hessian of an energy, so major symmetric.
 * workspace: device memory of commet_const_update_host_workspace(m, mesh, chunk, A != NULL)
 * bytes, 256-byte aligned, owned by the caller and not used by anything else until the
 * call has completed on `stream`.
 * The call returns once the work is queued; the host outputs are complete when `stream`
 * reaches that point. The copies run on two side streams (with nine events) that the
 * model handle creates with the model, on its device, and releases with it; a call
 * creates and allocates nothing. Calls on one model from several host threads are
 * ordered by a lock while they queue their work. On every return, error or not,
 * `stream` waits for every copy the call queued, so once `stream` reaches that point
 * nothing of the call still reads the workspace or F or writes the host outputs.
 * No status word: bad points come back as NaN.
 * Errors: INVALID_ARG (NULL, sizes, alignment, workspace too small), UNSUPPORTED (as the
 * device calls), CUDA. The model must belong to the current device.
 */
size_t commet_const_update_host_workspace(const commet_model *m, const commet_mesh *mesh, int64_t chunk,
                                          int32_t want_A);
int commet_const_update_host(const commet_model *m, const commet_mesh *mesh, int64_t n_qp, const void *F, void *psi,
                             void *P, void *A, void *f_e, void *K_e, void *workspace, size_t ws_bytes, int64_t chunk,
                             void *stream);

/*
 * Constitutive update in spatial form (App. A.1, the paper's own storage): for every qp
 *   tau[:, q] = Kirchhoff stress tau_ij = P_iJ F_jJ in Voigt order (11, 22, 33, 23, 13, 12),
 *   c[:, q]   = spatial stiffness c_ijkl = F_jJ A_iJkL F_lL - delta_ik tau_jl as the 21
 *               entries C_IJ (I <= J, row-major upper triangle) of the 6 x 6 Voigt matrix,
 *               C_IJ = c_{ij kl} with (i, j) the pair of slot I and (k, l) that of slot J,
 * both symmetric, so 27 values per point leave the GPU instead of P and A's 90.
 * F [9][n_qp] in; psi [n_qp] out or NULL; tau [6][n_qp] out (required); c [21][n_qp] out
 * or NULL (stress only). Every precision of the model; status, alignment and errors as
 * commet_const_update.
 */
int commet_const_update_spatial(const commet_model *m, int64_t n_qp, const void *F, void *psi, void *tau, void *c,
                                int32_t *status, void *stream);

/*
 * Mesh of hex8 elements (App. -: deal.II-style Q1 bricks). X (host, double [n_nodes][3])
 * and conn (host, int32 [n_el][8], lexicographic node order) are copied to the device.
 * want_csr = 1 also builds, on the host, the CSR pattern of the global stiffness
 * (rows 3*node+i; columns of every node sharing an element, 3 per node, sorted),
 * an element -> CSR position map (one int32 per element node pair), and an element
 * colouring in which no two elements of one colour share a node (greedy, in element
 * order). Synchronous. Errors: INVALID_ARG (node index out of range, NULL, sizes),
 * UNSUPPORTED (nnz >= 2^31), CUDA.
 */
int commet_mesh_create(int64_t n_nodes, const double *X, int64_t n_el, const int32_t *conn, int32_t want_csr,
                       commet_mesh **out);
int commet_mesh_destroy(commet_mesh *mesh);
/* Sizes of the CSR pattern and colouring: n_rows = 3 n_nodes, nnz, n_colours. */
int commet_mesh_info(const commet_mesh *mesh, int64_t *n_rows, int64_t *nnz, int32_t *n_colours);
/* Copy the CSR pattern to HOST arrays rowptr[n_rows + 1] (int64) and col[nnz] (int32). */
int commet_mesh_csr(const commet_mesh *mesh, int64_t *rowptr, int32_t *col);

/*
 * Deformation gradient at every qp (Algorithm 1, "trial F"):
 *   F_q = I + sum_I u^I (x) grad_X phi^I(xi_q), grad_X phi = Je^{-T} grad_xi phi.
 * u [3][n_nodes] in (precision of `precision`: COMMET_F64 -> double, else float);
 * F [9][8 n_el] out.
 */
int commet_compute_F(const commet_mesh *mesh, int32_t precision, const void *u, void *F, void *stream);

/*
 * Element integrals (eq. r-quad, k-quad, in material form via App. A.1):
 *   f_e[3I+i]       = sum_q w_q P_iJ dphi_I/dX_J
 *   K_e[3I+i][3K+k] = sum_q w_q dphi_I/dX_J A_iJkL dphi_K/dX_L,  w_q = det Je (Gauss weight 1)
 * and, optionally, their sums over elements into the global residual and CSR
 * stiffness (Algorithm 1; race-free by element colouring, one launch per colour).
 * P [9][8 n_el], A [81][8 n_el] in (A may be NULL only when K_e and K_vals are NULL).
 * f_e [24][n_el], K_e [576][n_el] out or NULL.
 * r [3 n_nodes], K_vals [nnz] out or NULL: OVERWRITTEN (zeroed first, in stream order).
 * Errors: NO_CSR when r or K_vals is given for a mesh built without the CSR pattern.
 */
int commet_elem_assemble(const commet_mesh *mesh, int32_t precision, const void *P, const void *A, void *f_e,
                         void *K_e, void *r, void *K_vals, void *stream);

/*
 * The same element integrals for a major-symmetric A (A_iJkL = A_kLiJ: the tangent of every
 * hyperelastic energy, eq. nncm-chain, and so every A that commet_const_update writes).
 * K_e is then symmetric, and it is formed from its upper node blocks (36 of 64, each node
 * pair once) and written whole, its other blocks as transposes: in FP64 about a quarter
 * fewer multiply-adds. The result for a non-symmetric A is K_e of its symmetrised upper
 * blocks, not eq. k-quad: call commet_elem_assemble for such an A. Arguments, outputs,
 * scatter and errors as commet_elem_assemble; the FP32 form without scatter is the same
 * kernel as there (bound by memory, not by arithmetic).
 */
int commet_elem_assemble_symmetric(const commet_mesh *mesh, int32_t precision, const void *P, const void *A,
                                   void *f_e, void *K_e, void *r, void *K_vals, void *stream);

/*
 * Element integrals in the spatial form of eq. r-quad and k-quad:
 *   f_e[3I+i]       = sum_q w_q tau_ij grad phi_I,j
 *   K_e[3I+i][3K+k] = sum_q w_q grad phi_I,m (delta_ik tau_ml + c_imkl) grad phi_K,l
 * with grad phi_I,m = dphi_I/dX_M (F^{-1})_Mm (spatial gradients) and w_q = det Je; equal
 * to the material form of commet_elem_assemble for the same point (App. A.1).
 * F [9][8 n_el], tau [6][8 n_el], c [21][8 n_el] in (layouts of
 * commet_const_update_spatial; c may be NULL only when K_e and K_vals are NULL);
 * outputs, scatter and errors as commet_elem_assemble.
 */
int commet_elem_assemble_spatial(const commet_mesh *mesh, int32_t precision, const void *F, const void *tau,
                                 const void *c, void *f_e, void *K_e, void *r, void *K_vals, void *stream);

/*
 * Adjoints of the assembly chain, for gradients of a loss of the global residual (eq. loss of
 * App. C, the NN-EUCLID objective) through commet_const_backward:
 *   commet_residual_adjoint:   G[:, q] = dL/dP_q = w_q sum_I lam_I (x) grad_X phi_I(xi_q), the
 *                              transpose of eq. r-quad and the scatter; lam = dL/dr [3 n_nodes]
 *                              (dof 3 node + i), G [9][8 n_el] out.
 *   commet_compute_F_adjoint:  du[i][node] = dL/du = sum over the node's elements and points of
 *                              dL/dF_iJ dphi/dX_J, the transpose of the trial F; dF [9][8 n_el]
 *                              in, du [3][n_nodes] OVERWRITTEN. Summed by element colour
 *                              (deterministic): needs a mesh built with want_csr (else NO_CSR).
 */
int commet_residual_adjoint(const commet_mesh *mesh, int32_t precision, const void *lam, void *G, void *stream);
int commet_compute_F_adjoint(const commet_mesh *mesh, int32_t precision, const void *dF, void *du, void *stream);

/*
 * Fused Newton-iteration assembly: u -> F -> (Psi, P, A) -> f_e, K_e -> r, K_vals for
 * every element in one pass per colour, with P and A kept on chip (Algorithm 3 with
 * the constitutive call fused into the element loop). r [3 n_nodes], K_vals [nnz]
 * OVERWRITTEN; u [3][n_nodes]; types follow the model's precision (F32 or F64).
 */
int commet_newton_assemble(const commet_model *m, const commet_mesh *mesh, const void *u, void *r, void *K_vals,
                           int32_t *status, void *stream);

/*
 * ---- The Newton step after assembly (Sec. 4.3: CG with a Jacobi preconditioner) ----
 * These calls act on a mesh built with want_csr. Each mesh holds one small FP64
 * reduction array that the solver calls below share: calls on one mesh must not overlap
 * on the GPU (use one stream per mesh). Dofs are numbered 3 node + i (the CSR rows).
 */
/* Fixed (Dirichlet) dofs: a strictly increasing HOST list of n_fixed dofs, copied; 0
 * clears them. Synchronous. Errors: INVALID_ARG (out of range, not increasing). */
int commet_mesh_set_dirichlet(commet_mesh *mesh, int64_t n_fixed, const int64_t *dofs);
/* u[i][node] = values[j] for fixed dof j = 3 node + i; u [3][n_nodes] on the device,
 * values a HOST double array [n_fixed] read before the call returns. */
int commet_set_dirichlet_values(const commet_mesh *mesh, int32_t precision, const double *values, void *u,
                                void *stream);
/* Dirichlet conditions on the system K du = r of the update u <- u - du: rows and columns
 * of the fixed dofs in K_vals zeroed with 1 on their diagonal (the matrix stays symmetric).
 * delta NULL: r of the fixed dofs zeroed, so they keep their values (r or K_vals may be NULL).
 * delta a HOST double array [n_fixed] (prescribed increments, in the order of the fixed
 * dofs, read before the call returns): r_c = -delta_c and every free row adds the coupling
 * it loses, r_f += K_fc delta_c, so the update moves the fixed dofs by delta (the predictor
 * of a load step); r and K_vals are then required. Errors: NO_CSR, INVALID_ARG. */
int commet_apply_dirichlet(const commet_mesh *mesh, int32_t precision, void *r, void *K_vals, const double *delta,
                           void *stream);
/*
 * x = K^{-1} b by conjugate gradients (Hestenes-Stiefel) preconditioned by the inverse
 * diagonal of K, from x = 0, until |b - K x| <= rtol |b| (recursively updated residual)
 * or max_iter iterations. K_vals [nnz] (symmetric positive definite, e.g. after
 * commet_apply_dirichlet), b, x [3 n_nodes] in the precision; dot products in FP64.
 * workspace: device scratch of commet_cg_workspace() bytes, 256-byte aligned.
 * Synchronous: returns after the solve with *iters and *rel_res (HOST, may be NULL); a
 * breakdown (p.Kp = 0) ends the solve with a NaN rel_res. Deterministic for a device.
 */
size_t commet_cg_workspace(const commet_mesh *mesh, int32_t precision);
int commet_cg_solve(const commet_mesh *mesh, int32_t precision, const void *K_vals, const void *b, void *x,
                    double rtol, int32_t max_iter, void *workspace, size_t ws_bytes, int32_t *iters, double *rel_res,
                    void *stream);
/* u[i][node] += alpha du[3 node + i]: a dof-ordered increment into the [3][n_nodes] field. */
int commet_add_increment(const commet_mesh *mesh, int32_t precision, const void *du, double alpha, void *u,
                         void *stream);
/* *out (HOST) = |x|_2 of a device vector of n entries, summed in FP64 in a fixed order. */
int commet_norm2(const commet_mesh *mesh, int32_t precision, int64_t n, const void *x, double *out, void *stream);

/*
 * Backward of the constitutive update for an upstream gradient G = dL/dP [9][n_qp]:
 *   dL_dF[:, q]   = sum_iJ G_iJ A_iJkL            (A of the forward at F_q)
 *   dL_dtheta[p]  = sum_q d/dtheta_p [ G_q : P_q ]  (all network parameters, order as
 *                   commet_model_n_params), summed over q in a fixed order
 * For a CANN model (eq. cann-def) theta is its weights in the order of cann_w,
 * [d][n][2] = (w1, w2) per input and term (App. C's calibration of the CANN).
 * Recomputes the forward per qp; stores no activations. dL_dF may be NULL.
 * workspace: device scratch of commet_const_backward_workspace() bytes, 256-byte aligned.
 * Deterministic: the same inputs give bitwise the same dL_dtheta.
 * F, dL_dP, dL_dF in the model's precision, [9][n_qp], 16-byte aligned; dL_dtheta
 * [n_params] is OVERWRITTEN (zeroed when n_qp = 0). A point with a non-finite F or G or
 * J <= 0 gets NaN in dL_dF and adds nothing to dL_dtheta; for a CANN model so does a
 * point whose dL_dF or weight-gradient terms leave the precision's number range (its
 * exponential terms at large stretches, in FP32 mostly).
 * Errors: INVALID_ARG (null, misaligned or short workspace); UNSUPPORTED for the bf16
 * precision, the Gent-Thomas and KAN inner functions, stress-free models (the shift n0
 * depends on theta), 64-wide networks with one fibre, and networks whose weights,
 * gradient accumulators and per-point slabs do not fit in shared memory even at half the
 * tile (64-wide with three or more layers). Nothing is launched when INVALID_ARG or
 * UNSUPPORTED is returned.
 */
size_t commet_const_backward_workspace(const commet_model *m, int64_t n_qp);
int commet_const_backward(const commet_model *m, int64_t n_qp, const void *F, const void *dL_dP, void *dL_dF,
                          void *dL_dtheta, void *workspace, size_t ws_bytes, void *stream);

/*
 * Backward that allocates nothing (no counterpart in the paper; it exists for callers
 * whose host application owns all device memory and cannot hand the library a
 * workspace). Same computation and arguments as commet_const_backward, minus the
 * workspace: the per-CTA partial sums go to a fixed array of
 * COMMET_NOALLOC_SCRATCH_BYTES compiled into the library, which every GPU that loads the
 * library holds until the process exits.
 *  - The first call on a device looks up that array's device address
 *    (cudaGetSymbolAddress) with the device current; make it before any stream capture.
 *  - All calls share the array: calls whose kernels may overlap on the GPU race and must
 *    be serialised by the caller. Nothing in it needs to be zero before a call.
 *  - Returns COMMET_ERR_UNSUPPORTED, launching nothing, when the call would need more
 *    scratch than COMMET_NOALLOC_SCRATCH_BYTES (commet_const_backward_workspace() tells
 *    the need; FP64 d7 W32 L3 needs about 7 MB, W64 networks do not fit), and for models
 *    other than the MICNN (the CANN's backward takes a workspace).
 *  - The looked-up address is kept per device ordinal for the life of the process. A
 *    device reset (cudaDeviceReset, or anything else that destroys the primary context)
 *    can move the array, so after one this entry point must not be called again until the
 *    library has been unloaded and loaded anew.
 */
#define COMMET_NOALLOC_SCRATCH_BYTES (8u * 1024u * 1024u)
int commet_const_backward_noalloc(const commet_model *m, int64_t n_qp, const void *F, const void *dL_dP,
                                  void *dL_dF, void *dL_dtheta, void *stream);

/*
 * Target stress of a closed-form Neo-Hookean-plus-fibre model, used as synthetic
 * training data for the backward:
 *   Psi_t = mu/2 (Ibar1 - 3) + kappa (J - 1)^2 + sum_f k1/(2 k2) (exp(k2 (I4_ff - 1)^2) - 1)
 * fibres: HOST double [n_fibres][3]; F [9][n_qp] in, P [9][n_qp] out (precision as given).
 */
int commet_target_stress(int32_t precision, int64_t n_qp, const void *F, int32_t n_fibres, const double *fibres,
                         double mu, double k1, double k2, double kappa, void *P, void *stream);

/* Human-readable text for a return code (static storage). */
const char *commet_status_string(int code);

#ifdef __cplusplus
}
#endif

#endif /* COMMET_H */
