// Internal declarations shared by the CUDA translation units of libcommet.
// Not installed; the public boundary is include/commet.h.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <mutex>

#include "../../include/commet.h"

namespace commet {

constexpr int kMaxFibres = 2;
constexpr int kRedBlocks = 4096;  // partial sums per reduction slot of the solver
constexpr int kRedDoubles = 16 + 4 * kRedBlocks;
constexpr int kMaxD = 3 + 2 * kMaxFibres;

// Offsets (in elements of the path's scalar type) of the packed weight block that
// every constitutive kernel copies into shared memory once per CTA.
struct NetLayout {
    int d, W, L;
    int W1t;  // [d][W]       W1 transposed (forward: contiguous over neurons)
    int W1r;  // [W][dp]      W1 row-major, rows padded to dp (tangent seed)
    int Bt;   // [L-1][d][W]  B_k transposed
    int At;   // [L-1][W][W]  A_k transposed: At[i][j] = A_k[j][i]
    int M;    // FP64 models with L >= 2: [W][W][dp] M[i][c][m] = A_2[c][i] W1[i][m], the first
              // hidden tangent's weight product (the layer-2 tangent is then sum_i s_1[i] M[i]);
              // 0 otherwise. At, M and Ar are the last three blocks, in this order
    int Ar;   // [L-1][W][W]  A_k row-major (reverse pass); the last block
    int c;    // [L][W]
    int a;    // [W]
    int b;    // [d]
    int n0;   // [d] stress-free shift (zeros when off)
    int K0;   // [d] K at F = I
    int tab;  // FP64 models: activation tables (actdf::kSlots float pairs); 0 otherwise
    // CANN (inner == COMMET_INNER_CANN): cn terms, weights cw [d][cn][2], kinds ck [cn][3]
    int inner, cn, cw, ck;
    // ICKAN: kR layers, B-spline degree kdeg, kG intervals; offsets of the widths [kR + 1]
    // (as numbers), grid ranges lo/hi [kR] and the spline parameters
    int kR, kdeg, kG, kwid, klo, khi, kpar, kwmax;
    int total;
};

// Kinematic layer constants.
struct KinParams {
    int kin;       // COMMET_KIN_*
    int nf;        // fibres
    double fib[kMaxFibres][3];
    double kappa;  // volumetric penalty
    int stress_free;
};

// Side streams and events of the host-buffer pipeline (host_pipeline.cu), created with the
// model on its device and released with it, so that a pipeline call creates nothing. The
// mutex orders the enqueueing of concurrent calls on one model: each call records and
// waits on these events before the next call records them again.
struct PipelineRes {
    cudaStream_t in = nullptr, out = nullptr;
    cudaEvent_t start = nullptr, end_in = nullptr, end_out = nullptr;
    cudaEvent_t ev_in[2] = {}, ev_done[2] = {}, ev_free[2] = {};
    std::mutex mu;
};

}  // namespace commet

struct commet_model {
    int precision;
    int inner = COMMET_INNER_MICNN;
    int d, W, L;
    commet::KinParams kp;
    commet::NetLayout lay;
    int64_t n_params;      // parameters of the caller's network (theta of commet_model_n_params)
    int64_t n_params_net = 0;  // parameters of the network the kernels run (padded width)
    int W_user = 0;            // the caller's width; W is the padded one the kernels run
    int32_t *d_theta_map = nullptr;  // [n_params_net] padded -> caller theta index, -1 for padding
    void *d_weights = nullptr;     // packed block, element type of the precision (float for BF16_MLP)
    void *d_theta64 = nullptr;     // flat theta (double) for reference
    void *d_bf16 = nullptr;        // hidden-layer weights in bf16 fragments (BF16_MLP only)
    size_t bf16_bytes = 0;
    commet::PipelineRes *pipe = nullptr;  // host-buffer pipeline streams and events
    int device = 0;
};

struct commet_mesh {
    int64_t n_nodes = 0, n_el = 0;
    double *d_X = nullptr;          // [n_nodes][3]
    float *d_Xf = nullptr;          // [n_nodes][3] float copy
    int32_t *d_conn = nullptr;      // [n_el][8]
    // CSR pattern and colouring (want_csr)
    int64_t n_rows = 0, nnz = 0;
    int64_t *d_rowptr = nullptr;    // [n_rows + 1]
    int32_t *d_col = nullptr;       // [nnz]
    uint32_t *d_emap = nullptr;     // [n_el][8][8] CSR position of (3*gI, 3*gK)
    int32_t *d_rowlen = nullptr;    // [n_nodes] entries per dof row of a node (3 * neighbours)
    int32_t n_colours = 0;
    int32_t *d_colour_el = nullptr; // elements sorted by colour
    int64_t colour_off[65] = {0};   // offsets into d_colour_el
    // host copies for commet_mesh_csr
    int64_t *h_rowptr = nullptr;
    int32_t *h_col = nullptr;
    // solver state: Dirichlet dofs (mask over the 3 n_nodes dofs, the sorted list and a
    // value buffer) and the FP64 reduction array of the CG scalars and partial sums
    int64_t n_fixed = 0;
    uint8_t *d_fixed = nullptr;
    int64_t *d_fixed_dofs = nullptr;
    double *d_fixed_vals = nullptr;
    double *d_delta = nullptr;  // [n_rows] prescribed increments, dense
    double *d_red = nullptr;
    unsigned int *d_err = nullptr;  // [16]: [0] tiles whose bulk copies did not complete in time,
                                    // [1..2] last-block counters of the CG kernels (zero between launches)
    int device = 0;
};

namespace commet {

// Host-buffer pipeline (host_pipeline.cu): chunked copies in, kernels, copies out.
int pipeline_res_create(commet_model *m);   // on the current device, at model creation
void pipeline_res_destroy(commet_model *m);
size_t host_pipeline_workspace(const commet_model *m, const commet_mesh *mesh, int64_t chunk, bool want_A);
int run_host_pipeline(const commet_model *m, const commet_mesh *mesh, int64_t n_qp, const void *F, void *psi, void *P,
                      void *A, void *f_e, void *K_e, void *ws, size_t ws_bytes, int64_t chunk, cudaStream_t s);

// Launchers (return COMMET_* codes). Pointers already validated.
int launch_const_update(const commet_model *m, int64_t n_qp, const void *F, void *psi, void *P, void *A,
                        int32_t *status, cudaStream_t s, void *dN_out = nullptr);
int launch_const_update_bf16(const commet_model *m, int64_t n_qp, const void *F, void *psi, void *P, void *A,
                             int32_t *status, cudaStream_t s, bool spatial = false);
// Spatial form (App. A.1): tau [6][n], c [21][n] (Voigt) instead of P, A; all precisions.
int launch_const_update_spatial(const commet_model *m, int64_t n_qp, const void *F, void *psi, void *tau, void *c,
                                int32_t *status, cudaStream_t s);
// Adjoints of the residual assembly and of the trial F (elem.cu): G = dL/dP from lam = dL/dr
// (lam may be null), du = dL/du from dF = dL/dF (dF may be null; needs the colouring).
int launch_assembly_adjoints(const commet_mesh *mesh, int precision, const void *lam, void *G, const void *dF,
                             void *du, cudaStream_t s);
// Newton step after assembly (solver.cu)
size_t cg_workspace_bytes(const commet_mesh *mesh, int precision);
int launch_cg_solve(const commet_mesh *mesh, int precision, const void *K_vals, const void *b, void *x, double rtol,
                    int max_iter, void *ws, int32_t *iters, double *rel_res, cudaStream_t s);
int launch_apply_dirichlet(const commet_mesh *mesh, int precision, void *r, void *K_vals, const double *delta_host,
                           cudaStream_t s);
int launch_set_dirichlet_values(const commet_mesh *mesh, int precision, const double *vals_host, void *u,
                                cudaStream_t s);
int launch_add_increment(const commet_mesh *mesh, int precision, const void *du, double alpha, void *u,
                         cudaStream_t s);
int launch_norm2(const commet_mesh *mesh, int precision, int64_t n, const void *x, double *out, cudaStream_t s);
int launch_elem_assemble_spatial(const commet_mesh *mesh, int precision, const void *F, const void *tau,
                                 const void *c, void *f_e, void *K_e, void *r, void *K_vals, cudaStream_t s);
int launch_status_init(int32_t *status, cudaStream_t s);
int launch_target_stress(int precision, int64_t n_qp, const void *F, int nf, const double *fib, double mu,
                         double k1, double k2, double kappa, void *P, cudaStream_t s);
int launch_compute_F(const commet_mesh *mesh, int precision, const void *u, void *F, cudaStream_t s);
// symmetric: A is major symmetric (every hyperelastic tangent); K_e from its upper blocks
int launch_elem_assemble(const commet_mesh *mesh, int precision, const void *P, const void *A, void *f_e,
                         void *K_e, void *r, void *K_vals, cudaStream_t s, bool symmetric = false);
int launch_newton_assemble(const commet_model *m, const commet_mesh *mesh, const void *u, void *r, void *K_vals,
                           int32_t *status, cudaStream_t s);
int prepare_bf16_weights(commet_model *m);
size_t backward_workspace_bytes(const commet_model *m, int64_t n_qp);
int launch_const_backward(const commet_model *m, int64_t n_qp, const void *F, const void *G, void *dF, void *dtheta,
                          void *ws, size_t ws_bytes, cudaStream_t s);

// Host-side mesh graph construction (mesh_host.cpp).
int build_csr_and_colouring(int64_t n_nodes, int64_t n_el, const int32_t *conn, commet_mesh *mesh);

// SM count of the current device (cached per device ordinal).
int sm_count();

}  // namespace commet

#define COMMET_CUDA_TRY(expr)                                   \
    do {                                                        \
        cudaError_t _e = (expr);                                \
        if (_e != cudaSuccess) return COMMET_ERR_CUDA;          \
    } while (0)
