// The Newton step after assembly (Sec. 4.3): Dirichlet conditions on the assembled CSR
// system, the Jacobi-preconditioned conjugate gradient solve the paper uses (CG with
// Jacobi relaxation as the preconditioner), and the displacement update.
//
// CG layout: every vector lives in the workspace ([5][n] of the precision's type) and the
// scalars of the recurrence in the mesh's reduction array, so that an iteration is three
// launches with no host round trip: SpMV with the p.Ap partial sums, whose last block to
// finish forms alpha; the x / r / z update with the r.z and r.r partial sums, whose last
// block forms beta and the stopping test; and the p update. Every kernel first reads the
// `done` word and returns at once after convergence, so the host reads that word only once
// per chunk of iterations. Dot products are summed in FP64 in a fixed order (per-block
// partials, then one tree in index order): a solve is bitwise reproducible for a given
// device and grid.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "internal.h"

namespace commet {

namespace {

constexpr int kSolveThreads = 256;
constexpr int kChunk = 16;  // iterations between host checks of the stopping word

// reduction array layout (doubles): scalars, then partial sums [2][kRedBlocks]
// PART_A / PART_B are two partial-sum regions (2 x kRedBlocks each).
enum { S_RZ = 0, S_RR, S_BB, S_ALPHA, S_BETA, S_DONE, S_ITERS, S_RTOL2, S_COUNT = 16 };
constexpr int PART_A = S_COUNT, PART_B = S_COUNT + 2 * kRedBlocks;

// True in the block that finishes last: every block publishes its partial sums, then
// counts itself in; the last one sums all partials (in index order, so the result does not
// depend on which block it is) and resets the counter for the next launch. No block waits.
__device__ __forceinline__ bool last_block(unsigned int *counter) {
    __shared__ bool is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (is_last) __threadfence();
    return is_last;
}

int red_blocks() { return std::min(kRedBlocks, 16 * sm_count()); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block sum of (a, b) written to part[blockIdx.x], part[kRedBlocks + blockIdx.x].
__device__ __forceinline__ void block_sum2(double a, double b, double *part) {
    __shared__ double s[2][kSolveThreads / 32];
    a = warp_sum(a);
    b = warp_sum(b);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        s[0][w] = a;
        s[1][w] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0.0, y = 0.0;
        for (int i = 0; i < kSolveThreads / 32; ++i) {
            x += s[0][i];
            y += s[1][i];
        }
        part[blockIdx.x] = x;
        part[kRedBlocks + blockIdx.x] = y;
    }
}

// One block sums the nb partials of both slots in index order.
__device__ __forceinline__ void sum_partials(const double *part, int nb, double &a, double &b) {
    __shared__ double s[2][kSolveThreads];
    double x = 0.0, y = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        x += part[i];
        y += part[kRedBlocks + i];
    }
    s[0][threadIdx.x] = x;
    s[1][threadIdx.x] = y;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            s[0][threadIdx.x] += s[0][threadIdx.x + h];
            s[1][threadIdx.x] += s[1][threadIdx.x + h];
        }
        __syncthreads();
    }
    a = s[0][0];
    b = s[1][0];
}

// ------------------------------------------------------------- Dirichlet
// One warp per row. delta (dense over the dofs, zero at free ones) or null: with delta the
// fixed dofs move by it in the next update u <- u - du, so r_c = -delta_c and a free row
// keeps the coupling it loses, r_f += K_fc delta_c, summed before the K_fc entries are zeroed.
template <typename T>
__global__ void dirichlet_kernel(int64_t n_rows, const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                                 const uint8_t *__restrict__ fixed, const double *__restrict__ delta,
                                 T *__restrict__ K_vals, T *__restrict__ r) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n_rows) return;
    const bool frow = fixed[row] != 0;
    double coupling = 0.0;
    if (K_vals != nullptr) {
        for (int64_t k = rowptr[row] + lane; k < rowptr[row + 1]; k += 32) {
            const int32_t c = col[k];
            if (frow) {
                K_vals[k] = (c == row) ? T(1) : T(0);
            } else if (fixed[c]) {
                if (delta != nullptr) coupling += (double)K_vals[k] * delta[c];
                K_vals[k] = T(0);
            }
        }
    }
    coupling = warp_sum(coupling);
    if (r != nullptr && lane == 0) {
        if (frow)
            r[row] = delta != nullptr ? (T)(-delta[row]) : T(0);
        else if (delta != nullptr)
            r[row] = (T)((double)r[row] + coupling);
    }
}

__global__ void scatter_delta_kernel(int64_t n_fixed, const int64_t *__restrict__ dofs,
                                     const double *__restrict__ vals, double *__restrict__ dense) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_fixed) dense[dofs[i]] = vals[i];
}

template <typename T>
__global__ void set_values_kernel(int64_t n_fixed, const int64_t *__restrict__ dofs, const double *__restrict__ vals,
                                  int64_t n_nodes, T *__restrict__ u) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_fixed) return;
    const int64_t d = dofs[i];
    u[(d % 3) * n_nodes + d / 3] = (T)vals[i];
}

template <typename T>
__global__ void add_increment_kernel(int64_t n_nodes, const T *__restrict__ du, double alpha, T *__restrict__ u) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * n_nodes) return;
    u[(i % 3) * n_nodes + i / 3] += (T)(alpha * (double)du[i]);
}

template <typename T>
__global__ void norm2_partial_kernel(int64_t n, const T *__restrict__ x, double *__restrict__ part) {
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = (double)x[i];
        s += v * v;
    }
    block_sum2(s, 0.0, part);
}

__global__ void norm2_final_kernel(const double *__restrict__ part, int nb, double *__restrict__ out) {
    double a, b;
    sum_partials(part, nb, a, b);
    if (threadIdx.x == 0) *out = sqrt(a);
}

// ------------------------------------------------------------------- CG
// x = 0, r = b, dinv = 1 / diag(K), z = dinv r, p = z; partials of r.z and b.b
template <typename T>
__global__ void cg_init_kernel(int64_t n, const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                               const T *__restrict__ K_vals, const T *__restrict__ b, T *__restrict__ x,
                               T *__restrict__ r, T *__restrict__ z, T *__restrict__ p, T *__restrict__ dinv,
                               double *__restrict__ red) {
    double rz = 0.0, bb = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        // diagonal by binary search in the sorted row
        int64_t lo = rowptr[i], hi = rowptr[i + 1] - 1;
        T diag = T(0);
        while (lo <= hi) {
            const int64_t mid = (lo + hi) >> 1;
            const int32_t c = col[mid];
            if (c == i) {
                diag = K_vals[mid];
                break;
            }
            if (c < i)
                lo = mid + 1;
            else
                hi = mid - 1;
        }
        const T di = (diag != T(0)) ? T(1) / diag : T(0);
        const T bi = b[i];
        x[i] = T(0);
        r[i] = bi;
        dinv[i] = di;
        z[i] = di * bi;
        p[i] = di * bi;
        rz += (double)bi * (double)(di * bi);
        bb += (double)bi * (double)bi;
    }
    block_sum2(rz, bb, red + PART_A);
}

__global__ void cg_start_kernel(double *__restrict__ red, int nb, double rtol) {
    double rz, bb;
    sum_partials(red + PART_A, nb, rz, bb);
    if (threadIdx.x == 0) {
        red[S_RZ] = rz;
        red[S_BB] = bb;
        red[S_RR] = bb;
        red[S_RTOL2] = rtol * rtol;
        red[S_ITERS] = 0.0;
        red[S_DONE] = (bb == 0.0) ? 1.0 : 0.0;
    }
}

// Ap = K p with 4 lanes per row (8 rows per warp). GB300 charges every FP64 warp
// instruction in full, so the row sums are split where they cost fewest FP64 instructions:
// about nnz / 32 DFMAs plus two shuffle additions per 8 rows (a warp per row would spend
// 5 shuffle additions per row on its reduction). The 4 lanes of a row read 4 consecutive
// values (one 32-byte sector). Partial sums of p.Ap per block.
template <typename T>
__global__ void cg_spmv_kernel(int64_t n_rows, const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                               const T *__restrict__ K_vals, const T *__restrict__ p, T *__restrict__ Ap,
                               double *__restrict__ red, unsigned int *__restrict__ counter) {
    if (red[S_DONE] != 0.0) return;
    const int lane = threadIdx.x & 31, sub = lane & 3;
    const int64_t stride = ((int64_t)gridDim.x * blockDim.x) >> 2;  // rows per grid pass
    double pap = 0.0;
    // base is uniform over the warp, so every lane reaches the shuffles together
    for (int64_t base = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 8; base < n_rows; base += stride) {
        const int64_t row = base + (lane >> 2);
        double a = 0.0;
        if (row < n_rows) {
            const int64_t e = rowptr[row + 1];
            for (int64_t k = rowptr[row] + sub; k < e; k += 4) a += (double)K_vals[k] * (double)p[col[k]];
        }
        a += __shfl_xor_sync(0xffffffffu, a, 1);
        a += __shfl_xor_sync(0xffffffffu, a, 2);
        if (sub == 0 && row < n_rows) {
            Ap[row] = (T)a;
            pap += a * (double)p[row];
        }
    }
    block_sum2(pap, 0.0, red + PART_A);
    if (last_block(counter)) {
        double s_pap, unused;
        sum_partials(red + PART_A, gridDim.x, s_pap, unused);
        if (threadIdx.x == 0) {
            red[S_ALPHA] = red[S_RZ] / s_pap;
            *counter = 0u;
        }
    }
}

// x += alpha p, r -= alpha Ap, z = dinv r; partials of the new r.z and r.r, from which the
// last block forms beta and the stopping test.
template <typename T>
__global__ void cg_update_kernel(int64_t n, T *__restrict__ x, T *__restrict__ r, T *__restrict__ z,
                                 const T *__restrict__ p, const T *__restrict__ Ap, const T *__restrict__ dinv,
                                 double *__restrict__ red, unsigned int *__restrict__ counter) {
    if (red[S_DONE] != 0.0) return;
    const T alpha = (T)red[S_ALPHA];
    double rz = 0.0, rr = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        x[i] += alpha * p[i];
        const T ri = r[i] - alpha * Ap[i];
        r[i] = ri;
        const T zi = dinv[i] * ri;
        z[i] = zi;
        rz += (double)ri * (double)zi;
        rr += (double)ri * (double)ri;
    }
    block_sum2(rz, rr, red + PART_B);
    if (last_block(counter)) {
        double rz_new, s_rr;
        sum_partials(red + PART_B, gridDim.x, rz_new, s_rr);
        if (threadIdx.x == 0) {
            red[S_BETA] = rz_new / red[S_RZ];
            red[S_RZ] = rz_new;
            red[S_RR] = s_rr;
            red[S_ITERS] += 1.0;
            if (s_rr <= red[S_RTOL2] * red[S_BB] || !(s_rr == s_rr)) red[S_DONE] = 1.0;
            *counter = 0u;
        }
    }
}

template <typename T>
__global__ void cg_p_kernel(int64_t n, const T *__restrict__ z, T *__restrict__ p, const double *__restrict__ red) {
    if (red[S_DONE] != 0.0) return;
    const T beta = (T)red[S_BETA];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = z[i] + beta * p[i];
}

template <typename T>
int cg_typed(const commet_mesh *mesh, const void *K_vals_v, const void *b_v, void *x_v, double rtol, int max_iter,
             void *ws, int32_t *iters, double *rel_res, cudaStream_t s) {
    const int64_t n = mesh->n_rows;
    const T *K_vals = (const T *)K_vals_v;
    const T *b = (const T *)b_v;
    T *x = (T *)x_v;
    T *r = (T *)ws, *z = r + n, *p = z + n, *Ap = p + n, *dinv = Ap + n;
    double *red = mesh->d_red;
    unsigned int *counters = mesh->d_err + 1;  // [2], zero between launches
    const int nb = red_blocks();
    const int spmv_blocks = (int)std::min<int64_t>(nb, (n * 4 + kSolveThreads - 1) / kSolveThreads);
    const int vec_blocks = (int)std::min<int64_t>(nb, (n + kSolveThreads - 1) / kSolveThreads);
    cg_init_kernel<T><<<vec_blocks, kSolveThreads, 0, s>>>(n, mesh->d_rowptr, mesh->d_col, K_vals, b, x, r, z, p,
                                                           dinv, red);
    cg_start_kernel<<<1, kSolveThreads, 0, s>>>(red, vec_blocks, rtol);
    COMMET_CUDA_TRY(cudaGetLastError());
    auto iterations = [&](int m, cudaStream_t st) {
        for (int k = 0; k < m; ++k) {
            cg_spmv_kernel<T><<<spmv_blocks, kSolveThreads, 0, st>>>(n, mesh->d_rowptr, mesh->d_col, K_vals, p, Ap,
                                                                     red, counters);
            cg_update_kernel<T><<<vec_blocks, kSolveThreads, 0, st>>>(n, x, r, z, p, Ap, dinv, red, counters + 1);
            cg_p_kernel<T><<<vec_blocks, kSolveThreads, 0, st>>>(n, z, p, red);
        }
    };
    // A chunk of kChunk iterations (3 kChunk launches with the same arguments) is captured
    // once as a CUDA graph and replayed, which removes the per-launch overhead that bounds
    // the iteration on small meshes. If capture is not available the launches go directly.
    cudaGraphExec_t chunk_exec = nullptr;
    if (max_iter >= kChunk) {
        cudaStream_t cs = nullptr;
        cudaGraph_t graph = nullptr;
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess) {
            if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                iterations(kChunk, cs);
                if (cudaStreamEndCapture(cs, &graph) == cudaSuccess && graph != nullptr) {
                    if (cudaGraphInstantiate(&chunk_exec, graph, 0) != cudaSuccess) chunk_exec = nullptr;
                    cudaGraphDestroy(graph);
                }
            }
            cudaStreamDestroy(cs);
        }
        (void)cudaGetLastError();  // a failed capture leaves the direct launches below
    }
    double host[S_COUNT];
    int done_iters = 0;
    int rc = COMMET_OK;
    for (int it0 = 0; it0 < max_iter; it0 += kChunk) {
        const int m = std::min(kChunk, max_iter - it0);
        if (m == kChunk && chunk_exec != nullptr) {
            if (cudaGraphLaunch(chunk_exec, s) != cudaSuccess) {
                rc = COMMET_ERR_CUDA;
                break;
            }
        } else {
            iterations(m, s);
        }
        if (cudaGetLastError() != cudaSuccess) {
            rc = COMMET_ERR_CUDA;
            break;
        }
        if (cudaMemcpyAsync(host, red, sizeof(host), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            rc = COMMET_ERR_CUDA;
            break;
        }
        done_iters = (int)host[S_ITERS];
        if (host[S_DONE] != 0.0) break;
    }
    if (chunk_exec != nullptr) {
        cudaStreamSynchronize(s);
        cudaGraphExecDestroy(chunk_exec);
    }
    if (rc != COMMET_OK) return rc;
    if (iters) *iters = done_iters;
    if (rel_res) *rel_res = host[S_BB] > 0.0 ? std::sqrt(host[S_RR] / host[S_BB]) : 0.0;
    return COMMET_OK;
}

}  // namespace

size_t cg_workspace_bytes(const commet_mesh *mesh, int precision) {
    const size_t es = precision == COMMET_F64 ? 8 : 4;
    return ((size_t)5 * mesh->n_rows * es + 255) / 256 * 256;
}

int launch_cg_solve(const commet_mesh *mesh, int precision, const void *K_vals, const void *b, void *x, double rtol,
                    int max_iter, void *ws, int32_t *iters, double *rel_res, cudaStream_t s) {
    if (precision == COMMET_F64) return cg_typed<double>(mesh, K_vals, b, x, rtol, max_iter, ws, iters, rel_res, s);
    return cg_typed<float>(mesh, K_vals, b, x, rtol, max_iter, ws, iters, rel_res, s);
}

int launch_apply_dirichlet(const commet_mesh *mesh, int precision, void *r, void *K_vals, const double *delta_host,
                           cudaStream_t s) {
    if (mesh->n_rows == 0 || mesh->d_fixed == nullptr) return COMMET_OK;
    const double *delta = nullptr;
    if (delta_host != nullptr) {
        // prescribed increments, dense over the dofs (zero at the free ones)
        const int64_t nf = mesh->n_fixed;
        COMMET_CUDA_TRY(cudaMemsetAsync(mesh->d_delta, 0, sizeof(double) * mesh->n_rows, s));
        COMMET_CUDA_TRY(
            cudaMemcpyAsync(mesh->d_fixed_vals, delta_host, sizeof(double) * nf, cudaMemcpyHostToDevice, s));
        scatter_delta_kernel<<<(unsigned)((nf + kSolveThreads - 1) / kSolveThreads), kSolveThreads, 0, s>>>(
            nf, mesh->d_fixed_dofs, mesh->d_fixed_vals, mesh->d_delta);
        delta = mesh->d_delta;
    }
    const int64_t blocks = (mesh->n_rows * 32 + kSolveThreads - 1) / kSolveThreads;
    if (precision == COMMET_F64)
        dirichlet_kernel<double><<<(unsigned)blocks, kSolveThreads, 0, s>>>(
            mesh->n_rows, mesh->d_rowptr, mesh->d_col, mesh->d_fixed, delta, (double *)K_vals, (double *)r);
    else
        dirichlet_kernel<float><<<(unsigned)blocks, kSolveThreads, 0, s>>>(
            mesh->n_rows, mesh->d_rowptr, mesh->d_col, mesh->d_fixed, delta, (float *)K_vals, (float *)r);
    COMMET_CUDA_TRY(cudaGetLastError());
    // the host increments are read by the copy before the call returns
    if (delta_host != nullptr) COMMET_CUDA_TRY(cudaStreamSynchronize(s));
    return COMMET_OK;
}

int launch_set_dirichlet_values(const commet_mesh *mesh, int precision, const double *vals_host, void *u,
                                cudaStream_t s) {
    const int64_t nf = mesh->n_fixed;
    if (nf == 0) return COMMET_OK;
    COMMET_CUDA_TRY(cudaMemcpyAsync(mesh->d_fixed_vals, vals_host, sizeof(double) * nf, cudaMemcpyHostToDevice, s));
    const int64_t blocks = (nf + kSolveThreads - 1) / kSolveThreads;
    if (precision == COMMET_F64)
        set_values_kernel<double><<<(unsigned)blocks, kSolveThreads, 0, s>>>(nf, mesh->d_fixed_dofs,
                                                                             mesh->d_fixed_vals, mesh->n_nodes,
                                                                             (double *)u);
    else
        set_values_kernel<float><<<(unsigned)blocks, kSolveThreads, 0, s>>>(nf, mesh->d_fixed_dofs, mesh->d_fixed_vals,
                                                                            mesh->n_nodes, (float *)u);
    COMMET_CUDA_TRY(cudaGetLastError());
    // the host values are read by the copy before the call returns
    COMMET_CUDA_TRY(cudaStreamSynchronize(s));
    return COMMET_OK;
}

int launch_add_increment(const commet_mesh *mesh, int precision, const void *du, double alpha, void *u,
                         cudaStream_t s) {
    const int64_t n = 3 * mesh->n_nodes;
    if (n == 0) return COMMET_OK;
    const int64_t blocks = (n + kSolveThreads - 1) / kSolveThreads;
    if (precision == COMMET_F64)
        add_increment_kernel<double><<<(unsigned)blocks, kSolveThreads, 0, s>>>(mesh->n_nodes, (const double *)du,
                                                                                alpha, (double *)u);
    else
        add_increment_kernel<float><<<(unsigned)blocks, kSolveThreads, 0, s>>>(mesh->n_nodes, (const float *)du, alpha,
                                                                               (float *)u);
    return cudaGetLastError() == cudaSuccess ? COMMET_OK : COMMET_ERR_CUDA;
}

int launch_norm2(const commet_mesh *mesh, int precision, int64_t n, const void *x, double *out, cudaStream_t s) {
    double *red = mesh->d_red;
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(red_blocks(), (n + kSolveThreads - 1) / kSolveThreads));
    if (precision == COMMET_F64)
        norm2_partial_kernel<double><<<nb, kSolveThreads, 0, s>>>(n, (const double *)x, red + PART_A);
    else
        norm2_partial_kernel<float><<<nb, kSolveThreads, 0, s>>>(n, (const float *)x, red + PART_A);
    norm2_final_kernel<<<1, kSolveThreads, 0, s>>>(red + PART_A, nb, red + S_COUNT - 1);
    COMMET_CUDA_TRY(cudaGetLastError());
    COMMET_CUDA_TRY(cudaMemcpyAsync(out, red + S_COUNT - 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    COMMET_CUDA_TRY(cudaStreamSynchronize(s));
    return COMMET_OK;
}

}  // namespace commet
