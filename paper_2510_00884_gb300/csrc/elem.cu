// Hex8 element kernels: trial F at the Gauss points (Algorithm 1), the element
// residual and stiffness integrals (eq. r-quad, k-quad in material form, App. A.1),
// and their race-free sum into the global residual and CSR stiffness by element colour.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "hex8.cuh"
#include "internal.h"
#include "tma.cuh"

namespace commet {

template <typename T>
__device__ __forceinline__ T node_coord(const double *X, int64_t n, int a) {
    return (T)X[3 * n + a];
}

// ------------------------------------------------------------------ compute_F
template <typename T>
__global__ void compute_F_kernel(int64_t n_el, int64_t n_nodes, const int32_t *__restrict__ conn,
                                 const double *__restrict__ X, const T *__restrict__ u, T *__restrict__ F) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= 8 * n_el) return;
    const int64_t e = gid >> 3;
    const int q = (int)(gid & 7);
    T Xe[8][3], ue[8][3];
#pragma unroll
    for (int I = 0; I < 8; ++I) {
        const int64_t n = conn[8 * e + I];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            Xe[I][a] = node_coord<T>(X, n, a);
            ue[I][a] = u[a * n_nodes + n];
        }
    }
    T gX[8][3], w;
    physical_grads<T>(Xe, q, gX, w);
    const int64_t n_qp = 8 * n_el;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int J = 0; J < 3; ++J) {
            T s = (i == J) ? T(1) : T(0);
#pragma unroll
            for (int I = 0; I < 8; ++I) s += ue[I][i] * gX[I][J];
            F[(3 * i + J) * n_qp + gid] = s;
        }
}

int launch_compute_F(const commet_mesh *mesh, int precision, const void *u, void *F, cudaStream_t s) {
    const int64_t n = 8 * mesh->n_el;
    if (n == 0) return COMMET_OK;
    const int tpb = 256;
    const int64_t blocks = (n + tpb - 1) / tpb;
    if (precision == COMMET_F64)
        compute_F_kernel<double><<<(unsigned)blocks, tpb, 0, s>>>(mesh->n_el, mesh->n_nodes, mesh->d_conn, mesh->d_X,
                                                                   (const double *)u, (double *)F);
    else
        compute_F_kernel<float><<<(unsigned)blocks, tpb, 0, s>>>(mesh->n_el, mesh->n_nodes, mesh->d_conn, mesh->d_X,
                                                                  (const float *)u, (float *)F);
    return cudaGetLastError() == cudaSuccess ? COMMET_OK : COMMET_ERR_CUDA;
}

// -------------------------------------------------------------- elem_assemble
// 8 lanes per element (lane I = element node I, which owns dof rows 3I..3I+2);
// 16 elements per 128-thread CTA. Per Gauss point the element's P and A (90 values)
// are staged in shared memory and read by its 8 lanes.
constexpr int kElPerCta = 16;

// SYM (a major-symmetric A, A_iJkL = A_kLiJ, as every hyperelastic tangent): K_e is
// symmetric, and lane I forms only the blocks (I, K) with K = I, I + 1, I + 2, I + 3 and,
// for I < 4, I + 4 (mod 8): each unordered node pair once, at most 5 blocks per lane
// instead of 8; every block other than (I, I) is also written transposed as (K, I).
template <typename T, bool SCATTER, bool SYM = false>
__global__ void __launch_bounds__(128)
    elem_assemble_kernel(int64_t n_el, const int32_t *__restrict__ el_list, int64_t n_list,
                         const int32_t *__restrict__ conn, const double *__restrict__ X, const T *__restrict__ P,
                         const T *__restrict__ A, T *__restrict__ f_e, T *__restrict__ K_e, T *__restrict__ r,
                         T *__restrict__ K_vals, const uint32_t *__restrict__ emap,
                         const int32_t *__restrict__ rowlen) {
    __shared__ T s_g[kElPerCta][8][8][3];  // [el][qp][node][dir]
    __shared__ T s_w[kElPerCta][8];
    __shared__ T s_pa[kElPerCta][90];      // P (9) then A (81) of the current qp
    const int le = threadIdx.x >> 3, I = threadIdx.x & 7;
    const int64_t li = (int64_t)blockIdx.x * kElPerCta + le;
    const bool valid = li < n_list;
    const int64_t e = valid ? (el_list ? (int64_t)el_list[li] : li) : 0;
    const int64_t n_qp = 8 * n_el;
    {
        // lane I computes the gradients at Gauss point I
        T Xe[8][3];
#pragma unroll
        for (int K = 0; K < 8; ++K) {
            const int64_t n = conn[8 * e + K];
#pragma unroll
            for (int a = 0; a < 3; ++a) Xe[K][a] = (T)X[3 * n + a];
        }
        T gX[8][3], w;
        physical_grads<T>(Xe, I, gX, w);
#pragma unroll
        for (int K = 0; K < 8; ++K)
#pragma unroll
            for (int a = 0; a < 3; ++a) s_g[le][I][K][a] = gX[K][a];
        s_w[le][I] = w;
    }
    constexpr int NB = SYM ? 5 : 8;  // blocks per lane: slot b is node K = (I + b) mod 8 (SYM) or b
    T f[3] = {T(0), T(0), T(0)};
    T Kr[3][NB][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int K = 0; K < NB; ++K)
#pragma unroll
            for (int k = 0; k < 3; ++k) Kr[i][K][k] = T(0);
    const bool want_K = (A != nullptr);
    for (int q = 0; q < 8; ++q) {
        __syncthreads();
        const int64_t qq = 8 * e + q;
        for (int c = I; c < 90; c += 8) {
            T v = T(0);
            if (c < 9)
                v = P[c * n_qp + qq];
            else if (want_K)
                v = A[(c - 9) * n_qp + qq];
            s_pa[le][c] = v;
        }
        __syncthreads();
        const T w = s_w[le][q];
        T wg[3];
#pragma unroll
        for (int J = 0; J < 3; ++J) wg[J] = w * s_g[le][q][I][J];
        const T *Pq = &s_pa[le][0];
        const T *Aq = &s_pa[le][9];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            f[i] += Pq[3 * i] * wg[0];
            f[i] += Pq[3 * i + 1] * wg[1];
            f[i] += Pq[3 * i + 2] * wg[2];
        }
        if (want_K) {
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                T T3[3][3];  // [k][L] = sum_J wg_J A_iJkL
#pragma unroll
                for (int k = 0; k < 3; ++k)
#pragma unroll
                    for (int L = 0; L < 3; ++L)
                        T3[k][L] = wg[0] * Aq[(3 * i) * 9 + 3 * k + L] + wg[1] * Aq[(3 * i + 1) * 9 + 3 * k + L] +
                                   wg[2] * Aq[(3 * i + 2) * 9 + 3 * k + L];
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    if (SYM && b == 4 && I >= 4) continue;
                    const int K = SYM ? ((I + b) & 7) : b;
                    const T g0 = s_g[le][q][K][0], g1 = s_g[le][q][K][1], g2 = s_g[le][q][K][2];
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        // one fused multiply-add per product, accumulated in place
                        Kr[i][b][k] += T3[k][0] * g0;
                        Kr[i][b][k] += T3[k][1] * g1;
                        Kr[i][b][k] += T3[k][2] * g2;
                    }
                }
            }
        }
    }
    if (!valid) return;
    if (f_e != nullptr) {
#pragma unroll
        for (int i = 0; i < 3; ++i) f_e[(3 * I + i) * n_el + e] = f[i];
    }
    if (K_e != nullptr && want_K) {
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            if (SYM && b == 4 && I >= 4) continue;
            const int K = SYM ? ((I + b) & 7) : b;
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    K_e[((3 * I + i) * 24 + 3 * K + k) * n_el + e] = Kr[i][b][k];
                    if (SYM && b > 0) K_e[((3 * K + k) * 24 + 3 * I + i) * n_el + e] = Kr[i][b][k];
                }
        }
    }
    if (SCATTER) {
        const int64_t gI = conn[8 * e + I];
        if (r != nullptr) {
#pragma unroll
            for (int i = 0; i < 3; ++i) r[3 * gI + i] += f[i];
        }
        if (K_vals != nullptr && want_K) {
            const int64_t rl = rowlen[gI];
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                if (SYM && b == 4 && I >= 4) continue;
                const int K = SYM ? ((I + b) & 7) : b;
                const int64_t base = emap[(8 * e + I) * 8 + K];
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int k = 0; k < 3; ++k) K_vals[base + i * rl + k] += Kr[i][b][k];
                if (SYM && b > 0) {
                    // the transposed block into the rows of node K (no other element of this
                    // colour touches them)
                    const int64_t base2 = emap[(8 * e + K) * 8 + I];
                    const int64_t rl2 = rowlen[conn[8 * e + K]];
#pragma unroll
                    for (int i = 0; i < 3; ++i)
#pragma unroll
                        for (int k = 0; k < 3; ++k) K_vals[base2 + k * rl2 + i] += Kr[i][b][k];
                }
            }
        }
    }
}

// ------------------------------------------------- TMA-fed element integrals
// The same integrals with the P and A of a tile of 16 consecutive elements (128 points)
// brought into shared memory by two 2D tensor copies ([9][128] and [81][128] boxes of the
// component-major tables) instead of per-lane strided loads: the copies overlap the
// gradient computation and arrive as whole 512-byte rows. Used for FP32, where the kernel
// is bound by HBM; FP64 is bound by its FP64 pipe and keeps the kernel above.
constexpr int kTmaQP = kElPerCta * 8;
constexpr int kTmaTries = 1 << 20;

template <typename T>
__global__ void __launch_bounds__(128)
    elem_tma_kernel(int64_t n_el, const __grid_constant__ CUtensorMap tmP, const __grid_constant__ CUtensorMap tmA,
                    int want_K, const int32_t *__restrict__ conn, const double *__restrict__ X, T *__restrict__ f_e,
                    T *__restrict__ K_e, unsigned int *__restrict__ err) {
    extern __shared__ __align__(128) unsigned char dsm[];
    T *s_p = reinterpret_cast<T *>(dsm);  // [9][128]
    T *s_a = s_p + 9 * kTmaQP;            // [81][128]
    __shared__ __align__(8) uint64_t bar;
    __shared__ T s_g[kElPerCta][8][8][3];
    __shared__ T s_w[kElPerCta][8];
    const int le = threadIdx.x >> 3, I = threadIdx.x & 7;
    const int64_t el0 = (int64_t)blockIdx.x * kElPerCta;
    const int64_t e = el0 + le;
    const bool valid = e < n_el;
    const int64_t ec = valid ? e : n_el - 1;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t bytes = (uint32_t)((9 + (want_K ? 81 : 0)) * kTmaQP * sizeof(T));
        mbar_expect_tx(&bar, bytes);
        tma_load_2d(s_p, &tmP, (int)(el0 * 8), 0, &bar);
        if (want_K) tma_load_2d(s_a, &tmA, (int)(el0 * 8), 0, &bar);
    }
    {
        // lane I: the gradients at Gauss point I, while the copies are in flight
        T Xe[8][3];
#pragma unroll
        for (int K = 0; K < 8; ++K) {
            const int64_t n = conn[8 * ec + K];
#pragma unroll
            for (int a = 0; a < 3; ++a) Xe[K][a] = (T)X[3 * n + a];
        }
        T gX[8][3], w;
        physical_grads<T>(Xe, I, gX, w);
#pragma unroll
        for (int K = 0; K < 8; ++K)
#pragma unroll
            for (int a = 0; a < 3; ++a) s_g[le][I][K][a] = gX[K][a];
        s_w[le][I] = w;
    }
    __syncthreads();
    if (!mbar_wait_bounded(&bar, 0, kTmaTries)) {
        // cannot happen in a correct run; flag it, let the copies land, and mark the tile
        if (threadIdx.x == 0) atomicAdd(err, 1u);
        mbar_wait_bounded(&bar, 0, kTmaTries);
        if (valid) {
            const T nanv = T(NAN);
            if (f_e != nullptr)
                for (int i = 0; i < 3; ++i) f_e[(3 * I + i) * n_el + e] = nanv;
            if (K_e != nullptr && want_K)
                for (int c = 0; c < 72; ++c) K_e[((3 * I + c / 24) * 24 + c % 24) * n_el + e] = nanv;
        }
        return;
    }
    T f[3] = {T(0), T(0), T(0)};
    T Kr[3][8][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int K = 0; K < 8; ++K)
#pragma unroll
            for (int k = 0; k < 3; ++k) Kr[i][K][k] = T(0);
    for (int q = 0; q < 8; ++q) {
        const int col = le * 8 + q;
        const T w = s_w[le][q];
        T wg[3];
#pragma unroll
        for (int J = 0; J < 3; ++J) wg[J] = w * s_g[le][q][I][J];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            f[i] += s_p[(3 * i) * kTmaQP + col] * wg[0];
            f[i] += s_p[(3 * i + 1) * kTmaQP + col] * wg[1];
            f[i] += s_p[(3 * i + 2) * kTmaQP + col] * wg[2];
        }
        if (want_K) {
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                T T3[3][3];
#pragma unroll
                for (int k = 0; k < 3; ++k)
#pragma unroll
                    for (int L = 0; L < 3; ++L)
                        T3[k][L] = wg[0] * s_a[((3 * i) * 9 + 3 * k + L) * kTmaQP + col] +
                                   wg[1] * s_a[((3 * i + 1) * 9 + 3 * k + L) * kTmaQP + col] +
                                   wg[2] * s_a[((3 * i + 2) * 9 + 3 * k + L) * kTmaQP + col];
#pragma unroll
                for (int K = 0; K < 8; ++K) {
                    const T g0 = s_g[le][q][K][0], g1 = s_g[le][q][K][1], g2 = s_g[le][q][K][2];
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        // one fused multiply-add per product, accumulated in place
                        Kr[i][K][k] += T3[k][0] * g0;
                        Kr[i][K][k] += T3[k][1] * g1;
                        Kr[i][K][k] += T3[k][2] * g2;
                    }
                }
            }
        }
    }
    if (!valid) return;
    if (f_e != nullptr) {
#pragma unroll
        for (int i = 0; i < 3; ++i) f_e[(3 * I + i) * n_el + e] = f[i];
    }
    if (K_e != nullptr && want_K) {
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int K = 0; K < 8; ++K)
#pragma unroll
                for (int k = 0; k < 3; ++k) K_e[((3 * I + i) * 24 + 3 * K + k) * n_el + e] = Kr[i][K][k];
    }
}

bool encode_tensor_map_2d(CUtensorMap *map, const void *base, int elem_bytes, uint64_t rows, uint64_t cols,
                          uint32_t box_rows, uint32_t box_cols) {
    using encode_fn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static encode_fn fn = nullptr;
    if (fn == nullptr) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || p == nullptr)
            return false;
        fn = reinterpret_cast<encode_fn>(p);
    }
    if ((reinterpret_cast<uintptr_t>(base) & 15u) != 0 || (cols * elem_bytes) % 16 != 0 ||
        (box_cols * (uint32_t)elem_bytes) % 16 != 0)
        return false;
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {cols * (uint64_t)elem_bytes};
    const cuuint32_t box[2] = {box_cols, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, elem_bytes == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
              const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Launches the TMA-fed kernel; COMMET_ERR_UNSUPPORTED when a tensor map cannot be encoded
// (the caller then uses the per-lane kernel).
template <typename T>
static int launch_elem_tma(const commet_mesh *mesh, const void *P, const void *A, void *f_e, void *K_e,
                           cudaStream_t s) {
    const int64_t n_el = mesh->n_el, n_qp = 8 * n_el;
    if (n_qp > 0x7fffffffLL) return COMMET_ERR_UNSUPPORTED;
    CUtensorMap tmP{}, tmA{};
    const bool want_K = (A != nullptr);
    if (!encode_tensor_map_2d(&tmP, P, (int)sizeof(T), 9, (uint64_t)n_qp, 9, kTmaQP)) return COMMET_ERR_UNSUPPORTED;
    if (want_K && !encode_tensor_map_2d(&tmA, A, (int)sizeof(T), 81, (uint64_t)n_qp, 81, kTmaQP))
        return COMMET_ERR_UNSUPPORTED;
    const size_t dyn = (size_t)(9 + 81) * kTmaQP * sizeof(T);
    if (cudaFuncSetAttribute(elem_tma_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) != cudaSuccess)
        return COMMET_ERR_CUDA;
    const int64_t blocks = (n_el + kElPerCta - 1) / kElPerCta;
    elem_tma_kernel<T><<<(unsigned)blocks, 128, dyn, s>>>(n_el, tmP, tmA, want_K ? 1 : 0, mesh->d_conn, mesh->d_X,
                                                          (T *)f_e, (T *)K_e, mesh->d_err);
    return cudaGetLastError() == cudaSuccess ? COMMET_OK : COMMET_ERR_CUDA;
}

template <typename T, bool SYM>
static int elem_typed(const commet_mesh *mesh, const void *P, const void *A, void *f_e, void *K_e, void *r,
                      void *K_vals, cudaStream_t s) {
    const int64_t n_el = mesh->n_el;
    if (n_el == 0) return COMMET_OK;
    const bool scatter = (r != nullptr) || (K_vals != nullptr);
    if (!scatter) {
        if constexpr (sizeof(T) == 4) {
            // HBM-bound: the full contraction costs no more than the symmetric one
            const int rc = launch_elem_tma<T>(mesh, P, A, f_e, K_e, s);
            if (rc != COMMET_ERR_UNSUPPORTED) return rc;
        }
        const int64_t blocks = (n_el + kElPerCta - 1) / kElPerCta;
        elem_assemble_kernel<T, false, SYM><<<(unsigned)blocks, 128, 0, s>>>(
            n_el, nullptr, n_el, mesh->d_conn, mesh->d_X, (const T *)P, (const T *)A, (T *)f_e, (T *)K_e, nullptr,
            nullptr, nullptr, nullptr);
        return cudaGetLastError() == cudaSuccess ? COMMET_OK : COMMET_ERR_CUDA;
    }
    if (r != nullptr) COMMET_CUDA_TRY(cudaMemsetAsync(r, 0, sizeof(T) * 3 * mesh->n_nodes, s));
    if (K_vals != nullptr) COMMET_CUDA_TRY(cudaMemsetAsync(K_vals, 0, sizeof(T) * mesh->nnz, s));
    for (int c = 0; c < mesh->n_colours; ++c) {
        const int64_t off = mesh->colour_off[c], cnt = mesh->colour_off[c + 1] - off;
        if (cnt == 0) continue;
        const int64_t blocks = (cnt + kElPerCta - 1) / kElPerCta;
        elem_assemble_kernel<T, true, SYM><<<(unsigned)blocks, 128, 0, s>>>(
            n_el, mesh->d_colour_el + off, cnt, mesh->d_conn, mesh->d_X, (const T *)P, (const T *)A, (T *)f_e,
            (T *)K_e, (T *)r, (T *)K_vals, mesh->d_emap, mesh->d_rowlen);
        if (cudaGetLastError() != cudaSuccess) return COMMET_ERR_CUDA;
    }
    return COMMET_OK;
}

// ------------------------------------------------------------------ adjoints
// For a loss of the global residual (eq. loss): G = dL/dP from lam = dL/dr, the transpose of
// eq. r-quad and of the scatter (a gather of lam at the element's nodes): one thread per
// (element, Gauss point), as compute_F.
template <typename T>
__global__ void residual_adjoint_kernel(int64_t n_el, const int32_t *__restrict__ conn, const double *__restrict__ X,
                                        const T *__restrict__ lam, T *__restrict__ G) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= 8 * n_el) return;
    const int64_t e = gid >> 3;
    const int q = (int)(gid & 7);
    T Xe[8][3], le[8][3];
#pragma unroll
    for (int I = 0; I < 8; ++I) {
        const int64_t n = conn[8 * e + I];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            Xe[I][a] = (T)X[3 * n + a];
            le[I][a] = lam[3 * n + a];
        }
    }
    T gX[8][3], w;
    physical_grads<T>(Xe, q, gX, w);
    const int64_t n_qp = 8 * n_el;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int J = 0; J < 3; ++J) {
            T s = T(0);
#pragma unroll
            for (int I = 0; I < 8; ++I) s += le[I][i] * gX[I][J];
            G[(3 * i + J) * n_qp + gid] = w * s;
        }
}

// du = dL/du from dF = dL/dF, the transpose of the trial F: element e adds
// sum_q dF_q,iJ dphi_I/dX_J to node I. 8 lanes per element (lane I: node I), 16 elements
// per CTA, one launch per element colour so that no two lanes add to one node.
template <typename T>
__global__ void __launch_bounds__(128)
    compute_F_adjoint_kernel(int64_t n_el, int64_t n_nodes, const int32_t *__restrict__ el_list, int64_t n_list,
                             const int32_t *__restrict__ conn, const double *__restrict__ X,
                             const T *__restrict__ dF, T *__restrict__ du) {
    __shared__ T s_g[kElPerCta][8][8][3];
    const int le = threadIdx.x >> 3, I = threadIdx.x & 7;
    const int64_t li = (int64_t)blockIdx.x * kElPerCta + le;
    const bool valid = li < n_list;
    const int64_t e = valid ? (int64_t)el_list[li] : 0;
    {
        T Xe[8][3];
#pragma unroll
        for (int K = 0; K < 8; ++K) {
            const int64_t n = conn[8 * e + K];
#pragma unroll
            for (int a = 0; a < 3; ++a) Xe[K][a] = (T)X[3 * n + a];
        }
        T gX[8][3], w;
        physical_grads<T>(Xe, I, gX, w);
#pragma unroll
        for (int K = 0; K < 8; ++K)
#pragma unroll
            for (int a = 0; a < 3; ++a) s_g[le][I][K][a] = gX[K][a];
    }
    __syncthreads();
    if (!valid) return;
    const int64_t n_qp = 8 * n_el;
    T acc[3] = {T(0), T(0), T(0)};
    for (int q = 0; q < 8; ++q) {
        const int64_t qq = 8 * e + q;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int J = 0; J < 3; ++J) acc[i] += dF[(3 * i + J) * n_qp + qq] * s_g[le][q][I][J];
    }
    const int64_t gI = conn[8 * e + I];
#pragma unroll
    for (int i = 0; i < 3; ++i) du[i * n_nodes + gI] += acc[i];
}

template <typename T>
static int adjoints_typed(const commet_mesh *mesh, const void *lam, void *G, const void *dF, void *du, cudaStream_t s) {
    const int64_t n_el = mesh->n_el;
    if (lam != nullptr && n_el > 0) {
        const int tpb = 256;
        residual_adjoint_kernel<T><<<(unsigned)((8 * n_el + tpb - 1) / tpb), tpb, 0, s>>>(
            n_el, mesh->d_conn, mesh->d_X, (const T *)lam, (T *)G);
        COMMET_CUDA_TRY(cudaGetLastError());
    }
    if (dF != nullptr) {
        COMMET_CUDA_TRY(cudaMemsetAsync(du, 0, sizeof(T) * 3 * mesh->n_nodes, s));
        for (int c = 0; c < mesh->n_colours; ++c) {
            const int64_t off = mesh->colour_off[c], cnt = mesh->colour_off[c + 1] - off;
            if (cnt == 0) continue;
            compute_F_adjoint_kernel<T><<<(unsigned)((cnt + kElPerCta - 1) / kElPerCta), 128, 0, s>>>(
                n_el, mesh->n_nodes, mesh->d_colour_el + off, cnt, mesh->d_conn, mesh->d_X, (const T *)dF, (T *)du);
            COMMET_CUDA_TRY(cudaGetLastError());
        }
    }
    return COMMET_OK;
}

int launch_assembly_adjoints(const commet_mesh *mesh, int precision, const void *lam, void *G, const void *dF,
                             void *du, cudaStream_t s) {
    if (precision == COMMET_F64) return adjoints_typed<double>(mesh, lam, G, dF, du, s);
    return adjoints_typed<float>(mesh, lam, G, dF, du, s);
}

int launch_elem_assemble(const commet_mesh *mesh, int precision, const void *P, const void *A, void *f_e,
                         void *K_e, void *r, void *K_vals, cudaStream_t s, bool symmetric) {
    if (symmetric) {
        if (precision == COMMET_F64) return elem_typed<double, true>(mesh, P, A, f_e, K_e, r, K_vals, s);
        return elem_typed<float, true>(mesh, P, A, f_e, K_e, r, K_vals, s);
    }
    if (precision == COMMET_F64) return elem_typed<double, false>(mesh, P, A, f_e, K_e, r, K_vals, s);
    return elem_typed<float, false>(mesh, P, A, f_e, K_e, r, K_vals, s);
}

}  // namespace commet
