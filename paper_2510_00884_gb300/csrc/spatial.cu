// Spatial (Voigt) form of the constitutive outputs and of the element integrals.
//
// App. A.1: the Kirchhoff stress tau_ij = P_iJ F_jJ and the spatial stiffness
// c_ijkl = F_jJ A_iJkL F_lL - delta_ik tau_jl are symmetric (c in both index pairs and
// between them), so a point needs 6 + 21 values instead of the 9 + 81 of P and A.
// The update kernel forms P and A on chip as in the material form and pushes them
// forward before anything leaves the SM; the element kernel evaluates eq. r-quad and
// k-quad directly in the spatial form with grad phi = Grad phi F^{-1}, reading F, tau, c
// (36 values per point instead of 90).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "hex8.cuh"
#include "update_kernel.cuh"

namespace commet {

int launch_const_update_spatial(const commet_model *m, int64_t n_qp, const void *F, void *psi, void *tau, void *c,
                                int32_t *status, cudaStream_t s) {
    if (status != nullptr) {
        int rc = launch_status_init(status, s);
        if (rc != COMMET_OK) return rc;
    }
    if (n_qp == 0) return COMMET_OK;
    if (m->precision == COMMET_F64) return dispatch<double, true>(m, n_qp, F, psi, tau, c, status, s, nullptr);
    if (m->precision == COMMET_F32) return dispatch<float, true>(m, n_qp, F, psi, tau, c, status, s, nullptr);
    if (m->precision == COMMET_BF16_MLP) return launch_const_update_bf16(m, n_qp, F, psi, tau, c, status, s, true);
    return COMMET_ERR_UNSUPPORTED;
}

// ------------------------------------------------------------ element integrals
// 8 lanes per element (lane I = node I, dof rows 3I..3I+2), 16 elements per CTA, as the
// material-form kernel. Per Gauss point the element's F, tau, c (36 values) are staged
// in shared memory; every lane forms F^{-1} and the spatial gradient of its own node,
// which the element's lanes share through shared memory.
constexpr int kSpElPerCta = 16;

template <typename T, bool SCATTER>
__global__ void __launch_bounds__(128)
    elem_spatial_kernel(int64_t n_el, const int32_t *__restrict__ el_list, int64_t n_list,
                        const int32_t *__restrict__ conn, const double *__restrict__ X, const T *__restrict__ Fg,
                        const T *__restrict__ tau, const T *__restrict__ cg, T *__restrict__ f_e, T *__restrict__ K_e,
                        T *__restrict__ r, T *__restrict__ K_vals, const uint32_t *__restrict__ emap,
                        const int32_t *__restrict__ rowlen) {
    __shared__ T s_gX[kSpElPerCta][8][8][3];  // [el][qp][node][dir] material gradients
    __shared__ T s_w[kSpElPerCta][8];
    __shared__ T s_v[kSpElPerCta][36];        // F (9), tau (6), c (21) of the current qp
    __shared__ T s_gx[kSpElPerCta][8][3];     // spatial gradients of the current qp
    const int le = threadIdx.x >> 3, I = threadIdx.x & 7;
    const int64_t li = (int64_t)blockIdx.x * kSpElPerCta + le;
    const bool valid = li < n_list;
    const int64_t e = valid ? (el_list ? (int64_t)el_list[li] : li) : 0;
    const int64_t n_qp = 8 * n_el;
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
            for (int a = 0; a < 3; ++a) s_gX[le][I][K][a] = gX[K][a];
        s_w[le][I] = w;
    }
    T f[3] = {T(0), T(0), T(0)};
    T Kr[3][8][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int K = 0; K < 8; ++K)
#pragma unroll
            for (int k = 0; k < 3; ++k) Kr[i][K][k] = T(0);
    const bool want_K = (cg != nullptr);
    for (int q = 0; q < 8; ++q) {
        __syncthreads();
        const int64_t qq = 8 * e + q;
        for (int c = I; c < 36; c += 8) {
            T v = T(0);
            if (c < 9)
                v = Fg[c * n_qp + qq];
            else if (c < 15)
                v = tau[(c - 9) * n_qp + qq];
            else if (want_K)
                v = cg[(c - 15) * n_qp + qq];
            s_v[le][c] = v;
        }
        __syncthreads();
        const T *Fq = &s_v[le][0];
        const T *tq = &s_v[le][9];
        const T *cq = &s_v[le][15];
        {
            // F^{-1}_Mm = cof(F)_mM / det F; grad phi_I,m = dphi_I/dX_M F^{-1}_Mm
            T cof[9];
            cof[0] = Fq[4] * Fq[8] - Fq[5] * Fq[7];
            cof[1] = Fq[5] * Fq[6] - Fq[3] * Fq[8];
            cof[2] = Fq[3] * Fq[7] - Fq[4] * Fq[6];
            cof[3] = Fq[2] * Fq[7] - Fq[1] * Fq[8];
            cof[4] = Fq[0] * Fq[8] - Fq[2] * Fq[6];
            cof[5] = Fq[1] * Fq[6] - Fq[0] * Fq[7];
            cof[6] = Fq[1] * Fq[5] - Fq[2] * Fq[4];
            cof[7] = Fq[2] * Fq[3] - Fq[0] * Fq[5];
            cof[8] = Fq[0] * Fq[4] - Fq[1] * Fq[3];
            const T id = T(1) / (Fq[0] * cof[0] + Fq[1] * cof[1] + Fq[2] * cof[2]);
            const T *gI = s_gX[le][q][I];
#pragma unroll
            for (int m = 0; m < 3; ++m)
                s_gx[le][I][m] = (gI[0] * cof[3 * m] + gI[1] * cof[3 * m + 1] + gI[2] * cof[3 * m + 2]) * id;
        }
        __syncthreads();
        const T w = s_w[le][q];
        T wg[3];
#pragma unroll
        for (int m = 0; m < 3; ++m) wg[m] = w * s_gx[le][I][m];
        // eq. r-quad: f_I,i += w tau_ij grad phi_I,j
#pragma unroll
        for (int i = 0; i < 3; ++i)
        {
            f[i] += tq[voigt_of(i, 0)] * wg[0];
            f[i] += tq[voigt_of(i, 1)] * wg[1];
            f[i] += tq[voigt_of(i, 2)] * wg[2];
        }
        if (want_K) {
            // eq. k-quad: K_(I,i)(K,k) += w grad phi_I,m (delta_ik tau_ml + c_imkl) grad phi_K,l
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                T T3[3][3];  // [k][l]
#pragma unroll
                for (int k = 0; k < 3; ++k)
#pragma unroll
                    for (int l = 0; l < 3; ++l) {
                        T s = T(0);
#pragma unroll
                        for (int m = 0; m < 3; ++m) {
                            T v = cq[voigt_upper_pos(voigt_of(i, m), voigt_of(k, l))];
                            if (i == k) v += tq[voigt_of(m, l)];
                            s += wg[m] * v;
                        }
                        T3[k][l] = s;
                    }
#pragma unroll
                for (int K = 0; K < 8; ++K) {
                    const T g0 = s_gx[le][K][0], g1 = s_gx[le][K][1], g2 = s_gx[le][K][2];
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
    if (SCATTER) {
        const int64_t gI = conn[8 * e + I];
        if (r != nullptr) {
#pragma unroll
            for (int i = 0; i < 3; ++i) r[3 * gI + i] += f[i];
        }
        if (K_vals != nullptr && want_K) {
            const int64_t rl = rowlen[gI];
#pragma unroll
            for (int K = 0; K < 8; ++K) {
                const int64_t base = emap[(8 * e + I) * 8 + K];
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int k = 0; k < 3; ++k) K_vals[base + i * rl + k] += Kr[i][K][k];
            }
        }
    }
}

template <typename T>
static int elem_spatial_typed(const commet_mesh *mesh, const void *F, const void *tau, const void *c, void *f_e,
                              void *K_e, void *r, void *K_vals, cudaStream_t s) {
    const int64_t n_el = mesh->n_el;
    if (n_el == 0) return COMMET_OK;
    const bool scatter = (r != nullptr) || (K_vals != nullptr);
    if (!scatter) {
        const int64_t blocks = (n_el + kSpElPerCta - 1) / kSpElPerCta;
        elem_spatial_kernel<T, false><<<(unsigned)blocks, 128, 0, s>>>(
            n_el, nullptr, n_el, mesh->d_conn, mesh->d_X, (const T *)F, (const T *)tau, (const T *)c, (T *)f_e,
            (T *)K_e, nullptr, nullptr, nullptr, nullptr);
        return cudaGetLastError() == cudaSuccess ? COMMET_OK : COMMET_ERR_CUDA;
    }
    if (r != nullptr) COMMET_CUDA_TRY(cudaMemsetAsync(r, 0, sizeof(T) * 3 * mesh->n_nodes, s));
    if (K_vals != nullptr) COMMET_CUDA_TRY(cudaMemsetAsync(K_vals, 0, sizeof(T) * mesh->nnz, s));
    for (int col = 0; col < mesh->n_colours; ++col) {
        const int64_t off = mesh->colour_off[col], cnt = mesh->colour_off[col + 1] - off;
        if (cnt == 0) continue;
        const int64_t blocks = (cnt + kSpElPerCta - 1) / kSpElPerCta;
        elem_spatial_kernel<T, true><<<(unsigned)blocks, 128, 0, s>>>(
            n_el, mesh->d_colour_el + off, cnt, mesh->d_conn, mesh->d_X, (const T *)F, (const T *)tau,
            (const T *)c, (T *)f_e, (T *)K_e, (T *)r, (T *)K_vals, mesh->d_emap, mesh->d_rowlen);
        if (cudaGetLastError() != cudaSuccess) return COMMET_ERR_CUDA;
    }
    return COMMET_OK;
}

int launch_elem_assemble_spatial(const commet_mesh *mesh, int precision, const void *F, const void *tau,
                                 const void *c, void *f_e, void *K_e, void *r, void *K_vals, cudaStream_t s) {
    if (precision == COMMET_F64) return elem_spatial_typed<double>(mesh, F, tau, c, f_e, K_e, r, K_vals, s);
    return elem_spatial_typed<float>(mesh, F, tau, c, f_e, K_e, r, K_vals, s);
}

}  // namespace commet
