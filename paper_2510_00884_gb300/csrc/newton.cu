// Fused Newton-iteration assembly: for every element of one colour,
//   gather X, u -> F at the 8 Gauss points (Algorithm 1) -> constitutive update
//   (qp_group_update) -> f_int, K_e (eq. r-quad, k-quad in material form)
//   -> += into r and the CSR values,
// with P and A kept in shared memory (they never reach HBM). One warp owns one
// element at a time: its 8 lane groups are the element's 8 Gauss points during the
// constitutive update, then lane (I, jb) forms dof rows 3I..3I+2 against the columns
// of nodes 2jb, 2jb+1. No two elements of a colour share a node, so the scatter is a
// plain read-modify-write; colours are launched one after another on the stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>

#include "qp_body.cuh"

namespace commet {

namespace {

// per-warp element area (elements of T)
constexpr int kEX = 0;              // X [8][3]
constexpr int kEU = 24;             // u [8][3]
constexpr int kEG = 48;             // grad_X phi [8 qp][8 nodes][3]
constexpr int kEW = 48 + 192;       // w [8]
constexpr int kEPA = 48 + 192 + 8;  // P (9) then A (81) per qp: [8][90]
constexpr int kEArea = kEPA + 8 * 90;

template <typename T>
__device__ __forceinline__ void gauss_grads(const T *Xe, int q, T *gX, T &w) {
    const T gp = T(0.57735026918962576451);
    T g[8][3];
#pragma unroll
    for (int I = 0; I < 8; ++I) {
        T xi[3], zq[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            xi[a] = ((I >> a) & 1) ? T(1) : T(-1);
            zq[a] = ((q >> a) & 1) ? gp : -gp;
        }
        const T f0 = T(1) + xi[0] * zq[0], f1 = T(1) + xi[1] * zq[1], f2 = T(1) + xi[2] * zq[2];
        g[I][0] = T(0.125) * xi[0] * f1 * f2;
        g[I][1] = T(0.125) * xi[1] * f0 * f2;
        g[I][2] = T(0.125) * xi[2] * f0 * f1;
    }
    T Je[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            T s = T(0);
#pragma unroll
            for (int I = 0; I < 8; ++I) s += Xe[3 * I + a] * g[I][b];
            Je[3 * a + b] = s;
        }
    T cof[9], det;
    cof_det(Je, cof, det);
    const T id = T(1) / det;
#pragma unroll
    for (int I = 0; I < 8; ++I)
#pragma unroll
        for (int a = 0; a < 3; ++a)
            gX[3 * I + a] = (cof[3 * a] * g[I][0] + cof[3 * a + 1] * g[I][1] + cof[3 * a + 2] * g[I][2]) * id;
    w = det;
}

}  // namespace

template <typename T, int NF, int W>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 256 : 384)
    newton_kernel(const T *__restrict__ gw, NetLayout lay, KinConst<T> kc, const int32_t *__restrict__ el_list,
                  int64_t n_list, const int32_t *__restrict__ conn, const double *__restrict__ X,
                  const T *__restrict__ u, int64_t n_nodes, T *__restrict__ r, T *__restrict__ K_vals,
                  const uint32_t *__restrict__ emap, const int32_t *__restrict__ rowlen,
                  int32_t *__restrict__ status, int qstride) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sw = reinterpret_cast<T *>(smem_raw);
    // every packed block but the layer-2 tangent weights M goes to shared memory (this
    // kernel folds s_1 into A_2 instead); A_k row-major, the last block, moves down by M
    const int msz = lay.M ? lay.Ar - lay.M : 0;
    const int wbytes = ((lay.total - msz) * (int)sizeof(T) + 15) / 16 * 16;
    {
        const int n16 = wbytes / 16;
        const int cut16 = msz ? lay.M * (int)sizeof(T) / 16 : n16;
        const int skip16 = msz * (int)sizeof(T) / 16;
        const int4 *src = reinterpret_cast<const int4 *>(gw);
        int4 *dst = reinterpret_cast<int4 *>(sw);
        for (int i = threadIdx.x; i < n16; i += blockDim.x) dst[i] = src[i < cut16 ? i : i + skip16];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int qi = lane >> 2, jb = lane & 3;
    const int per_warp = kQPW * qstride + (kEArea + 3) / 4 * 4;
    T *wbase = sw + wbytes / (int)sizeof(T) + (size_t)warp * per_warp;
    T *qs = wbase + qi * qstride;
    T *ea = wbase + kQPW * qstride;
    const int64_t n_gwarps = (int64_t)gridDim.x * (blockDim.x >> 5);

    for (int64_t li = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; li < n_list; li += n_gwarps) {
        const int64_t e = el_list[li];
        if (lane < 24) {
            const int I = lane / 3, a = lane % 3;
            const int64_t n = conn[8 * e + I];
            ea[kEX + lane] = (T)X[3 * n + a];
            ea[kEU + lane] = u[a * n_nodes + n];
        }
        __syncwarp();
        // Gauss point qi: gradients, weight, F
        T gX[24], w;
        gauss_grads<T>(ea + kEX, qi, gX, w);
        if (jb == 0) {
#pragma unroll
            for (int c = 0; c < 24; ++c) ea[kEG + 24 * qi + c] = gX[c];
            ea[kEW + qi] = w;
        }
        T F[9];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int J = 0; J < 3; ++J) {
                T s = (i == J) ? T(1) : T(0);
#pragma unroll
                for (int I = 0; I < 8; ++I) s += ea[kEU + 3 * I + i] * gX[3 * I + J];
                F[3 * i + J] = s;
            }
        T psi_val;
        bool report;
        T *pa = ea + kEPA + 90 * qi;
        qp_group_update<T, NF, W>(sw, lay, nullptr, sw + lay.At, sw + lay.Ar - msz, kc, qs, qi, jb, F, true, pa, 1, pa + 9, 1, nullptr, 0, psi_val,
                                  report);
        if (report && jb == 0 && status != nullptr) {
            const int64_t q = 8 * e + qi;
            atomicAdd(&status[0], 1);
            atomicMin(&status[1], (int32_t)(q < INT32_MAX ? q : INT32_MAX));
        }
        __syncwarp();
        // element integrals: lane (I = qi, jb) -> rows 3I..3I+2, column nodes 2jb, 2jb+1
        const int I = qi;
        T f[3] = {T(0), T(0), T(0)};
        T Kr[3][2][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int kk = 0; kk < 2; ++kk)
#pragma unroll
                for (int k = 0; k < 3; ++k) Kr[i][kk][k] = T(0);
#pragma unroll 1
        for (int q = 0; q < 8; ++q) {
            const T wq = ea[kEW + q];
            const T *gq = ea + kEG + 24 * q;
            const T wg0 = wq * gq[3 * I], wg1 = wq * gq[3 * I + 1], wg2 = wq * gq[3 * I + 2];
            const T *Pq = ea + kEPA + 90 * q;
            const T *Aq = Pq + 9;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                f[i] += Pq[3 * i] * wg0;
                f[i] += Pq[3 * i + 1] * wg1;
                f[i] += Pq[3 * i + 2] * wg2;
                T T3[3][3];
#pragma unroll
                for (int k = 0; k < 3; ++k)
#pragma unroll
                    for (int L = 0; L < 3; ++L)
                        T3[k][L] = wg0 * Aq[(3 * i) * 9 + 3 * k + L] + wg1 * Aq[(3 * i + 1) * 9 + 3 * k + L] +
                                   wg2 * Aq[(3 * i + 2) * 9 + 3 * k + L];
#pragma unroll
                for (int kk = 0; kk < 2; ++kk) {
                    const int K = 2 * jb + kk;
                    const T g0 = gq[3 * K], g1 = gq[3 * K + 1], g2 = gq[3 * K + 2];
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        Kr[i][kk][k] += T3[k][0] * g0;
                        Kr[i][kk][k] += T3[k][1] * g1;
                        Kr[i][kk][k] += T3[k][2] * g2;
                    }
                }
            }
        }
        const int64_t gI = conn[8 * e + I];
        if (jb == 0) {
#pragma unroll
            for (int i = 0; i < 3; ++i) r[3 * gI + i] += f[i];
        }
        const int64_t rl = rowlen[gI];
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
            const int K = 2 * jb + kk;
            const int64_t base = emap[(8 * e + I) * 8 + K];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int k = 0; k < 3; ++k) K_vals[base + i * rl + k] += Kr[i][kk][k];
        }
        __syncwarp();
    }
}

template <typename T, int NF, int W>
static int newton_typed(const commet_model *m, const commet_mesh *mesh, const void *u, void *r, void *K_vals,
                        int32_t *status, cudaStream_t s) {
    using Cf = CUConf<T, NF, W>;
    KinConst<T> kc{};
    kc.kin = m->kp.kin;
    kc.stress_free = m->kp.stress_free;
    kc.kappa = (T)m->kp.kappa;
    for (int f = 0; f < 2; ++f)
        for (int c = 0; c < 3; ++c) kc.fib[f][c] = (T)m->kp.fib[f][c];
    const int qstride = qp_slab_elems<T>(Cf::D, W, m->L, NF);
    const int msz = m->lay.M ? m->lay.Ar - m->lay.M : 0;  // M stays in global memory (unused here)
    const size_t wbytes = ((size_t)(m->lay.total - msz) * sizeof(T) + 15) / 16 * 16;
    const size_t per_warp = ((size_t)kQPW * qstride + (kEArea + 3) / 4 * 4) * sizeof(T);
    int dev = 0, smem_max = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if ((size_t)smem_max < wbytes + per_warp) return COMMET_ERR_UNSUPPORTED;
    const int max_threads = sizeof(T) == 8 ? 256 : 384;
    const int warps = (int)std::min<size_t>((size_t)max_threads / 32, (smem_max - wbytes) / per_warp);
    const size_t smem = wbytes + warps * per_warp;
    auto kern = newton_kernel<T, NF, W>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return COMMET_ERR_CUDA;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem);
    if (per_sm < 1) per_sm = 1;
    COMMET_CUDA_TRY(cudaMemsetAsync(r, 0, sizeof(T) * 3 * mesh->n_nodes, s));
    COMMET_CUDA_TRY(cudaMemsetAsync(K_vals, 0, sizeof(T) * mesh->nnz, s));
    for (int c = 0; c < mesh->n_colours; ++c) {
        const int64_t off = mesh->colour_off[c], cnt = mesh->colour_off[c + 1] - off;
        if (cnt == 0) continue;
        const int64_t want = (cnt + warps - 1) / warps;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sm_count() * per_sm));
        kern<<<grid, warps * 32, smem, s>>>((const T *)m->d_weights, m->lay, kc, mesh->d_colour_el + off, cnt,
                                            mesh->d_conn, mesh->d_X, (const T *)u, mesh->n_nodes, (T *)r,
                                            (T *)K_vals, mesh->d_emap, mesh->d_rowlen, status, qstride);
        if (cudaGetLastError() != cudaSuccess) return COMMET_ERR_CUDA;
    }
    return COMMET_OK;
}

template <typename T>
static int newton_dispatch(const commet_model *m, const commet_mesh *mesh, const void *u, void *r, void *K_vals,
                           int32_t *status, cudaStream_t s) {
    const int nf = m->kp.nf, W = m->W;
#define COMMET_CASE(NF_, W_) \
    if (nf == NF_ && W == W_) return newton_typed<T, NF_, W_>(m, mesh, u, r, K_vals, status, s);
    COMMET_CASE(0, 16)
    COMMET_CASE(0, 32)
    COMMET_CASE(2, 32)
#undef COMMET_CASE
    return COMMET_ERR_UNSUPPORTED;
}

int launch_newton_assemble(const commet_model *m, const commet_mesh *mesh, const void *u, void *r, void *K_vals,
                           int32_t *status, cudaStream_t s) {
    if (m->inner != COMMET_INNER_MICNN) return COMMET_ERR_UNSUPPORTED;
    if (mesh->n_el == 0) {
        const size_t es = m->precision == COMMET_F64 ? 8 : 4;
        if (mesh->n_nodes > 0) COMMET_CUDA_TRY(cudaMemsetAsync(r, 0, es * 3 * mesh->n_nodes, s));
        if (mesh->nnz > 0) COMMET_CUDA_TRY(cudaMemsetAsync(K_vals, 0, es * mesh->nnz, s));
        return COMMET_OK;
    }
    if (m->precision == COMMET_F64) return newton_dispatch<double>(m, mesh, u, r, K_vals, status, s);
    if (m->precision == COMMET_F32) return newton_dispatch<float>(m, mesh, u, r, K_vals, status, s);
    return COMMET_ERR_UNSUPPORTED;
}

}  // namespace commet
