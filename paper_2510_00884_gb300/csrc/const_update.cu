// Fused constitutive update (Algorithm 2's constitutive call in material form):
// F -> kinematic scalars K -> MICNN value, gradient and Hessian -> P, A, Psi.
//
// Work mapping. A group of 4 consecutive lanes owns one quadrature point; lane jb of
// the group owns neurons [jb*W/4, (jb+1)*W/4) of every hidden layer. A warp handles 8
// points at a time; CTAs are persistent and hold the whole network in shared memory.
// Per-point activations live in a padded shared-memory slab of the group (the pad
// puts the 8 points of a warp in different banks).
//
// Network derivatives. Algorithm 4 propagates 1 + d + d(d+1)/2 channels through each
// layer. This kernel computes the same exact Hessian with fewer operations:
//   forward values     y_k, z_k = F(y_k), s_k = F'(y_k), t_k = F''(y_k)
//   reverse adjoints   zbar_L = a, ybar_k = s_k zbar_k, zbar_{k-1} = A_k^T ybar_k,
//                      dN/dK = b + sum_k B_k^T ybar_k  (B_1 := W1)
//   forward tangents   J_1 = W1, J_k = A_k diag(s_{k-1}) J_{k-1} + B_k
//   Hessian            d2N/dK2 = sum_k J_k^T diag(t_k zbar_k) J_k
// (the second-order adjoint identity; the J_k of a layer is consumed as soon as it is
// formed, so only one W x d tangent block per point is stored).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>

#include "device_math.cuh"
#include "internal.h"

namespace commet {

constexpr int kG = 4;    // lanes per quadrature point
constexpr int kQPW = 8;  // quadrature points per warp

template <typename T, int NF, int W>
struct CUConf {
    static constexpr int D = 3 + 2 * NF;
    static constexpr int DP = (D + 3) / 4 * 4;
    static constexpr int NH = D * (D + 1) / 2;
    static constexpr int NJ = W / kG;
    static constexpr int NC0 = sizeof(T) == 8 ? 4 : 8;
    static constexpr int NC = NC0 < NJ ? NC0 : NJ;
};

// Per-qp slab size in elements of T for the given network (host and device agree).
template <typename T>
__host__ __device__ inline int qp_slab_elems(int D, int W, int L, int NF) {
    const int DP = (D + 3) / 4 * 4;
    const int nbuf = L >= 4 ? 2 : (L == 3 ? 1 : 0);
    int work = 2 * W;
    if (nbuf * W * DP > work) work = nbuf * W * DP;
    int raw = 2 * L * W + work;
    const int stage = 9 * D + 54 + 18 * NF + 5 + NF;
    if (stage > raw) raw = stage;
    int words = raw * (int)sizeof(T) / 4;
    words = (words + 31) / 32 * 32 + 4;
    return words * 4 / (int)sizeof(T);
}

template <typename T>
__device__ __forceinline__ T shfl_xor(T v, int m) {
    return __shfl_xor_sync(0xffffffffu, v, m);
}

template <typename T, int NF, int W>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 256 : 512)
    const_update_kernel(const T *__restrict__ gw, NetLayout lay, KinConst<T> kc, int64_t n_qp,
                        const T *__restrict__ Fg, T *__restrict__ psi, T *__restrict__ P, T *__restrict__ A,
                        int32_t *__restrict__ status, T *__restrict__ dN_out, int qstride) {
    using Cf = CUConf<T, NF, W>;
    constexpr int D = Cf::D, DP = Cf::DP, NH = Cf::NH, NJ = Cf::NJ, NC = Cf::NC;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sw = reinterpret_cast<T *>(smem_raw);
    const int wbytes = (lay.total * (int)sizeof(T) + 15) / 16 * 16;
    {
        const int n16 = wbytes / 16;
        const int4 *src = reinterpret_cast<const int4 *>(gw);
        int4 *dst = reinterpret_cast<int4 *>(sw);
        for (int i = threadIdx.x; i < n16; i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int qi = lane >> 2, jb = lane & 3;
    const int L = lay.L;
    T *qs = sw + wbytes / (int)sizeof(T) + (size_t)(warp * kQPW + qi) * qstride;
    T *sd = qs;              // s_k at (k-1) W, t_k / D_k at (L+k-1) W
    T *wk = qs + 2 * L * W;  // work area
    const int j0 = jb * NJ;
    const int64_t n_tiles = (n_qp + kQPW - 1) / kQPW;
    const int64_t n_gwarps = (int64_t)gridDim.x * (blockDim.x >> 5);

    for (int64_t tile = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; tile < n_tiles; tile += n_gwarps) {
        const int64_t q = tile * kQPW + qi;
        const bool valid = q < n_qp;
        T F[9];
#pragma unroll
        for (int cpt = 0; cpt < 9; ++cpt) F[cpt] = valid ? Fg[cpt * n_qp + q] : ((cpt % 4) == 0 ? T(1) : T(0));
        T K[D], Jm1;
        bool bad = !kin_scalars<T, NF>(F, kc, K, Jm1);
        if (bad) {
#pragma unroll
            for (int cpt = 0; cpt < 9; ++cpt) F[cpt] = (cpt % 4) == 0 ? T(1) : T(0);
            kin_scalars<T, NF>(F, kc, K, Jm1);
        }

        // ---- forward values
        T npart = T(0);
        for (int k = 1; k <= L; ++k) {
            T y[NJ];
#pragma unroll
            for (int jj = 0; jj < NJ; ++jj) y[jj] = sw[lay.c + (k - 1) * W + j0 + jj];
            if (k == 1) {
#pragma unroll
                for (int m = 0; m < D; ++m) {
                    const T *wr = sw + lay.W1t + m * W + j0;
#pragma unroll
                    for (int jj = 0; jj < NJ; ++jj) y[jj] += wr[jj] * K[m];
                }
            } else {
                const T *zin = wk + ((k - 1) & 1) * W;
                const T *At = sw + lay.At + (k - 2) * W * W + j0;
#pragma unroll 4
                for (int i = 0; i < W; ++i) {
                    const T zi = zin[i];
#pragma unroll
                    for (int jj = 0; jj < NJ; ++jj) y[jj] += At[i * W + jj] * zi;
                }
                const T *Bt = sw + lay.Bt + (k - 2) * D * W + j0;
#pragma unroll
                for (int m = 0; m < D; ++m)
#pragma unroll
                    for (int jj = 0; jj < NJ; ++jj) y[jj] += Bt[m * W + jj] * K[m];
            }
            T *sk = sd + (k - 1) * W + j0;
            T *tk = sd + (L + k - 1) * W + j0;
            T *zout = wk + (k & 1) * W + j0;
#pragma unroll
            for (int jj = 0; jj < NJ; ++jj) {
                T z, s, t;
                act(y[jj], z, s, t);
                sk[jj] = s;
                tk[jj] = t;
                if (k < L)
                    zout[jj] = z;
                else
                    npart += sw[lay.a + j0 + jj] * z;
            }
            __syncwarp();
        }
        if (jb == 0) {
#pragma unroll
            for (int m = 0; m < D; ++m) npart += sw[lay.b + m] * K[m];
        }

        // ---- reverse adjoints and gradient
        T dN[D];
#pragma unroll
        for (int m = 0; m < D; ++m) dN[m] = (jb == 0) ? sw[lay.b + m] : T(0);
        T *yb = wk;
        {
            const T *Bt = (L == 1) ? (sw + lay.W1t + j0) : (sw + lay.Bt + (L - 2) * D * W + j0);
#pragma unroll
            for (int jj = 0; jj < NJ; ++jj) {
                const int j = j0 + jj;
                const T aj = sw[lay.a + j];
                const T ybar = sd[(L - 1) * W + j] * aj;
                sd[(2 * L - 1) * W + j] *= aj;
                yb[j] = ybar;
#pragma unroll
                for (int m = 0; m < D; ++m) dN[m] += Bt[m * W + jj] * ybar;
            }
            __syncwarp();
        }
        for (int k = L; k >= 2; --k) {
            T zb[NJ];
#pragma unroll
            for (int ii = 0; ii < NJ; ++ii) zb[ii] = T(0);
            const T *Ar = sw + lay.Ar + (k - 2) * W * W + j0;
#pragma unroll 4
            for (int j = 0; j < W; ++j) {
                const T ybj = yb[j];
#pragma unroll
                for (int ii = 0; ii < NJ; ++ii) zb[ii] += Ar[j * W + ii] * ybj;
            }
            __syncwarp();
            const T *Bt = (k - 1 == 1) ? (sw + lay.W1t + j0) : (sw + lay.Bt + (k - 3) * D * W + j0);
#pragma unroll
            for (int ii = 0; ii < NJ; ++ii) {
                const int i = j0 + ii;
                const T ybar = sd[(k - 2) * W + i] * zb[ii];
                sd[(L + k - 2) * W + i] *= zb[ii];
                yb[i] = ybar;
#pragma unroll
                for (int m = 0; m < D; ++m) dN[m] += Bt[m * W + ii] * ybar;
            }
            __syncwarp();
        }

        // ---- forward tangents and Hessian
        T Hs[NH];
#pragma unroll
        for (int h = 0; h < NH; ++h) Hs[h] = T(0);
#pragma unroll
        for (int jj = 0; jj < NJ; ++jj) {
            const int j = j0 + jj;
            const T *w1 = sw + lay.W1r + j * DP;
            const T Dj = sd[L * W + j];
#pragma unroll
            for (int m = 0; m < D; ++m) {
                const T dm = Dj * w1[m];
#pragma unroll
                for (int n = 0; n <= m; ++n) Hs[m * (m + 1) / 2 + n] += dm * w1[n];
            }
        }
        for (int k = 2; k <= L; ++k) {
            const T *At = sw + lay.At + (k - 2) * W * W + j0;
            const T *Bt = sw + lay.Bt + (k - 2) * D * W + j0;
            const T *sin = wk + ((k - 1) & 1) * W * DP;
            T *sout = wk + (k & 1) * W * DP;
#pragma unroll 1
            for (int c0 = 0; c0 < NJ; c0 += NC) {
                T acc[NC][D];
#pragma unroll
                for (int cc = 0; cc < NC; ++cc)
#pragma unroll
                    for (int m = 0; m < D; ++m) acc[cc][m] = Bt[m * W + c0 + cc];
                if (k == 2) {
#pragma unroll 2
                    for (int i = 0; i < W; ++i) {
                        const T si = sd[i];
                        const T *w1 = sw + lay.W1r + i * DP;
                        T sv[D];
#pragma unroll
                        for (int m = 0; m < D; ++m) sv[m] = si * w1[m];
#pragma unroll
                        for (int cc = 0; cc < NC; ++cc) {
                            const T wv = At[i * W + c0 + cc];
#pragma unroll
                            for (int m = 0; m < D; ++m) acc[cc][m] += wv * sv[m];
                        }
                    }
                } else {
#pragma unroll 2
                    for (int i = 0; i < W; ++i) {
                        const T *p = sin + i * DP;
                        T sv[D];
#pragma unroll
                        for (int m = 0; m < D; ++m) sv[m] = p[m];
#pragma unroll
                        for (int cc = 0; cc < NC; ++cc) {
                            const T wv = At[i * W + c0 + cc];
#pragma unroll
                            for (int m = 0; m < D; ++m) acc[cc][m] += wv * sv[m];
                        }
                    }
                }
#pragma unroll
                for (int cc = 0; cc < NC; ++cc) {
                    const int j = j0 + c0 + cc;
                    const T Dj = sd[(L + k - 1) * W + j];
#pragma unroll
                    for (int m = 0; m < D; ++m) {
                        const T dm = Dj * acc[cc][m];
#pragma unroll
                        for (int n = 0; n <= m; ++n) Hs[m * (m + 1) / 2 + n] += dm * acc[cc][n];
                    }
                    if (k < L) {
                        const T sj = sd[(k - 1) * W + j];
                        T *o = sout + j * DP;
#pragma unroll
                        for (int m = 0; m < D; ++m) o[m] = sj * acc[cc][m];
                    }
                }
            }
            __syncwarp();
        }

        // ---- reduce the group's partial sums
#pragma unroll
        for (int msk = 1; msk <= 2; msk <<= 1) {
            npart += shfl_xor(npart, msk);
#pragma unroll
            for (int m = 0; m < D; ++m) dN[m] += shfl_xor(dN[m], msk);
#pragma unroll
            for (int h = 0; h < NH; ++h) Hs[h] += shfl_xor(Hs[h], msk);
        }
        if (dN_out != nullptr && valid && jb == 0) {
#pragma unroll
            for (int m = 0; m < D; ++m) {
                dN_out[m * n_qp + q] = dN[m];
                dN_out[(D + m) * n_qp + q] = K[m];
            }
        }

        // ---- kinematic derivatives, P, A, Psi
        T cvec[D];
#pragma unroll
        for (int m = 0; m < D; ++m) cvec[m] = dN[m] - sw[lay.n0 + m];
        stage_kinematics<T, NF>(F, kc, cvec, Jm1, jb, qs);
        __syncwarp();
        bool nonfinite = false;
        for (int a = jb; a < 9; a += kG) {
            T Pa, Arow[9];
            assemble_row<T, NF>(a, qs, Hs, cvec, Pa, Arow);
            bool fin = dev_finite(Pa);
#pragma unroll
            for (int b = 0; b < 9; ++b) fin = fin && dev_finite(Arow[b]);
            nonfinite |= !fin;
            const bool nan_out = bad || !fin;
            if (valid) {
                const T nanv = T(NAN);
                P[a * n_qp + q] = nan_out ? nanv : Pa;
                if (A != nullptr) {
#pragma unroll
                    for (int b = 0; b < 9; ++b) A[(9 * a + b) * n_qp + q] = nan_out ? nanv : Arow[b];
                }
            }
        }
        // a point is reported if J <= 0 / bad input, or any of its rows was not finite
        const unsigned nf_mask = __ballot_sync(0xffffffffu, nonfinite);
        const bool grp_nonfinite = ((nf_mask >> (qi * 4)) & 0xFu) != 0u;
        if (valid && jb == 0) {
            T Psi = npart + kc.kappa * Jm1 * Jm1;
#pragma unroll
            for (int m = 0; m < D; ++m) Psi -= sw[lay.n0 + m] * (K[m] - sw[lay.K0 + m]);
            const bool rep = bad || grp_nonfinite || !dev_finite(Psi);
            if (psi != nullptr) psi[q] = rep ? T(NAN) : Psi;
            if (rep && status != nullptr) {
                atomicAdd(&status[0], 1);
                atomicMin(&status[1], (int32_t)(q < INT32_MAX ? q : INT32_MAX));
            }
        }
        __syncwarp();
    }
}

__global__ void status_init_kernel(int32_t *status) {
    status[0] = 0;
    status[1] = INT32_MAX;
}

int launch_status_init(int32_t *status, cudaStream_t s) {
    status_init_kernel<<<1, 1, 0, s>>>(status);
    return cudaGetLastError() == cudaSuccess ? COMMET_OK : COMMET_ERR_CUDA;
}

int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

template <typename T, int NF, int W>
static int launch_typed(const commet_model *m, int64_t n_qp, const void *F, void *psi, void *P, void *A,
                        int32_t *status, cudaStream_t s, void *dN_out) {
    using Cf = CUConf<T, NF, W>;
    KinConst<T> kc{};
    kc.kin = m->kp.kin;
    kc.stress_free = m->kp.stress_free;
    kc.kappa = (T)m->kp.kappa;
    for (int f = 0; f < 2; ++f)
        for (int c = 0; c < 3; ++c) kc.fib[f][c] = (T)m->kp.fib[f][c];
    const int qstride = qp_slab_elems<T>(Cf::D, W, m->L, NF);
    const size_t wbytes = ((size_t)m->lay.total * sizeof(T) + 15) / 16 * 16;
    const size_t per_warp = (size_t)kQPW * qstride * sizeof(T);
    int dev = 0;
    cudaGetDevice(&dev);
    int smem_max = 0;
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int max_threads = sizeof(T) == 8 ? 256 : 512;
    int warps = (int)std::min<size_t>((size_t)max_threads / 32, (smem_max - wbytes) / per_warp);
    if (smem_max < (int)wbytes || warps < 1) return COMMET_ERR_UNSUPPORTED;
    const size_t smem = wbytes + warps * per_warp;
    auto kern = const_update_kernel<T, NF, W>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return COMMET_ERR_CUDA;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem);
    if (per_sm < 1) per_sm = 1;
    const int64_t n_tiles = (n_qp + kQPW - 1) / kQPW;
    const int64_t want = (n_tiles + warps - 1) / warps;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sm_count() * per_sm));
    kern<<<grid, warps * 32, smem, s>>>((const T *)m->d_weights, m->lay, kc, n_qp, (const T *)F, (T *)psi, (T *)P,
                                        (T *)A, status, (T *)dN_out, qstride);
    return cudaGetLastError() == cudaSuccess ? COMMET_OK : COMMET_ERR_CUDA;
}

template <typename T>
static int dispatch(const commet_model *m, int64_t n_qp, const void *F, void *psi, void *P, void *A,
                    int32_t *status, cudaStream_t s, void *dN_out) {
    const int nf = m->kp.nf, W = m->W;
#define COMMET_CASE(NF_, W_) \
    if (nf == NF_ && W == W_) return launch_typed<T, NF_, W_>(m, n_qp, F, psi, P, A, status, s, dN_out);
    COMMET_CASE(0, 16)
    COMMET_CASE(0, 32)
    COMMET_CASE(0, 64)
    COMMET_CASE(1, 16)
    COMMET_CASE(1, 32)
    COMMET_CASE(2, 16)
    COMMET_CASE(2, 32)
    COMMET_CASE(2, 64)
#undef COMMET_CASE
    return COMMET_ERR_UNSUPPORTED;
}

int launch_const_update(const commet_model *m, int64_t n_qp, const void *F, void *psi, void *P, void *A,
                        int32_t *status, cudaStream_t s, void *dN_out) {
    if (status != nullptr) {
        int rc = launch_status_init(status, s);
        if (rc != COMMET_OK) return rc;
    }
    if (n_qp == 0) return COMMET_OK;
    if (m->precision == COMMET_F64) return dispatch<double>(m, n_qp, F, psi, P, A, status, s, dN_out);
    if (m->precision == COMMET_F32) return dispatch<float>(m, n_qp, F, psi, P, A, status, s, dN_out);
    return COMMET_ERR_UNSUPPORTED;
}

}  // namespace commet
