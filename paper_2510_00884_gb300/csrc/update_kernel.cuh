// The fused constitutive-update kernel and its launcher, shared by the material-form
// entry (const_update.cu: P, A) and the spatial-form entry (spatial.cu: tau, c in Voigt
// form, App. A.1); each translation unit instantiates one form.
//
// Fused constitutive update (Algorithm 2's constitutive call): F -> kinematic scalars K ->
// MICNN value, gradient and Hessian -> P, A, Psi, one persistent kernel over all points.
// The per-point work is qp_group_update (qp_body.cuh): a group of 4 lanes per point,
// 8 points per warp, the whole network in shared memory.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>

#include "closed_form.cuh"
#include "qp_body.cuh"

namespace commet {

int sm_count();

// Instantiations that batch the kinematic scalars where the records fit: FP64 networks
// without fibres or at most 16 wide (the two-fibre 32- and 64-wide ones have no room for
// the records beside their warps' slabs, and carry no code for them).
template <typename T, int NF, int W>
constexpr bool update_batches() {
    return sizeof(T) == 8 && (NF == 0 || W <= 16);
}

template <typename T, int NF, int W, bool SPATIAL>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 256 : 384)
    const_update_kernel(const T *__restrict__ gw, NetLayout lay, KinConst<T> kc, int64_t n_qp,
                        const T *__restrict__ Fg, T *__restrict__ psi, T *__restrict__ P, T *__restrict__ A,
                        int32_t *__restrict__ status, T *__restrict__ dN_out, int qstride, int wcount, bool batch) {
    using Cf = CUConf<T, NF, W>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sw = reinterpret_cast<T *>(smem_raw);
    // the packed weights up to wcount elements go to shared memory; the hidden weights
    // (the last blocks: A_k transposed, M, A_k row-major) are read from global memory when
    // wcount stops before them
    const int wbytes = (wcount * (int)sizeof(T) + 15) / 16 * 16;
    const T *at = (wcount > lay.At) ? sw + lay.At : gw + lay.At;
    const T *mt = (lay.M == 0) ? nullptr : ((wcount > lay.M) ? sw + lay.M : gw + lay.M);
    const T *ar = (wcount >= lay.total) ? sw + lay.Ar : gw + lay.Ar;
    {
        const int n16 = wbytes / 16;
        const int4 *src = reinterpret_cast<const int4 *>(gw);
        int4 *dst = reinterpret_cast<int4 *>(sw);
        for (int i = threadIdx.x; i < n16; i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int qi = lane >> 2, jb = lane & 3;
    T *qs = sw + wbytes / (int)sizeof(T) + (size_t)(warp * kQPW + qi) * qstride;
    const int64_t n_tiles = (n_qp + kQPW - 1) / kQPW;
    const int64_t n_gwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    // FP64 with batch: the kinematic scalars of the warp's next kKinTiles tiles, one point
    // per lane (kin_batch), in the warp's records after the point slabs
    T *rec = sw + wbytes / (int)sizeof(T) + (size_t)(blockDim.x >> 5) * kQPW * qstride +
             (size_t)warp * kinrec_size<NF, true>() * 32;
    const bool use_rec = update_batches<T, NF, W>() && batch;

    for (int64_t tile0 = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; tile0 < n_tiles;
         tile0 += kKinTiles * n_gwarps) {
        if (use_rec) kin_batch<T, NF, false, true>(Fg, nullptr, n_qp, tile0, n_gwarps, n_tiles, kc, rec, lane);
        __syncwarp();
        for (int sub = 0; sub < kKinTiles; ++sub) {
            const int64_t tile = tile0 + sub * n_gwarps;
            if (tile >= n_tiles) break;
            const T *krec = use_rec ? rec : nullptr;
            const int kr = sub * kQPW + qi;
            const int64_t q = tile * kQPW + qi;
            const bool valid = q < n_qp;
            T F[9];
#pragma unroll
            for (int cpt = 0; cpt < 9; ++cpt) F[cpt] = valid ? Fg[cpt * n_qp + q] : ((cpt % 4) == 0 ? T(1) : T(0));
            const int64_t qo = valid ? q : 0;
            T psi_val;
            bool report;
            if constexpr (SPATIAL) {
                // P and A of the point go to its slab, then are pushed forward to tau (P) and c (A)
                T *pa = qs + qp_stage_end(Cf::D, NF);
                qp_group_update<T, NF, W>(sw, lay, mt, at, ar, kc, qs, qi, jb, F, valid, pa, 1,
                                          A ? pa + 9 : nullptr, 1, nullptr, 0, psi_val, report, krec, kr);
                __syncwarp();
                push_forward_group<T>(qs + Stage<Cf::D, NF>::F, pa, pa + 9, jb, valid, P + qo,
                                      A ? A + qo : nullptr, n_qp);
            } else {
                qp_group_update<T, NF, W>(sw, lay, mt, at, ar, kc, qs, qi, jb, F, valid, P + qo, n_qp,
                                          A ? A + qo : nullptr, n_qp, dN_out ? dN_out + qo : nullptr, n_qp, psi_val,
                                          report, krec, kr);
            }
            if (valid && jb == 0) {
                if (psi != nullptr) psi[q] = psi_val;
                if (report && status != nullptr) {
                    atomicAdd(&status[0], 1);
                    atomicMin(&status[1], (int32_t)(q < INT32_MAX ? q : INT32_MAX));
                }
            }
            __syncwarp();
        }
    }
}

template <typename T, int NF, int W, bool SPATIAL>
static int launch_typed(const commet_model *m, int64_t n_qp, const void *F, void *psi, void *P, void *A,
                        int32_t *status, cudaStream_t s, void *dN_out) {
    using Cf = CUConf<T, NF, W>;
    KinConst<T> kc{};
    kc.kin = m->kp.kin;
    kc.stress_free = m->kp.stress_free;
    kc.kappa = (T)m->kp.kappa;
    for (int f = 0; f < 2; ++f)
        for (int c = 0; c < 3; ++c) kc.fib[f][c] = (T)m->kp.fib[f][c];
    const int qstride = qp_slab_elems<T>(Cf::D, W, m->L, NF, SPATIAL);
    const size_t per_warp = (size_t)kQPW * qstride * sizeof(T);
    int dev = 0;
    cudaGetDevice(&dev);
    int smem_max = 0;
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int max_threads = sizeof(T) == 8 ? 256 : 384;
    // all weights in shared memory, unless leaving A_k row-major, or the last two or three
    // blocks (A_k transposed, M, A_k row-major), in global memory lets more warps fit
    // beside the point slabs; FP64 warps are worth most in multiples of four, one per
    // scheduler, each of which has its own share of the FP64 pipe
    auto fit = [&](size_t wb) -> int {
        return wb + per_warp > (size_t)smem_max
                   ? 0
                   : (int)std::min<size_t>((size_t)max_threads / 32, (smem_max - wb) / per_warp);
    };
    int wcount = m->lay.total;
    int warps = fit(((size_t)m->lay.total * sizeof(T) + 15) / 16 * 16);
    // (FP32 is bound by latency: A_k transposed stays in shared memory there)
    for (const int wc : {m->lay.Ar, m->lay.M > 0 ? m->lay.M : m->lay.Ar, sizeof(T) == 8 ? m->lay.At : m->lay.Ar}) {
        const int w = fit(((size_t)wc * sizeof(T) + 15) / 16 * 16);
        if (w > warps) {
            warps = w;
            wcount = wc;
        }
    }
    const size_t wbytes = ((size_t)wcount * sizeof(T) + 15) / 16 * 16;
    if (warps < 1) return COMMET_ERR_UNSUPPORTED;
    // FP64: the batched kinematic scalars' records, where they fit beside the same warps
    const size_t rec_bytes = (size_t)kinrec_size<NF, true>() * 32 * sizeof(T);
    const bool batch = update_batches<T, NF, W>() && wbytes + warps * (per_warp + rec_bytes) <= (size_t)smem_max;
    const size_t smem = wbytes + warps * (per_warp + (batch ? rec_bytes : 0));
    auto kern = const_update_kernel<T, NF, W, SPATIAL>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return COMMET_ERR_CUDA;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem);
    if (per_sm < 1) per_sm = 1;
    const int64_t n_tiles = (n_qp + kQPW - 1) / kQPW;
    const int64_t want = (n_tiles + warps - 1) / warps;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sm_count() * per_sm));
    kern<<<grid, warps * 32, smem, s>>>((const T *)m->d_weights, m->lay, kc, n_qp, (const T *)F, (T *)psi, (T *)P,
                                        (T *)A, status, (T *)dN_out, qstride, wcount, batch);
    return cudaGetLastError() == cudaSuccess ? COMMET_OK : COMMET_ERR_CUDA;
}

template <typename T, bool SPATIAL>
static int dispatch(const commet_model *m, int64_t n_qp, const void *F, void *psi, void *P, void *A,
                    int32_t *status, cudaStream_t s, void *dN_out) {
    if (m->inner != COMMET_INNER_MICNN) return dispatch_closed<T, SPATIAL>(m, n_qp, F, psi, P, A, status, s, dN_out);
    const int nf = m->kp.nf, W = m->W;
#define COMMET_CASE(NF_, W_) \
    if (nf == NF_ && W == W_) return launch_typed<T, NF_, W_, SPATIAL>(m, n_qp, F, psi, P, A, status, s, dN_out);
    COMMET_CASE(0, 4)
    COMMET_CASE(0, 8)
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

}  // namespace commet
