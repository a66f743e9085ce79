// Constitutive update for the inner functions that are not networks: the CANN of
// eq. cann-def and the closed-form Gent-Thomas energy of eq. gt. The point's inner
// value, gradient and (diagonal) Hessian are formed by its 4-lane group; everything
// after that (polyconvex chain rule, kinematic staging, P and A, Psi) is the shared
// qp_group_finish of the network kernels.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>

#include "qp_body.cuh"

namespace commet {

int sm_count();

__device__ __forceinline__ double dev_exp(double x) { return exp(x); }
__device__ __forceinline__ float dev_exp(float x) { return expf(x); }
__device__ __forceinline__ double dev_log(double x) { return log(x); }
__device__ __forceinline__ float dev_log(float x) { return logf(x); }

// One CANN term of eq. cann-def at input value x, with its first and second derivative
// by the chain rule of eq. cann-chain-rule: v = w2 f2(f1(f0(x))), g = dv/dx, h = d2v/dx2.
// f0'' = 0 for every f0 of the menu; the second derivative of -ln(1 - w1 y) is
// +(w1 / (1 - w1 y))^2.
template <typename T>
__device__ __forceinline__ void cann_term(T x, int f0, int p, int f2, T w1, T w2, T &v, T &g, T &h) {
    T a, ad;
    if (f0 == COMMET_CANN_F0_MACAULAY) {
        a = x > T(0) ? x : T(0);
        ad = x > T(0) ? T(1) : (x < T(0) ? T(0) : T(0.5));
    } else if (f0 == COMMET_CANN_F0_ABS) {
        a = x < T(0) ? -x : x;
        ad = x > T(0) ? T(1) : (x < T(0) ? T(-1) : T(0));
    } else {
        a = x;
        ad = T(1);
    }
    T y, yd, ydd;
    if (p == 1) {
        y = a;
        yd = T(1);
        ydd = T(0);
    } else if (p == 2) {
        y = a * a;
        yd = T(2) * a;
        ydd = T(2);
    } else {
        y = a * a * a;
        yd = T(3) * a * a;
        ydd = T(6) * a;
    }
    T f, fd, fdd;
    if (f2 == COMMET_CANN_F2_EXP) {
        const T e = dev_exp(w1 * y);
        f = e - T(1);
        fd = w1 * e;
        fdd = w1 * w1 * e;
    } else if (f2 == COMMET_CANN_F2_LOG) {
        const T q = T(1) - w1 * y;  // q <= 0 gives a non-finite value: the point is reported
        f = -dev_log(q);
        fd = w1 / q;
        fdd = fd * fd;
    } else {
        f = w1 * y;
        fd = w1;
        fdd = T(0);
    }
    v = w2 * f;
    g = w2 * fd * yd * ad;
    h = w2 * (fdd * yd * yd + fd * ydd) * ad * ad;
}

// Derivatives of one CANN term's dv/dx = w2 f2'(f1(f0(x)); w1) f1'(f0(x)) f0'(x) with
// respect to its weights (the backward's parameter gradients): g2 = d/dw2 = f2' f1' f0',
// g1 = d/dw1 = w2 (d f2'/d w1) f1' f0', with d f2'/d w1 = 1 (w1 y), exp(w1 y) (1 + w1 y)
// (exp(w1 y) - 1) and 1/(1 - w1 y)^2 (-ln(1 - w1 y)).
template <typename T>
__device__ __forceinline__ void cann_term_wgrad(T x, int f0, int p, int f2, T w1, T w2, T &g1, T &g2) {
    T a, ad;
    if (f0 == COMMET_CANN_F0_MACAULAY) {
        a = x > T(0) ? x : T(0);
        ad = x > T(0) ? T(1) : (x < T(0) ? T(0) : T(0.5));
    } else if (f0 == COMMET_CANN_F0_ABS) {
        a = x < T(0) ? -x : x;
        ad = x > T(0) ? T(1) : (x < T(0) ? T(-1) : T(0));
    } else {
        a = x;
        ad = T(1);
    }
    const T y = p == 1 ? a : (p == 2 ? a * a : a * a * a);
    const T yd = p == 1 ? T(1) : (p == 2 ? T(2) * a : T(3) * a * a);
    T fd, fdw;
    if (f2 == COMMET_CANN_F2_EXP) {
        const T e = dev_exp(w1 * y);
        fd = w1 * e;
        fdw = e * (T(1) + w1 * y);
    } else if (f2 == COMMET_CANN_F2_LOG) {
        const T qi = T(1) / (T(1) - w1 * y);
        fd = w1 * qi;
        fdw = qi * qi;
    } else {
        fd = w1;
        fdw = T(1);
    }
    const T c = yd * ad;
    g2 = fd * c;
    g1 = w2 * fdw * c;
}

// The CANN's N, dN/dK and diagonal Hessian at K for one point: the D n terms (input m,
// term k) go round-robin over the point's 4 lanes, each lane holding partial sums.
template <typename T, int D>
__device__ __forceinline__ void cann_point(const T *sw, const NetLayout &lay, const T *K, int jb, T &npart, T *dN,
                                           T *Hs) {
    const int n = lay.cn, nt = D * n;
    for (int t0 = 0; t0 < nt; t0 += kG) {
        const int t = t0 + jb;
        if (t < nt) {
            const int m = t / n, k = t - m * n;
            T x = T(0);
#pragma unroll
            for (int mm = 0; mm < D; ++mm) x = (mm == m) ? K[mm] : x;
            T v, g, h;
            cann_term<T>(x, (int)sw[lay.ck + 3 * k], (int)sw[lay.ck + 3 * k + 1], (int)sw[lay.ck + 3 * k + 2],
                         sw[lay.cw + 2 * t], sw[lay.cw + 2 * t + 1], v, g, h);
            npart += v;
#pragma unroll
            for (int mm = 0; mm < D; ++mm) {
                dN[mm] += (mm == m) ? g : T(0);
                Hs[mm * (mm + 1) / 2 + mm] += (mm == m) ? h : T(0);
            }
        }
    }
}

// One weighted B-spline phi = w psi of an ICKAN layer (App. B) at x, with phi' and phi'':
// degree KD on uniform knots t_m = lo + (m - KD) h. In knot units x sits in span m with
// offset u; the KD + 1 non-zero basis functions follow from de Boor's triangle on uniform
// knots (every denominator of the recursion is the stage number j), and the derivatives
// from the lower-degree stages of the same triangle:
//   psi'  = (1/h)   sum_l (c_l - c_{l-1}) B_l,KD-1
//   psi'' = (1/h^2) sum_l (c_l - 2 c_{l-1} + c_{l-2}) B_l,KD-2
// (control points outside 0 .. nb - 1 are zero; outside the knots everything is zero).
template <typename T, int KD>
__device__ __forceinline__ void kan_spline(T x, T lo, T inv_h, int G, const T *__restrict__ wc, T &f, T &f1,
                                           T &f2) {
    const int nb = G + KD;
    const T s = (x - lo) * inv_h + T(KD);
    f = f1 = f2 = T(0);
    if (!(s >= T(0)) || !(s < T(G + 2 * KD))) return;
    const int m = (int)floor(s);
    const T u = s - T(m);
    T N[KD + 1], N1[KD], N2[KD - 1];
    N[0] = T(1);
    if constexpr (KD == 2) N2[0] = T(1);  // the degree-0 stage is the single indicator
#pragma unroll
    for (int j = 1; j <= KD; ++j) {
        T saved = T(0);
#pragma unroll
        for (int r = 0; r < j; ++r) {
            const T temp = N[r] * (T(1) / T(j));
            N[r] = saved + (T(r + 1) - u) * temp;
            saved = (u + T(j - r - 1)) * temp;
        }
        N[j] = saved;
        if (j == KD - 2) {
#pragma unroll
            for (int r = 0; r <= KD - 2; ++r) N2[r] = N[r];
        }
        if (j == KD - 1) {
#pragma unroll
            for (int r = 0; r <= KD - 1; ++r) N1[r] = N[r];
        }
    }
    const T ws = wc[0];
    const T *c = wc + 1;
    auto cp = [&](int l) -> T { return (l >= 0 && l < nb) ? c[l] : T(0); };
    T v = T(0), d1 = T(0), d2 = T(0);
#pragma unroll
    for (int r = 0; r <= KD; ++r) v += cp(m - KD + r) * N[r];
#pragma unroll
    for (int r = 0; r < KD; ++r) {
        const int l = m - KD + 1 + r;
        d1 += (cp(l) - cp(l - 1)) * N1[r];
    }
#pragma unroll
    for (int r = 0; r < KD - 1; ++r) {
        const int l = m - KD + 2 + r;
        d2 += (cp(l) - T(2) * cp(l - 1) + cp(l - 2)) * N2[r];
    }
    f = ws * v;
    f1 = ws * inv_h * d1;
    f2 = ws * inv_h * inv_h * d2;
}

// ICKAN value, gradient and packed Hessian of one point on its 4-lane group: the outputs
// of a hidden layer go round-robin over the lanes (each propagates z, dz/dK, d2z/dK2 of its
// outputs by the chain rule and writes them to the point's slab); the last layer's single
// output is split over its inputs, leaving per-lane partial sums for qp_group_finish.
template <typename T, int D, int KD>
__device__ __forceinline__ void kan_point(const T *__restrict__ sw, const NetLayout &lay, const T *K, T *qs, int jb,
                                          T &npart, T *dN, T *Hs) {
    constexpr int NH = D * (D + 1) / 2, S = 1 + D + NH;  // z, dz, d2z per neuron
    const int R = lay.kR, G = lay.kG, nb = G + KD;
    const int stride = lay.kwmax * S;
    const T *par = sw + lay.kpar;
    for (int r = 0; r < R; ++r) {
        const int nin = (int)sw[lay.kwid + r], nout = (int)sw[lay.kwid + r + 1];
        const T lo = sw[lay.klo + r], inv_h = T(G) / (sw[lay.khi + r] - lo);
        const T *zin = qs + ((r + 1) & 1) * stride;  // layer r - 1's outputs
        T *zout = qs + (r & 1) * stride;
        const bool last = (r == R - 1);
        // outputs (hidden layers) or inputs (last layer) of this lane
        for (int t = jb; t < (last ? nin : nout); t += kG) {
            T z = T(0), dz[D], d2z[NH];
#pragma unroll
            for (int a = 0; a < D; ++a) dz[a] = T(0);
#pragma unroll
            for (int h = 0; h < NH; ++h) d2z[h] = T(0);
            const int i = last ? 0 : t;
            const int j0 = last ? t : 0, j1 = last ? t + 1 : nin;
            for (int j = j0; j < j1; ++j) {
                const T *wc = par + (size_t)(i * nin + j) * (1 + nb);
                if (r == 0) {
                    // inputs are K itself: dz_j = e_j, d2z_j = 0
                    T x = T(0);
#pragma unroll
                    for (int a = 0; a < D; ++a) x = (a == j) ? K[a] : x;
                    T f, f1, f2;
                    kan_spline<T, KD>(x, lo, inv_h, G, wc, f, f1, f2);
                    z += f;
#pragma unroll
                    for (int a = 0; a < D; ++a) {
                        dz[a] += (a == j) ? f1 : T(0);
                        d2z[a * (a + 1) / 2 + a] += (a == j) ? f2 : T(0);
                    }
                } else {
                    const T *in = zin + j * S;
                    T f, f1, f2;
                    kan_spline<T, KD>(in[0], lo, inv_h, G, wc, f, f1, f2);
                    z += f;
#pragma unroll
                    for (int a = 0; a < D; ++a) {
                        const T da = in[1 + a];
                        dz[a] += f1 * da;
#pragma unroll
                        for (int b = 0; b <= a; ++b) d2z[a * (a + 1) / 2 + b] += f2 * da * in[1 + b];
                    }
#pragma unroll
                    for (int h = 0; h < NH; ++h) d2z[h] += f1 * in[1 + D + h];
                }
            }
            if (last) {
                npart += z;
#pragma unroll
                for (int a = 0; a < D; ++a) dN[a] += dz[a];
#pragma unroll
                for (int h = 0; h < NH; ++h) Hs[h] += d2z[h];
            } else {
                T *out = zout + t * S;
                out[0] = z;
#pragma unroll
                for (int a = 0; a < D; ++a) out[1 + a] = dz[a];
#pragma unroll
                for (int h = 0; h < NH; ++h) out[1 + D + h] = d2z[h];
            }
        }
        par += (size_t)nin * nout * (1 + nb);
        __syncwarp();
    }
}

template <typename T, int NF, int INNER, bool SPATIAL, int KD = 3>
__global__ void __launch_bounds__(256)
    closed_update_kernel(const T *__restrict__ gw, NetLayout lay, KinConst<T> kc, int64_t n_qp,
                         const T *__restrict__ Fg, T *__restrict__ psi, T *__restrict__ P, T *__restrict__ A,
                         int32_t *__restrict__ status, T *__restrict__ dN_out, int qstride, bool batch) {
    constexpr int D = 3 + 2 * NF, NH = D * (D + 1) / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sw = reinterpret_cast<T *>(smem_raw);
    const int wbytes = (lay.total * (int)sizeof(T) + 15) / 16 * 16;
    {
        const int4 *src = reinterpret_cast<const int4 *>(gw);
        int4 *dst = reinterpret_cast<int4 *>(sw);
        for (int i = threadIdx.x; i < wbytes / 16; i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int qi = lane >> 2, jb = lane & 3;
    T *qs = sw + wbytes / (int)sizeof(T) + (size_t)(warp * kQPW + qi) * qstride;
    const int64_t n_tiles = (n_qp + kQPW - 1) / kQPW;
    const int64_t n_gwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const bool want_A = (A != nullptr);
    // the warp's kinematic records after the point slabs (batch: when they fit in shared
    // memory; otherwise the scalars are formed per point)
    T *rec = sw + wbytes / (int)sizeof(T) + (size_t)(blockDim.x >> 5) * kQPW * qstride +
             (size_t)warp * kinrec_size<NF, sizeof(T) == 8>() * 32;

    for (int64_t tile0 = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; tile0 < n_tiles;
         tile0 += kKinTiles * n_gwarps) {
        if (batch) kin_batch<T, NF, false, sizeof(T) == 8>(Fg, nullptr, n_qp, tile0, n_gwarps, n_tiles, kc, rec, lane);
        __syncwarp();
        for (int sub = 0; sub < kKinTiles; ++sub) {
            const int64_t tile = tile0 + sub * n_gwarps;
            if (tile >= n_tiles) break;
            const int64_t q = tile * kQPW + qi;
            const bool valid = q < n_qp;
            const int64_t qo = valid ? q : 0;
            T F[9];
#pragma unroll
            for (int c = 0; c < 9; ++c) F[c] = valid ? Fg[c * n_qp + q] : ((c % 4) == 0 ? T(1) : T(0));
            T K[D], Jm1;
            PolyChain<T> ch;
            const bool bad = batch ? kin_read<T, NF>(rec, sub * kQPW + qi, K, Jm1, ch)
                                   : !kin_scalars_k64<T, NF>(F, kc, K, Jm1, ch);
            if (bad) {
#pragma unroll
                for (int c = 0; c < 9; ++c) F[c] = (c % 4) == 0 ? T(1) : T(0);
                if (!batch) kin_scalars_k64<T, NF>(F, kc, K, Jm1, ch);
            }
            T npart = T(0), dN[D], Hs[NH];
#pragma unroll
            for (int m = 0; m < D; ++m) dN[m] = T(0);
#pragma unroll
            for (int h = 0; h < NH; ++h) Hs[h] = T(0);
            if constexpr (INNER == COMMET_INNER_ICKAN) {
                kan_point<T, 3 + 2 * NF, KD>(sw, lay, K, qs, jb, npart, dN, Hs);
            } else if constexpr (INNER == COMMET_INNER_CANN) {
                cann_point<T, D>(sw, lay, K, jb, npart, dN, Hs);
            } else {
                // eq. gt on raw (Ibar1, Ibar2, J); J - 1 from det_minus_one
                if (jb == 0) {
                    const T r2 = T(1) / K[1];
                    npart = T(0.5) * (K[0] - T(3)) + dev_log(K[1] * T(1.0 / 3.0)) + Jm1 * Jm1;
                    dN[0] = T(0.5);
                    dN[1] = r2;
                    dN[2] = T(2) * Jm1;
                    Hs[2] = -r2 * r2;
                    Hs[5] = T(2);
                }
            }
            T psi_val;
            bool report;
            const T *pre = (sizeof(T) == 8 && batch) ? kin_pre<T, NF>(rec, sub * kQPW + qi) : nullptr;
            if constexpr (SPATIAL) {
                T *pa = qs + qp_stage_end(D, NF);
                qp_group_finish<T, NF>(sw + lay.n0, sw + lay.K0, kc, qs, qi, jb, F, K, Jm1, ch, bad, valid, npart, dN,
                                       Hs, want_A, pa, 1, want_A ? pa + 9 : nullptr, 1, nullptr, 0, psi_val, report,
                                       pre);
                __syncwarp();
                push_forward_group<T>(qs + Stage<D, NF>::F, pa, pa + 9, jb, valid, P + qo, want_A ? A + qo : nullptr,
                                      n_qp);
            } else {
                qp_group_finish<T, NF>(sw + lay.n0, sw + lay.K0, kc, qs, qi, jb, F, K, Jm1, ch, bad, valid, npart, dN,
                                       Hs, want_A, P + qo, n_qp, want_A ? A + qo : nullptr, n_qp,
                                       dN_out ? dN_out + qo : nullptr, n_qp, psi_val, report, pre);
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

template <typename T, int NF, int INNER, bool SPATIAL, int KD = 3>
static int launch_closed(const commet_model *m, int64_t n_qp, const void *F, void *psi, void *P, void *A,
                         int32_t *status, cudaStream_t s, void *dN_out) {
    constexpr int D = 3 + 2 * NF;
    KinConst<T> kc{};
    kc.kin = m->kp.kin;
    kc.stress_free = m->kp.stress_free;
    kc.kappa = (T)m->kp.kappa;
    for (int f = 0; f < 2; ++f)
        for (int c = 0; c < 3; ++c) kc.fib[f][c] = (T)m->kp.fib[f][c];
    const int net = (INNER == COMMET_INNER_ICKAN) ? 2 * m->lay.kwmax * (1 + D + D * (D + 1) / 2) : 0;
    const int qstride = qp_slab_elems<T>(D, 0, 0, NF, SPATIAL, net);
    const size_t wbytes = ((size_t)m->lay.total * sizeof(T) + 15) / 16 * 16;
    const int warps = 8;
    const size_t smem_pt = wbytes + (size_t)warps * kQPW * qstride * sizeof(T);
    const size_t smem_b = smem_pt + (size_t)warps * kinrec_size<NF, sizeof(T) == 8>() * 32 * sizeof(T);
    int dev = 0, smem_max = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const bool batch = smem_b <= (size_t)smem_max;  // kinematic records beside the slabs
    const size_t smem = batch ? smem_b : smem_pt;
    auto kern = closed_update_kernel<T, NF, INNER, SPATIAL, KD>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return COMMET_ERR_CUDA;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem);
    if (per_sm < 1) per_sm = 1;
    const int64_t n_tiles = (n_qp + kQPW - 1) / kQPW;
    const int64_t want = (n_tiles + warps - 1) / warps;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sm_count() * per_sm));
    kern<<<grid, warps * 32, smem, s>>>((const T *)m->d_weights, m->lay, kc, n_qp, (const T *)F, (T *)psi, (T *)P,
                                        (T *)A, status, (T *)dN_out, qstride, batch);
    return cudaGetLastError() == cudaSuccess ? COMMET_OK : COMMET_ERR_CUDA;
}

template <typename T, bool SPATIAL>
static int dispatch_closed(const commet_model *m, int64_t n_qp, const void *F, void *psi, void *P, void *A,
                           int32_t *status, cudaStream_t s, void *dN_out) {
    const int nf = m->kp.nf;
    if (m->inner == COMMET_INNER_ICKAN && nf == 0) {
        if (m->lay.kdeg == 2)
            return launch_closed<T, 0, COMMET_INNER_ICKAN, SPATIAL, 2>(m, n_qp, F, psi, P, A, status, s, dN_out);
        if (m->lay.kdeg == 3)
            return launch_closed<T, 0, COMMET_INNER_ICKAN, SPATIAL, 3>(m, n_qp, F, psi, P, A, status, s, dN_out);
        if (m->lay.kdeg == 4)
            return launch_closed<T, 0, COMMET_INNER_ICKAN, SPATIAL, 4>(m, n_qp, F, psi, P, A, status, s, dN_out);
        return COMMET_ERR_UNSUPPORTED;
    }
    if (m->inner == COMMET_INNER_GENT_THOMAS && nf == 0)
        return launch_closed<T, 0, COMMET_INNER_GENT_THOMAS, SPATIAL>(m, n_qp, F, psi, P, A, status, s, dN_out);
    if (m->inner == COMMET_INNER_CANN) {
        if (nf == 0) return launch_closed<T, 0, COMMET_INNER_CANN, SPATIAL>(m, n_qp, F, psi, P, A, status, s, dN_out);
        if (nf == 1) return launch_closed<T, 1, COMMET_INNER_CANN, SPATIAL>(m, n_qp, F, psi, P, A, status, s, dN_out);
        if (nf == 2) return launch_closed<T, 2, COMMET_INNER_CANN, SPATIAL>(m, n_qp, F, psi, P, A, status, s, dN_out);
    }
    return COMMET_ERR_UNSUPPORTED;
}

}  // namespace commet
