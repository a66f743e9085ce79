// Per-point body of the fused constitutive update, shared by the constitutive kernel
// and the fused Newton assembly kernel.
//
// A group of 4 consecutive lanes owns one quadrature point; lane jb of the group owns
// neurons [jb*W/4, (jb+1)*W/4) of every hidden layer. The network sits in shared
// memory (`sw`, packed as described by NetLayout) and the point's activations in its
// padded shared-memory slab `qs`.
//
// Network derivatives. Algorithm 4 propagates 1 + d + d(d+1)/2 channels through each
// layer. This code computes the same exact Hessian with fewer operations:
//   forward values     y_k, z_k = F(y_k), s_k = F'(y_k), t_k = F''(y_k)
//   reverse adjoints   zbar_L = a, ybar_k = s_k zbar_k, zbar_{k-1} = A_k^T ybar_k,
//                      dN/dK = b + sum_k B_k^T ybar_k  (B_1 := W1)
//   forward tangents   J_1 = W1, J_k = A_k diag(s_{k-1}) J_{k-1} + B_k
//   Hessian            d2N/dK2 = sum_k J_k^T diag(t_k zbar_k) J_k
// (the second-order adjoint identity; the J_k of a layer is consumed as soon as it is
// formed, so only one W x d tangent block per point is stored).
#pragma once

#include <cuda_runtime.h>

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

// One point on its 4-lane group (all 32 lanes of the warp call this together).
//  F      the point's deformation gradient (replaced by I when it is not admissible)
//  valid  false for padding points: computed on F = I, nothing written
//  Pq, pst / Aq, ast   where row a of P and entry (a, b) of A go: Pq[a*pst], Aq[(9a+b)*ast]
//                      (Aq may be null)
//  dNq, dst            optional: dN/dK and K written to dNq[m*dst], dNq[(D+m)*dst]
//  psi_val, report     the point's Psi (NaN if reported) and whether it is reported
//                      (J <= 0, non-finite input or result); valid in every lane
template <typename T, int NF, int W>
__device__ __forceinline__ void qp_group_update(const T *__restrict__ sw, const NetLayout &lay,
                                                const KinConst<T> &kc, T *qs, int qi, int jb, T (&F)[9],
                                                bool valid, T *Pq, int64_t pst, T *Aq, int64_t ast, T *dNq,
                                                int64_t dst, T &psi_val, bool &report) {
    using Cf = CUConf<T, NF, W>;
    constexpr int D = Cf::D, DP = Cf::DP, NH = Cf::NH, NJ = Cf::NJ, NC = Cf::NC;
    const int L = lay.L;
    T *sd = qs;              // s_k at (k-1) W, t_k / D_k at (L+k-1) W
    T *wk = qs + 2 * L * W;  // work area
    const int j0 = jb * NJ;
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

    // ---- forward tangents and Hessian (only when A is wanted: P needs dN/dK alone)
    const bool want_A = (Aq != nullptr);
    T Hs[NH];
#pragma unroll
    for (int h = 0; h < NH; ++h) Hs[h] = T(0);
    if (want_A) {
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

    }  // want_A

    // ---- reduce the group's partial sums
#pragma unroll
    for (int msk = 1; msk <= 2; msk <<= 1) {
        npart += shfl_xor(npart, msk);
#pragma unroll
        for (int m = 0; m < D; ++m) dN[m] += shfl_xor(dN[m], msk);
#pragma unroll
        for (int h = 0; h < NH; ++h) Hs[h] += shfl_xor(Hs[h], msk);
    }
    if (dNq != nullptr && valid && jb == 0) {
#pragma unroll
        for (int m = 0; m < D; ++m) {
            dNq[m * dst] = dN[m];
            dNq[(D + m) * dst] = K[m];
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
        if (want_A) {
            assemble_row<T, NF>(a, qs, Hs, cvec, Pa, Arow);
        } else {
            Pa = assemble_P<T, NF>(a, qs, cvec);
#pragma unroll
            for (int b = 0; b < 9; ++b) Arow[b] = T(0);
        }
        bool fin = dev_finite(Pa);
#pragma unroll
        for (int b = 0; b < 9; ++b) fin = fin && dev_finite(Arow[b]);
        nonfinite |= !fin;
        const bool nan_out = bad || !fin;
        if (valid) {
            const T nanv = T(NAN);
            Pq[a * pst] = nan_out ? nanv : Pa;
            if (Aq != nullptr) {
#pragma unroll
                for (int b = 0; b < 9; ++b) Aq[(9 * a + b) * ast] = nan_out ? nanv : Arow[b];
            }
        }
    }
    // a point is reported if J <= 0 / bad input, or any of its rows was not finite
    const unsigned nf_mask = __ballot_sync(0xffffffffu, nonfinite);
    const bool grp_nonfinite = ((nf_mask >> (qi * 4)) & 0xFu) != 0u;
    {
        T Psi = npart + kc.kappa * Jm1 * Jm1;
#pragma unroll
        for (int m = 0; m < D; ++m) Psi -= sw[lay.n0 + m] * (K[m] - sw[lay.K0 + m]);
        report = bad || grp_nonfinite || !dev_finite(Psi);
        psi_val = report ? T(NAN) : Psi;
    }
}

}  // namespace commet
