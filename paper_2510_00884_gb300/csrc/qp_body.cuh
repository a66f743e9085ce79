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

// End of the staging area in a point's slab (elements of T): staged kinematics, then
// u[9][DP] and d2N/dK2 [D][DP] (see qp_group_update). The spatial-output kernels put the
// point's P (9) and A (81) right after it.
__host__ __device__ inline int qp_stage_end(int D, int NF) {
    const int DP = (D + 3) / 4 * 4;
    return (9 * D + 54 + 18 * NF + 5 + NF + 3) / 4 * 4 + 9 * DP + D * DP;
}

// FP64 only: the per-point prescaled vectors of A's structured terms (see
// prescale_structured), right after the staging area; in the spatial kernels the same
// room later holds the point's P and A (every A entry is formed before any is stored).
__host__ __device__ inline int qp_pre_elems(int NF) { return (45 + 18 * NF + 3) / 4 * 4; }

// Per-qp slab size in elements of T for the given network (host and device agree);
// with `spatial`, room for P and A after the staging area; `net` elements at least.
template <typename T>
__host__ __device__ inline int qp_slab_elems(int D, int W, int L, int NF, bool spatial = false, int net = 0) {
    const int DP = (D + 3) / 4 * 4;
    const int nbuf = L >= 4 ? 2 : (L == 3 ? 1 : 0);
    int work = 2 * W;
    if (nbuf * W * DP > work) work = nbuf * W * DP;
    int raw = 2 * L * W + work;
    int after = spatial ? 90 : 0;
    if (sizeof(T) == 8 && qp_pre_elems(NF) > after) after = qp_pre_elems(NF);
    const int stage = qp_stage_end(D, NF) + after;
    if (stage > raw) raw = stage;
    if (net > raw) raw = net;  // per-point network area of the non-MLP inner functions
    int words = raw * (int)sizeof(T) / 4;
    words = (words + 31) / 32 * 32 + 4;
    return words * 4 / (int)sizeof(T);
}

template <typename T>
__device__ __forceinline__ T shfl_xor(T v, int m) {
    return __shfl_xor_sync(0xffffffffu, v, m);
}

// Vector shared-memory loads/stores of N consecutive elements: 128-bit when N is a
// multiple of 16 / sizeof(T) (p 16-byte aligned), 64-bit float pairs when N is even
// (p 8-byte aligned), scalar otherwise (the narrow networks, W = 4 and 8).
template <int N, typename T>
__device__ __forceinline__ void ldv(const T *p, T *r) {
    if constexpr (sizeof(T) == 8 && N % 2 == 0) {
#pragma unroll
        for (int v = 0; v < N / 2; ++v) {
            const double2 x = reinterpret_cast<const double2 *>(p)[v];
            r[2 * v] = x.x;
            r[2 * v + 1] = x.y;
        }
    } else if constexpr (sizeof(T) == 4 && N % 4 == 0) {
#pragma unroll
        for (int v = 0; v < N / 4; ++v) {
            const float4 x = reinterpret_cast<const float4 *>(p)[v];
            r[4 * v] = x.x;
            r[4 * v + 1] = x.y;
            r[4 * v + 2] = x.z;
            r[4 * v + 3] = x.w;
        }
    } else if constexpr (sizeof(T) == 4 && N % 2 == 0) {
#pragma unroll
        for (int v = 0; v < N / 2; ++v) {
            const float2 x = reinterpret_cast<const float2 *>(p)[v];
            r[2 * v] = x.x;
            r[2 * v + 1] = x.y;
        }
    } else {
#pragma unroll
        for (int v = 0; v < N; ++v) r[v] = p[v];
    }
}
template <int N, typename T>
__device__ __forceinline__ void stv(T *p, const T *r) {
    if constexpr (sizeof(T) == 8 && N % 2 == 0) {
#pragma unroll
        for (int v = 0; v < N / 2; ++v) reinterpret_cast<double2 *>(p)[v] = make_double2(r[2 * v], r[2 * v + 1]);
    } else if constexpr (sizeof(T) == 4 && N % 4 == 0) {
#pragma unroll
        for (int v = 0; v < N / 4; ++v)
            reinterpret_cast<float4 *>(p)[v] = make_float4(r[4 * v], r[4 * v + 1], r[4 * v + 2], r[4 * v + 3]);
    } else if constexpr (sizeof(T) == 4 && N % 2 == 0) {
#pragma unroll
        for (int v = 0; v < N / 2; ++v) reinterpret_cast<float2 *>(p)[v] = make_float2(r[2 * v], r[2 * v + 1]);
    } else {
#pragma unroll
        for (int v = 0; v < N; ++v) p[v] = r[v];
    }
}

// K in FP64 whatever T is. The CANN's polynomial terms make dN/dK proportional to K,
// and a shifted invariant such as Ibar2 - 3 formed in FP32 carries an absolute error of
// a few ulp(3) ~ 1e-6, a large relative error when K is small; with FP64 kinematic
// scalars the FP32 path keeps its 1e-5 bound. (A network's dN/dK varies slowly with K,
// so the network kernels form K in T.)
template <typename T, int NF>
__device__ __forceinline__ bool kin_scalars_k64(const T (&F)[9], const KinConst<T> &kc, T *K, T &Jm1,
                                                PolyChain<T> &ch) {
    if constexpr (sizeof(T) == 8) {
        return kin_scalars<T, NF>(F, kc, K, Jm1, &ch);
    } else {
        constexpr int D = 3 + 2 * NF;
        KinConst<double> kd{};
        kd.kin = kc.kin;
        kd.stress_free = kc.stress_free;
        kd.kappa = (double)kc.kappa;
        for (int f = 0; f < 2; ++f)
            for (int c = 0; c < 3; ++c) kd.fib[f][c] = (double)kc.fib[f][c];
        double Fd[9], Kd[D], Jd;
        PolyChain<double> chd;
#pragma unroll
        for (int c = 0; c < 9; ++c) Fd[c] = (double)F[c];
        const bool ok = kin_scalars<double, NF>(Fd, kd, Kd, Jd, &chd);
#pragma unroll
        for (int m = 0; m < D; ++m) K[m] = (T)Kd[m];
        Jm1 = (T)Jd;
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            ch.d1[m] = (T)chd.d1[m];
            ch.d2[m] = (T)chd.d2[m];
        }
        return ok;
    }
}

// Kinematic scalars of a warp's next kKinTiles tiles (kKinTiles x kQPW = 32 points), one
// point per lane. In the per-point code the four lanes of a point's group would each form
// the same FP64 scalars, and GB300 bills an FP64 warp instruction to all 32 lanes whatever
// the mask: formed here, once per point, they take a quarter of the FP64 instructions.
// With PRE (FP64) the record also holds, after those, C[9], I1, I2 and J^(-1/3) of the
// same F for stage_kinematics. Lane l takes point off + l % kQPW of tile tile0 + (l / kQPW) tstep (tiles of tile_pts
// points: kQPW for a warp's own tiles, the CTA's for a CTA tile) and writes, component-major
// at rec[c * 32 + l]: K[D], J - 1, phi'[3], phi''[3] and 1 where F (or, WITH_G, G = dL/dP)
// was inadmissible and the scalars are those of F = I (0 otherwise).
constexpr int kKinTiles = 32 / kQPW;

// Record layout (component-major, stride 32): K[D] at 0, J - 1 at D, then phi'[3] and
// phi''[3] (the polyconvex layer: networks without fibres only), the replaced-input flag,
// and with PRE the staging's C[9], I1, I2, J^(-1/3).
template <int NF>
__host__ __device__ constexpr int kinrec_chain() {
    return 3 + 2 * NF + 1;
}
template <int NF>
__host__ __device__ constexpr int kinrec_flag() {
    return kinrec_chain<NF>() + (NF == 0 ? 6 : 0);
}
template <int NF, bool PRE = false>
__host__ __device__ constexpr int kinrec_size() {
    return kinrec_flag<NF>() + 1 + (PRE ? 12 : 0);
}

template <typename T, int NF, bool WITH_G, bool PRE = false>
__device__ __forceinline__ void kin_batch(const T *__restrict__ Fg, const T *__restrict__ Gg, int64_t n_qp,
                                          int64_t tile0, int64_t tstep, int64_t n_tiles, const KinConst<T> &kc,
                                          T *rec, int lane, int tile_pts = kQPW, int off = 0) {
    constexpr int D = 3 + 2 * NF, oc = kinrec_chain<NF>(), of = kinrec_flag<NF>();
    const int64_t tile = tile0 + (int64_t)(lane / kQPW) * tstep;
    const int64_t q = tile * tile_pts + off + (lane % kQPW);
    const bool valid = tile < n_tiles && q < n_qp;
    T F[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) F[c] = valid ? Fg[c * n_qp + q] : ((c % 4) == 0 ? T(1) : T(0));
    bool gbad = false;
    if constexpr (WITH_G) {
#pragma unroll
        for (int c = 0; c < 9; ++c) gbad = gbad || (valid && !dev_finite(Gg[c * n_qp + q]));
    }
    T K[D], Jm1;
    PolyChain<T> ch{};
    const bool bad = !kin_scalars_k64<T, NF>(F, kc, K, Jm1, ch) || gbad;
    if (bad) {
#pragma unroll
        for (int c = 0; c < 9; ++c) F[c] = (c % 4) == 0 ? T(1) : T(0);
        kin_scalars_k64<T, NF>(F, kc, K, Jm1, ch);
    }
#pragma unroll
    for (int m = 0; m < D; ++m) rec[m * 32 + lane] = K[m];
    rec[D * 32 + lane] = Jm1;
    if constexpr (NF == 0) {
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            rec[(oc + m) * 32 + lane] = ch.d1[m];
            rec[(oc + 3 + m) * 32 + lane] = ch.d2[m];
        }
    }
    rec[of * 32 + lane] = bad ? T(1) : T(0);
    if constexpr (PRE) {
        // as stage_kinematics forms them (the same F, replaced by I where bad)
        T C[9];
        right_cg(F, C);
#pragma unroll
        for (int i = 0; i < 9; ++i) rec[(of + 1 + i) * 32 + lane] = C[i];
        rec[(of + 10) * 32 + lane] = C[0] + C[4] + C[8];
        rec[(of + 11) * 32 + lane] = second_invariant(C);
        rec[(of + 12) * 32 + lane] = dev_rcbrt(T(1) + Jm1);
    }
}

// Where point r's stage_kinematics values sit in a PRE record (stride 32).
template <typename T, int NF>
__device__ __forceinline__ const T *kin_pre(const T *rec, int r) {
    return rec + (kinrec_flag<NF>() + 1) * 32 + r;
}

// The record of point r (0..31) of the last kin_batch; returns whether F = I was used.
// (phi', phi'' are zero for networks with fibres, which have no polyconvex layer.)
template <typename T, int NF>
__device__ __forceinline__ bool kin_read(const T *rec, int r, T *K, T &Jm1, PolyChain<T> &ch) {
    constexpr int D = 3 + 2 * NF, oc = kinrec_chain<NF>();
#pragma unroll
    for (int m = 0; m < D; ++m) K[m] = rec[m * 32 + r];
    Jm1 = rec[D * 32 + r];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        ch.d1[m] = NF == 0 ? rec[(oc + m) * 32 + r] : T(0);
        ch.d2[m] = NF == 0 ? rec[(oc + 3 + m) * 32 + r] : T(0);
    }
    return rec[kinrec_flag<NF>() * 32 + r] != T(0);
}

// One input neuron's contribution to a lane's block of the layer tangent:
//   acc[cc][m] += (w[cc] * scale) * v[m]      (scaled: k = 2, s_1 folded into the weight)
//   acc[cc][m] +=  w[cc] * v[m]               (otherwise)
// FP32 with 8 output neurons per lane runs on output pairs, one fma.rn.f32x2 (two FMAs,
// one issue slot, the same correctly rounded result per lane) per pair and input entry.
// Measured on d7 W32 L3 (4.24 -> 3.73 ms on 2^21 points); with 4 outputs per lane the
// scalar form was the faster one, so it is kept there and in FP64.
template <typename T, int NC, int D>
__device__ __forceinline__ void tangent_step(T (&acc)[NC][D], const T *w, const T *v, T scale, bool scaled = true) {
    if constexpr (sizeof(T) == 4 && NC >= 8 && NC % 2 == 0) {
#pragma unroll
        for (int p = 0; p < NC / 2; ++p) {
            float2 w2 = make_float2(w[2 * p], w[2 * p + 1]);
            if (scaled) w2 = __fmul2_rn(w2, make_float2(scale, scale));
#pragma unroll
            for (int m = 0; m < D; ++m) {
                const float2 r = __ffma2_rn(w2, make_float2(v[m], v[m]), make_float2(acc[2 * p][m], acc[2 * p + 1][m]));
                acc[2 * p][m] = r.x;
                acc[2 * p + 1][m] = r.y;
            }
        }
    } else {
#pragma unroll
        for (int cc = 0; cc < NC; ++cc) {
            const T ws = scaled ? w[cc] * scale : w[cc];
#pragma unroll
            for (int m = 0; m < D; ++m) acc[cc][m] += ws * v[m];
        }
    }
}

// Second half of a point's update, shared by every inner function: the 4-lane group
// reduction of the partial sums (npart, dN, Hs: N, dN/dK and the packed lower triangle
// of d2N/dK2, each lane holding its share), the polyconvex chain rule, the kinematic
// staging and the assembly of P and A (eq. nncm-chain, material form), and Psi.
//  n0s, K0s  the stress-free shift n0 and K(I) (zeros when off)
//  K, Jm1, ch, bad   from kin_scalars at the (possibly replaced) F
// Outputs as qp_group_update.
template <typename T, int NF>
__device__ __forceinline__ void qp_group_finish(const T *n0s, const T *K0s, const KinConst<T> &kc, T *qs, int qi,
                                                int jb, const T (&F)[9], const T *K, T Jm1,
                                                const PolyChain<T> &ch, bool bad, bool valid, T npart, T *dN,
                                                T *Hs, bool want_A, T *Pq, int64_t pst, T *Aq, int64_t ast,
                                                T *dNq, int64_t dst, T &psi_val, bool &report,
                                                const T *pre = nullptr) {
    constexpr int D = 3 + 2 * NF, DP = (D + 3) / 4 * 4, NH = D * (D + 1) / 2;
    // ---- reduce the group's partial sums
#pragma unroll
    for (int msk = 1; msk <= 2; msk <<= 1) {
        npart += shfl_xor(npart, msk);
#pragma unroll
        for (int m = 0; m < D; ++m) dN[m] += shfl_xor(dN[m], msk);
        if (want_A) {  // the Hessian is zero and unused when only P is wanted
#pragma unroll
            for (int h = 0; h < NH; ++h) Hs[h] += shfl_xor(Hs[h], msk);
        }
    }
    if (dNq != nullptr && valid && jb == 0) {
#pragma unroll
        for (int m = 0; m < D; ++m) {
            dNq[m * dst] = dN[m];
            dNq[(D + m) * dst] = K[m];
        }
    }

    // ---- Psi first: a point whose energy is not finite (an inner function outside its
    // domain) is reported with all of its outputs NaN, like an inadmissible F
    T Psi = npart + kc.kappa * Jm1 * Jm1;
#pragma unroll
    for (int m = 0; m < D; ++m) Psi -= n0s[m] * (K[m] - K0s[m]);
    bad = bad || !dev_finite(Psi);

    // ---- kinematic derivatives, P, A
    T cvec[D];
#pragma unroll
    for (int m = 0; m < D; ++m) cvec[m] = dN[m] - n0s[m];
    if constexpr (NF == 0) {
        if (kc.kin == COMMET_KIN_POLYCONVEX) poly_to_invariants<T>(ch, cvec, Hs);
    }
    if (want_A)
        stage_kinematics<T, NF>(F, kc, cvec, Jm1, jb, qs, pre);
    else
        stage_kinematics<T, NF, true>(F, kc, cvec, Jm1, jb, qs, pre);  // what P (and tau) need
    using S = Stage<D, NF>;
    constexpr int UOFF = (S::size + 3) / 4 * 4;  // u_a = sum_m g_m[a] N_mn : [9][DP]
    constexpr int HOFF = UOFF + 9 * DP;          // d2N/dK2, full: [D][DP]
    constexpr int NPL = (D + kG - 1) / kG;       // u columns per lane
    if (want_A && jb == 0) {
#pragma unroll
        for (int m = 0; m < D; ++m)
#pragma unroll
            for (int n = 0; n < D; ++n)
                qs[HOFF + m * DP + n] = Hs[(m >= n) ? (m * (m + 1) / 2 + n) : (n * (n + 1) / 2 + m)];
    }
    __syncwarp();
    bool group_nonfinite = false;
    if constexpr (sizeof(T) != 8) {
        // FP32: each lane forms whole rows a = jb, jb + 4, jb + 8 (fewer live registers)
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
                if (want_A) {
#pragma unroll
                    for (int b = 0; b < 9; ++b) Aq[(9 * a + b) * ast] = nan_out ? nanv : Arow[b];
                }
            }
        }
        const unsigned m0 = __ballot_sync(0xffffffffu, nonfinite);
        group_nonfinite = ((m0 >> (qi * 4)) & 0xFu) != 0u;
    } else {
        // FP64: the FP64 pipe is charged per warp instruction, so the work is spread evenly:
        // P rows a = jb, jb + 4, jb + 8 and, with A, the 45 upper entries round-robin over the
        // group's four lanes; every value is formed before any is stored so that a point with
        // a non-finite entry is written as NaN throughout.
        T Pv[3];
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            const int a = jb + kG * t;
            Pv[t] = (a < 9) ? assemble_P<T, NF>(a, qs, cvec) : T(0);
        }
        T Av[12];
#pragma unroll
        for (int t = 0; t < 12; ++t) Av[t] = T(0);
        if (want_A) {
#pragma unroll 1
            for (int a = 0; a < 9; ++a) {
#pragma unroll
                for (int nn = 0; nn < NPL; ++nn) {
                    const int n = jb * NPL + nn;
                    const int nc = n < D ? n : D - 1;
                    T acc = T(0);
#pragma unroll
                    for (int m = 0; m < D; ++m) acc += qs[S::g + 9 * m + a] * qs[HOFF + m * DP + nc];
                    if (n < D) qs[UOFF + a * DP + n] = acc;
                }
            }
            T *pre = qs + qp_stage_end(D, NF);
            prescale_structured<T, NF>(qs, jb, pre);
            __syncwarp();
#pragma unroll
            for (int t = 0; t < 12; ++t) {
                const int e = jb + kG * t;
                if (e < 45) {
                    int a, b;
                    upper_index(e, a, b);
                    Av[t] = assemble_entry_pre<T, NF, DP>(a, b, qs, qs + UOFF, pre);
                }
            }
        }
        bool nonfinite = false;
#pragma unroll
        for (int t = 0; t < 3; ++t) nonfinite |= !dev_finite(Pv[t]);
#pragma unroll
        for (int t = 0; t < 12; ++t) nonfinite |= !dev_finite(Av[t]);
        {
            const unsigned m0 = __ballot_sync(0xffffffffu, nonfinite);
            nonfinite = ((m0 >> (qi * 4)) & 0xFu) != 0u;
            group_nonfinite = nonfinite;
        }
        if (valid) {
            const bool nan_out = bad || nonfinite;
            const T nanv = T(NAN);
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                const int a = jb + kG * t;
                if (a < 9) Pq[a * pst] = nan_out ? nanv : Pv[t];
            }
            if (want_A) {
#pragma unroll
                for (int t = 0; t < 12; ++t) {
                    const int e = jb + kG * t;
                    if (e < 45) {
                        int a, b;
                        upper_index(e, a, b);
                        const T v = nan_out ? nanv : Av[t];
                        Aq[(9 * a + b) * ast] = v;
                        if (a != b) Aq[(9 * b + a) * ast] = v;
                    }
                }
            }
        }
    }
    // a point is reported if J <= 0 / bad input, or any of its values was not finite
    const bool grp_nonfinite = group_nonfinite;
    report = bad || grp_nonfinite;
    psi_val = report ? T(NAN) : Psi;
}

// One point on its 4-lane group (all 32 lanes of the warp call this together).
//  mt     the layer-2 tangent weights M (lay.M), in shared or global memory, or null: the
//         layer-2 tangent then folds s_1 into A_2 (one multiply per neuron pair)
//  at     the transposed A_k block (lay.At of the packed weights), in shared memory or,
//         for networks too large for it, in global memory
//  ar     the row-major A_k block (lay.Ar of the packed weights), in shared memory or,
//         for networks too large for it, in global memory
//  F      the point's deformation gradient (replaced by I when it is not admissible)
//  valid  false for padding points: computed on F = I, nothing written
//  Pq, pst / Aq, ast   where row a of P and entry (a, b) of A go: Pq[a*pst], Aq[(9a+b)*ast]
//                      (Aq may be null)
//  dNq, dst            optional: dN/dK and K written to dNq[m*dst], dNq[(D+m)*dst]
//  psi_val, report     the point's Psi (NaN if reported) and whether it is reported
//                      (J <= 0, non-finite input or result); valid in every lane
template <typename T, int NF, int W>
__device__ __forceinline__ void qp_group_update(const T *__restrict__ sw, const NetLayout &lay,
                                                const T *__restrict__ mt, const T *__restrict__ at,
                                                const T *__restrict__ ar, const KinConst<T> &kc, T *qs, int qi,
                                                int jb, T (&F)[9],
                                                bool valid, T *Pq, int64_t pst, T *Aq, int64_t ast, T *dNq,
                                                int64_t dst, T &psi_val, bool &report, const T *krec = nullptr,
                                                int kr = 0) {
    using Cf = CUConf<T, NF, W>;
    constexpr int D = Cf::D, DP = Cf::DP, NH = Cf::NH, NJ = Cf::NJ, NC = Cf::NC;
    const int L = lay.L;
    T *sd = qs;              // s_k at (k-1) W, t_k / D_k at (L+k-1) W
    T *wk = qs + 2 * L * W;  // work area
    const int j0 = jb * NJ;
    T K[D], Jm1;
    PolyChain<T> ch;
    // the kinematic scalars: from the warp's batch record krec[.. kr ..] (kin_batch, FP64),
    // else formed here
    bool bad = krec != nullptr ? kin_read<T, NF>(krec, kr, K, Jm1, ch) : !kin_scalars<T, NF>(F, kc, K, Jm1, &ch);
    if (bad) {
#pragma unroll
        for (int cpt = 0; cpt < 9; ++cpt) F[cpt] = (cpt % 4) == 0 ? T(1) : T(0);
        if (krec == nullptr) kin_scalars<T, NF>(F, kc, K, Jm1, &ch);
    }

    const bool want_A = (Aq != nullptr);  // P alone needs neither F'' nor the tangents
    // ---- forward values
    constexpr int V = 16 / (int)sizeof(T);  // elements per 128-bit shared load
    T npart = T(0);
    for (int k = 1; k <= L; ++k) {
        T y[NJ];
        ldv<NJ>(sw + lay.c + (k - 1) * W + j0, y);
        if (k == 1) {
#pragma unroll
            for (int m = 0; m < D; ++m) {
                T w[NJ];
                ldv<NJ>(sw + lay.W1t + m * W + j0, w);
#pragma unroll
                for (int jj = 0; jj < NJ; ++jj) y[jj] += w[jj] * K[m];
            }
        } else {
            const T *zin = wk + ((k - 1) & 1) * W;
            const T *At = (sizeof(T) == 8 ? at : sw + lay.At) + (k - 2) * W * W + j0;
#pragma unroll 2
            for (int i = 0; i < W; i += V) {
                T zv[V];
                ldv<V>(zin + i, zv);
#pragma unroll
                for (int u = 0; u < V; ++u) {
                    T w[NJ];
                    ldv<NJ>(At + (i + u) * W, w);
#pragma unroll
                    for (int jj = 0; jj < NJ; ++jj) y[jj] += w[jj] * zv[u];
                }
            }
            const T *Bt = sw + lay.Bt + (k - 2) * D * W + j0;
#pragma unroll
            for (int m = 0; m < D; ++m) {
                T w[NJ];
                ldv<NJ>(Bt + m * W, w);
#pragma unroll
                for (int jj = 0; jj < NJ; ++jj) y[jj] += w[jj] * K[m];
            }
        }
        T sv[NJ], tv[NJ], zv[NJ];
#pragma unroll
        for (int jj = 0; jj < NJ; ++jj) {
            if constexpr (sizeof(T) == 8)
                act_tab(y[jj], zv[jj], sv[jj], tv[jj], sw + lay.tab);
            else
                act(y[jj], zv[jj], sv[jj], tv[jj]);
        }
        stv<NJ>(sd + (k - 1) * W + j0, sv);
        if (want_A) stv<NJ>(sd + (L + k - 1) * W + j0, tv);
        if (k < L) {
            stv<NJ>(wk + (k & 1) * W + j0, zv);
        } else {
            T av[NJ];
            ldv<NJ>(sw + lay.a + j0, av);
#pragma unroll
            for (int jj = 0; jj < NJ; ++jj) npart += av[jj] * zv[jj];
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
        T av[NJ], sv[NJ], ybar[NJ];
        ldv<NJ>(sw + lay.a + j0, av);
        ldv<NJ>(sd + (L - 1) * W + j0, sv);
#pragma unroll
        for (int jj = 0; jj < NJ; ++jj) ybar[jj] = sv[jj] * av[jj];
        if (want_A) {  // D_L = F''(y_L) zbar_L for the Hessian
            T tv[NJ];
            ldv<NJ>(sd + (2 * L - 1) * W + j0, tv);
#pragma unroll
            for (int jj = 0; jj < NJ; ++jj) tv[jj] *= av[jj];
            stv<NJ>(sd + (2 * L - 1) * W + j0, tv);
        }
        stv<NJ>(yb + j0, ybar);
#pragma unroll
        for (int m = 0; m < D; ++m) {
            T w[NJ];
            ldv<NJ>(Bt + m * W, w);
#pragma unroll
            for (int jj = 0; jj < NJ; ++jj) dN[m] += w[jj] * ybar[jj];
        }
        __syncwarp();
    }
    for (int k = L; k >= 2; --k) {
        T zb[NJ];
#pragma unroll
        for (int ii = 0; ii < NJ; ++ii) zb[ii] = T(0);
        const T *Ar = ar + (k - 2) * W * W + j0;
#pragma unroll 2
        for (int j = 0; j < W; j += V) {
            T yv[V];
            ldv<V>(yb + j, yv);
#pragma unroll
            for (int u = 0; u < V; ++u) {
                T w[NJ];
                ldv<NJ>(Ar + (j + u) * W, w);
#pragma unroll
                for (int ii = 0; ii < NJ; ++ii) zb[ii] += w[ii] * yv[u];
            }
        }
        __syncwarp();
        const T *Bt = (k - 1 == 1) ? (sw + lay.W1t + j0) : (sw + lay.Bt + (k - 3) * D * W + j0);
        T sv[NJ], ybar[NJ];
        ldv<NJ>(sd + (k - 2) * W + j0, sv);
#pragma unroll
        for (int ii = 0; ii < NJ; ++ii) ybar[ii] = sv[ii] * zb[ii];
        if (want_A) {
            T tv[NJ];
            ldv<NJ>(sd + (L + k - 2) * W + j0, tv);
#pragma unroll
            for (int ii = 0; ii < NJ; ++ii) tv[ii] *= zb[ii];
            stv<NJ>(sd + (L + k - 2) * W + j0, tv);
        }
        stv<NJ>(yb + j0, ybar);
#pragma unroll
        for (int m = 0; m < D; ++m) {
            T w[NJ];
            ldv<NJ>(Bt + m * W, w);
#pragma unroll
            for (int ii = 0; ii < NJ; ++ii) dN[m] += w[ii] * ybar[ii];
        }
        __syncwarp();
    }

    // ---- forward tangents and Hessian (only when A is wanted: P needs dN/dK alone)
    T Hs[NH];
#pragma unroll
    for (int h = 0; h < NH; ++h) Hs[h] = T(0);
    if (want_A) {
        {
            T Dv[NJ];
            ldv<NJ>(sd + L * W + j0, Dv);
#pragma unroll
            for (int jj = 0; jj < NJ; ++jj) {
                T w1[DP];
                ldv<DP>(sw + lay.W1r + (j0 + jj) * DP, w1);
#pragma unroll
                for (int m = 0; m < D; ++m) {
                    const T dm = Dv[jj] * w1[m];
#pragma unroll
                    for (int n = 0; n <= m; ++n) Hs[m * (m + 1) / 2 + n] += dm * w1[n];
                }
            }
        }
        for (int k = 2; k <= L; ++k) {
            const T *At = (sizeof(T) == 8 ? at : sw + lay.At) + (k - 2) * W * W + j0;
            const T *Bt = sw + lay.Bt + (k - 2) * D * W + j0;
            const T *sin = wk + ((k - 1) & 1) * W * DP;
            T *sout = wk + (k & 1) * W * DP;
#pragma unroll 1
            for (int c0 = 0; c0 < NJ; c0 += NC) {
                T acc[NC][D];
#pragma unroll
                for (int m = 0; m < D; ++m) {
                    T w[NC];
                    ldv<NC>(Bt + m * W + c0, w);
#pragma unroll
                    for (int cc = 0; cc < NC; ++cc) acc[cc][m] = w[cc];
                }
                bool use_m = false;
                if constexpr (sizeof(T) == 8) use_m = (k == 2 && mt != nullptr);
                if (use_m) {
                    // J_2 = B_2 + sum_i s_1[i] M[i]: one multiply-add per entry
#pragma unroll 2
                    for (int i = 0; i < W; ++i) {
                        const T s1 = sd[i];
                        T mv[NC * DP];
                        ldv<NC * DP>(mt + ((size_t)i * W + j0 + c0) * DP, mv);
#pragma unroll
                        for (int cc = 0; cc < NC; ++cc)
#pragma unroll
                            for (int m = 0; m < D; ++m) acc[cc][m] += s1 * mv[cc * DP + m];
                    }
                } else if (k == 2) {
#pragma unroll 1
                    for (int i = 0; i < W; i += V) {
                        T s1[V];
                        ldv<V>(sd + i, s1);
#pragma unroll
                        for (int u = 0; u < V; ++u) {
                            // s_1 folded into the weight: NC multiplies instead of D
                            T w1[DP], w[NC];
                            ldv<DP>(sw + lay.W1r + (i + u) * DP, w1);
                            ldv<NC>(At + (i + u) * W + c0, w);
                            tangent_step<T, NC, D>(acc, w, w1, s1[u]);
                        }
                    }
                } else {
#pragma unroll 2
                    for (int i = 0; i < W; ++i) {
                        T sv[DP], w[NC];
                        ldv<DP>(sin + i * DP, sv);
                        ldv<NC>(At + i * W + c0, w);
                        tangent_step<T, NC, D>(acc, w, sv, T(1), false);
                    }
                }
                T Dv[NC], sjv[NC];
                ldv<NC>(sd + (L + k - 1) * W + j0 + c0, Dv);
                ldv<NC>(sd + (k - 1) * W + j0 + c0, sjv);
#pragma unroll
                for (int cc = 0; cc < NC; ++cc) {
#pragma unroll
                    for (int m = 0; m < D; ++m) {
                        const T dm = Dv[cc] * acc[cc][m];
#pragma unroll
                        for (int n = 0; n <= m; ++n) Hs[m * (m + 1) / 2 + n] += dm * acc[cc][n];
                    }
                    if (k < L) {
                        T o[DP];
#pragma unroll
                        for (int m = 0; m < DP; ++m) o[m] = (m < D) ? sjv[cc] * acc[cc][m] : T(0);
                        stv<DP>(sout + (j0 + c0 + cc) * DP, o);
                    }
                }
            }
            __syncwarp();
        }
    }  // want_A

    // an FP64 batch record (PRE) also holds the staging's C, I1, I2 and J^(-1/3)
    const T *pre = (sizeof(T) == 8 && krec != nullptr) ? kin_pre<T, NF>(krec, kr) : nullptr;
    qp_group_finish<T, NF>(sw + lay.n0, sw + lay.K0, kc, qs, qi, jb, F, K, Jm1, ch, bad, valid, npart, dN, Hs,
                           want_A, Pq, pst, Aq, ast, dNq, dst, psi_val, report, pre);
}

}  // namespace commet
