// Device-side kinematics and activation helpers shared by the constitutive kernels.
//
// The kinematic layer (Sec. 2.2, eq. comp-se; invariants eq. 454; isochoric
// invariants App. A.2) is evaluated in material form: K_m(F), g_m = dK_m/dF and the
// second derivatives contracted with the network gradient, sum_m c_m d2K_m/dF dF,
// which is written as a short sum of structured terms instead of d 81-entry tensors:
//
//   A_iJkL = sum_mn N_mn g_m[iJ] g_n[kL]
//          + U_iJ H_kL + H_iJ U_kL + beta H_iJ H_kL + gamma F_iJ F_kL        (rank one)
//          - eta H_iL H_kJ + zeta F_iL F_kJ
//          + sum_f 2 c5f (F_iL a_k A_J + a_i A_L F_kJ)                        (index swap)
//          + d_ik X_JL + Y_ik d_JL + sum_f 2 c5f B_ik A_J A_L                 (products)
//
// with H = F^{-T}, B = F F^T, a = F A, v = C A, and coefficients built from
// c_m = dN/dK_m, J, I1, I2, kappa (see stage_kinematics below).
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "../../include/commet.h"
#include "act_df.cuh"

namespace commet {

template <typename T>
struct KinConst {
    int kin;          // COMMET_KIN_*
    int stress_free;  // shift by n0
    T kappa;
    T fib[2][3];
};

// ---------------------------------------------------------------- activation
// softplus z = log(1 + e^y), s = z' = logistic(y), t = z'' = s (1 - s) = e/(1+e)^2
// with e = exp(-|y|) so that nothing overflows.
__device__ __forceinline__ void act(double y, double &z, double &s, double &t) {
    const double e = exp(-fabs(y));
    const double r = 1.0 / (1.0 + e);
    z = fmax(y, 0.0) + log1p(e);
    s = (y >= 0.0) ? r : e * r;
    t = e * r * r;
}
__device__ __forceinline__ void act(float y, float &z, float &s, float &t) {
    const float e = __expf(-fabsf(y));
    const float r = __fdividef(1.0f, 1.0f + e);  // 1 + e in [1, 2]: the approximate reciprocal is within 2 ulp
    z = fmaxf(y, 0.0f) + __logf(1.0f + e);  // absolute error ~1e-7: within the FP32 tolerance
    s = (y >= 0.0f) ? r : e * r;
    t = e * r * r;
}
__device__ __forceinline__ void act_value_slope(double y, double &z, double &s) {
    const double e = exp(-fabs(y));
    const double r = 1.0 / (1.0 + e);
    z = fmax(y, 0.0) + log1p(e);
    s = (y >= 0.0) ? r : e * r;
}
__device__ __forceinline__ void act_value_slope(float y, float &z, float &s) {
    const float e = __expf(-fabsf(y));
    const float r = __fdividef(1.0f, 1.0f + e);  // 1 + e in [1, 2]: the approximate reciprocal is within 2 ulp
    z = fmaxf(y, 0.0f) + log1pf(e);
    s = (y >= 0.0f) ? r : e * r;
}

// FP64 softplus triple from float-pair tables in shared memory: act_df.cuh
__device__ __forceinline__ void act_tab(double y, double &z, double &s, double &t, const double *tab) {
    actdf::softplus3(y, z, s, t, reinterpret_cast<const actdf::f2 *>(tab));
}

// x^(-1/3) for x > 0: an FP32 seed 2^(-log2(x)/3) from the MUFU (relative error about
// 2^-21) and two Newton steps y <- y + y (1 - x y^3)/3 in FP64 (2^-42, then rounding
// level): 10 FP64 operations, where libm's rcbrt costs several times that on the FP64
// pipe. Arguments outside [2^-126, 2^120) take libm's rcbrt.
__device__ __forceinline__ double dev_rcbrt(double x) {
    const int hi = __double2hiint(x);
    if (hi < 0x38100000 || hi >= 0x47700000) return rcbrt(x);
    // truncated FP32 copy of x (exponent rebiased from 1023 to 127); the seed converted to
    // double exactly with integer operations
    const float xf = __int_as_float((int)((unsigned)(hi - 0x38000000) << 3));
    double y = actdf::f_to_d(__expf(-0.33333334f * __logf(xf)));
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const double y3 = y * y * y;
        const double r = fma(-x, y3, 1.0);
        y = fma(y * (1.0 / 3.0), r, y);
    }
    return y;
}
__device__ __forceinline__ float dev_rcbrt(float x) { return rcbrtf(x); }
__device__ __forceinline__ bool dev_finite(double x) { return isfinite(x); }
__device__ __forceinline__ bool dev_finite(float x) { return isfinite(x); }

// ------------------------------------------------------------ basic kinematics

// cofactor of F (cof F = J F^{-T}) and J = det F
template <typename T>
__device__ __forceinline__ void cof_det(const T *F, T *cof, T &J) {
    cof[0] = F[4] * F[8] - F[5] * F[7];
    cof[1] = F[5] * F[6] - F[3] * F[8];
    cof[2] = F[3] * F[7] - F[4] * F[6];
    cof[3] = F[2] * F[7] - F[1] * F[8];
    cof[4] = F[0] * F[8] - F[2] * F[6];
    cof[5] = F[1] * F[6] - F[0] * F[7];
    cof[6] = F[1] * F[5] - F[2] * F[4];
    cof[7] = F[2] * F[3] - F[0] * F[5];
    cof[8] = F[0] * F[4] - F[1] * F[3];
    J = F[0] * cof[0] + F[1] * cof[1] + F[2] * cof[2];
}

// C = F^T F (full 3x3)
template <typename T>
__device__ __forceinline__ void right_cg(const T *F, T *C) {
#pragma unroll
    for (int I = 0; I < 3; ++I)
#pragma unroll
        for (int J = I; J < 3; ++J) {
            T s = F[I] * F[J] + F[3 + I] * F[3 + J] + F[6 + I] * F[6 + J];
            C[3 * I + J] = s;
            C[3 * J + I] = s;
        }
}

// I2 = (tr^2 C - tr C^2)/2 as the sum of the principal 2x2 minors of the symmetric C:
// six operations instead of eleven
template <typename T>
__device__ __forceinline__ T second_invariant(const T *C) {
    T s = C[0] * C[4];
    s += C[0] * C[8];
    s += C[4] * C[8];
    s -= C[1] * C[1];
    s -= C[2] * C[2];
    s -= C[5] * C[5];
    return s;
}

// B = F F^T (full 3x3)
template <typename T>
__device__ __forceinline__ void left_cg(const T *F, T *B) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            T s = F[3 * i] * F[3 * j] + F[3 * i + 1] * F[3 * j + 1] + F[3 * i + 2] * F[3 * j + 2];
            B[3 * i + j] = s;
            B[3 * j + i] = s;
        }
}

// J - 1 = det F - 1 in double precision. The volumetric penalty 2 kappa (J - 1) and
// the J - 1 network input cancel to a small difference near J = 1, so the FP32 path
// also evaluates this one quantity in FP64 (a few dozen DFMA per point).
__device__ __forceinline__ double det_minus_one(const double *F) {
    double cof[9], J;
    cof_det(F, cof, J);
    return J - 1.0;
}
__device__ __forceinline__ float det_minus_one(const float *F) {
    double Fd[9], cof[9], J;
#pragma unroll
    for (int a = 0; a < 9; ++a) Fd[a] = (double)F[a];
    cof_det(Fd, cof, J);
    return (float)(J - 1.0);
}

// Polyconvex kinematic layer (App. C): K_m = phi_m(I_m) of the invariants
// I = (Ibar1, Ibar2, J), phi = (I - 3, I^{3/2} - 3^{3/2}, (I - 1)^2). The staged kinematic
// derivatives are those of I_m, so the network's gradient c and Hessian N are carried over
// to invariant space by the chain rule:
//   dPsi/dI_m = phi'_m c_m,   d2Psi/dI_m dI_n = phi'_m phi'_n N_mn + delta_mn phi''_m c_m.
template <typename T>
struct PolyChain {
    T d1[3], d2[3];  // phi'_m, phi''_m at the point
};

template <typename T>
__device__ __forceinline__ void poly_inputs(T *K, T Jm1, PolyChain<T> *ch) {
    const T Ib2 = K[1];
    const T sq = sqrt(Ib2);  // Ibar2 >= 3 for every admissible F
    K[0] -= T(3);
    K[1] = Ib2 * sq - T(5.196152422706632);  // 3^{3/2}
    K[2] = Jm1 * Jm1;
    if (ch != nullptr) {
        ch->d1[0] = T(1);
        ch->d1[1] = T(1.5) * sq;
        ch->d1[2] = T(2) * Jm1;
        ch->d2[0] = T(0);
        ch->d2[1] = T(0.75) / sq;
        ch->d2[2] = T(2);
    }
}

// c <- phi' c and the packed lower triangle Hs (Hs[m (m + 1) / 2 + n], n <= m) <- the
// invariant-space Hessian, both in place (D = 3).
template <typename T>
__device__ __forceinline__ void poly_to_invariants(const PolyChain<T> &ch, T *c, T *Hs) {
#pragma unroll
    for (int m = 0; m < 3; ++m) {
#pragma unroll
        for (int n = 0; n <= m; ++n) Hs[m * (m + 1) / 2 + n] *= ch.d1[m] * ch.d1[n];
        Hs[m * (m + 1) / 2 + m] += ch.d2[m] * c[m];
    }
#pragma unroll
    for (int m = 0; m < 3; ++m) c[m] *= ch.d1[m];
}

// Kinematic scalars K (D = 3 + 2 NF entries) and Jm1 = J - 1. Returns false if
// J <= 0 or F is not finite. With the polyconvex layer, ch (if given) receives phi', phi''.
template <typename T, int NF>
__device__ __forceinline__ bool kin_scalars(const T *F, const KinConst<T> &kc, T *K, T &Jm1,
                                            PolyChain<T> *ch = nullptr) {
    Jm1 = det_minus_one(F);
    const T J = T(1) + Jm1;
    T C[9];
    right_cg(F, C);
    const T I1 = C[0] + C[4] + C[8];
    const T I2 = second_invariant(C);
    const bool ok = (J > T(0)) && dev_finite(Jm1) && dev_finite(I1);
    const T r3 = dev_rcbrt(ok ? J : T(1));
    const T jm23 = r3 * r3;
    K[0] = jm23 * I1;
    K[1] = jm23 * jm23 * I2;
    K[2] = J;
    if (kc.kin == COMMET_KIN_ISO_SHIFTED) {
        K[0] -= T(3);
        K[1] -= T(3);
        K[2] = Jm1;
    } else if (NF == 0 && kc.kin == COMMET_KIN_POLYCONVEX) {
        poly_inputs<T>(K, Jm1, ch);
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        T v[3];
#pragma unroll
        for (int I = 0; I < 3; ++I) v[I] = C[3 * I] * kc.fib[f][0] + C[3 * I + 1] * kc.fib[f][1] + C[3 * I + 2] * kc.fib[f][2];
        K[3 + f] = v[0] * kc.fib[f][0] + v[1] * kc.fib[f][1] + v[2] * kc.fib[f][2];
        K[3 + NF + f] = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    }
    return ok;
}

// Layout of the per-qp staging area written by stage_kinematics (units of T).
template <int D, int NF>
struct Stage {
    static constexpr int g = 0;             // [D][9] g_m = dK_m/dF
    static constexpr int F = 9 * D;         // [9]
    static constexpr int H = F + 9;         // [9] F^{-T}
    static constexpr int U = H + 9;         // [9]
    static constexpr int X = U + 9;         // [9] (J, L)
    static constexpr int Y = X + 9;         // [9] (i, k)
    static constexpr int Bm = Y + 9;        // [9] left Cauchy-Green
    static constexpr int aA = Bm + 9;       // [NF][9] a_f (x) A_f, [3k+J] = a_k A_J
    static constexpr int AA = aA + 9 * NF;  // [NF][9] A_f (x) A_f
    static constexpr int sc = AA + 9 * NF;  // beta, gamma, eta, zeta, 2 c5f (NF), 2 kappa (J-1) J
    static constexpr int size = sc + 5 + NF;
};

// Writes the quantities every entry of P and A needs into the point's staging area.
// The four lanes of a point's group call it together; lane `lane4` (0..3) writes the
// components a = lane4, lane4 + 4, lane4 + 8 of every 9-component quantity, so that all
// lanes run the same instructions (GB300 bills a divergent branch's FP64 instructions to
// every lane of the warp). Scalars and the fibre vectors a = F A, v = C A, F v are formed
// in every lane. c[] = dN/dK - n0; Jm1 = J - 1 from det_minus_one. With G_ONLY, only what
// P needs is staged: the kinematic gradients g_m, F, F^{-T} and 2 kappa (J - 1) J.
// pre (FP64, optional): C[9], I1, I2 and J^(-1/3) of this F already formed, at stride 32
// (a batch record, see kin_batch), instead of forming them in every lane.
template <typename T, int NF, bool G_ONLY = false>
__device__ __forceinline__ void stage_kinematics(const T *F, const KinConst<T> &kc, const T *c, T Jm1, int lane4,
                                                 T *st, const T *pre = nullptr) {
    constexpr int D = 3 + 2 * NF;
    using S = Stage<D, NF>;
    T C[9];
    // FP32 (bound by latency, not by FP64 instructions) forms the cofactor matrix in
    // straight-line code; FP64 lanes form only their own entries below
    T cof[9], Jc;
    if constexpr (sizeof(T) != 8) cof_det(F, cof, Jc);
    const T J = T(1) + Jm1;
    T I1, I2, r3;
    if (pre != nullptr) {
#pragma unroll
        for (int i = 0; i < 9; ++i) C[i] = pre[i * 32];
        I1 = pre[9 * 32];
        I2 = pre[10 * 32];
        r3 = pre[11 * 32];
    } else {
        right_cg(F, C);
        I1 = C[0] + C[4] + C[8];
        I2 = second_invariant(C);
        r3 = dev_rcbrt(J);
    }
    const T jm23 = r3 * r3, jm43 = jm23 * jm23;
    const T iJ = jm23 * r3;  // 1/J = (J^(-1/3))^3
    const T p1 = T(-2) / T(3), p2 = T(-4) / T(3);
    const T c1 = c[0], c2 = c[1], c3 = c[2];
    const T k2 = T(2) * kc.kappa;
    T af[NF > 0 ? NF : 1][3], vf[NF > 0 ? NF : 1][3], Fvf[NF > 0 ? NF : 1][3];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        const T *A0 = kc.fib[f];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            af[f][i] = F[3 * i] * A0[0] + F[3 * i + 1] * A0[1] + F[3 * i + 2] * A0[2];
            vf[f][i] = C[3 * i] * A0[0] + C[3 * i + 1] * A0[1] + C[3 * i + 2] * A0[2];
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) Fvf[f][i] = F[3 * i] * vf[f][0] + F[3 * i + 1] * vf[f][1] + F[3 * i + 2] * vf[f][2];
    }
    const T x0 = T(2) * c1 * jm23 + T(2) * I1 * c2 * jm43;
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        const int a = lane4 + 4 * t;
        if (a < 9) {
            const int p = a / 3, q = a - 3 * p;  // a = 3 p + q
            // FP64: this lane's cofactor entry only (the lanes share one instruction stream)
            T cofa;
            if constexpr (sizeof(T) == 8) {
                const int pa1 = p == 2 ? 0 : p + 1, pa2 = p == 0 ? 2 : p - 1;
                const int qa1 = q == 2 ? 0 : q + 1, qa2 = q == 0 ? 2 : q - 1;
                cofa = F[3 * pa1 + qa1] * F[3 * pa2 + qa2] - F[3 * pa1 + qa2] * F[3 * pa2 + qa1];
            } else {
                cofa = cof[a];
            }
            const T Fa = F[a], Ha = cofa * iJ;
            const T FC = F[3 * p] * C[q] + F[3 * p + 1] * C[3 + q] + F[3 * p + 2] * C[6 + q];
            const T gI2 = T(2) * (I1 * Fa - FC);  // raw dI2/dF = 2 (I1 F - F C)
            st[S::g + a] = jm23 * (T(2) * Fa + p1 * I1 * Ha);
            st[S::g + 9 + a] = jm43 * (gI2 + p2 * I2 * Ha);
            st[S::g + 18 + a] = cofa;
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                const T *A0 = kc.fib[f];
                st[S::g + 9 * (3 + f) + a] = T(2) * af[f][p] * A0[q];
                st[S::g + 9 * (3 + NF + f) + a] = T(2) * (af[f][p] * vf[f][q] + Fvf[f][p] * A0[q]);
            }
            st[S::F + a] = Fa;
            st[S::H + a] = Ha;
            if (!G_ONLY) {
                const T Bpq = F[3 * p] * F[3 * q] + F[3 * p + 1] * F[3 * q + 1] + F[3 * p + 2] * F[3 * q + 2];
                st[S::U + a] = c1 * jm23 * p1 * T(2) * Fa + c2 * jm43 * p2 * gI2;
                st[S::Bm + a] = Bpq;
                T X = (p == q ? x0 : T(0)) - T(2) * c2 * jm43 * C[a];
                T Y = -T(2) * c2 * jm43 * Bpq;
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    const T *A0 = kc.fib[f];
                    const T c4 = c[3 + f], c5 = c[3 + NF + f];
                    X += T(2) * c4 * A0[p] * A0[q] + T(2) * c5 * (A0[p] * vf[f][q] + vf[f][p] * A0[q]);
                    Y += T(2) * c5 * af[f][p] * af[f][q];
                    st[S::aA + 9 * f + a] = af[f][p] * A0[q];
                    st[S::AA + 9 * f + a] = A0[p] * A0[q];
                }
                st[S::X + a] = X;
                st[S::Y + a] = Y;
            }
        }
    }
    if (G_ONLY && lane4 == 0) st[S::sc + 4 + NF] = k2 * Jm1 * J;
    if (!G_ONLY && lane4 == 0) {
        st[S::sc + 0] = c1 * jm23 * p1 * p1 * I1 + c2 * jm43 * p2 * p2 * I2 + c3 * J + k2 * J * J + k2 * Jm1 * J;
        st[S::sc + 1] = T(4) * c2 * jm43;
        st[S::sc + 2] = c1 * jm23 * p1 * I1 + c2 * jm43 * p2 * I2 + c3 * J + k2 * Jm1 * J;
        st[S::sc + 3] = -T(2) * c2 * jm43;
#pragma unroll
        for (int f = 0; f < NF; ++f) st[S::sc + 4 + f] = T(2) * c[3 + NF + f];
        st[S::sc + 4 + NF] = k2 * Jm1 * J;
    }
}

// ------------------------------------------------------------ spatial form
// Voigt pairs in the order (11, 22, 33, 23, 13, 12).
__host__ __device__ constexpr int voigt_i(int v) { return v < 3 ? v : (v == 3 ? 1 : 0); }
__host__ __device__ constexpr int voigt_j(int v) { return v < 3 ? v : (v == 5 ? 1 : 2); }
// Voigt slot of the symmetric index pair (i, j).
__host__ __device__ constexpr int voigt_of(int i, int j) {
    return i == j ? i : ((i + j) == 3 ? 3 : ((i + j) == 2 ? 4 : 5));
}
// Position of the Voigt pair (I, J) in the row-major upper triangle of the 6 x 6 matrix.
__host__ __device__ constexpr int voigt_upper_pos(int I, int J) {
    return I <= J ? I * 6 - I * (I - 1) / 2 + (J - I) : J * 6 - J * (J - 1) / 2 + (I - J);
}
// Inverse of voigt_upper_pos for e in [0, 21).
__device__ __forceinline__ void voigt_upper_pair(int e, int &I, int &J) {
    I = 0;
    int rem = e;
#pragma unroll
    for (int r = 0; r < 5; ++r)
        if (rem >= 6 - I) {
            rem -= 6 - I;
            ++I;
        }
    J = I + rem;
}

// Push-forward of one point's P (9) and A (81) to the Kirchhoff stress and the spatial
// stiffness in Voigt form (App. A.1):
//   tau_ij = P_iJ F_jJ,   c_ijkl = F_jJ A_iJkL F_lL - delta_ik tau_jl,
// tau[v] for the 6 Voigt pairs, c[e] for the 21 upper-triangle pairs (I, J) of the 6 x 6
// Voigt matrix. Fs, Ps, As are in shared memory; the 4 lanes of the point's group share
// the 27 outputs (lane4 takes o = lane4 + 4 t) and write them at tau[o * stride],
// c[(o - 6) * stride] (c may be null: stress only).
template <typename T>
__device__ __forceinline__ void push_forward_group(const T *Fs, const T *Ps, const T *As, int lane4, bool valid,
                                                   T *tau, T *c, int64_t stride) {
#pragma unroll
    for (int t = 0; t < 7; ++t) {
        const int o = lane4 + 4 * t;
        if (o >= 27 || (o >= 6 && c == nullptr)) continue;
        int i, j, k = 0, l = 0;
        if (o < 6) {
            i = voigt_i(o);
            j = voigt_j(o);
        } else {
            int I, J;
            voigt_upper_pair(o - 6, I, J);
            i = voigt_i(I);
            j = voigt_j(I);
            k = voigt_i(J);
            l = voigt_j(J);
        }
        T v;
        if (o < 6) {
            v = Ps[3 * i] * Fs[3 * j] + Ps[3 * i + 1] * Fs[3 * j + 1] + Ps[3 * i + 2] * Fs[3 * j + 2];
        } else {
            v = T(0);
#pragma unroll
            for (int Jc = 0; Jc < 3; ++Jc) {
                const T *Ar = As + (3 * i + Jc) * 9 + 3 * k;
                v += Fs[3 * j + Jc] * (Ar[0] * Fs[3 * l] + Ar[1] * Fs[3 * l + 1] + Ar[2] * Fs[3 * l + 2]);
            }
            if (i == k) v -= Ps[3 * j] * Fs[3 * l] + Ps[3 * j + 1] * Fs[3 * l + 1] + Ps[3 * j + 2] * Fs[3 * l + 2];
        }
        if (valid) {
            if (o < 6)
                tau[o * stride] = v;
            else
                c[(o - 6) * stride] = v;
        }
    }
}

// P_a alone (no tangent): sum_m c_m g_m[a] + 2 kappa (J - 1) J H_a.
template <typename T, int NF>
__device__ __forceinline__ T assemble_P(int a, const T *st, const T *c) {
    constexpr int D = 3 + 2 * NF;
    using S = Stage<D, NF>;
    T p = T(0);
#pragma unroll
    for (int m = 0; m < D; ++m) p += c[m] * st[S::g + 9 * m + a];
    return p + st[S::sc + 4 + NF] * st[S::H + a];
}

// Row a = 3i + J of P and A from the staged quantities; Hs is the packed lower
// triangle of d2N/dK2 (index m*(m+1)/2 + n, n <= m), c = dN/dK - n0.
template <typename T, int NF>
__device__ __forceinline__ void assemble_row(int a, const T *st, const T *Hs, const T *c, T &Pa, T *Arow) {
    constexpr int D = 3 + 2 * NF;
    using S = Stage<D, NF>;
    const int i = a / 3, J_ = a % 3;
    T u[D];
#pragma unroll
    for (int n = 0; n < D; ++n) u[n] = T(0);
    T p = T(0);
#pragma unroll
    for (int m = 0; m < D; ++m) {
        const T gma = st[S::g + 9 * m + a];
        p += c[m] * gma;
#pragma unroll
        for (int n = 0; n < D; ++n) {
            const int idx = (m >= n) ? (m * (m + 1) / 2 + n) : (n * (n + 1) / 2 + m);
            u[n] += gma * Hs[idx];
        }
    }
    const T Ha = st[S::H + a], Fa = st[S::F + a], Ua = st[S::U + a];
    Pa = p + st[S::sc + 4 + NF] * Ha;
    const T beta = st[S::sc + 0], gamma = st[S::sc + 1], eta = st[S::sc + 2], zeta = st[S::sc + 3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int L = 0; L < 3; ++L) {
            const int b = 3 * k + L;
            T s = T(0);
#pragma unroll
            for (int n = 0; n < D; ++n) s += u[n] * st[S::g + 9 * n + b];
            const T Hb = st[S::H + b];
            s += Ua * Hb;
            s += Ha * st[S::U + b];
            s += (beta * Ha) * Hb;
            s += (gamma * Fa) * st[S::F + b];
            const T FiL = st[S::F + 3 * i + L], FkJ = st[S::F + 3 * k + J_];
            s += (-eta * st[S::H + 3 * i + L]) * st[S::H + 3 * k + J_];
            s += (zeta * FiL) * FkJ;
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                const T c5x2 = st[S::sc + 4 + f];
                s += c5x2 * (FiL * st[S::aA + 9 * f + 3 * k + J_] + st[S::aA + 9 * f + 3 * i + L] * FkJ +
                             st[S::Bm + 3 * i + k] * st[S::AA + 9 * f + 3 * J_ + L]);
            }
            if (i == k) s += st[S::X + 3 * J_ + L];
            if (J_ == L) s += st[S::Y + 3 * i + k];
            Arow[b] = s;
        }
}


// FP64 A assembly with the structured terms' scalars folded into per-point vectors, so
// that each term of an entry is one fused multiply-add (GB300 bills every FP64 warp
// instruction 16 SM clocks): lane4 writes components a = lane4, lane4 + 4, lane4 + 8 of
//   V = U + (beta/2) H, G = gamma F, E = -eta H, Z = zeta F,
//   XY[3i + J] = X[3J + J] + Y[3i + i]      (the two Kronecker terms of a diagonal entry)
//   per fibre f: aA'_f = 2 c5f aA_f, Bm'_f = 2 c5f Bm
// at pre[0, 9, 18, 27, 36] and pre[45 + 18 f], pre[54 + 18 f]. Then
//   A_ab = d_ik d_JL XY + d_ik (1 - d_JL) X_JL + (1 - d_ik) d_JL Y_ik + u_a . g_b
//        + V_a H_b + H_a V_b + G_a F_b + E_iL H_kJ + Z_iL F_kJ
//        + sum_f (F_iL aA'_f,kJ + aA'_f,iL F_kJ + Bm'_f,ik AA_f,JL),
// the same sum as assemble_entry with D + 5 + 3 NF FP64 operations instead of D + 12 + 4 NF.
template <typename T, int NF>
__device__ __forceinline__ void prescale_structured(const T *st, int lane4, T *pre) {
    constexpr int D = 3 + 2 * NF;
    using S = Stage<D, NF>;
    const T hb = T(0.5) * st[S::sc + 0], gamma = st[S::sc + 1], meta = -st[S::sc + 2], zeta = st[S::sc + 3];
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        const int a = lane4 + 4 * t;
        if (a < 9) {
            const int i = a / 3, J_ = a - 3 * i;
            const T Ha = st[S::H + a], Fa = st[S::F + a];
            pre[a] = hb * Ha + st[S::U + a];
            pre[9 + a] = gamma * Fa;
            pre[18 + a] = meta * Ha;
            pre[27 + a] = zeta * Fa;
            pre[36 + a] = st[S::X + 4 * J_] + st[S::Y + 4 * i];
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                const T c5x2 = st[S::sc + 4 + f];
                pre[45 + 18 * f + a] = c5x2 * st[S::aA + 9 * f + a];
                pre[54 + 18 * f + a] = c5x2 * st[S::Bm + a];
            }
        }
    }
}

template <typename T, int NF, int DP>
__device__ __forceinline__ T assemble_entry_pre(int a, int b, const T *st, const T *ust, const T *pre) {
    constexpr int D = 3 + 2 * NF;
    using S = Stage<D, NF>;
    const int i = a / 3, J_ = a - 3 * i, k = b / 3, L = b - 3 * k;
    const int iL = 3 * i + L, kJ = 3 * k + J_;
    T s = (i == k) ? ((J_ == L) ? pre[36 + a] : st[S::X + 3 * J_ + L]) : ((J_ == L) ? st[S::Y + 3 * i + k] : T(0));
#pragma unroll
    for (int n = 0; n < D; ++n) s += ust[a * DP + n] * st[S::g + 9 * n + b];
    s += pre[a] * st[S::H + b];
    s += st[S::H + a] * pre[b];
    s += pre[9 + a] * st[S::F + b];
    s += pre[18 + iL] * st[S::H + kJ];
    const T FiL = st[S::F + iL], FkJ = st[S::F + kJ];
    s += pre[27 + iL] * FkJ;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        s += FiL * pre[45 + 18 * f + kJ];
        s += pre[45 + 18 * f + iL] * FkJ;
        s += pre[54 + 18 * f + 3 * i + k] * st[S::AA + 9 * f + 3 * J_ + L];
    }
    return s;
}

// The e-th (0 <= e < 45) entry of the upper triangle of a symmetric 9 x 9 matrix, row by row.
__device__ __forceinline__ void upper_index(int e, int &a, int &b) {
    int r = 0;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const bool step = e >= 9 - r;
        e -= step ? 9 - r : 0;
        r += step ? 1 : 0;
    }
    a = r;
    b = r + e;
}

}  // namespace commet
