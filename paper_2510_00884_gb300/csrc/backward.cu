// Backward (adjoint) of the constitutive update for an upstream G = dL/dP per point:
//   dL/dF_q     = G_q : A_q
//   dL/dtheta   = sum_q d/dtheta [ G_q : P_q(theta) ] = sum_q d/dtheta [ grad_K N . r_q ],
//                 r_q,m = G_q : dK_m/dF
// (the network's weights enter P only through grad_K N; the volumetric penalty does
// not depend on theta). Nothing is stored between forward and backward: each point's
// forward is recomputed here.
//
// Per point (a group of 4 lanes, as in the forward kernel): the network is evaluated
// with a forward tangent along r (zdot_k = F'(y_k) ydot_k, ydot_k = A_k zdot_{k-1} + B_k r),
// then differentiated in reverse:
//   ydotbar_k = s_k zdotbar_k,  ybar_k = s_k zbar_k + t_k ydot_k zdotbar_k,
//   zbar_{k-1} = A_k^T ybar_k,  zdotbar_{k-1} = A_k^T ydotbar_k,  zdotbar_L = a, zbar_L = 0,
//   dA_k += ybar_k z_{k-1}^T + ydotbar_k zdot_{k-1}^T, dB_k += ybar_k K^T + ydotbar_k r^T,
//   dc_k += ybar_k, da += zdot_L, db += r.
// zdotbar follows the plain adjoint recursion, so ydotbar also gives dN/dK, and
// sum_k B_k^T ybar_k is the Hessian-vector product (d2N/dK2) r; with them
//   dL/dF = sum_n ((d2N/dK2) r)_n g_n + sum_a G_a S_ab,
// S being the structured (non rank-one) part of A.
//
// The sums over points of the weight gradients are formed per CTA tile as small
// outer-product GEMMs into shared-memory accumulators owned by fixed threads, written
// once per CTA, and reduced over CTAs in index order by a second kernel: the result is
// bitwise reproducible for a given device.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "closed_form.cuh"
#include "device_math.cuh"
#include "internal.h"
#include "qp_body.cuh"

namespace commet {

namespace {

// kG (lanes per point) and kQPW (points per warp) come from qp_body.cuh

// Warps per CTA (8 points each: the CTA tile): 4 in FP64, 8 in FP32; 64-wide networks,
// whose weights, accumulators and slabs would not fit, run half as many.
template <typename T>
struct BwConf {
    static constexpr int warps = sizeof(T) == 8 ? 4 : 8;
    static constexpr int min_warps = warps / 2;
    static constexpr int least_warps = sizeof(T) == 8 ? 1 : 2;  // smallest tile of any launch
};

// Per-point slab (elements of T): K[d] then 1, r[d] then 0 (the bias column of the W x d
// weight-gradient sums), z_k/zdot_k (k = 1..L-1), zdot_L, and per layer s_k, t_k, ydot_k;
// then ybar, ydotbar of the current layer; padded.
struct BwSlab {
    int K, r, z, zd, zdL, s, t, yd, yb, ydb, size;
};

__host__ __device__ inline int bw_round4(int x) { return (x + 3) / 4 * 4; }

__host__ __device__ inline BwSlab bw_slab(int d, int W, int L, int NF, int tsize) {
    BwSlab b{};
    int o = 0;  // every array starts on a 4-element boundary (128-bit shared loads)
    b.K = o; o = bw_round4(o + d + 1);
    b.r = o; o = bw_round4(o + d + 1);
    b.z = o; o = bw_round4(o + (L - 1) * W);
    b.zd = o; o = bw_round4(o + (L - 1) * W);
    b.zdL = o; o = bw_round4(o + W);
    b.s = o; o = bw_round4(o + L * W);
    b.t = o; o = bw_round4(o + L * W);
    b.yd = o; o = bw_round4(o + L * W);
    b.yb = o; o = bw_round4(o + W);
    b.ydb = o; o = bw_round4(o + W);
    // staged kinematics, then G and its precomputed contractions (BwPre below)
    const int stage = 9 * d + 54 + 18 * NF + 5 + NF + 30 + 9 * NF;
    int raw = o > stage ? o : stage;
    int words = raw * tsize / 4;
    words = (words + 31) / 32 * 32 + 4;
    b.size = words * 4 / tsize;
    return b;
}

// Offsets (units of T) of G = dL/dP and of the contractions of G with the staged
// kinematics that every row of G : S uses, placed after the staged kinematics.
template <int D, int NF>
struct BwPre {
    static constexpr int G = Stage<D, NF>::size;  // [9]
    static constexpr int Nh = G + 9;              // [9] (G^T H)_JL at 3 J + L
    static constexpr int Nf = Nh + 9;             // [9] (G^T F)_JL
    static constexpr int sc = Nf + 9;             // G : U, G : H, G : F
    static constexpr int a = sc + 3;              // [NF][3] a_f = F A_f
    static constexpr int v1 = a + 3 * NF;         // [NF][3] F^T G A_f
    static constexpr int v23 = v1 + 3 * NF;       // [NF][3] F G^T a_f + B G A_f
    static constexpr int size = v23 + 3 * NF;
};

// The group of 4 lanes (lane4) of a point writes G and the contractions above; lanes
// split the components (a = lane4 + 4 t) and, with two fibres, the fibres, so that the
// group's FP64 instructions are shared rather than repeated.
template <typename T, int NF>
__device__ __forceinline__ void structured_pre(T *st, const T (&G)[9], const KinConst<T> &kc, int lane4) {
    constexpr int D = 3 + 2 * NF;
    using S = Stage<D, NF>;
    using R = BwPre<D, NF>;
    const T *F = st + S::F, *H = st + S::H, *U = st + S::U, *Bm = st + S::Bm;
    T *Gs = st + R::G;
#pragma unroll
    for (int a = 0; a < 9; ++a)
        if ((a & 3) == lane4) Gs[a] = G[a];
    __syncwarp();
    T gu = 0, gh = 0, gf = 0;
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        const int e = lane4 + 4 * t;
        if (e < 9) {
            const T g = Gs[e];
            gu += g * U[e];
            gh += g * H[e];
            gf += g * F[e];
            const int J = e / 3, L = e - 3 * J;
            T nh = 0, nf = 0;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                nh += Gs[3 * i + J] * H[3 * i + L];
                nf += Gs[3 * i + J] * F[3 * i + L];
            }
            st[R::Nh + e] = nh;
            st[R::Nf + e] = nf;
        }
    }
#pragma unroll
    for (int msk = 1; msk <= 2; msk <<= 1) {
        gu += __shfl_xor_sync(0xffffffffu, gu, msk);
        gh += __shfl_xor_sync(0xffffffffu, gh, msk);
        gf += __shfl_xor_sync(0xffffffffu, gf, msk);
    }
    if (lane4 == 0) {
        st[R::sc + 0] = gu;
        st[R::sc + 1] = gh;
        st[R::sc + 2] = gf;
    }
    if constexpr (NF > 0) {
        // fibre f = lane4 / 2 (lanes 0, 2 write): a = F A, GA = G A, v1 = F^T GA,
        // w = G^T a, v23 = F w + B GA (B symmetric)
        const int f = lane4 >> 1;
        if (f < NF) {
            const T *A0 = kc.fib[f];
            T a[3], GA[3], w[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                a[i] = F[3 * i] * A0[0] + F[3 * i + 1] * A0[1] + F[3 * i + 2] * A0[2];
                GA[i] = Gs[3 * i] * A0[0] + Gs[3 * i + 1] * A0[1] + Gs[3 * i + 2] * A0[2];
            }
#pragma unroll
            for (int J = 0; J < 3; ++J) w[J] = Gs[J] * a[0] + Gs[3 + J] * a[1] + Gs[6 + J] * a[2];
            if ((lane4 & 1) == 0) {
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    st[R::a + 3 * f + i] = a[i];
                    st[R::v1 + 3 * f + i] = F[i] * GA[0] + F[3 + i] * GA[1] + F[6 + i] * GA[2];
                    st[R::v23 + 3 * f + i] = F[3 * i] * w[0] + F[3 * i + 1] * w[1] + F[3 * i + 2] * w[2] +
                                             Bm[i] * GA[0] + Bm[3 + i] * GA[1] + Bm[6 + i] * GA[2];
                }
            }
        }
    }
}

// sum_a G_a S_ab for the structured part S of A (see device_math.cuh) and row b, from
// the staged kinematics and structured_pre:
//   (G:U) H_b + (G:H) U_b + beta (G:H) H_b + gamma (G:F) F_b - eta (H G^T H)_b
//   + zeta (F G^T F)_b + (G X)_b + (Y G)_b
//   + sum_f 2 c5_f [a_k (F^T G A)_L + A_L (F G^T a + B G A)_k],   b = 3 k + L.
template <typename T, int NF>
__device__ __forceinline__ T contract_structured(int b, const T *st, const KinConst<T> &kc) {
    constexpr int D = 3 + 2 * NF;
    using S = Stage<D, NF>;
    using R = BwPre<D, NF>;
    const int k = b / 3, L = b % 3;
    const T *F = st + S::F, *H = st + S::H, *U = st + S::U, *X = st + S::X, *Y = st + S::Y;
    const T *Gs = st + R::G;
    const T GU = st[R::sc + 0], GH = st[R::sc + 1], GF = st[R::sc + 2];
    const T beta = st[S::sc + 0], gamma = st[S::sc + 1], eta = st[S::sc + 2], zeta = st[S::sc + 3];
    T v = GU * H[b] + GH * U[b] + beta * GH * H[b] + gamma * GF * F[b];
    T hgh = 0, fgf = 0, gx = 0, yg = 0;
#pragma unroll
    for (int J = 0; J < 3; ++J) {
        hgh += H[3 * k + J] * st[R::Nh + 3 * J + L];
        fgf += F[3 * k + J] * st[R::Nf + 3 * J + L];
        gx += Gs[3 * k + J] * X[3 * J + L];
        yg += Y[3 * k + J] * Gs[3 * J + L];
    }
    v += -eta * hgh + zeta * fgf + gx + yg;
#pragma unroll
    for (int f = 0; f < NF; ++f)
        v += st[S::sc + 4 + f] *
             (st[R::a + 3 * f + k] * st[R::v1 + 3 * f + L] + kc.fib[f][L] * st[R::v23 + 3 * f + k]);
    return v;
}

// Weight-gradient sums over the CTA tile's Q points (slab stride qstride):
//   acc[row * cols + col] += sum_q U1[q][row] V1[q][col] + U2[q][row] V2[q][col],
// with the U, V vectors at offsets u1, v1, u2, v2 of each point's slab, in register blocks.
// The square W x W case (W even) in 2 x 2 register
// blocks: per point, four paired loads feed eight multiply-adds where the scalar form needs
// four loads for two. Slab offsets and the slab stride are even, so the pairs are aligned.
template <typename T>
__device__ __forceinline__ void tile_outer_sq(T *acc, int W, const T *base, int qstride, int u1, int v1, int u2,
                                              int v2, int Q) {
    using T2 = typename std::conditional<sizeof(T) == 8, double2, float2>::type;
    const int hw = W >> 1, nb = hw * hw;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        const int jb = b / hw;
        const int j0 = 2 * jb, i0 = 2 * (b - jb * hw);
        T s00 = T(0), s01 = T(0), s10 = T(0), s11 = T(0);
        for (int q = 0; q < Q; ++q) {
            const T *p = base + (size_t)q * qstride;
            const T2 a = *reinterpret_cast<const T2 *>(p + u1 + j0);
            const T2 c = *reinterpret_cast<const T2 *>(p + v1 + i0);
            const T2 a2 = *reinterpret_cast<const T2 *>(p + u2 + j0);
            const T2 c2 = *reinterpret_cast<const T2 *>(p + v2 + i0);
            s00 += a.x * c.x;
            s01 += a.x * c.y;
            s10 += a.y * c.x;
            s11 += a.y * c.y;
            s00 += a2.x * c2.x;
            s01 += a2.x * c2.y;
            s10 += a2.y * c2.x;
            s11 += a2.y * c2.y;
        }
        T *r0 = acc + j0 * W + i0, *r1 = r0 + W;
        r0[0] += s00;
        r0[1] += s01;
        r1[0] += s10;
        r1[1] += s11;
    }
}

// The W x d blocks (rows W even, both products present) with rows in pairs: per point,
// two paired row loads and two column loads feed four multiply-adds. Column `cols` is the
// bias: the slabs hold 1 after V1 and 0 after V2, so it sums U1 alone (x * 1 + y * 0 adds
// exactly x), into acc[rows * cols + row]. The W x d block and the bias vector are
// adjacent in the parameter order, and the extra column fills threads that the W x d
// blocks alone leave idle.
template <typename T>
__device__ __forceinline__ void tile_outer_rows2(T *acc, int rows, int cols, const T *base, int qstride, int u1,
                                                 int v1, int u2, int v2, int Q) {
    using T2 = typename std::conditional<sizeof(T) == 8, double2, float2>::type;
    const int nc = cols + 1, nb = (rows >> 1) * nc;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        const int jb = b / nc, i = b - jb * nc, j0 = 2 * jb;
        T s0 = T(0), s1 = T(0);
        for (int q = 0; q < Q; ++q) {
            const T *p = base + (size_t)q * qstride;
            const T2 a = *reinterpret_cast<const T2 *>(p + u1 + j0);
            const T2 a2 = *reinterpret_cast<const T2 *>(p + u2 + j0);
            const T c = p[v1 + i], c2 = p[v2 + i];
            s0 += a.x * c;
            s1 += a.y * c;
            s0 += a2.x * c2;
            s1 += a2.y * c2;
        }
        T *r0 = (i < cols) ? acc + j0 * cols + i : acc + rows * cols + j0;
        T *r1 = (i < cols) ? r0 + cols : r0 + 1;
        *r0 += s0;
        *r1 += s1;
    }
}

// acc[j] += sum_q U[q][j], on the threads from t0 on (independent sums start on
// different warps, so that they run side by side)
template <typename T>
__device__ __forceinline__ void tile_sum(T *acc, int n, const T *base, int qstride, int u, int Q, int t0) {
    const int nt = (int)blockDim.x - t0;
    for (int j = (int)threadIdx.x - t0; j >= 0 && j < n; j += nt) {
        T s = T(0);
        for (int q = 0; q < Q; ++q) s += base[(size_t)q * qstride + u + j];
        acc[j] += s;
    }
}

}  // namespace

// GACC: the network is too large for its weights, the parameter-gradient accumulators
// and the point slabs to share the shared memory (64-wide networks with three or more
// layers). The CTA then accumulates straight into its own slice of the workspace (each
// entry still owned by one fixed thread, so the sums keep their order) and reads the
// row-major A_k of the reverse pass from global memory (through L1).
// Resident CTAs per SM the register allocation plans for: two (FP64, whose CTAs of at most
// 128 threads then keep up to 255 registers, their shared memory allowing no more than two;
// FP32 networks without fibres up to 32 wide, at most 128 registers), one elsewhere.
template <typename T, int NF, int W>
struct BwMinBlocks {
    static constexpr int value = (sizeof(T) == 8 || (NF == 0 && W <= 32)) ? 2 : 1;
};

template <typename T, int NF, int W, int WARPS, bool GACC = false>
__global__ void __launch_bounds__(WARPS * 32, (BwMinBlocks<T, NF, W>::value))
    const_backward_kernel(const T *__restrict__ gw, NetLayout lay, KinConst<T> kc, int64_t n_qp,
                          const T *__restrict__ Fg, const T *__restrict__ Gg, T *__restrict__ dFg,
                          T *__restrict__ partial, int np_pad, BwSlab sl, int batch) {
    constexpr int D = 3 + 2 * NF, NJ = W / kG;
    constexpr int Q = WARPS * kQPW;  // points per CTA tile
    static_assert(BwPre<D, NF>::size == 9 * D + 54 + 18 * NF + 5 + NF + 30 + 9 * NF,
                  "bw_slab reserves the staged kinematics and BwPre");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sw = reinterpret_cast<T *>(smem_raw);
    // the packed weights go to shared memory except the update's layer-2 tangent weights M
    // (A_k row-major, the last block, moves down by its size) and, with GACC, A_k
    // row-major, read from global memory
    const int msz = lay.M ? lay.Ar - lay.M : 0;
    const int wcount = (GACC ? lay.Ar : lay.total) - msz;
    const int wbytes = (wcount * (int)sizeof(T) + 15) / 16 * 16;
    {
        const int n16 = wbytes / 16;
        const int cut16 = msz ? lay.M * (int)sizeof(T) / 16 : n16;
        const int skip16 = msz * (int)sizeof(T) / 16;
        const int4 *src = reinterpret_cast<const int4 *>(gw);
        int4 *dst = reinterpret_cast<int4 *>(sw);
        for (int i = threadIdx.x; i < n16; i += blockDim.x) dst[i] = src[i < cut16 ? i : i + skip16];
    }
    const T *arw = GACC ? gw + lay.Ar : sw + lay.Ar - msz;
    // [np_pad] parameter-gradient accumulators: shared memory, or this CTA's workspace slice
    T *acc = GACC ? partial + (size_t)blockIdx.x * np_pad : sw + wbytes / (int)sizeof(T);
    T *slabs = GACC ? sw + wbytes / (int)sizeof(T) : acc + np_pad;
    for (int i = threadIdx.x; i < np_pad; i += blockDim.x) acc[i] = T(0);
    __syncthreads();

    const int L = lay.L;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int qi = lane >> 2, jb = lane & 3;
    const int ql = warp * kQPW + qi;  // point index within the tile
    T *qs = slabs + (size_t)ql * sl.size;
    const int j0 = jb * NJ;
    // offsets of the parameter blocks (theta order)
    const int oW1 = 0, oc1 = W * D, oL = oc1 + W;
    const int lsz = W * W + W * D + W;
    const int oa = oL + (L - 1) * lsz, ob = oa + W;

    const int64_t n_tiles = (n_qp + Q - 1) / Q;
    // FP64 with batch: the kinematic scalars of the warp's points in the CTA's next
    // kKinTiles tiles, one point per lane (kin_batch), in the warp's records after the slabs;
    // batch 2: with the staging's scalars too (PRE records), 1: without
    const bool use_rec = sizeof(T) == 8 && batch > 0;
    const int rsize = batch == 2 ? kinrec_size<NF, true>() : kinrec_size<NF>();
    T *rec = slabs + (size_t)Q * sl.size + (size_t)warp * rsize * 32;
    for (int64_t tile0 = blockIdx.x; tile0 < n_tiles; tile0 += (int64_t)kKinTiles * gridDim.x) {
        if (use_rec) {
            if (batch == 2)
                kin_batch<T, NF, true, true>(Fg, Gg, n_qp, tile0, gridDim.x, n_tiles, kc, rec, lane, Q, warp * kQPW);
            else
                kin_batch<T, NF, true>(Fg, Gg, n_qp, tile0, gridDim.x, n_tiles, kc, rec, lane, Q, warp * kQPW);
        }
        __syncwarp();
        for (int sub = 0; sub < kKinTiles; ++sub) {
            const int64_t tile = tile0 + (int64_t)sub * gridDim.x;
            if (tile >= n_tiles) break;
            const int64_t q = tile * Q + ql;
            const bool valid = q < n_qp;
            T F[9], G[9];
#pragma unroll
            for (int c = 0; c < 9; ++c) {
                F[c] = valid ? Fg[c * n_qp + q] : ((c % 4) == 0 ? T(1) : T(0));
                G[c] = valid ? Gg[c * n_qp + q] : T(0);
            }
            T K[D], Jm1;
            PolyChain<T> ch;
            bool bad;
            if (use_rec) {
                bad = kin_read<T, NF>(rec, sub * kQPW + qi, K, Jm1, ch);
            } else {
                bad = !kin_scalars<T, NF>(F, kc, K, Jm1, &ch);
#pragma unroll
                for (int c = 0; c < 9; ++c) bad = bad || !dev_finite(G[c]);
            }
            if (bad) {
#pragma unroll
                for (int c = 0; c < 9; ++c) {
                    F[c] = (c % 4) == 0 ? T(1) : T(0);
                    G[c] = T(0);
                }
                if (!use_rec) kin_scalars<T, NF>(F, kc, K, Jm1, &ch);
            }
            // the staging's C, I1, I2, J^(-1/3) from a PRE record
            const T *pre = (sizeof(T) == 8 && batch == 2) ? kin_pre<T, NF>(rec, sub * kQPW + qi) : nullptr;
            const bool poly = NF == 0 && kc.kin == COMMET_KIN_POLYCONVEX;
            // r_m = G : g_m; the 4 lanes stage g (part 1, 2) and read it back
            {
                T zero[D];
#pragma unroll
                for (int m = 0; m < D; ++m) zero[m] = T(0);
                stage_kinematics<T, NF, true>(F, kc, zero, Jm1, jb, qs, pre);
            }
            T r[D];
            {
                // G goes next to the staged g_m (the F slot is free here); lane jb sums the
                // components a = jb + 4 t, and the group adds the four partial sums
                using S = Stage<D, NF>;
                T *Gs = qs + S::F;
#pragma unroll
                for (int a = 0; a < 9; ++a)
                    if ((a & 3) == jb) Gs[a] = G[a];
                __syncwarp();
#pragma unroll
                for (int m = 0; m < D; ++m) r[m] = T(0);
#pragma unroll
                for (int t = 0; t < 3; ++t) {
                    const int a = jb + 4 * t;
                    if (a < 9) {
                        const T g = Gs[a];
#pragma unroll
                        for (int m = 0; m < D; ++m) r[m] += g * qs[S::g + 9 * m + a];
                    }
                }
#pragma unroll
                for (int msk = 1; msk <= 2; msk <<= 1)
#pragma unroll
                    for (int m = 0; m < D; ++m) r[m] += __shfl_xor_sync(0xffffffffu, r[m], msk);
            }
            // polyconvex layer: g_m above are invariant derivatives; the network sees
            // r_K = phi' r_I, and r_I is kept for the chain rule's second-order term
            T rI[D];
#pragma unroll
            for (int m = 0; m < D; ++m) rI[m] = r[m];
            if (poly) {
#pragma unroll
                for (int m = 0; m < 3; ++m) r[m] *= ch.d1[m];
            }
            __syncwarp();
            if (jb == 0) {
#pragma unroll
                for (int m = 0; m < D; ++m) {
                    qs[sl.K + m] = K[m];
                    qs[sl.r + m] = r[m];
                }
                qs[sl.K + D] = T(1);  // the bias column of tile_outer_rows2
                qs[sl.r + D] = T(0);
            }
            __syncwarp();

            // ---- forward: values and tangents along r
            constexpr int V = 16 / (int)sizeof(T);  // elements per 128-bit shared load
            for (int k = 1; k <= L; ++k) {
                T y[NJ], yd[NJ];
                ldv<NJ>(sw + lay.c + (k - 1) * W + j0, y);
#pragma unroll
                for (int jj = 0; jj < NJ; ++jj) yd[jj] = T(0);
                if (k == 1) {
#pragma unroll
                    for (int m = 0; m < D; ++m) {
                        T w[NJ];
                        ldv<NJ>(sw + lay.W1t + m * W + j0, w);
#pragma unroll
                        for (int jj = 0; jj < NJ; ++jj) {
                            y[jj] += w[jj] * K[m];
                            yd[jj] += w[jj] * r[m];
                        }
                    }
                } else {
                    const T *zin = qs + sl.z + (k - 2) * W, *zdin = qs + sl.zd + (k - 2) * W;
                    const T *At = sw + lay.At + (k - 2) * W * W + j0;
#pragma unroll 2
                    for (int i = 0; i < W; i += V) {
                        T zv[V], zdv[V];
                        ldv<V>(zin + i, zv);
                        ldv<V>(zdin + i, zdv);
#pragma unroll
                        for (int u = 0; u < V; ++u) {
                            T w[NJ];
                            ldv<NJ>(At + (i + u) * W, w);
#pragma unroll
                            for (int jj = 0; jj < NJ; ++jj) {
                                y[jj] += w[jj] * zv[u];
                                yd[jj] += w[jj] * zdv[u];
                            }
                        }
                    }
                    const T *Bt = sw + lay.Bt + (k - 2) * D * W + j0;
#pragma unroll
                    for (int m = 0; m < D; ++m) {
                        T w[NJ];
                        ldv<NJ>(Bt + m * W, w);
#pragma unroll
                        for (int jj = 0; jj < NJ; ++jj) {
                            y[jj] += w[jj] * K[m];
                            yd[jj] += w[jj] * r[m];
                        }
                    }
                }
                T zv[NJ], sv[NJ], tv[NJ], zdv[NJ];
#pragma unroll
                for (int jj = 0; jj < NJ; ++jj) {
                    if constexpr (sizeof(T) == 8)
                        act_tab(y[jj], zv[jj], sv[jj], tv[jj], sw + lay.tab);
                    else
                        act(y[jj], zv[jj], sv[jj], tv[jj]);
                    zdv[jj] = sv[jj] * yd[jj];
                }
                stv<NJ>(qs + sl.s + (k - 1) * W + j0, sv);
                stv<NJ>(qs + sl.t + (k - 1) * W + j0, tv);
                stv<NJ>(qs + sl.yd + (k - 1) * W + j0, yd);
                if (k < L) {
                    stv<NJ>(qs + sl.z + (k - 1) * W + j0, zv);
                    stv<NJ>(qs + sl.zd + (k - 1) * W + j0, zdv);
                } else {
                    stv<NJ>(qs + sl.zdL + j0, zdv);
                }
                __syncwarp();
            }

            // ---- reverse over the tangent computation
            T zb[NJ], zdb[NJ];
            ldv<NJ>(sw + lay.a + j0, zdb);
#pragma unroll
            for (int jj = 0; jj < NJ; ++jj) zb[jj] = T(0);
            T Hr[D], dN[D];
#pragma unroll
            for (int m = 0; m < D; ++m) {
                Hr[m] = T(0);
                dN[m] = (jb == 0) ? sw[lay.b + m] : T(0);
            }
            for (int k = L; k >= 1; --k) {
                const T *Bt = (k == 1) ? (sw + lay.W1t + j0) : (sw + lay.Bt + (k - 2) * D * W + j0);
                {
                    T sv[NJ], tv[NJ], ydv[NJ], ybv[NJ], ydbv[NJ];
                    ldv<NJ>(qs + sl.s + (k - 1) * W + j0, sv);
                    ldv<NJ>(qs + sl.t + (k - 1) * W + j0, tv);
                    ldv<NJ>(qs + sl.yd + (k - 1) * W + j0, ydv);
#pragma unroll
                    for (int jj = 0; jj < NJ; ++jj) {
                        ydbv[jj] = sv[jj] * zdb[jj];
                        ybv[jj] = sv[jj] * zb[jj] + tv[jj] * ydv[jj] * zdb[jj];
                    }
                    stv<NJ>(qs + sl.yb + j0, ybv);
                    stv<NJ>(qs + sl.ydb + j0, ydbv);
#pragma unroll
                    for (int m = 0; m < D; ++m) {
                        T w[NJ];
                        ldv<NJ>(Bt + m * W, w);
#pragma unroll
                        for (int jj = 0; jj < NJ; ++jj) {
                            Hr[m] += w[jj] * ybv[jj];
                            dN[m] += w[jj] * ydbv[jj];
                        }
                    }
                }
                __syncthreads();
                // tile reductions of this layer's weight gradients
                const T *base = slabs;
                if (k == 1) {
                    // W1 and c_1 (adjacent: oc1 = oW1 + W D)
                    tile_outer_rows2<T>(acc + oW1, W, D, base, sl.size, sl.yb, sl.K, sl.ydb, sl.r, Q);
                } else {
                    const int o = oL + (k - 2) * lsz;
                    tile_outer_sq<T>(acc + o, W, base, sl.size, sl.yb, sl.z + (k - 2) * W, sl.ydb,
                                     sl.zd + (k - 2) * W, Q);
                    // B_k and c_k
                    tile_outer_rows2<T>(acc + o + W * W, W, D, base, sl.size, sl.yb, sl.K, sl.ydb, sl.r, Q);
                    // zbar_{k-1} = A_k^T ybar_k, zdotbar_{k-1} = A_k^T ydotbar_k for own neurons
                    const T *Ar = arw + (k - 2) * W * W + j0;
#pragma unroll
                    for (int ii = 0; ii < NJ; ++ii) {
                        zb[ii] = T(0);
                        zdb[ii] = T(0);
                    }
#pragma unroll 2
                    for (int j = 0; j < W; j += V) {
                        T ybv[V], ydbv[V];
                        ldv<V>(qs + sl.yb + j, ybv);
                        ldv<V>(qs + sl.ydb + j, ydbv);
#pragma unroll
                        for (int u = 0; u < V; ++u) {
                            T w[NJ];
                            ldv<NJ>(Ar + (j + u) * W, w);
#pragma unroll
                            for (int ii = 0; ii < NJ; ++ii) {
                                zb[ii] += w[ii] * ybv[u];
                                zdb[ii] += w[ii] * ydbv[u];
                            }
                        }
                    }
                }
                __syncthreads();
            }
            tile_sum<T>(acc + oa, W, slabs, sl.size, sl.zdL, Q, 0);
            tile_sum<T>(acc + ob, D, slabs, sl.size, sl.r, Q, blockDim.x > 32 ? 32 : 0);

            // ---- dL/dF = sum_n (Hr)_n g_n + G : S (structured part)
#pragma unroll
            for (int msk = 1; msk <= 2; msk <<= 1)
#pragma unroll
                for (int m = 0; m < D; ++m) {
                    Hr[m] += __shfl_xor_sync(0xffffffffu, Hr[m], msk);
                    dN[m] += __shfl_xor_sync(0xffffffffu, dN[m], msk);
                }
            __syncthreads();  // slabs are reused as staging below
            T cvec[D];
#pragma unroll
            for (int m = 0; m < D; ++m) cvec[m] = dN[m] - sw[lay.n0 + m];
            if (poly) {
                // (d2Psi/dI2) r_I = phi' (N r_K) + phi'' c r_I;  dPsi/dI = phi' c
#pragma unroll
                for (int m = 0; m < 3; ++m) {
                    Hr[m] = ch.d1[m] * Hr[m] + ch.d2[m] * cvec[m] * rI[m];
                    cvec[m] *= ch.d1[m];
                }
            }
            stage_kinematics<T, NF>(F, kc, cvec, Jm1, jb, qs, pre);
            __syncwarp();
            if (dFg != nullptr) {
                using S = Stage<D, NF>;
                structured_pre<T, NF>(qs, G, kc, jb);
                __syncwarp();
                for (int b = jb; b < 9; b += kG) {
                    T v = contract_structured<T, NF>(b, qs, kc);
#pragma unroll
                    for (int n = 0; n < D; ++n) v += Hr[n] * qs[S::g + 9 * n + b];
                    if (valid) dFg[b * n_qp + q] = bad ? T(NAN) : v;
                }
            }
            __syncthreads();
        }
    }
    // write this CTA's partial sums (GACC: already in place)
    if constexpr (!GACC) {
        T *dst = partial + (size_t)blockIdx.x * np_pad;
        for (int i = threadIdx.x; i < np_pad; i += blockDim.x) dst[i] = acc[i];
    }
}

// Sums the per-CTA partials of parameter p in CTA order; with a map (padded networks) the
// sum goes to the caller's theta index map[p], and padding parameters (map -1) are dropped.
template <typename T>
__global__ void reduce_partials_kernel(const T *__restrict__ partial, int n_blocks, int np, int np_pad,
                                       T *__restrict__ out, const int32_t *__restrict__ map) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const int dst = map ? map[p] : p;
    if (dst < 0) return;
    T s = T(0);
    for (int b = 0; b < n_blocks; ++b) s += partial[(size_t)b * np_pad + p];
    out[dst] = s;
}

static int bw_grid(const commet_model *m, int64_t n_qp, int Q) {
    const int64_t n_tiles = (n_qp + Q - 1) / Q;
    return (int)std::max<int64_t>(1, std::min<int64_t>(n_tiles, 2 * (int64_t)sm_count()));
}

static int64_t np_net(const commet_model *m) { return m->n_params_net > 0 ? m->n_params_net : m->n_params; }
static int np_padded(const commet_model *m) { return (int)((np_net(m) + 3) / 4 * 4); }

// Backward of the CANN (eq. cann-def), theta = its weights (w1, w2) per input m and term k:
// with r_m = G : dK_m/dF (times phi'_m on the polyconvex layer, whose staged gradients are
// those of the invariants),
//   dL/dF = G : A,   dL/dw2_mk = sum_q r_m f2' f1' f0',   dL/dw1_mk = sum_q r_m w2 (d f2'/d w1) f1' f0'.
// Per point (4 lanes, 8 points per warp) the forward of the closed-form update leaves P and
// A in the point's slab; the lanes contract A with G by columns, then take the D n terms
// round-robin. Each term's gradient is summed over the warp's 8 points by shuffles and
// added to the warp's accumulators in shared memory (one lane per term); the CTA's sum over
// its warps, in warp order, goes to the workspace, reduced over CTAs by reduce_partials_kernel.
constexpr int kCannBwWarps = 8;

// Whether the CANN backward forms the kinematic scalars in batches (kin_batch): not in
// FP64 with fibres, whose point slabs leave no room for the records.
template <typename T, int NF>
__host__ __device__ constexpr bool cann_bw_batches() {
    return sizeof(T) == 4 || NF == 0;
}

template <typename T, int NF>
__global__ void __launch_bounds__(kCannBwWarps * 32, (sizeof(T) == 4 && NF == 0) ? 2 : 1)
    cann_backward_kernel(const T *__restrict__ gw, NetLayout lay, KinConst<T> kc, int64_t n_qp,
                         const T *__restrict__ Fg, const T *__restrict__ Gg, T *__restrict__ dFg,
                         T *__restrict__ partial, int np_pad, int qstride) {
    constexpr int D = 3 + 2 * NF, NH = D * (D + 1) / 2;
    using S = Stage<D, NF>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sw = reinterpret_cast<T *>(smem_raw);
    const int wbytes = (lay.total * (int)sizeof(T) + 15) / 16 * 16;
    {
        const int4 *src = reinterpret_cast<const int4 *>(gw);
        int4 *dst = reinterpret_cast<int4 *>(sw);
        for (int i = threadIdx.x; i < wbytes / 16; i += blockDim.x) dst[i] = src[i];
    }
    T *acc = sw + wbytes / (int)sizeof(T);  // [kCannBwWarps][np_pad]
    T *slabs = acc + kCannBwWarps * np_pad;
    for (int i = threadIdx.x; i < kCannBwWarps * np_pad; i += blockDim.x) acc[i] = T(0);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int qi = lane >> 2, jb = lane & 3;
    T *qs = slabs + (size_t)(warp * kQPW + qi) * qstride;
    T *wacc = acc + warp * np_pad;
    const int n = lay.cn, nt = D * n;
    const int64_t n_tiles = (n_qp + kQPW - 1) / kQPW;
    const int64_t n_gwarps = (int64_t)gridDim.x * kCannBwWarps;
    // the warp's kinematic records after the point slabs (FP64 with fibres: no room beside
    // its slabs, the scalars are formed per point)
    constexpr bool kBatch = cann_bw_batches<T, NF>();
    constexpr bool kPre = kBatch && sizeof(T) == 8;  // FP64 records also hold the staging's scalars
    T *rec = slabs + (size_t)kCannBwWarps * kQPW * qstride + (size_t)warp * kinrec_size<NF, kPre>() * 32;

    for (int64_t tile0 = (int64_t)blockIdx.x * kCannBwWarps + warp; tile0 < n_tiles; tile0 += kKinTiles * n_gwarps) {
        if constexpr (kBatch) kin_batch<T, NF, true, kPre>(Fg, Gg, n_qp, tile0, n_gwarps, n_tiles, kc, rec, lane);
        __syncwarp();
        for (int sub = 0; sub < kKinTiles; ++sub) {
            const int64_t tile = tile0 + sub * n_gwarps;
            if (tile >= n_tiles) break;
            const int64_t q = tile * kQPW + qi;
            const bool valid = q < n_qp;
            T F[9], G[9];
#pragma unroll
            for (int c = 0; c < 9; ++c) {
                F[c] = valid ? Fg[c * n_qp + q] : ((c % 4) == 0 ? T(1) : T(0));
                G[c] = valid ? Gg[c * n_qp + q] : T(0);
            }
            T K[D], Jm1;
            PolyChain<T> ch;
            bool bad;
            if constexpr (kBatch) {
                bad = kin_read<T, NF>(rec, sub * kQPW + qi, K, Jm1, ch);
            } else {
                bad = !kin_scalars_k64<T, NF>(F, kc, K, Jm1, ch);
#pragma unroll
                for (int c = 0; c < 9; ++c) bad = bad || !dev_finite(G[c]);
            }
            if (bad) {
#pragma unroll
                for (int c = 0; c < 9; ++c) {
                    F[c] = (c % 4) == 0 ? T(1) : T(0);
                    G[c] = T(0);
                }
                if constexpr (!kBatch) kin_scalars_k64<T, NF>(F, kc, K, Jm1, ch);
            }
            T npart = T(0), dN[D], Hs[NH];
#pragma unroll
            for (int m = 0; m < D; ++m) dN[m] = T(0);
#pragma unroll
            for (int h = 0; h < NH; ++h) Hs[h] = T(0);
            cann_point<T, D>(sw, lay, K, jb, npart, dN, Hs);
            T *pa = qs + qp_stage_end(D, NF);  // the point's P (9) and A (81)
            T psi_val;
            bool report;
            qp_group_finish<T, NF>(sw + lay.n0, sw + lay.K0, kc, qs, qi, jb, F, K, Jm1, ch, bad, valid, npart, dN, Hs,
                                   true, pa, 1, pa + 9, 1, nullptr, 0, psi_val, report,
                                   kPre ? kin_pre<T, NF>(rec, sub * kQPW + qi) : nullptr);
            __syncwarp();
            // dL/dF by columns b = jb, jb + 4, jb + 8
            T dfv[3];
            bool fin = true;
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                const int b = jb + kG * t;
                T v = T(0);
                if (b < 9) {
#pragma unroll
                    for (int a = 0; a < 9; ++a) v += G[a] * pa[9 + 9 * a + b];
                }
                dfv[t] = v;
                fin = fin && dev_finite(v);
            }
            // r_m = G : dK_m/dF from the staged kinematic gradients
            T r[D];
#pragma unroll
            for (int m = 0; m < D; ++m) {
                T v = T(0);
#pragma unroll
                for (int a = 0; a < 9; ++a) v += G[a] * qs[S::g + 9 * m + a];
                r[m] = v;
            }
            if constexpr (NF == 0) {
                if (kc.kin == COMMET_KIN_POLYCONVEX) {
#pragma unroll
                    for (int m = 0; m < 3; ++m) r[m] *= ch.d1[m];
                }
            }
            // the point's weight-gradient terms, d n of them round-robin over its 4 lanes
            auto term = [&](int t, T &g1, T &g2) {
                const int m = t / n, k = t - m * n;
                T x = T(0), rm = T(0);
#pragma unroll
                for (int mm = 0; mm < D; ++mm) {
                    x = (mm == m) ? K[mm] : x;
                    rm = (mm == m) ? r[mm] : rm;
                }
                cann_term_wgrad<T>(x, (int)sw[lay.ck + 3 * k], (int)sw[lay.ck + 3 * k + 1], (int)sw[lay.ck + 3 * k + 2],
                                   sw[lay.cw + 2 * t], sw[lay.cw + 2 * t + 1], g1, g2);
                g1 *= rm;
                g2 *= rm;
            };
            // FP64: the lane's first kTermRegs terms stay in registers for the sums below (their
            // exponentials cost FP64 work); any further ones, and all FP32 ones, are evaluated
            // again there
            constexpr int kTermRegs = sizeof(T) == 8 ? 4 : 0;
            T c1[kTermRegs > 0 ? kTermRegs : 1], c2[kTermRegs > 0 ? kTermRegs : 1];
#pragma unroll
            for (int i = 0; i < kTermRegs; ++i) {
                c1[i] = c2[i] = T(0);
                if (jb + kG * i < nt) {
                    term(jb + kG * i, c1[i], c2[i]);
                    fin = fin && dev_finite(c1[i]) && dev_finite(c2[i]);
                }
            }
            for (int t0 = kG * kTermRegs; t0 < nt; t0 += kG) {
                if (t0 + jb < nt) {
                    T g1, g2;
                    term(t0 + jb, g1, g2);
                    fin = fin && dev_finite(g1) && dev_finite(g2);
                }
            }
            // a point outside the energy's domain (reported by the forward) or whose dL/dF or
            // gradient terms leave the number range (the CANN's exponentials, mostly in FP32)
            // is treated as J <= 0: NaN in dL/dF, nothing in dL/dw
            const unsigned nonfin = __ballot_sync(0xffffffffu, !fin);
            const bool drop = report || !valid || ((nonfin >> (qi * 4)) & 0xFu) != 0u;
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                const int b = jb + kG * t;
                if (b < 9 && valid && dFg != nullptr) dFg[b * n_qp + q] = drop ? T(NAN) : dfv[t];
            }
            for (int t0 = 0; t0 < nt; t0 += kG) {
                const int t = t0 + jb, i = t0 / kG;
                T g1 = T(0), g2 = T(0);
                if (kTermRegs > 0 && i < kTermRegs) {
#pragma unroll
                    for (int r2 = 0; r2 < kTermRegs; ++r2) {
                        g1 = (r2 == i) ? c1[r2] : g1;
                        g2 = (r2 == i) ? c2[r2] : g2;
                    }
                    if (drop) g1 = g2 = T(0);
                } else if (t < nt && !drop) {
                    term(t, g1, g2);
                }
                // the same term over the warp's 8 points (lanes with the same jb)
#pragma unroll
                for (int msk = 4; msk <= 16; msk <<= 1) {
                    g1 += shfl_xor(g1, msk);
                    g2 += shfl_xor(g2, msk);
                }
                if (qi == 0 && t < nt) {
                    wacc[2 * t] += g1;
                    wacc[2 * t + 1] += g2;
                }
            }
            __syncwarp();
        }
    }
    __syncthreads();
    for (int p = threadIdx.x; p < np_pad; p += blockDim.x) {
        T v = T(0);
        for (int w = 0; w < kCannBwWarps; ++w) v += acc[w * np_pad + p];
        partial[(size_t)blockIdx.x * np_pad + p] = v;
    }
}

size_t backward_workspace_bytes(const commet_model *m, int64_t n_qp) {
    if (m->precision != COMMET_F64 && m->precision != COMMET_F32) return 0;
    if (m->inner == COMMET_INNER_CANN) {
        const size_t es = m->precision == COMMET_F64 ? 8 : 4;
        const size_t bytes = (size_t)bw_grid(m, n_qp, kCannBwWarps * kQPW) * np_padded(m) * es;
        return (bytes + 255) / 256 * 256;
    }
    if (m->inner != COMMET_INNER_MICNN) return 0;
    const size_t es = m->precision == COMMET_F64 ? 8 : 4;
    // sized for the smallest tile any launch may use (the largest grid)
    const int Q = (m->precision == COMMET_F64 ? BwConf<double>::least_warps : BwConf<float>::least_warps) * kQPW;
    const size_t bytes = (size_t)bw_grid(m, n_qp, Q) * np_padded(m) * es;
    return (bytes + 255) / 256 * 256;
}

template <typename T, int NF, int W, int WARPS, bool GACC = false>
static int bw_launch(const commet_model *m, int64_t n_qp, const void *F, const void *G, void *dF, void *dth,
                     void *ws, cudaStream_t s) {
    KinConst<T> kc{};
    kc.kin = m->kp.kin;
    kc.stress_free = m->kp.stress_free;
    kc.kappa = (T)m->kp.kappa;
    for (int f = 0; f < 2; ++f)
        for (int c = 0; c < 3; ++c) kc.fib[f][c] = (T)m->kp.fib[f][c];
    const int D = 3 + 2 * NF;
    const BwSlab sl = bw_slab(D, W, m->L, NF, (int)sizeof(T));
    const int Q = WARPS * kQPW;
    const int np_pad = np_padded(m);
    const int msz = m->lay.M ? m->lay.Ar - m->lay.M : 0;  // M is not used here (global memory)
    const size_t wbytes = ((size_t)((GACC ? m->lay.Ar : m->lay.total) - msz) * sizeof(T) + 15) / 16 * 16;
    const size_t smem0 = wbytes + (GACC ? 0 : (size_t)np_pad * sizeof(T)) + (size_t)Q * sl.size * sizeof(T);
    int dev = 0, smem_max = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (smem0 > (size_t)smem_max) return COMMET_ERR_UNSUPPORTED;
    // FP64: the batched kinematic scalars' records, where they fit beside the slabs
    const size_t rec_long = (size_t)WARPS * kinrec_size<NF, true>() * 32 * sizeof(T);
    const size_t rec_short = (size_t)WARPS * kinrec_size<NF>() * 32 * sizeof(T);
    const int batch = sizeof(T) != 8                            ? 0
                      : smem0 + rec_long <= (size_t)smem_max  ? 2
                      : smem0 + rec_short <= (size_t)smem_max ? 1
                                                              : 0;
    const size_t smem = smem0 + (batch == 2 ? rec_long : batch == 1 ? rec_short : 0);
    auto kern = const_backward_kernel<T, NF, W, WARPS, GACC>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return COMMET_ERR_CUDA;
    const int grid = bw_grid(m, n_qp, Q);
    kern<<<grid, WARPS * 32, smem, s>>>((const T *)m->d_weights, m->lay, kc, n_qp, (const T *)F,
                                                   (const T *)G, (T *)dF, (T *)ws, np_pad, sl, batch);
    if (cudaGetLastError() != cudaSuccess) return COMMET_ERR_CUDA;
    const int np = (int)np_net(m);
    reduce_partials_kernel<T><<<(np + 255) / 256, 256, 0, s>>>((const T *)ws, grid, np, np_pad, (T *)dth,
                                                               m->d_theta_map);
    return cudaGetLastError() == cudaSuccess ? COMMET_OK : COMMET_ERR_CUDA;
}

template <typename T, int NF, int W>
static int bw_typed(const commet_model *m, int64_t n_qp, const void *F, const void *G, void *dF, void *dth,
                    void *ws, cudaStream_t s) {
    int rc = bw_launch<T, NF, W, BwConf<T>::warps>(m, n_qp, F, G, dF, dth, ws, s);
    if constexpr (W == 64) {
        // half the tile; then accumulators in the workspace and A_k row-major from global
        // memory, at the full, half and (FP64) quarter tile
        if (rc == COMMET_ERR_UNSUPPORTED) rc = bw_launch<T, NF, W, BwConf<T>::min_warps>(m, n_qp, F, G, dF, dth, ws, s);
        if (rc == COMMET_ERR_UNSUPPORTED) rc = bw_launch<T, NF, W, BwConf<T>::warps, true>(m, n_qp, F, G, dF, dth, ws, s);
        if (rc == COMMET_ERR_UNSUPPORTED)
            rc = bw_launch<T, NF, W, BwConf<T>::min_warps, true>(m, n_qp, F, G, dF, dth, ws, s);
        if (rc == COMMET_ERR_UNSUPPORTED && BwConf<T>::least_warps < BwConf<T>::min_warps)
            rc = bw_launch<T, NF, W, BwConf<T>::least_warps, true>(m, n_qp, F, G, dF, dth, ws, s);
    }
    return rc;
}

template <typename T>
static int bw_dispatch(const commet_model *m, int64_t n_qp, const void *F, const void *G, void *dF, void *dth,
                       void *ws, cudaStream_t s) {
    const int nf = m->kp.nf, W = m->W;
#define COMMET_CASE(NF_, W_) \
    if (nf == NF_ && W == W_) return bw_typed<T, NF_, W_>(m, n_qp, F, G, dF, dth, ws, s);
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

template <typename T, int NF>
static int cann_bw_launch(const commet_model *m, int64_t n_qp, const void *F, const void *G, void *dF, void *dth,
                          void *ws, cudaStream_t s) {
    constexpr int D = 3 + 2 * NF;
    KinConst<T> kc{};
    kc.kin = m->kp.kin;
    kc.stress_free = m->kp.stress_free;
    kc.kappa = (T)m->kp.kappa;
    for (int f = 0; f < 2; ++f)
        for (int c = 0; c < 3; ++c) kc.fib[f][c] = (T)m->kp.fib[f][c];
    const int qstride = qp_slab_elems<T>(D, 0, 0, NF, true);  // room for P and A after the staging
    const int np_pad = np_padded(m);
    const size_t wbytes = ((size_t)m->lay.total * sizeof(T) + 15) / 16 * 16;
    // the point slabs, then (where the scalars are batched) the kinematic records, FP64
    // with the staging's scalars
    constexpr bool batch = cann_bw_batches<T, NF>();
    constexpr int rec = batch ? kinrec_size<NF, batch && sizeof(T) == 8>() * 32 : 0;
    const size_t smem = wbytes + (size_t)kCannBwWarps * np_pad * sizeof(T) +
                        (size_t)kCannBwWarps * (kQPW * qstride + rec) * sizeof(T);
    int dev = 0, smem_max = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (smem > (size_t)smem_max) return COMMET_ERR_UNSUPPORTED;
    auto kern = cann_backward_kernel<T, NF>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return COMMET_ERR_CUDA;
    const int grid = bw_grid(m, n_qp, kCannBwWarps * kQPW);
    kern<<<grid, kCannBwWarps * 32, smem, s>>>((const T *)m->d_weights, m->lay, kc, n_qp, (const T *)F, (const T *)G,
                                                (T *)dF, (T *)ws, np_pad, qstride);
    if (cudaGetLastError() != cudaSuccess) return COMMET_ERR_CUDA;
    const int np = (int)np_net(m);
    reduce_partials_kernel<T><<<(np + 255) / 256, 256, 0, s>>>((const T *)ws, grid, np, np_pad, (T *)dth, nullptr);
    return cudaGetLastError() == cudaSuccess ? COMMET_OK : COMMET_ERR_CUDA;
}

template <typename T>
static int cann_bw_dispatch(const commet_model *m, int64_t n_qp, const void *F, const void *G, void *dF, void *dth,
                            void *ws, cudaStream_t s) {
    if (m->kp.nf == 0) return cann_bw_launch<T, 0>(m, n_qp, F, G, dF, dth, ws, s);
    if (m->kp.nf == 1) return cann_bw_launch<T, 1>(m, n_qp, F, G, dF, dth, ws, s);
    if (m->kp.nf == 2) return cann_bw_launch<T, 2>(m, n_qp, F, G, dF, dth, ws, s);
    return COMMET_ERR_UNSUPPORTED;
}

int launch_const_backward(const commet_model *m, int64_t n_qp, const void *F, const void *G, void *dF, void *dth,
                          void *ws, size_t ws_bytes, cudaStream_t s) {
    (void)ws_bytes;
    if (m->inner != COMMET_INNER_MICNN && m->inner != COMMET_INNER_CANN) return COMMET_ERR_UNSUPPORTED;
    if (n_qp == 0) {
        const size_t es = m->precision == COMMET_F64 ? 8 : 4;
        return cudaMemsetAsync(dth, 0, es * m->n_params, s) == cudaSuccess ? COMMET_OK : COMMET_ERR_CUDA;
    }
    if (m->inner == COMMET_INNER_CANN) {
        if (m->precision == COMMET_F64) return cann_bw_dispatch<double>(m, n_qp, F, G, dF, dth, ws, s);
        if (m->precision == COMMET_F32) return cann_bw_dispatch<float>(m, n_qp, F, G, dF, dth, ws, s);
        return COMMET_ERR_UNSUPPORTED;
    }
    if (m->precision == COMMET_F64) return bw_dispatch<double>(m, n_qp, F, G, dF, dth, ws, s);
    if (m->precision == COMMET_F32) return bw_dispatch<float>(m, n_qp, F, G, dF, dth, ws, s);
    return COMMET_ERR_UNSUPPORTED;
}

}  // namespace commet
