// Constitutive update with the hidden W x W layers on the fifth-generation tensor cores
// (tcgen05: bf16 operands in shared memory, fp32 accumulators in tensor memory): the
// COMMET_BF16_MLP precision. The network derivatives follow the scheme of the FP64/FP32
// kernel (forward values, reverse adjoints, forward tangents consumed into the Hessian).
//
// One CTA of 128 SPLIT threads takes a tile of 128 points: point i is lane i of tensor
// memory and row i of every MMA (M = 128), held by threads i + 128 p, p < SPLIT (warps w,
// w + 4, ... reach the same TMEM lanes), each taking W / SPLIT of every layer's neurons
// (SPLIT = 2). Per tile and hidden layer k:
//     values    Y_k      = Z_{k-1} A_k^T                [128 x W] = [128 x W][W x W]
//     adjoints  Zb_{k-1} = Yb_k A_k                     [128 x W]
//     tangents  J_k^(m)  = T_{k-1}^(m) A_k^T, m < d,    T = F'(y) (.) J
// are tcgen05.mma kind::f16 instructions issued by one thread from operand tiles that
// the threads write row by row (bf16, K-major core-matrix layout) and from the weights,
// staged once per CTA in the same layout; the accumulators are read back with
// tcgen05.ld. F'(y) and F''(y) of every layer are kept in the point's TMEM lane as fp16
// pairs (tcgen05.st), F'' later replaced by the adjoint weight D_k = F''(y) zbar_k. Layer
// 1 (d inputs), biases and skip terms, activations, the output layer and the Hessian sums
// run in fp32 in the point's threads, whose partial sums meet in shared memory. The
// kinematics (fp32, J - 1 without cancellation) and the P/A assembly run in groups of 4
// lanes as in the other kernels, each warp taking 4 / SPLIT rounds of 8 of its 32
// points, their data passed by warp shuffles.
//
// Tensor memory per CTA: d W columns of accumulators (values and adjoints use the first
// W) plus L W columns of (F', F''/D) pairs: (d + L) W <= 512.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>

#include "device_math.cuh"
#include "internal.h"
#include "tma.cuh"
#include "umma.cuh"

namespace commet {

namespace {

constexpr int kTile = 128;           // points per CTA tile = MMA M = TMEM lanes
constexpr int kWaitTries = 1 << 22;  // bounded mbarrier polls per MMA batch

// Offsets of the bf16-path weight block: an fp32 part (units of float) followed by a
// bf16 part (bytes) holding, per hidden layer k >= 2, A_k (rows j, K = i) and A_k^T
// (rows i, K = j) in the core-matrix layout, W * W * 2 bytes each.
struct TcLayout {
    int d, dp, W, L;
    int W1t, Bkt, c, a, b, n0, K0, f32_total;  // float offsets; W1t [d][W], Bkt [L-1][d][W]
    int Ab, Atb, b16_bytes;                     // byte offsets from the start of the bf16 part
};

// J - 1 = det(I + H) - 1 = tr H + (principal 2x2 minors of H) + det H, H = F - I:
// free of the cancellation of det F - 1 near J = 1 (accurate to a few ulp of |H|).
__device__ __forceinline__ float det_minus_one_f32(const float *F) {
    const float h0 = F[0] - 1.f, h4 = F[4] - 1.f, h8 = F[8] - 1.f;
    const float tr = h0 + h4 + h8;
    const float m2 = (h0 * h4 - F[1] * F[3]) + (h0 * h8 - F[2] * F[6]) + (h4 * h8 - F[5] * F[7]);
    const float d3 = h0 * (h4 * h8 - F[5] * F[7]) - F[1] * (F[3] * h8 - F[5] * F[6]) + F[2] * (F[3] * F[7] - h4 * F[6]);
    return tr + m2 + d3;
}

template <int NF>
__device__ __forceinline__ bool kin_scalars_f32(const float *F, const KinConst<float> &kc, float *K, float &Jm1,
                                                PolyChain<float> *ch) {
    Jm1 = det_minus_one_f32(F);
    const float J = 1.f + Jm1;
    float C[9];
    right_cg(F, C);
    const float I1 = C[0] + C[4] + C[8];
    float trC2 = 0.f;
#pragma unroll
    for (int a = 0; a < 9; ++a) trC2 += C[a] * C[a];
    const float I2 = 0.5f * (I1 * I1 - trC2);
    const bool ok = (J > 0.f) && isfinite(Jm1) && isfinite(I1);
    const float r3 = rcbrtf(ok ? J : 1.f);
    const float jm23 = r3 * r3;
    K[0] = jm23 * I1;
    K[1] = jm23 * jm23 * I2;
    K[2] = J;
    if (kc.kin == COMMET_KIN_ISO_SHIFTED) {
        K[0] -= 3.f;
        K[1] -= 3.f;
        K[2] = Jm1;
    } else if (NF == 0 && kc.kin == COMMET_KIN_POLYCONVEX) {
        poly_inputs<float>(K, Jm1, ch);
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        float v[3];
#pragma unroll
        for (int I = 0; I < 3; ++I)
            v[I] = C[3 * I] * kc.fib[f][0] + C[3 * I + 1] * kc.fib[f][1] + C[3 * I + 2] * kc.fib[f][2];
        K[3 + f] = v[0] * kc.fib[f][0] + v[1] * kc.fib[f][1] + v[2] * kc.fib[f][2];
        K[3 + NF + f] = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    }
    return ok;
}

__device__ __forceinline__ uint32_t pack_half2(float lo, float hi) {
    __half2 v = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}
__device__ __forceinline__ float2 unpack_half2(uint32_t u) {
    return __half22float2(*reinterpret_cast<__half2 *>(&u));
}
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

// 8 consecutive columns j0..j0+7 (j0 % 8 == 0) of row r of an operand tile with K = W.
template <int W>
__device__ __forceinline__ void store_row8(unsigned char *op, int r, int j0, const float *v) {
    uint4 u;
    u.x = pack_bf16x2(v[0], v[1]);
    u.y = pack_bf16x2(v[2], v[3]);
    u.z = pack_bf16x2(v[4], v[5]);
    u.w = pack_bf16x2(v[6], v[7]);
    *reinterpret_cast<uint4 *>(op + cm_byte(r, j0, W)) = u;
}

// ---- neuron pairs in packed FP32 (fma/mul/add.rn.f32x2: two lanes per instruction)
__device__ __forceinline__ float2 bc2(float x) { return make_float2(x, x); }
__device__ __forceinline__ float mufu_ex2(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float mufu_rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float mufu_lg2(float x) {
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// Softplus of two pre-activations: z = log(1 + e^y), s = z' = logistic(y), t = z'' =
// e / (1 + e)^2 with e = exp(-|y|) = 2^(-|y| log2 e), all from three MUFU operations per
// neuron (2^x, 1/x, log2 x); 1 + e lies in (1, 2], where the approximate reciprocal and
// logarithm are within a few ulp, far inside the bf16 path's tolerance.
__device__ __forceinline__ void act2(float2 y, float2 &z, float2 &s, float2 &t) {
    constexpr float kLog2e = 1.4426950408889634f, kLn2 = 0.6931471805599453f;
    const float2 m = __fmul2_rn(make_float2(-fabsf(y.x), -fabsf(y.y)), bc2(kLog2e));
    const float2 e = make_float2(mufu_ex2(m.x), mufu_ex2(m.y));
    const float2 u = __fadd2_rn(e, bc2(1.f));
    const float2 r = make_float2(mufu_rcp(u.x), mufu_rcp(u.y));
    const float2 lg = make_float2(mufu_lg2(u.x), mufu_lg2(u.y));
    z = __ffma2_rn(lg, bc2(kLn2), make_float2(fmaxf(y.x, 0.f), fmaxf(y.y, 0.f)));
    const float2 er = __fmul2_rn(e, r);
    s = make_float2(y.x >= 0.f ? r.x : er.x, y.y >= 0.f ? r.y : er.y);
    t = __fmul2_rn(er, r);
}

// Pair h (0: neurons 0, 1; 1: neurons 2, 3) of a quad of neurons loaded as one float4.
__device__ __forceinline__ float2 qh(const float4 &q, int h) { return h ? make_float2(q.z, q.w) : make_float2(q.x, q.y); }
__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }

// sum_m w[m] K[m] with w 16-byte aligned in shared memory (broadcast loads).
template <int D>
__device__ __forceinline__ float dot_w(const float *w, const float *K) {
    float s = 0.f;
#pragma unroll
    for (int m0 = 0; m0 < D; m0 += 4) {
        const float4 v = *reinterpret_cast<const float4 *>(w + m0);
        s += v.x * K[m0];
        if (m0 + 1 < D) s += v.y * K[m0 + 1];
        if (m0 + 2 < D) s += v.z * K[m0 + 2];
        if (m0 + 3 < D) s += v.w * K[m0 + 3];
    }
    return s;
}

// One GEMM D[128 x W] = Op[128 x W] * Bw[W x W]^T (Bw rows = output columns), K = W.
template <int W>
__device__ __forceinline__ void issue_gemm(uint32_t d_tmem, uint32_t op_saddr, uint32_t w_saddr) {
    constexpr uint32_t idesc = umma_idesc_bf16(kTile, W);
#pragma unroll
    for (int s = 0; s < W / 16; ++s)
        umma_bf16(d_tmem, umma_desc(op_saddr + 256u * s, 128u, 16u * W), umma_desc(w_saddr + 256u * s, 128u, 16u * W),
                  idesc, s > 0);
}

// Makes this tile's operand rows and TMEM stores visible, lets thread 0 issue the batch
// (issue() runs on thread 0 only), and waits for its completion. False on timeout (every
// thread returns the same answer).
template <typename Issue>
__device__ __forceinline__ bool mma_round(uint64_t *bar, uint32_t &phase, Issue issue) {
    fence_async_smem();
    tmem_wait_st();
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
        tc_fence_after();
        issue();
        umma_commit(bar);
    }
    const bool ok = mbar_wait_bounded(bar, phase, kWaitTries);
    phase ^= 1u;
    const bool any_fail = __syncthreads_or(!ok) != 0;
    tc_fence_after();
    return !any_fail;
}

}  // namespace

// Threads per point. 4 (16 warps, at most 128 registers) measured the same as 2 on the
// d3 W64 L3 network: the kernel is bound by the issue of its per-point scalar work.
template <int NF> struct TcSplit { static constexpr int value = 2; };

template <int NF, int W, bool SPATIAL, int SPLIT = TcSplit<NF>::value>
__global__ void __launch_bounds__(kTile * SPLIT, 1)
    bf16_tc_kernel(const float *__restrict__ gw32, const unsigned char *__restrict__ gw16, TcLayout lay,
                   KinConst<float> kc, int64_t n_qp, const float *__restrict__ Fg, float *__restrict__ psi,
                   float *__restrict__ P, float *__restrict__ A, int32_t *__restrict__ status, int *__restrict__ err,
                   uint32_t tmem_cols, int stage_stride) {
    constexpr int D = 3 + 2 * NF, NH = D * (D + 1) / 2;
    constexpr int kThreads = kTile * SPLIT;
    constexpr int WH = W / SPLIT;       // neurons per thread
    constexpr int CH = (D > 3 || WH < 16) ? 8 : 16;  // TMEM columns per load / store
    constexpr int NCH = WH / CH;
    constexpr int NRED = 1 + D + NH;    // partial sums a thread hands to its partner
    constexpr int OPB = kTile * W * 2;  // bytes of one operand tile
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_bar;

    // shared memory: [bf16 weights][operand Z][operands T^(0..D-1)][fp32 weights]
    //                [partial sums NRED x 128 SPLIT][stage areas 32 SPLIT x stage_stride]
    unsigned char *w16 = smem_raw;
    unsigned char *opZ = w16 + lay.b16_bytes;
    unsigned char *opT = opZ + OPB;
    float *s32 = reinterpret_cast<float *>(opT + D * OPB);
    const int f32_bytes = (lay.f32_total * 4 + 15) / 16 * 16;
    float *red = reinterpret_cast<float *>(reinterpret_cast<unsigned char *>(s32) + f32_bytes);
    float *stage_base = red + kThreads * NRED;
    {
        const int4 *src = reinterpret_cast<const int4 *>(gw16);
        int4 *dst = reinterpret_cast<int4 *>(w16);
        for (int i = threadIdx.x; i < lay.b16_bytes / 16; i += blockDim.x) dst[i] = src[i];
        const int4 *src32 = reinterpret_cast<const int4 *>(gw32);
        int4 *dst32 = reinterpret_cast<int4 *>(s32);
        for (int i = threadIdx.x; i < f32_bytes / 16; i += blockDim.x) dst32[i] = src32[i];
    }
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row = tid & (kTile - 1), part = tid >> 7;  // point in the tile, neuron block
    const int j0 = part * WH;
    if (warp == 0) {
        tmem_alloc(&s_tmem, tmem_cols);
        tmem_relinquish();
    }
    if (tid == 0) mbar_init(&s_bar, 1);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t tl = tmem + ((uint32_t)((warp & 3) * 32) << 16);  // this thread's lane, column 0
    const uint32_t col_st = (uint32_t)(D * W);                  // (F', F''/D) pairs of layer k at col_st + (k-1) W
    const uint32_t sa_opZ = smem_addr(opZ), sa_opT = smem_addr(opT), sa_w = smem_addr(w16);
    const int L = lay.L;
    const bool want_A = A != nullptr;
    const int g = lane >> 2, t4 = lane & 3;
    float *st = stage_base + (size_t)(warp * 8 + g) * stage_stride;
    uint32_t phase = 0;
    bool aborted = false;

    const int64_t n_tiles = (n_qp + kTile - 1) / kTile;
    int64_t tile = blockIdx.x;
    // F of the next tile is loaded while the current one is in the network passes
    float Fn[9];
    auto load_F = [&](int64_t t, float (&dst)[9]) {
        const int64_t qq = t * kTile + row;
        const bool v = t < n_tiles && qq < n_qp;
#pragma unroll
        for (int c = 0; c < 9; ++c) dst[c] = v ? Fg[c * n_qp + qq] : ((c % 4) == 0 ? 1.f : 0.f);
    };
    load_F(tile, Fn);
    for (; tile < n_tiles; tile += gridDim.x) {
        float F[9], K[D], Jm1;
        PolyChain<float> ch;
#pragma unroll
        for (int c = 0; c < 9; ++c) F[c] = Fn[c];
        load_F(tile + gridDim.x, Fn);
        bool bad = !kin_scalars_f32<NF>(F, kc, K, Jm1, &ch);
        if (bad) {
#pragma unroll
            for (int c = 0; c < 9; ++c) F[c] = (c % 4) == 0 ? 1.f : 0.f;
            kin_scalars_f32<NF>(F, kc, K, Jm1, &ch);
        }

        // ---- forward values; layer 1 in fp32. Neurons go in pairs (packed FP32); tensor
        // memory holds, for the pair (j, j + 1), half2(s_j, s_j+1) in column j and
        // half2(t_j, t_j+1) in column j + 1 (t later replaced by D = t zbar).
        float2 np2 = make_float2(0.f, 0.f);
#pragma unroll 1
        for (int c = 0; c < NCH; ++c) {
            float zz[CH];
            uint32_t sv[CH];
#pragma unroll
            for (int u = 0; u < CH; u += 4) {  // a quad of neurons: two pairs, 128-bit loads
                const int j = j0 + c * CH + u;
                const float4 cq = ld4(s32 + lay.c + j);
                const float4 aq = (L == 1) ? ld4(s32 + lay.a + j) : make_float4(0.f, 0.f, 0.f, 0.f);
                float4 wq[D];
#pragma unroll
                for (int m = 0; m < D; ++m) wq[m] = ld4(s32 + lay.W1t + m * W + j);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int uu = u + 2 * h;
                    float2 y2 = qh(cq, h);
#pragma unroll
                    for (int m = 0; m < D; ++m) y2 = __ffma2_rn(qh(wq[m], h), bc2(K[m]), y2);
                    float2 z2, s2, t2;
                    act2(y2, z2, s2, t2);
                    sv[uu] = pack_half2(s2.x, s2.y);
                    sv[uu + 1] = pack_half2(t2.x, t2.y);
                    zz[uu] = z2.x;
                    zz[uu + 1] = z2.y;
                    if (L == 1) np2 = __ffma2_rn(qh(aq, h), z2, np2);
                }
            }
            tmem_st<CH>(tl + col_st + j0 + c * CH, sv);
            if (L > 1) {
#pragma unroll
                for (int u = 0; u < CH; u += 8) store_row8<W>(opZ, row, j0 + c * CH + u, zz + u);
            }
        }
        for (int k = 2; k <= L; ++k) {
            const uint32_t wk = sa_w + (uint32_t)(lay.Ab + (k - 2) * W * W * 2);
            if (!mma_round(&s_bar, phase, [&] { issue_gemm<W>(tmem, sa_opZ, wk); })) {
                aborted = true;
                break;
            }
            const float *ck = s32 + lay.c + (k - 1) * W;
            const float *Bk = s32 + lay.Bkt + (k - 2) * D * W;
#pragma unroll 1
            for (int c = 0; c < NCH; ++c) {
                uint32_t acc[CH], sv[CH];
                float zz[CH];
                tmem_ld<CH>(tl + j0 + c * CH, acc);
                tmem_wait_ld();
#pragma unroll
                for (int u = 0; u < CH; u += 4) {
                    const int j = j0 + c * CH + u;
                    const float4 cq = ld4(ck + j);
                    const float4 aq = (k == L) ? ld4(s32 + lay.a + j) : make_float4(0.f, 0.f, 0.f, 0.f);
                    float4 bq[D];
#pragma unroll
                    for (int m = 0; m < D; ++m) bq[m] = ld4(Bk + m * W + j);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int uu = u + 2 * h;
                        float2 y2 = __fadd2_rn(make_float2(__uint_as_float(acc[uu]), __uint_as_float(acc[uu + 1])),
                                               qh(cq, h));
#pragma unroll
                        for (int m = 0; m < D; ++m) y2 = __ffma2_rn(qh(bq[m], h), bc2(K[m]), y2);
                        float2 z2, s2, t2;
                        act2(y2, z2, s2, t2);
                        sv[uu] = pack_half2(s2.x, s2.y);
                        sv[uu + 1] = pack_half2(t2.x, t2.y);
                        zz[uu] = z2.x;
                        zz[uu + 1] = z2.y;
                        if (k == L) np2 = __ffma2_rn(qh(aq, h), z2, np2);
                    }
                }
                tmem_st<CH>(tl + col_st + (k - 1) * W + j0 + c * CH, sv);
                if (k < L) {
#pragma unroll
                    for (int u = 0; u < CH; u += 8) store_row8<W>(opZ, row, j0 + c * CH + u, zz + u);
                }
            }
        }
        if (aborted) break;
        float npart = np2.x + np2.y;
        if (part == 0) npart += dot_w<D>(s32 + lay.b, K);

        // ---- reverse adjoints: zbar_L = a; ybar = F' zbar; D = F'' zbar; zbar_{k-1} = ybar_k A_k
        // two accumulator sets (even and odd pair of a quad) shorten the dependency chains
        float2 dN2[2][D];
#pragma unroll
        for (int m = 0; m < D; ++m) {
            dN2[0][m] = make_float2(part == 0 ? s32[lay.b + m] : 0.f, 0.f);
            dN2[1][m] = make_float2(0.f, 0.f);
        }
        tmem_wait_st();  // layer L's (F', F'') pairs are read back below
        for (int k = L; k >= 1; --k) {
            if (k < L) {
                const uint32_t wt = sa_w + (uint32_t)(lay.Atb + (k - 1) * W * W * 2);  // A_{k+1}^T
                if (!mma_round(&s_bar, phase, [&] { issue_gemm<W>(tmem, sa_opZ, wt); })) {
                    aborted = true;
                    break;
                }
            }
            const float *Bw = (k == 1) ? (s32 + lay.W1t) : (s32 + lay.Bkt + (k - 2) * D * W);
#pragma unroll 1
            for (int c = 0; c < NCH; ++c) {
                uint32_t sv[CH], acc[CH];
                float yv[CH];
                tmem_ld<CH>(tl + col_st + (k - 1) * W + j0 + c * CH, sv);
                if (k < L) tmem_ld<CH>(tl + j0 + c * CH, acc);
                tmem_wait_ld();
#pragma unroll
                for (int u = 0; u < CH; u += 4) {
                    const int j = j0 + c * CH + u;
                    const float4 aq = (k < L) ? make_float4(0.f, 0.f, 0.f, 0.f) : ld4(s32 + lay.a + j);
                    float4 bq[D];
#pragma unroll
                    for (int m = 0; m < D; ++m) bq[m] = ld4(Bw + m * W + j);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int uu = u + 2 * h;
                        const float2 zb2 = (k < L) ? make_float2(__uint_as_float(acc[uu]), __uint_as_float(acc[uu + 1]))
                                                   : qh(aq, h);
                        const float2 s2 = unpack_half2(sv[uu]), t2 = unpack_half2(sv[uu + 1]);
                        const float2 yb2 = __fmul2_rn(s2, zb2);
                        const float2 d2 = __fmul2_rn(t2, zb2);
                        sv[uu + 1] = pack_half2(d2.x, d2.y);
#pragma unroll
                        for (int m = 0; m < D; ++m) dN2[h][m] = __ffma2_rn(qh(bq[m], h), yb2, dN2[h][m]);
                        yv[uu] = yb2.x;
                        yv[uu + 1] = yb2.y;
                    }
                }
                tmem_st<CH>(tl + col_st + (k - 1) * W + j0 + c * CH, sv);
                if (k >= 2) {
#pragma unroll
                    for (int u = 0; u < CH; u += 8) store_row8<W>(opZ, row, j0 + c * CH + u, yv + u);
                }
            }
        }
        if (aborted) break;
        float dN[D];
#pragma unroll
        for (int m = 0; m < D; ++m) dN[m] = (dN2[0][m].x + dN2[0][m].y) + (dN2[1][m].x + dN2[1][m].y);

        // ---- forward tangents and the Hessian H = sum_k J_k^T diag(D_k) J_k, on neuron
        // pairs: H2 holds the even and the odd neurons' partial sums
        constexpr int NHA = D == 3 ? 2 : 1;  // Hessian accumulator sets (registers allow two for d = 3)
        float2 H2[NHA][NH];
#pragma unroll
        for (int a2 = 0; a2 < NHA; ++a2)
#pragma unroll
            for (int i = 0; i < NH; ++i) H2[a2][i] = make_float2(0.f, 0.f);
        if (want_A) {
            tmem_wait_st();
#pragma unroll 1
            for (int c = 0; c < NCH; ++c) {
                uint32_t sv[CH];
                float tv[D][CH];
                tmem_ld<CH>(tl + col_st + j0 + c * CH, sv);
                tmem_wait_ld();
#pragma unroll
                for (int u = 0; u < CH; u += 4) {
                    const int j = j0 + c * CH + u;
                    float4 wq[D];
#pragma unroll
                    for (int m = 0; m < D; ++m) wq[m] = ld4(s32 + lay.W1t + m * W + j);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int uu = u + 2 * h;
                        float2(&Hh)[NH] = H2[h % NHA];
                        const float2 s2 = unpack_half2(sv[uu]), d2 = unpack_half2(sv[uu + 1]);
#pragma unroll
                        for (int m = 0; m < D; ++m) {
                            const float2 wm = qh(wq[m], h);
                            const float2 dm = __fmul2_rn(d2, wm);
#pragma unroll
                            for (int n = 0; n <= m; ++n)
                                Hh[m * (m + 1) / 2 + n] = __ffma2_rn(dm, qh(wq[n], h), Hh[m * (m + 1) / 2 + n]);
                            const float2 t2 = __fmul2_rn(s2, wm);
                            tv[m][uu] = t2.x;
                            tv[m][uu + 1] = t2.y;
                        }
                    }
                }
                if (L > 1) {
#pragma unroll
                    for (int m = 0; m < D; ++m)
#pragma unroll
                        for (int u = 0; u < CH; u += 8) store_row8<W>(opT + m * OPB, row, j0 + c * CH + u, tv[m] + u);
                }
            }
            for (int k = 2; k <= L; ++k) {
                const uint32_t wk = sa_w + (uint32_t)(lay.Ab + (k - 2) * W * W * 2);
                if (!mma_round(&s_bar, phase, [&] {
#pragma unroll
                        for (int m = 0; m < D; ++m)
                            issue_gemm<W>(tmem + (uint32_t)(m * W), sa_opT + (uint32_t)(m * OPB), wk);
                    })) {
                    aborted = true;
                    break;
                }
                const float *Bk = s32 + lay.Bkt + (k - 2) * D * W;
#pragma unroll 1
                for (int c = 0; c < NCH; ++c) {
                    uint32_t jv[D][CH], sv[CH];
#pragma unroll
                    for (int m = 0; m < D; ++m) tmem_ld<CH>(tl + m * W + j0 + c * CH, jv[m]);
                    tmem_ld<CH>(tl + col_st + (k - 1) * W + j0 + c * CH, sv);
                    tmem_wait_ld();
                    float tv[D][CH];
#pragma unroll
                    for (int u = 0; u < CH; u += 4) {
                        const int j = j0 + c * CH + u;
                        float4 bq[D];
#pragma unroll
                        for (int m = 0; m < D; ++m) bq[m] = ld4(Bk + m * W + j);
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int uu = u + 2 * h;
                            float2(&Hh)[NH] = H2[h % NHA];
                            const float2 s2 = unpack_half2(sv[uu]), d2 = unpack_half2(sv[uu + 1]);
                            float2 Jm[D];
#pragma unroll
                            for (int m = 0; m < D; ++m)
                                Jm[m] = __fadd2_rn(make_float2(__uint_as_float(jv[m][uu]), __uint_as_float(jv[m][uu + 1])),
                                                   qh(bq[m], h));
#pragma unroll
                            for (int m = 0; m < D; ++m) {
                                const float2 dm = __fmul2_rn(d2, Jm[m]);
#pragma unroll
                                for (int n = 0; n <= m; ++n)
                                    Hh[m * (m + 1) / 2 + n] = __ffma2_rn(dm, Jm[n], Hh[m * (m + 1) / 2 + n]);
                                const float2 t2 = __fmul2_rn(s2, Jm[m]);
                                tv[m][uu] = t2.x;
                                tv[m][uu + 1] = t2.y;
                            }
                        }
                    }
                    if (k < L) {
#pragma unroll
                        for (int m = 0; m < D; ++m)
#pragma unroll
                            for (int u = 0; u < CH; u += 8) store_row8<W>(opT + m * OPB, row, j0 + c * CH + u, tv[m] + u);
                    }
                }
            }
            if (aborted) break;
        }
        float Hs[NH];
#pragma unroll
        for (int i = 0; i < NH; ++i) {
            Hs[i] = H2[0][i].x + H2[0][i].y;
            if constexpr (NHA > 1) Hs[i] += H2[NHA - 1][i].x + H2[NHA - 1][i].y;
        }

        // ---- the point's partial sums over its threads: npart, dN, Hs
        {
            float *mine = red + tid;  // entry i at mine[i * kThreads]
            mine[0] = npart;
#pragma unroll
            for (int m = 0; m < D; ++m) mine[(1 + m) * kThreads] = dN[m];
#pragma unroll
            for (int i = 0; i < NH; ++i) mine[(1 + D + i) * kThreads] = Hs[i];
            __syncthreads();
#pragma unroll
            for (int p = 1; p < SPLIT; ++p) {
                const float *other = red + row + ((part + p) % SPLIT) * kTile;
                npart += other[0];
#pragma unroll
                for (int m = 0; m < D; ++m) dN[m] += other[(1 + m) * kThreads];
#pragma unroll
                for (int i = 0; i < NH; ++i) Hs[i] += other[(1 + D + i) * kThreads];
            }
            __syncthreads();
        }

        // ---- P, A, Psi: the warp's 32 points in 4 rounds of 8 groups of 4 lanes
        float cvec[D];
#pragma unroll
        for (int m = 0; m < D; ++m) cvec[m] = dN[m] - s32[lay.n0 + m];
        if constexpr (NF == 0) {
            if (kc.kin == COMMET_KIN_POLYCONVEX) poly_to_invariants<float>(ch, cvec, Hs);
        }
        constexpr int kRounds = 4 / SPLIT;
#pragma unroll 1
        for (int r = kRounds * part; r < kRounds * part + kRounds; ++r) {
            const int src = 8 * r + g;
            float Fr[9], cr[D], Hr[NH], Kr[D];
#pragma unroll
            for (int c = 0; c < 9; ++c) Fr[c] = __shfl_sync(0xffffffffu, F[c], src);
#pragma unroll
            for (int m = 0; m < D; ++m) {
                cr[m] = __shfl_sync(0xffffffffu, cvec[m], src);
                Kr[m] = __shfl_sync(0xffffffffu, K[m], src);
            }
#pragma unroll
            for (int i = 0; i < NH; ++i) Hr[i] = want_A ? __shfl_sync(0xffffffffu, Hs[i], src) : 0.f;
            const float Jr = __shfl_sync(0xffffffffu, Jm1, src);
            const float npr = __shfl_sync(0xffffffffu, npart, src);
            const bool badr = __shfl_sync(0xffffffffu, bad ? 1 : 0, src) != 0;
            const int64_t qr = tile * kTile + (warp & 3) * 32 + src;
            const bool validr = qr < n_qp;
            __syncwarp();
            stage_kinematics<float, NF>(Fr, kc, cr, Jr, t4, st);
            __syncwarp();
            bool nonfinite = false;
            // spatial form: P and A go to the point's area after its staging, then are
            // pushed forward to tau (written through P) and c (through A)
            constexpr int kStageF = (9 * D + 54 + 18 * NF + 5 + NF + 3) / 4 * 4;
            float *pa = st + kStageF;
            for (int a = t4; a < 9; a += 4) {
                float Pa, Arow[9];
                if (want_A) {
                    assemble_row<float, NF>(a, st, Hr, cr, Pa, Arow);
                } else {
                    Pa = assemble_P<float, NF>(a, st, cr);
#pragma unroll
                    for (int b = 0; b < 9; ++b) Arow[b] = 0.f;
                }
                bool fin = isfinite(Pa);
#pragma unroll
                for (int b = 0; b < 9; ++b) fin = fin && isfinite(Arow[b]);
                nonfinite |= !fin;
                const bool nan_out = badr || !fin;
                if constexpr (SPATIAL) {
                    pa[a] = nan_out ? NAN : Pa;
                    if (want_A) {
#pragma unroll
                        for (int b = 0; b < 9; ++b) pa[9 + 9 * a + b] = nan_out ? NAN : Arow[b];
                    }
                } else if (validr) {
                    P[a * n_qp + qr] = nan_out ? NAN : Pa;
                    if (want_A) {
#pragma unroll
                        for (int b = 0; b < 9; ++b) A[(9 * a + b) * n_qp + qr] = nan_out ? NAN : Arow[b];
                    }
                }
            }
            if constexpr (SPATIAL) {
                __syncwarp();
                const int64_t qo = validr ? qr : 0;
                push_forward_group<float>(st + Stage<D, NF>::F, pa, pa + 9, t4, validr, P + qo,
                                          want_A ? A + qo : nullptr, n_qp);
            }
            const unsigned nf_mask = __ballot_sync(0xffffffffu, nonfinite);
            const bool grp_nonfinite = ((nf_mask >> (g * 4)) & 0xFu) != 0u;
            if (validr && t4 == 0) {
                float Psi = npr + kc.kappa * Jr * Jr;
#pragma unroll
                for (int m = 0; m < D; ++m) Psi -= s32[lay.n0 + m] * (Kr[m] - s32[lay.K0 + m]);
                const bool rep = badr || grp_nonfinite || !isfinite(Psi);
                if (psi != nullptr) psi[qr] = rep ? NAN : Psi;
                if (rep && status != nullptr) {
                    atomicAdd(&status[0], 1);
                    atomicMin(&status[1], (int32_t)(qr < INT32_MAX ? qr : INT32_MAX));
                }
            }
            __syncwarp();
        }
    }
    if (aborted) {
        // an MMA batch did not complete within the bound: report the points this CTA did not
        // produce, give the batch a last bounded wait, and release tensor memory
        if (tid == 0) {
            atomicOr(err, 1);
            if (status != nullptr) {
                int64_t missing = 0;
                for (int64_t t2 = tile; t2 < n_tiles; t2 += gridDim.x) {
                    const int64_t left = n_qp - t2 * kTile;
                    missing += left < kTile ? left : kTile;
                }
                const int64_t first = tile * kTile;
                atomicAdd(&status[0], (int32_t)(missing < INT32_MAX ? missing : INT32_MAX));
                atomicMin(&status[1], (int32_t)(first < INT32_MAX ? first : INT32_MAX));
            }
        }
        mbar_wait_bounded(&s_bar, phase ^ 1u, kWaitTries);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, tmem_cols);
}

// ------------------------------------------------------------------- host side

static TcLayout tc_layout(int d, int W, int L) {
    TcLayout l{};
    l.d = d;
    l.dp = (d + 3) / 4 * 4;
    l.W = W;
    l.L = L;
    int o = 0;
    // W1 and B_k transposed: row m holds input m's weights of all W neurons, so that the
    // weights of neighbouring neurons (a packed pair, a 128-bit load) are adjacent
    l.W1t = o; o += d * W;
    l.Bkt = o; o += (L - 1) * d * W;
    l.c = o; o += L * W;
    l.a = o; o += W;
    l.b = o; o += l.dp;
    l.n0 = o; o += l.dp;
    l.K0 = o; o += l.dp;
    l.f32_total = (o + 3) / 4 * 4;
    l.Ab = 0;
    l.Atb = (L - 1) * W * W * 2;
    l.b16_bytes = 2 * (L - 1) * W * W * 2;
    return l;
}

static size_t f32_part_bytes(const TcLayout &l) { return ((size_t)l.f32_total * 4 + 15) / 16 * 16; }

// Builds the bf16-path weight block from the fp32 packed block of the model (device to
// host copy at creation; kept in m->d_bf16, followed by a 16-byte device error word).
int prepare_bf16_weights(commet_model *m) {
    const int d = m->d, W = m->W, L = m->L;
    const NetLayout &nl = m->lay;
    const TcLayout tl = tc_layout(d, W, L);
    float *h = new float[nl.total];
    if (cudaMemcpy(h, m->d_weights, sizeof(float) * nl.total, cudaMemcpyDeviceToHost) != cudaSuccess) {
        delete[] h;
        return COMMET_ERR_CUDA;
    }
    const int dpn = (d + 3) / 4 * 4;
    const size_t f32_bytes = f32_part_bytes(tl);
    const size_t total = f32_bytes + (size_t)tl.b16_bytes + 16;
    unsigned char *buf = new unsigned char[total]();
    float *f = reinterpret_cast<float *>(buf);
    unsigned char *bb = buf + f32_bytes;
    for (int j = 0; j < W; ++j)
        for (int mm = 0; mm < d; ++mm) f[tl.W1t + mm * W + j] = h[nl.W1r + j * dpn + mm];
    for (int k = 0; k < L - 1; ++k)
        for (int j = 0; j < W; ++j) {
            for (int mm = 0; mm < d; ++mm) f[tl.Bkt + (k * d + mm) * W + j] = h[nl.Bt + k * d * W + mm * W + j];
            for (int i = 0; i < W; ++i) {
                const __nv_bfloat16 aji = __float2bfloat16_rn(h[nl.Ar + k * W * W + j * W + i]);
                *reinterpret_cast<__nv_bfloat16 *>(bb + tl.Ab + k * W * W * 2 + cm_byte(j, i, W)) = aji;
                *reinterpret_cast<__nv_bfloat16 *>(bb + tl.Atb + k * W * W * 2 + cm_byte(i, j, W)) = aji;
            }
        }
    for (int i = 0; i < L * W; ++i) f[tl.c + i] = h[nl.c + i];
    for (int j = 0; j < W; ++j) f[tl.a + j] = h[nl.a + j];
    for (int mm = 0; mm < d; ++mm) {
        f[tl.b + mm] = h[nl.b + mm];
        f[tl.n0 + mm] = h[nl.n0 + mm];
        f[tl.K0 + mm] = h[nl.K0 + mm];
    }
    delete[] h;
    cudaFree(m->d_bf16);
    m->d_bf16 = nullptr;
    int rc = COMMET_OK;
    if (cudaMalloc(&m->d_bf16, total) != cudaSuccess ||
        cudaMemcpy(m->d_bf16, buf, total, cudaMemcpyHostToDevice) != cudaSuccess)
        rc = COMMET_ERR_CUDA;
    m->bf16_bytes = total;
    delete[] buf;
    return rc;
}

template <int NF, int W, bool SPATIAL>
static int bf16_typed(const commet_model *m, int64_t n_qp, const void *F, void *psi, void *P, void *A,
                      int32_t *status, cudaStream_t s) {
    constexpr int D = 3 + 2 * NF;
    const int L = m->L;
    // tensor memory: D W accumulator columns + L W (F', F'') columns, a power of two >= 32
    const int need_cols = (D + L) * W;
    if (need_cols > 512) return COMMET_ERR_UNSUPPORTED;
    uint32_t cols = 32;
    while ((int)cols < need_cols) cols <<= 1;
    KinConst<float> kc{};
    kc.kin = m->kp.kin;
    kc.stress_free = m->kp.stress_free;
    kc.kappa = (float)m->kp.kappa;
    for (int f = 0; f < 2; ++f)
        for (int c = 0; c < 3; ++c) kc.fib[f][c] = (float)m->kp.fib[f][c];
    const TcLayout tl = tc_layout(m->d, W, L);
    const size_t f32_bytes = f32_part_bytes(tl);
    const int stage = (9 * D + 54 + 18 * NF + 5 + NF + 3) / 4 * 4 + (SPATIAL ? 90 : 0);
    const int stage_stride = stage | 1;  // odd: the 32 group areas fall on distinct banks
    const size_t opb = (size_t)kTile * W * 2;
    const int nred = 1 + D + D * (D + 1) / 2;
    constexpr int threads = kTile * TcSplit<NF>::value;
    size_t smem = (size_t)tl.b16_bytes + (1 + D) * opb + f32_bytes + (size_t)threads * nred * 4 +
                  (size_t)(threads / 32) * 8 * stage_stride * 4;
    int dev = 0, smem_max = 0, smem_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    // no more CTAs per SM than tensor memory holds: pad the request so that shared memory
    // admits at most 512 / cols of them
    const int ctas_tmem = 512 / (int)cols;
    const size_t floor_req = (size_t)smem_sm / (ctas_tmem + 1) + 1;
    smem = std::max(smem, floor_req);
    if ((size_t)smem_max < smem) return COMMET_ERR_UNSUPPORTED;
    auto kern = bf16_tc_kernel<NF, W, SPATIAL>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return COMMET_ERR_CUDA;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    per_sm = std::max(1, std::min(per_sm, ctas_tmem));
    const int64_t n_tiles = (n_qp + kTile - 1) / kTile;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(n_tiles, (int64_t)sm_count() * per_sm));
    const float *w32 = (const float *)m->d_bf16;
    const unsigned char *w16 = (const unsigned char *)m->d_bf16 + f32_bytes;
    int *err = (int *)((unsigned char *)m->d_bf16 + f32_bytes + tl.b16_bytes);
    kern<<<grid, threads, smem, s>>>(w32, w16, tl, kc, n_qp, (const float *)F, (float *)psi, (float *)P, (float *)A,
                                   status, err, cols, stage_stride);
    return cudaGetLastError() == cudaSuccess ? COMMET_OK : COMMET_ERR_CUDA;
}

template <bool SPATIAL>
static int bf16_dispatch(const commet_model *m, int64_t n_qp, const void *F, void *psi, void *P, void *A,
                         int32_t *status, cudaStream_t s) {
    if (n_qp == 0) return COMMET_OK;
    const int nf = m->kp.nf, W = m->W;
    if (nf == 0 && W == 64) return bf16_typed<0, 64, SPATIAL>(m, n_qp, F, psi, P, A, status, s);
    if (nf == 0 && W == 32) return bf16_typed<0, 32, SPATIAL>(m, n_qp, F, psi, P, A, status, s);
    if (nf == 2 && W == 32) return bf16_typed<2, 32, SPATIAL>(m, n_qp, F, psi, P, A, status, s);
    return COMMET_ERR_UNSUPPORTED;
}

int launch_const_update_bf16(const commet_model *m, int64_t n_qp, const void *F, void *psi, void *P, void *A,
                             int32_t *status, cudaStream_t s, bool spatial) {
    if (m->d_bf16 == nullptr) return COMMET_ERR_UNSUPPORTED;
    return spatial ? bf16_dispatch<true>(m, n_qp, F, psi, P, A, status, s)
                   : bf16_dispatch<false>(m, n_qp, F, psi, P, A, status, s);
}

}  // namespace commet
