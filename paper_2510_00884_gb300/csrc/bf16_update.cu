// Constitutive update with the hidden W x W layers on bf16 tensor cores (fp32
// accumulate): the COMMET_BF16_MLP precision. The network derivatives follow the same
// scheme as the FP64/FP32 kernel (forward values, reverse adjoints, forward tangents
// consumed into the Hessian); here every hidden-layer product
//     values    Y_k   = Z_{k-1} A_k^T       [16 points x W] = [16 x W][W x W]
//     adjoints  Zb_{k-1} = Yb_k A_k         [16 x W]
//     tangents  J_k^(m) = (s_{k-1} J_{k-1}^(m)) A_k^T   for each input m
// is a warp-level bf16 MMA (m16n8k16) with the 16 points of a warp along M. The fp32
// accumulator fragment of one layer is, element for element, the A-operand fragment of
// the next, so activations stay in registers; only F', F'' (s_k) and the adjoint
// weights (D_k) go to shared memory. Layer 1 (d inputs), the output layer, the
// activations, the Hessian sums and the kinematics/P/A assembly are fp32.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>

#include "device_math.cuh"
#include "internal.h"

namespace commet {

namespace {

// Offsets of the bf16-path weight block: an fp32 part (units of float) followed by a
// bf16 part (units of bf16) holding A_k row-major and A_k^T row-major with padded rows.
struct B16Layout {
    int d, dp, W, L, ld;
    int W1, Bk, c, a, b, n0, K0, f32_total;  // float offsets
    int Ab, Atb, b16_total;                   // bf16 offsets (from the start of the bf16 part)
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

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

constexpr int kPW = 16;  // points per warp (the MMA's M)

}  // namespace

// Per-warp shared memory: s_k and t_k/D_k in fp16 for 16 points x W neurons x L layers,
// point-major with a pad (pstride halves per point), reused at the end as the 16
// points' fp32 staging areas. fp16 keeps 11 bits, finer than the bf16 MMA inputs.
template <int NF, int W, bool SPATIAL>
__global__ void __launch_bounds__(256)
    bf16_update_kernel(const float *__restrict__ gw32, const __nv_bfloat16 *__restrict__ gw16, B16Layout lay,
                       KinConst<float> kc, int64_t n_qp, const float *__restrict__ Fg, float *__restrict__ psi,
                       float *__restrict__ P, float *__restrict__ A, int32_t *__restrict__ status, int pstride) {
    constexpr int D = 3 + 2 * NF, NH = D * (D + 1) / 2;
    constexpr int NT = W / 8;   // n-tiles (8 neurons)
    constexpr int KT = W / 16;  // k-tiles (16 neurons)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *s32 = reinterpret_cast<float *>(smem_raw);
    const int f32_bytes = (lay.f32_total * 4 + 15) / 16 * 16;
    __nv_bfloat16 *s16 = reinterpret_cast<__nv_bfloat16 *>(smem_raw + f32_bytes);
    const int b16_bytes = (lay.b16_total * 2 + 15) / 16 * 16;
    {
        const int4 *src = reinterpret_cast<const int4 *>(gw32);
        int4 *dst = reinterpret_cast<int4 *>(smem_raw);
        for (int i = threadIdx.x; i < f32_bytes / 16; i += blockDim.x) dst[i] = src[i];
        const int4 *src16 = reinterpret_cast<const int4 *>(gw16);
        int4 *dst16 = reinterpret_cast<int4 *>(smem_raw + f32_bytes);
        for (int i = threadIdx.x; i < b16_bytes / 16; i += blockDim.x) dst16[i] = src16[i];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const int L = lay.L;
    __half *ws = reinterpret_cast<__half *>(smem_raw + f32_bytes + b16_bytes) + (size_t)warp * kPW * pstride;
    // s_k of point p, neuron j: ws[p * pstride + (k-1) * W + j]; t_k / D_k at (L + k - 1) * W
    const int64_t n_tiles = (n_qp + kPW - 1) / kPW;
    const int64_t n_gwarps = (int64_t)gridDim.x * (blockDim.x >> 5);

    for (int64_t tile = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; tile < n_tiles; tile += n_gwarps) {
        // ---- kinematics of the two points this lane holds (rows g and g + 8)
        float F[2][9], K[2][D], Jm1[2];
        bool bad[2], valid[2];
        PolyChain<float> ch[2];
        int64_t q[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            q[h] = tile * kPW + g + 8 * h;
            valid[h] = q[h] < n_qp;
#pragma unroll
            for (int c = 0; c < 9; ++c) F[h][c] = valid[h] ? Fg[c * n_qp + q[h]] : ((c % 4) == 0 ? 1.f : 0.f);
            bad[h] = !kin_scalars_f32<NF>(F[h], kc, K[h], Jm1[h], &ch[h]);
            if (bad[h]) {
#pragma unroll
                for (int c = 0; c < 9; ++c) F[h][c] = (c % 4) == 0 ? 1.f : 0.f;
                kin_scalars_f32<NF>(F[h], kc, K[h], Jm1[h], &ch[h]);
            }
        }
        __half *wrow[2] = {ws + g * pstride, ws + (g + 8) * pstride};

        // ---- forward values
        float acc[NT][4];
        uint32_t af[KT][4];
        float npart[2] = {0.f, 0.f};
        for (int k = 1; k <= L; ++k) {
            if (k == 1) {
#pragma unroll
                for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int j = 8 * nt + 2 * t + (e & 1), h = e >> 1;
                        float y = s32[lay.c + j];
#pragma unroll
                        for (int m = 0; m < D; ++m) y += s32[lay.W1 + j * lay.dp + m] * K[h][m];
                        acc[nt][e] = y;
                    }
            } else {
                const __nv_bfloat16 *Ab = s16 + lay.Ab + (k - 2) * W * lay.ld;
#pragma unroll
                for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int j = 8 * nt + 2 * t + (e & 1), h = e >> 1;
                        float y = s32[lay.c + (k - 1) * W + j];
#pragma unroll
                        for (int m = 0; m < D; ++m) y += s32[lay.Bk + ((k - 2) * W + j) * lay.dp + m] * K[h][m];
                        acc[nt][e] = y;
                    }
#pragma unroll
                for (int kt = 0; kt < KT; ++kt)
#pragma unroll
                    for (int nt = 0; nt < NT; ++nt) {
                        const __nv_bfloat16 *bp = Ab + (8 * nt + g) * lay.ld + 16 * kt + 2 * t;
                        const uint32_t b0 = *reinterpret_cast<const uint32_t *>(bp);
                        const uint32_t b1 = *reinterpret_cast<const uint32_t *>(bp + 8);
                        mma_bf16(acc[nt], af[kt], b0, b1);
                    }
            }
            // activation; s_k, t_k to shared memory; z to the next layer's A fragments
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int j = 8 * nt + 2 * t + (e & 1), h = e >> 1;
                    float z, s, tt;
                    act(acc[nt][e], z, s, tt);
                    wrow[h][(k - 1) * W + j] = __float2half_rn(s);
                    wrow[h][(L + k - 1) * W + j] = __float2half_rn(tt);
                    if (k == L) npart[h] += s32[lay.a + j] * z;
                    acc[nt][e] = z;
                }
            if (k < L) {
#pragma unroll
                for (int kt = 0; kt < KT; ++kt) {
                    af[kt][0] = pack_bf16(acc[2 * kt][0], acc[2 * kt][1]);
                    af[kt][1] = pack_bf16(acc[2 * kt][2], acc[2 * kt][3]);
                    af[kt][2] = pack_bf16(acc[2 * kt + 1][0], acc[2 * kt + 1][1]);
                    af[kt][3] = pack_bf16(acc[2 * kt + 1][2], acc[2 * kt + 1][3]);
                }
            }
        }
        if (t == 0) {
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int m = 0; m < D; ++m) npart[h] += s32[lay.b + m] * K[h][m];
        }

        // ---- reverse adjoints: zbar_L = a; ybar = s zbar; D = t zbar; zbar_{k-1} = ybar_k A_k
        float dN[2][D];
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int m = 0; m < D; ++m) dN[h][m] = (t == 0) ? s32[lay.b + m] : 0.f;
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[nt][e] = s32[lay.a + 8 * nt + 2 * t + (e & 1)];  // zbar_L
        for (int k = L; k >= 1; --k) {
            const float *Bm = (k == 1) ? (s32 + lay.W1) : (s32 + lay.Bk + (k - 2) * W * lay.dp);
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int j = 8 * nt + 2 * t + (e & 1), h = e >> 1;
                    const float zb = acc[nt][e];
                    const float yb = __half2float(wrow[h][(k - 1) * W + j]) * zb;
                    wrow[h][(L + k - 1) * W + j] =
                        __float2half_rn(__half2float(wrow[h][(L + k - 1) * W + j]) * zb);  // D_k = t_k zbar_k
#pragma unroll
                    for (int m = 0; m < D; ++m) dN[h][m] += Bm[j * lay.dp + m] * yb;
                    acc[nt][e] = yb;
                }
            if (k == 1) break;
#pragma unroll
            for (int kt = 0; kt < KT; ++kt) {
                af[kt][0] = pack_bf16(acc[2 * kt][0], acc[2 * kt][1]);
                af[kt][1] = pack_bf16(acc[2 * kt][2], acc[2 * kt][3]);
                af[kt][2] = pack_bf16(acc[2 * kt + 1][0], acc[2 * kt + 1][1]);
                af[kt][3] = pack_bf16(acc[2 * kt + 1][2], acc[2 * kt + 1][3]);
            }
            const __nv_bfloat16 *Atb = s16 + lay.Atb + (k - 2) * W * lay.ld;
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[nt][e] = 0.f;
#pragma unroll
            for (int kt = 0; kt < KT; ++kt)
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) {
                    const __nv_bfloat16 *bp = Atb + (8 * nt + g) * lay.ld + 16 * kt + 2 * t;
                    const uint32_t b0 = *reinterpret_cast<const uint32_t *>(bp);
                    const uint32_t b1 = *reinterpret_cast<const uint32_t *>(bp + 8);
                    mma_bf16(acc[nt], af[kt], b0, b1);
                }
        }
        __syncwarp();

        // ---- forward tangents and Hessian: H = sum_k J_k^T diag(D_k) J_k
        float Hs[2][NH];
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int i = 0; i < NH; ++i) Hs[h][i] = 0.f;
        const bool want_A = (A != nullptr);  // P alone needs dN/dK, not the Hessian
        // layer 1: J_1 = W1
#pragma unroll
        for (int nt = 0; nt < NT && want_A; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int j = 8 * nt + 2 * t + (e & 1), h = e >> 1;
                const float Dj = __half2float(wrow[h][L * W + j]);
                const float *w1 = s32 + lay.W1 + j * lay.dp;
#pragma unroll
                for (int m = 0; m < D; ++m) {
                    const float dm = Dj * w1[m];
#pragma unroll
                    for (int n = 0; n <= m; ++n) Hs[h][m * (m + 1) / 2 + n] += dm * w1[n];
                }
            }
        if (L >= 2 && want_A) {
            // A fragments of s_1 (x) W1[:, m] for every input m
            uint32_t tf[D][KT][4];
#pragma unroll
            for (int m = 0; m < D; ++m)
#pragma unroll
                for (int kt = 0; kt < KT; ++kt) {
                    float v[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        // element e: nt = 2kt + (e >> 2), (e & 3) as in the C layout
                        const int nt = 2 * kt + (e >> 2), ee = e & 3;
                        const int j = 8 * nt + 2 * t + (ee & 1), h = ee >> 1;
                        v[e] = __half2float(wrow[h][j]) * s32[lay.W1 + j * lay.dp + m];
                    }
                    tf[m][kt][0] = pack_bf16(v[0], v[1]);
                    tf[m][kt][1] = pack_bf16(v[2], v[3]);
                    tf[m][kt][2] = pack_bf16(v[4], v[5]);
                    tf[m][kt][3] = pack_bf16(v[6], v[7]);
                }
            for (int k = 2; k <= L; ++k) {
                const __nv_bfloat16 *Ab = s16 + lay.Ab + (k - 2) * W * lay.ld;
                float jac[D][NT][4];
#pragma unroll
                for (int m = 0; m < D; ++m)
#pragma unroll
                    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            jac[m][nt][e] = s32[lay.Bk + ((k - 2) * W + 8 * nt + 2 * t + (e & 1)) * lay.dp + m];
#pragma unroll
                for (int kt = 0; kt < KT; ++kt)
#pragma unroll
                    for (int nt = 0; nt < NT; ++nt) {
                        const __nv_bfloat16 *bp = Ab + (8 * nt + g) * lay.ld + 16 * kt + 2 * t;
                        const uint32_t b0 = *reinterpret_cast<const uint32_t *>(bp);
                        const uint32_t b1 = *reinterpret_cast<const uint32_t *>(bp + 8);
#pragma unroll
                        for (int m = 0; m < D; ++m) mma_bf16(jac[m][nt], tf[m][kt], b0, b1);
                    }
#pragma unroll
                for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int j = 8 * nt + 2 * t + (e & 1), h = e >> 1;
                        const float Dj = __half2float(wrow[h][(L + k - 1) * W + j]);
#pragma unroll
                        for (int m = 0; m < D; ++m) {
                            const float dm = Dj * jac[m][nt][e];
#pragma unroll
                            for (int n = 0; n <= m; ++n) Hs[h][m * (m + 1) / 2 + n] += dm * jac[n][nt][e];
                        }
                    }
                if (k < L) {
#pragma unroll
                    for (int m = 0; m < D; ++m)
#pragma unroll
                        for (int kt = 0; kt < KT; ++kt) {
                            float v[8];
#pragma unroll
                            for (int e = 0; e < 8; ++e) {
                                const int nt = 2 * kt + (e >> 2), ee = e & 3;
                                const int j = 8 * nt + 2 * t + (ee & 1), h = ee >> 1;
                                v[e] = __half2float(wrow[h][(k - 1) * W + j]) * jac[m][nt][ee];
                            }
                            tf[m][kt][0] = pack_bf16(v[0], v[1]);
                            tf[m][kt][1] = pack_bf16(v[2], v[3]);
                            tf[m][kt][2] = pack_bf16(v[4], v[5]);
                            tf[m][kt][3] = pack_bf16(v[6], v[7]);
                        }
                }
            }
        }

        // ---- reduce over the 4 lanes that share rows g, g + 8
#pragma unroll
        for (int msk = 1; msk <= 2; msk <<= 1)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                npart[h] += __shfl_xor_sync(0xffffffffu, npart[h], msk);
#pragma unroll
                for (int m = 0; m < D; ++m) dN[h][m] += __shfl_xor_sync(0xffffffffu, dN[h][m], msk);
#pragma unroll
                for (int i = 0; i < NH; ++i) Hs[h][i] += __shfl_xor_sync(0xffffffffu, Hs[h][i], msk);
            }
        __syncwarp();

        // ---- P, A, Psi: the 4 lanes (t) of row g act as the point's group, twice
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float *st = reinterpret_cast<float *>(ws + (g + 8 * h) * pstride);  // reuses the s/D area
            float cvec[D];
#pragma unroll
            for (int m = 0; m < D; ++m) cvec[m] = dN[h][m] - s32[lay.n0 + m];
            if constexpr (NF == 0) {
                if (kc.kin == COMMET_KIN_POLYCONVEX) poly_to_invariants<float>(ch[h], cvec, Hs[h]);
            }
            __syncwarp();
            stage_kinematics<float, NF>(F[h], kc, cvec, Jm1[h], t, st);
            __syncwarp();
            bool nonfinite = false;
            // spatial form: P and A go to the point's area after its staging, then are
            // pushed forward to tau (written through P) and c (through A)
            constexpr int kStageF = (9 * D + 54 + 18 * NF + 5 + NF + 3) / 4 * 4;
            float *pa = st + kStageF;
            for (int a = t; a < 9; a += 4) {
                float Pa, Arow[9];
                if (want_A) {
                    assemble_row<float, NF>(a, st, Hs[h], cvec, Pa, Arow);
                } else {
                    Pa = assemble_P<float, NF>(a, st, cvec);
#pragma unroll
                    for (int b = 0; b < 9; ++b) Arow[b] = 0.f;
                }
                bool fin = isfinite(Pa);
#pragma unroll
                for (int b = 0; b < 9; ++b) fin = fin && isfinite(Arow[b]);
                nonfinite |= !fin;
                const bool nan_out = bad[h] || !fin;
                if constexpr (SPATIAL) {
                    pa[a] = nan_out ? NAN : Pa;
                    if (A != nullptr) {
#pragma unroll
                        for (int b = 0; b < 9; ++b) pa[9 + 9 * a + b] = nan_out ? NAN : Arow[b];
                    }
                } else if (valid[h]) {
                    P[a * n_qp + q[h]] = nan_out ? NAN : Pa;
                    if (A != nullptr) {
#pragma unroll
                        for (int b = 0; b < 9; ++b) A[(9 * a + b) * n_qp + q[h]] = nan_out ? NAN : Arow[b];
                    }
                }
            }
            if constexpr (SPATIAL) {
                __syncwarp();
                const int64_t qo = valid[h] ? q[h] : 0;
                push_forward_group<float>(st + Stage<D, NF>::F, pa, pa + 9, t, valid[h], P + qo,
                                          A != nullptr ? A + qo : nullptr, n_qp);
            }
            const unsigned nf_mask = __ballot_sync(0xffffffffu, nonfinite);
            const bool grp_nonfinite = ((nf_mask >> (g * 4)) & 0xFu) != 0u;
            if (valid[h] && t == 0) {
                float Psi = npart[h] + kc.kappa * Jm1[h] * Jm1[h];
#pragma unroll
                for (int m = 0; m < D; ++m) Psi -= s32[lay.n0 + m] * (K[h][m] - s32[lay.K0 + m]);
                const bool rep = bad[h] || grp_nonfinite || !isfinite(Psi);
                if (psi != nullptr) psi[q[h]] = rep ? NAN : Psi;
                if (rep && status != nullptr) {
                    atomicAdd(&status[0], 1);
                    atomicMin(&status[1], (int32_t)(q[h] < INT32_MAX ? q[h] : INT32_MAX));
                }
            }
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------- host side

static B16Layout b16_layout(int d, int W, int L) {
    B16Layout l{};
    l.d = d;
    l.dp = (d + 3) / 4 * 4;
    l.W = W;
    l.L = L;
    l.ld = W + 8;
    int o = 0;
    l.W1 = o; o += W * l.dp;
    l.Bk = o; o += (L - 1) * W * l.dp;
    l.c = o; o += L * W;
    l.a = o; o += W;
    l.b = o; o += l.dp;
    l.n0 = o; o += l.dp;
    l.K0 = o; o += l.dp;
    l.f32_total = (o + 3) / 4 * 4;
    int p = 0;
    l.Ab = p; p += (L - 1) * W * l.ld;
    l.Atb = p; p += (L - 1) * W * l.ld;
    l.b16_total = (p + 7) / 8 * 8;
    return l;
}

// Builds the bf16-path weight block from the fp32 packed block of the model (device
// to host copy at creation; kept in m->d_bf16).
int prepare_bf16_weights(commet_model *m) {
    const int d = m->d, W = m->W, L = m->L;
    const NetLayout &nl = m->lay;
    const B16Layout bl = b16_layout(d, W, L);
    float *h = new float[nl.total];
    if (cudaMemcpy(h, m->d_weights, sizeof(float) * nl.total, cudaMemcpyDeviceToHost) != cudaSuccess) {
        delete[] h;
        return COMMET_ERR_CUDA;
    }
    const int dpn = (d + 3) / 4 * 4;
    const size_t f32_bytes = ((size_t)bl.f32_total * 4 + 15) / 16 * 16;
    const size_t b16_bytes = ((size_t)bl.b16_total * 2 + 15) / 16 * 16;
    unsigned char *buf = new unsigned char[f32_bytes + b16_bytes]();
    float *f = reinterpret_cast<float *>(buf);
    __nv_bfloat16 *bb = reinterpret_cast<__nv_bfloat16 *>(buf + f32_bytes);
    for (int j = 0; j < W; ++j)
        for (int mm = 0; mm < d; ++mm) f[bl.W1 + j * bl.dp + mm] = h[nl.W1r + j * dpn + mm];
    for (int k = 0; k < L - 1; ++k)
        for (int j = 0; j < W; ++j) {
            for (int mm = 0; mm < d; ++mm) f[bl.Bk + (k * W + j) * bl.dp + mm] = h[nl.Bt + k * d * W + mm * W + j];
            for (int i = 0; i < W; ++i) {
                const float aji = h[nl.Ar + k * W * W + j * W + i];
                bb[bl.Ab + (k * W + j) * bl.ld + i] = __float2bfloat16_rn(aji);
                bb[bl.Atb + (k * W + i) * bl.ld + j] = __float2bfloat16_rn(aji);
            }
        }
    for (int i = 0; i < L * W; ++i) f[bl.c + i] = h[nl.c + i];
    for (int j = 0; j < W; ++j) f[bl.a + j] = h[nl.a + j];
    for (int mm = 0; mm < d; ++mm) {
        f[bl.b + mm] = h[nl.b + mm];
        f[bl.n0 + mm] = h[nl.n0 + mm];
        f[bl.K0 + mm] = h[nl.K0 + mm];
    }
    delete[] h;
    cudaFree(m->d_bf16);
    m->d_bf16 = nullptr;
    int rc = COMMET_OK;
    if (cudaMalloc(&m->d_bf16, f32_bytes + b16_bytes) != cudaSuccess ||
        cudaMemcpy(m->d_bf16, buf, f32_bytes + b16_bytes, cudaMemcpyHostToDevice) != cudaSuccess)
        rc = COMMET_ERR_CUDA;
    m->bf16_bytes = f32_bytes + b16_bytes;
    delete[] buf;
    return rc;
}

template <int NF, int W, bool SPATIAL>
static int bf16_typed(const commet_model *m, int64_t n_qp, const void *F, void *psi, void *P, void *A,
                      int32_t *status, cudaStream_t s) {
    KinConst<float> kc{};
    kc.kin = m->kp.kin;
    kc.stress_free = m->kp.stress_free;
    kc.kappa = (float)m->kp.kappa;
    for (int f = 0; f < 2; ++f)
        for (int c = 0; c < 3; ++c) kc.fib[f][c] = (float)m->kp.fib[f][c];
    const B16Layout bl = b16_layout(m->d, W, m->L);
    const size_t f32_bytes = ((size_t)bl.f32_total * 4 + 15) / 16 * 16;
    const size_t b16_bytes = ((size_t)bl.b16_total * 2 + 15) / 16 * 16;
    const int D = 3 + 2 * NF;
    const int stage = (9 * D + 54 + 18 * NF + 5 + NF + 3) / 4 * 4 + (SPATIAL ? 90 : 0);
    const int raw_halves = std::max(2 * m->L * W, 2 * stage);
    const int words = ((raw_halves + 1) / 2 + 31) / 32 * 32 + 4;  // 4-byte words per point
    const int pstride = 2 * words;                                // halves per point
    const size_t per_warp = (size_t)kPW * pstride * 2;
    int dev = 0, smem_max = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if ((size_t)smem_max < f32_bytes + b16_bytes + per_warp) return COMMET_ERR_UNSUPPORTED;
    const int warps = (int)std::min<size_t>(8, (smem_max - f32_bytes - b16_bytes) / per_warp);
    const size_t smem = f32_bytes + b16_bytes + warps * per_warp;
    auto kern = bf16_update_kernel<NF, W, SPATIAL>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return COMMET_ERR_CUDA;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem);
    if (per_sm < 1) per_sm = 1;
    const int64_t n_tiles = (n_qp + kPW - 1) / kPW;
    const int64_t want = (n_tiles + warps - 1) / warps;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sm_count() * per_sm));
    const float *w32 = (const float *)m->d_bf16;
    const __nv_bfloat16 *w16 = (const __nv_bfloat16 *)((const unsigned char *)m->d_bf16 + f32_bytes);
    kern<<<grid, warps * 32, smem, s>>>(w32, w16, bl, kc, n_qp, (const float *)F, (float *)psi, (float *)P,
                                        (float *)A, status, pstride);
    return cudaGetLastError() == cudaSuccess ? COMMET_OK : COMMET_ERR_CUDA;
}

template <bool SPATIAL>
static int bf16_dispatch(const commet_model *m, int64_t n_qp, const void *F, void *psi, void *P, void *A,
                         int32_t *status, cudaStream_t s) {
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
