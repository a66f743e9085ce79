// Closed-form target model used as synthetic training data for the backward pass:
// Psi_t = mu/2 (Ibar1 - 3) + kappa (J - 1)^2 + sum_f k1/(2 k2) (exp(k2 (I4_ff - 1)^2) - 1),
// whose first Piola-Kirchhoff stress is
//   P = mu/2 J^{-2/3} (2F - 2/3 I1 F^{-T}) + 2 kappa (J-1) J F^{-T}
//       + sum_f k1 (I4_f - 1) exp(k2 (I4_f - 1)^2) 2 a_f (x) A_f,   a_f = F A_f.
#include <cuda_runtime.h>

#include <cstdint>

#include "device_math.cuh"
#include "internal.h"

namespace commet {

template <typename T>
__global__ void target_stress_kernel(int64_t n_qp, const T *__restrict__ Fg, int nf, T f00, T f01, T f02, T f10,
                                     T f11, T f12, T mu, T k1, T k2, T kappa, T *__restrict__ P) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n_qp) return;
    T F[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) F[c] = Fg[c * n_qp + q];
    T cof[9], Jc;
    cof_det(F, cof, Jc);
    const T Jm1 = det_minus_one(F), J = T(1) + Jm1;
    T I1 = T(0);
#pragma unroll
    for (int c = 0; c < 9; ++c) I1 += F[c] * F[c];
    const T r3 = dev_rcbrt(J), jm23 = r3 * r3, iJ = T(1) / J;
    T Pq[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) {
        const T H = cof[c] * iJ;
        Pq[c] = T(0.5) * mu * jm23 * (T(2) * F[c] - T(2) / T(3) * I1 * H) + T(2) * kappa * Jm1 * cof[c];
    }
    const T fib[2][3] = {{f00, f01, f02}, {f10, f11, f12}};
    for (int f = 0; f < nf; ++f) {
        T a[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) a[i] = F[3 * i] * fib[f][0] + F[3 * i + 1] * fib[f][1] + F[3 * i + 2] * fib[f][2];
        const T x = a[0] * a[0] + a[1] * a[1] + a[2] * a[2] - T(1);
        const T coef = T(2) * k1 * x * exp(k2 * x * x);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int L = 0; L < 3; ++L) Pq[3 * i + L] += coef * a[i] * fib[f][L];
    }
#pragma unroll
    for (int c = 0; c < 9; ++c) P[c * n_qp + q] = Pq[c];
}

int launch_target_stress(int precision, int64_t n_qp, const void *F, int nf, const double *fib, double mu,
                         double k1, double k2, double kappa, void *P, cudaStream_t s) {
    double f[2][3] = {{0, 0, 0}, {0, 0, 0}};
    for (int i = 0; i < nf; ++i)
        for (int c = 0; c < 3; ++c) f[i][c] = fib[3 * i + c];
    const int tpb = 256;
    const unsigned blocks = (unsigned)((n_qp + tpb - 1) / tpb);
    if (precision == COMMET_F64)
        target_stress_kernel<double><<<blocks, tpb, 0, s>>>(n_qp, (const double *)F, nf, f[0][0], f[0][1], f[0][2],
                                                             f[1][0], f[1][1], f[1][2], mu, k1, k2, kappa,
                                                             (double *)P);
    else
        target_stress_kernel<float><<<blocks, tpb, 0, s>>>(n_qp, (const float *)F, nf, (float)f[0][0],
                                                            (float)f[0][1], (float)f[0][2], (float)f[1][0],
                                                            (float)f[1][1], (float)f[1][2], (float)mu, (float)k1,
                                                            (float)k2, (float)kappa, (float *)P);
    return cudaGetLastError() == cudaSuccess ? COMMET_OK : COMMET_ERR_CUDA;
}

}  // namespace commet
