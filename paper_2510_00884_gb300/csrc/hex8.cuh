// Hex8 reference-element data shared by the element kernels: shape-function gradients
// at the 2x2x2 Gauss points and their physical counterparts (Sec. 2.1 discretisation).
#pragma once

#include <cuda_runtime.h>

namespace commet {

// Reference-cube data: node I at (+-1,+-1,+-1) lexicographic (x fastest), Gauss point q
// at (+-1/sqrt3)^3 in the same order, weight 1.
template <typename T>
__device__ __forceinline__ void shape_grad_ref(int q, T g[8][3]) {
    const T gp = T(0.57735026918962576451);
#pragma unroll
    for (int I = 0; I < 8; ++I) {
        T xi[3], zq[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            xi[a] = ((I >> a) & 1) ? T(1) : T(-1);
            zq[a] = ((q >> a) & 1) ? gp : -gp;
        }
        const T f0 = T(1) + xi[0] * zq[0], f1 = T(1) + xi[1] * zq[1], f2 = T(1) + xi[2] * zq[2];
        g[I][0] = T(0.125) * xi[0] * f1 * f2;
        g[I][1] = T(0.125) * xi[1] * f0 * f2;
        g[I][2] = T(0.125) * xi[2] * f0 * f1;
    }
}

// grad_X phi_I = Je^{-T} grad_xi phi_I and w = det Je for one element/Gauss point.
template <typename T>
__device__ __forceinline__ void physical_grads(const T Xe[8][3], int q, T gX[8][3], T &w) {
    T g[8][3];
    shape_grad_ref<T>(q, g);
    T Je[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            T s = T(0);
#pragma unroll
            for (int I = 0; I < 8; ++I) s += Xe[I][a] * g[I][b];
            Je[3 * a + b] = s;
        }
    T cof[9];
    cof[0] = Je[4] * Je[8] - Je[5] * Je[7];
    cof[1] = Je[5] * Je[6] - Je[3] * Je[8];
    cof[2] = Je[3] * Je[7] - Je[4] * Je[6];
    cof[3] = Je[2] * Je[7] - Je[1] * Je[8];
    cof[4] = Je[0] * Je[8] - Je[2] * Je[6];
    cof[5] = Je[1] * Je[6] - Je[0] * Je[7];
    cof[6] = Je[1] * Je[5] - Je[2] * Je[4];
    cof[7] = Je[2] * Je[3] - Je[0] * Je[5];
    cof[8] = Je[0] * Je[4] - Je[1] * Je[3];
    const T det = Je[0] * cof[0] + Je[1] * cof[1] + Je[2] * cof[2];
    const T id = T(1) / det;
#pragma unroll
    for (int I = 0; I < 8; ++I)
#pragma unroll
        for (int a = 0; a < 3; ++a)
            gX[I][a] = (cof[3 * a] * g[I][0] + cof[3 * a + 1] * g[I][1] + cof[3 * a + 2] * g[I][2]) * id;
    w = det;
}

}  // namespace commet
