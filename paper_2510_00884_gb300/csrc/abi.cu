// extern "C" boundary of libcommet: argument checks, handle construction, dispatch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "device_math.cuh"
#include "internal.h"

using namespace commet;

namespace {

bool aligned16(const void *p) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

size_t elem_size(int precision) { return precision == COMMET_F64 ? sizeof(double) : sizeof(float); }

int round4(int x) { return (x + 3) / 4 * 4; }

// Build the packed-weight layout (offsets in elements, each block starting on a
// multiple of 4 elements so that it is 16-byte aligned for float and double).
NetLayout make_layout(int d, int W, int L, bool with_tab) {
    NetLayout l{};
    l.d = d;
    l.W = W;
    l.L = L;
    const int dp = (d + 3) / 4 * 4;
    int o = 0;
    l.W1t = o; o = round4(o + d * W);
    l.W1r = o; o = round4(o + W * dp);
    l.Bt = o; o = round4(o + (L - 1) * d * W);
    l.c = o; o = round4(o + L * W);
    l.a = o; o = round4(o + W);
    l.b = o; o = round4(o + d);
    l.n0 = o; o = round4(o + d);
    l.K0 = o; o = round4(o + d);
    l.tab = 0;
    if (with_tab) {
        l.tab = o;
        o = round4(o + actdf::kSlots);
    }
    // the hidden weights come last: A_k transposed (forward values and tangents), the
    // FP64 layer-2 tangent weights M and A_k row-major (reverse pass); networks whose
    // weights crowd the point slabs out of shared memory read the last one, two or three
    // of these blocks from global memory (L1/L2) instead
    l.At = o; o = round4(o + (L - 1) * W * W);
    l.M = 0;
    if (with_tab && L >= 2) {
        l.M = o;
        o = round4(o + W * W * dp);
    }
    l.Ar = o; o = round4(o + (L - 1) * W * W);
    l.total = o;
    return l;
}

template <typename T>
int upload(const std::vector<double> &h, void **dptr) {
    const size_t bytes = (h.size() * sizeof(T) + 15) / 16 * 16;
    std::vector<unsigned char> buf(bytes, 0);
    T *t = reinterpret_cast<T *>(buf.data());
    for (size_t i = 0; i < h.size(); ++i) t[i] = (T)h[i];
    COMMET_CUDA_TRY(cudaMalloc(dptr, bytes));
    COMMET_CUDA_TRY(cudaMemcpy(*dptr, buf.data(), bytes, cudaMemcpyHostToDevice));
    return COMMET_OK;
}

// n0 = dN/dK and K0 = K at F = I for the stress-free shift, evaluated by the
// constitutive kernel itself and written into the model's packed block.
int stress_free_shift(commet_model *m) {
    const int precision = m->precision, d = m->d;
    const NetLayout &l = m->lay;
    int rc;
    if (!m->kp.stress_free) return COMMET_OK;
    {
        // n0 = dN/dK and K0 = K at F = I, evaluated by the constitutive kernel itself
        const size_t es = elem_size(precision == COMMET_F64 ? COMMET_F64 : COMMET_F32);
        void *dF = nullptr, *dP = nullptr, *dN = nullptr;
        const double I9[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
        unsigned char Fbuf[9 * sizeof(double)];
        for (int c = 0; c < 9; ++c) {
            if (es == 8)
                reinterpret_cast<double *>(Fbuf)[c] = I9[c];
            else
                reinterpret_cast<float *>(Fbuf)[c] = (float)I9[c];
        }
        commet_model tmp = *m;
        tmp.precision = (precision == COMMET_F64) ? COMMET_F64 : COMMET_F32;
        rc = COMMET_ERR_CUDA;
        if (cudaMalloc(&dF, 16 * es) == cudaSuccess && cudaMalloc(&dP, 16 * es) == cudaSuccess &&
            cudaMalloc(&dN, 2 * kMaxD * es) == cudaSuccess &&
            cudaMemcpy(dF, Fbuf, 9 * es, cudaMemcpyHostToDevice) == cudaSuccess) {
            rc = launch_const_update(&tmp, 1, dF, nullptr, dP, nullptr, nullptr, 0, dN);
            if (rc == COMMET_OK && cudaDeviceSynchronize() != cudaSuccess) rc = COMMET_ERR_CUDA;
            if (rc == COMMET_OK) {
                unsigned char *wb = reinterpret_cast<unsigned char *>(m->d_weights);
                if (cudaMemcpy(wb + l.n0 * es, dN, d * es, cudaMemcpyDeviceToDevice) != cudaSuccess ||
                    cudaMemcpy(wb + l.K0 * es, (unsigned char *)dN + d * es, d * es, cudaMemcpyDeviceToDevice) !=
                        cudaSuccess)
                    rc = COMMET_ERR_CUDA;
            }
        }
        cudaFree(dF);
        cudaFree(dP);
        cudaFree(dN);
    }
    return rc;
}

// CANN (eq. cann-def) and Gent-Thomas (eq. gt) models: no network; the packed block holds
// the CANN weights [d][n][2], its kinds [n][3] (as numbers) and n0, K0.
int create_closed_form(const commet_model_desc *desc, int32_t precision, commet_model **out) {
    const int inner = desc->inner;
    if (desc->kinematics != COMMET_KIN_ISO_SHIFTED && desc->kinematics != COMMET_KIN_RAW &&
        desc->kinematics != COMMET_KIN_POLYCONVEX)
        return COMMET_ERR_INVALID_ARG;
    if (desc->n_fibres < 0 || desc->d < 1) return COMMET_ERR_INVALID_ARG;
    if (desc->kinematics != COMMET_KIN_RAW && desc->n_fibres != 0) return COMMET_ERR_INVALID_ARG;
    if (desc->n_fibres > kMaxFibres) return COMMET_ERR_UNSUPPORTED;
    if (desc->n_fibres > 0 && desc->fibres == nullptr) return COMMET_ERR_INVALID_ARG;
    const int d = desc->d;
    if (d != (desc->kinematics == COMMET_KIN_RAW ? 3 + 2 * desc->n_fibres : 3)) return COMMET_ERR_INVALID_ARG;
    if (!std::isfinite(desc->kappa)) return COMMET_ERR_INVALID_ARG;
    int n = 0;
    if (inner == COMMET_INNER_CANN) {
        n = desc->cann_terms;
        if (n < 1 || n > COMMET_CANN_MAX_TERMS || desc->cann_kind == nullptr || desc->cann_w == nullptr)
            return COMMET_ERR_INVALID_ARG;
        for (int k = 0; k < n; ++k) {
            const int f0 = desc->cann_kind[3 * k], p = desc->cann_kind[3 * k + 1], f2 = desc->cann_kind[3 * k + 2];
            if (f0 < COMMET_CANN_F0_ID || f0 > COMMET_CANN_F0_ABS || p < 1 || p > 3 || f2 < COMMET_CANN_F2_LINEAR ||
                f2 > COMMET_CANN_F2_LOG)
                return COMMET_ERR_INVALID_ARG;
        }
        for (int i = 0; i < 2 * d * n; ++i)
            if (!std::isfinite(desc->cann_w[i])) return COMMET_ERR_INVALID_ARG;
    } else if (inner == COMMET_INNER_ICKAN) {
        const int R = desc->kan_layers, k = desc->kan_degree, G = desc->kan_grid;
        if (R < 1 || R > COMMET_KAN_MAX_LAYERS || desc->kan_widths == nullptr || desc->kan_lo == nullptr ||
            desc->kan_hi == nullptr || desc->kan_params == nullptr || G < 1 || G > 128)
            return COMMET_ERR_INVALID_ARG;
        if (k < 2 || k > 4) return COMMET_ERR_UNSUPPORTED;
        if (desc->kan_widths[0] != d || desc->kan_widths[R] != 1 || desc->n_fibres != 0)
            return COMMET_ERR_INVALID_ARG;
        for (int r = 0; r <= R; ++r)
            if (desc->kan_widths[r] < 1 || desc->kan_widths[r] > COMMET_KAN_MAX_WIDTH) return COMMET_ERR_INVALID_ARG;
        for (int r = 0; r < R; ++r)
            if (!std::isfinite(desc->kan_lo[r]) || !std::isfinite(desc->kan_hi[r]) || !(desc->kan_hi[r] > desc->kan_lo[r]))
                return COMMET_ERR_INVALID_ARG;
    } else if (desc->kinematics != COMMET_KIN_RAW || desc->n_fibres != 0) {
        return COMMET_ERR_INVALID_ARG;  // eq. gt is written on raw (Ibar1, Ibar2, J)
    }
    if (precision == COMMET_BF16_MLP) return COMMET_ERR_UNSUPPORTED;

    commet_model *m = new (std::nothrow) commet_model();
    if (!m) return COMMET_ERR_CUDA;
    m->precision = precision;
    m->inner = inner;
    m->d = d;
    m->W = 0;
    m->L = 0;
    m->kp.kin = desc->kinematics;
    m->kp.nf = desc->n_fibres;
    for (int f = 0; f < desc->n_fibres; ++f)
        for (int c = 0; c < 3; ++c) m->kp.fib[f][c] = desc->fibres[3 * f + c];
    m->kp.kappa = desc->kappa;
    m->kp.stress_free = desc->stress_free ? 1 : 0;
    NetLayout l{};
    l.d = d;
    l.inner = inner;
    l.cn = n;
    int64_t n_kan = 0;  // ICKAN parameters
    if (inner == COMMET_INNER_ICKAN) {
        l.kR = desc->kan_layers;
        l.kdeg = desc->kan_degree;
        l.kG = desc->kan_grid;
        l.kwmax = 1;
        for (int r = 0; r <= l.kR; ++r) l.kwmax = std::max(l.kwmax, (int)desc->kan_widths[r]);
        for (int r = 0; r < l.kR; ++r) n_kan += (int64_t)desc->kan_widths[r] * desc->kan_widths[r + 1];
        n_kan *= 1 + l.kG + l.kdeg;
    }
    int o = 0;
    l.cw = o; o = round4(o + 2 * d * n);
    l.ck = o; o = round4(o + 3 * n);
    l.kwid = o; o = round4(o + (inner == COMMET_INNER_ICKAN ? l.kR + 1 : 0));
    l.klo = o; o = round4(o + l.kR);
    l.khi = o; o = round4(o + l.kR);
    l.kpar = o; o = round4(o + (int)n_kan);
    l.n0 = o; o = round4(o + d);
    l.K0 = o; o = round4(o + d);
    l.total = o;
    m->lay = l;
    m->n_params = inner == COMMET_INNER_ICKAN ? n_kan : (int64_t)2 * d * n;
    cudaGetDevice(&m->device);
    std::vector<double> h(l.total, 0.0);
    for (int i = 0; i < 2 * d * n; ++i) h[l.cw + i] = desc->cann_w[i];
    for (int i = 0; i < 3 * n; ++i) h[l.ck + i] = (double)desc->cann_kind[i];
    if (inner == COMMET_INNER_ICKAN) {
        for (int r = 0; r <= l.kR; ++r) h[l.kwid + r] = (double)desc->kan_widths[r];
        for (int r = 0; r < l.kR; ++r) {
            h[l.klo + r] = desc->kan_lo[r];
            h[l.khi + r] = desc->kan_hi[r];
        }
        for (int64_t i = 0; i < n_kan; ++i) {
            if (!std::isfinite(desc->kan_params[i])) {
                delete m;
                return COMMET_ERR_INVALID_ARG;
            }
            h[l.kpar + i] = desc->kan_params[i];
        }
    }
    int rc = (precision == COMMET_F64) ? upload<double>(h, &m->d_weights) : upload<float>(h, &m->d_weights);
    if (rc == COMMET_OK) rc = stress_free_shift(m);
    if (rc == COMMET_OK) rc = pipeline_res_create(m);
    if (rc != COMMET_OK) {
        commet_model_destroy(m);
        return rc;
    }
    *out = m;
    return COMMET_OK;
}

}  // namespace

extern "C" {

const char *commet_status_string(int code) {
    switch (code) {
        case COMMET_OK: return "ok";
        case COMMET_ERR_INVALID_ARG: return "invalid argument";
        case COMMET_ERR_UNSUPPORTED: return "unsupported shape, precision or kinematics";
        case COMMET_ERR_CUDA: return "CUDA error";
        case COMMET_ERR_NO_CSR: return "mesh has no CSR pattern";
        default: return "unknown status code";
    }
}

int commet_model_create(const commet_model_desc *desc, int32_t precision, commet_model **out) {
    if (desc == nullptr || out == nullptr) return COMMET_ERR_INVALID_ARG;
    if (precision != COMMET_F64 && precision != COMMET_F32 && precision != COMMET_BF16_MLP)
        return COMMET_ERR_INVALID_ARG;
    const int inner = desc->inner;
    if (inner != COMMET_INNER_MICNN && inner != COMMET_INNER_CANN && inner != COMMET_INNER_GENT_THOMAS &&
        inner != COMMET_INNER_ICKAN)
        return COMMET_ERR_INVALID_ARG;
    if (inner != COMMET_INNER_MICNN) return create_closed_form(desc, precision, out);
    if (desc->kinematics != COMMET_KIN_ISO_SHIFTED && desc->kinematics != COMMET_KIN_RAW &&
        desc->kinematics != COMMET_KIN_POLYCONVEX)
        return COMMET_ERR_INVALID_ARG;
    if (desc->n_fibres < 0 || desc->L < 1 || desc->W < 1 || desc->d < 1) return COMMET_ERR_INVALID_ARG;
    if (desc->kinematics != COMMET_KIN_RAW && desc->n_fibres != 0) return COMMET_ERR_INVALID_ARG;
    if (desc->n_fibres > kMaxFibres) return COMMET_ERR_UNSUPPORTED;
    const int d_expect = desc->kinematics == COMMET_KIN_RAW ? 3 + 2 * desc->n_fibres : 3;
    if (desc->d != d_expect) return COMMET_ERR_INVALID_ARG;
    if (desc->activation != COMMET_ACT_SOFTPLUS) return COMMET_ERR_UNSUPPORTED;
    if (desc->W1 == nullptr || desc->a_out == nullptr || desc->b_out == nullptr) return COMMET_ERR_INVALID_ARG;
    if (desc->L > 1 && (desc->A == nullptr || desc->B == nullptr)) return COMMET_ERR_INVALID_ARG;
    if (desc->n_fibres > 0 && desc->fibres == nullptr) return COMMET_ERR_INVALID_ARG;
    if (!(std::isfinite(desc->kappa))) return COMMET_ERR_INVALID_ARG;
    const int Wu = desc->W, d = desc->d, L = desc->L;
    if (Wu > 64 || L > 16) return COMMET_ERR_UNSUPPORTED;
    // Widths the kernels are built for: 4, 8 (no fibres), 16, 32, 64. Another width runs as the
    // next built one with zero rows and columns, an exact padding: a padded neuron gets no input
    // weight and no bias and feeds nothing, so N and all its derivatives are unchanged.
    int W = Wu <= 4 ? 4 : (Wu <= 8 ? 8 : (Wu <= 16 ? 16 : (Wu <= 32 ? 32 : 64)));
    if (W < 16 && desc->n_fibres != 0) W = 16;  // the narrow kernels take no fibres
    std::vector<double> pW1, pA, pB, pc, pa;
    std::vector<int32_t> theta_map;
    commet_model_desc padded;
    if (W != Wu) {
        pW1.assign((size_t)W * d, 0.0);
        pA.assign((size_t)(L - 1) * W * W, 0.0);
        pB.assign((size_t)(L - 1) * W * d, 0.0);
        pc.assign((size_t)L * W, 0.0);
        pa.assign(W, 0.0);
        for (int i = 0; i < Wu; ++i) {
            for (int mm = 0; mm < d; ++mm) pW1[i * d + mm] = desc->W1[i * d + mm];
            pa[i] = desc->a_out[i];
            for (int k = 0; k < L; ++k) pc[k * W + i] = desc->c ? desc->c[k * Wu + i] : 0.0;
            for (int k = 0; k < L - 1; ++k) {
                for (int j = 0; j < Wu; ++j) pA[((size_t)k * W + i) * W + j] = desc->A[((size_t)k * Wu + i) * Wu + j];
                for (int mm = 0; mm < d; ++mm) pB[((size_t)k * W + i) * d + mm] = desc->B[((size_t)k * Wu + i) * d + mm];
            }
        }
        padded = *desc;
        padded.W = W;
        padded.W1 = pW1.data();
        padded.A = L > 1 ? pA.data() : nullptr;
        padded.B = L > 1 ? pB.data() : nullptr;
        padded.c = pc.data();
        padded.a_out = pa.data();
        // padded theta [W1, c1, (A_k, B_k, c_k), a, b] -> the caller's theta index (or -1)
        int64_t ou = 0;
        auto block = [&](int rows, int cols, int urows, int ucols) {
            for (int i = 0; i < rows; ++i)
                for (int j = 0; j < cols; ++j)
                    theta_map.push_back((i < urows && j < ucols) ? (int32_t)(ou + (int64_t)i * ucols + j) : -1);
            ou += (int64_t)urows * ucols;
        };
        block(W, d, Wu, d);
        block(1, W, 1, Wu);
        for (int k = 0; k < L - 1; ++k) {
            block(W, W, Wu, Wu);
            block(W, d, Wu, d);
            block(1, W, 1, Wu);
        }
        block(1, W, 1, Wu);
        block(1, d, 1, d);
        desc = &padded;
    }

    commet_model *m = new (std::nothrow) commet_model();
    if (!m) return COMMET_ERR_CUDA;
    m->precision = precision;
    m->d = d;
    m->W = W;
    m->L = L;
    m->kp.kin = desc->kinematics;
    m->kp.nf = desc->n_fibres;
    for (int f = 0; f < desc->n_fibres; ++f)
        for (int c = 0; c < 3; ++c) m->kp.fib[f][c] = desc->fibres[3 * f + c];
    m->kp.kappa = desc->kappa;
    m->kp.stress_free = desc->stress_free ? 1 : 0;
    m->lay = make_layout(d, W, L, precision == COMMET_F64);
    m->lay.inner = COMMET_INNER_MICNN;
    m->W_user = Wu;
    m->n_params_net = (int64_t)W * d + W + (int64_t)(L - 1) * ((int64_t)W * W + (int64_t)W * d + W) + W + d;
    m->n_params = (int64_t)Wu * d + Wu + (int64_t)(L - 1) * ((int64_t)Wu * Wu + (int64_t)Wu * d + Wu) + Wu + d;
    cudaGetDevice(&m->device);
    if (!theta_map.empty()) {
        if (cudaMalloc(&m->d_theta_map, sizeof(int32_t) * theta_map.size()) != cudaSuccess ||
            cudaMemcpy(m->d_theta_map, theta_map.data(), sizeof(int32_t) * theta_map.size(), cudaMemcpyHostToDevice) !=
                cudaSuccess) {
            commet_model_destroy(m);
            return COMMET_ERR_CUDA;
        }
    }

    const NetLayout &l = m->lay;
    const int dp = (d + 3) / 4 * 4;
    std::vector<double> h(l.total, 0.0);
    for (int j = 0; j < W; ++j)
        for (int mm = 0; mm < d; ++mm) {
            h[l.W1t + mm * W + j] = desc->W1[j * d + mm];
            h[l.W1r + j * dp + mm] = desc->W1[j * d + mm];
        }
    for (int k = 0; k < L - 1; ++k) {
        const double *Ak = desc->A + (size_t)k * W * W;
        const double *Bk = desc->B + (size_t)k * W * d;
        for (int j = 0; j < W; ++j) {
            for (int i = 0; i < W; ++i) {
                h[l.At + k * W * W + i * W + j] = Ak[j * W + i];
                h[l.Ar + k * W * W + j * W + i] = Ak[j * W + i];
            }
            for (int mm = 0; mm < d; ++mm) h[l.Bt + k * d * W + mm * W + j] = Bk[j * d + mm];
        }
    }
    for (int k = 0; k < L; ++k)
        for (int j = 0; j < W; ++j) h[l.c + k * W + j] = desc->c ? desc->c[k * W + j] : 0.0;
    for (int j = 0; j < W; ++j) h[l.a + j] = desc->a_out[j];
    for (int mm = 0; mm < d; ++mm) h[l.b + mm] = desc->b_out[mm];
    if (l.M > 0) {
        // M[i][c][m] = A_2[c][i] W1[i][m] (rows of A_2 are the layer's output neurons)
        for (int i = 0; i < W; ++i)
            for (int c = 0; c < W; ++c)
                for (int mm = 0; mm < d; ++mm)
                    h[l.M + ((size_t)i * W + c) * dp + mm] = desc->A[(size_t)c * W + i] * desc->W1[i * d + mm];
    }
    if (l.tab > 0) {
        // float-pair tables of the FP64 activation (act_df.cuh), one pair per 8-byte slot
        std::vector<actdf::f2> tab(actdf::kSlots);
        actdf::make_table(tab.data());
        for (int i = 0; i < actdf::kSlots; ++i) std::memcpy(&h[l.tab + i], &tab[i], sizeof(double));
    }

    int rc;
    if (precision == COMMET_F64)
        rc = upload<double>(h, &m->d_weights);
    else
        rc = upload<float>(h, &m->d_weights);
    if (rc != COMMET_OK) {
        commet_model_destroy(m);
        return rc;
    }
    rc = stress_free_shift(m);
    if (rc != COMMET_OK) {
        commet_model_destroy(m);
        return rc;
    }
    if (precision == COMMET_BF16_MLP) {
        rc = prepare_bf16_weights(m);
        if (rc != COMMET_OK) {
            commet_model_destroy(m);
            return rc;
        }
    }
    rc = pipeline_res_create(m);
    if (rc != COMMET_OK) {
        commet_model_destroy(m);
        return rc;
    }
    *out = m;
    return COMMET_OK;
}

int commet_model_destroy(commet_model *m) {
    if (m == nullptr) return COMMET_ERR_INVALID_ARG;
    cudaFree(m->d_weights);
    cudaFree(m->d_theta64);
    cudaFree(m->d_bf16);
    cudaFree(m->d_theta_map);
    pipeline_res_destroy(m);
    delete m;
    return COMMET_OK;
}

int64_t commet_model_n_params(const commet_model *m) { return m ? m->n_params : -1; }

int commet_const_update(const commet_model *m, int64_t n_qp, const void *F, void *psi, void *P, void *A,
                        int32_t *status, void *stream) {
    if (m == nullptr || n_qp < 0) return COMMET_ERR_INVALID_ARG;
    if (n_qp > 0 && (F == nullptr || P == nullptr)) return COMMET_ERR_INVALID_ARG;
    if (!aligned16(F) || !aligned16(P) || !aligned16(A) || !aligned16(psi) ||
        (reinterpret_cast<uintptr_t>(status) & 7u) != 0)
        return COMMET_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (m->precision == COMMET_BF16_MLP) {
        if (status) {
            int rc = launch_status_init(status, s);
            if (rc != COMMET_OK) return rc;
        }
        if (n_qp == 0) return COMMET_OK;
        return launch_const_update_bf16(m, n_qp, F, psi, P, A, status, s);
    }
    return launch_const_update(m, n_qp, F, psi, P, A, status, s, nullptr);
}

size_t commet_const_update_host_workspace(const commet_model *m, const commet_mesh *mesh, int64_t chunk,
                                          int32_t want_A) {
    if (m == nullptr || chunk < 1) return 0;
    return host_pipeline_workspace(m, mesh, chunk, want_A != 0);
}

int commet_const_update_host(const commet_model *m, const commet_mesh *mesh, int64_t n_qp, const void *F, void *psi,
                             void *P, void *A, void *f_e, void *K_e, void *workspace, size_t ws_bytes, int64_t chunk,
                             void *stream) {
    if (m == nullptr || n_qp < 0 || chunk < 1) return COMMET_ERR_INVALID_ARG;
    if (n_qp > 0 && (F == nullptr || P == nullptr)) return COMMET_ERR_INVALID_ARG;
    if (mesh != nullptr && n_qp != 8 * mesh->n_el) return COMMET_ERR_INVALID_ARG;
    if (mesh == nullptr && (f_e != nullptr || K_e != nullptr)) return COMMET_ERR_INVALID_ARG;
    if (A == nullptr && K_e != nullptr) return COMMET_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(workspace) & 255u) != 0) return COMMET_ERR_INVALID_ARG;
    if (n_qp == 0) return COMMET_OK;
    if (workspace == nullptr || ws_bytes < host_pipeline_workspace(m, mesh, chunk, A != nullptr))
        return COMMET_ERR_INVALID_ARG;
    return run_host_pipeline(m, mesh, n_qp, F, psi, P, A, f_e, K_e, workspace, ws_bytes, chunk,
                             reinterpret_cast<cudaStream_t>(stream));
}

int commet_const_update_spatial(const commet_model *m, int64_t n_qp, const void *F, void *psi, void *tau, void *c,
                                int32_t *status, void *stream) {
    if (m == nullptr || n_qp < 0) return COMMET_ERR_INVALID_ARG;
    if (n_qp > 0 && (F == nullptr || tau == nullptr)) return COMMET_ERR_INVALID_ARG;
    if (!aligned16(F) || !aligned16(tau) || !aligned16(c) || !aligned16(psi) ||
        (reinterpret_cast<uintptr_t>(status) & 7u) != 0)
        return COMMET_ERR_INVALID_ARG;
    return launch_const_update_spatial(m, n_qp, F, psi, tau, c, status, reinterpret_cast<cudaStream_t>(stream));
}

int commet_target_stress(int32_t precision, int64_t n_qp, const void *F, int32_t n_fibres, const double *fibres,
                         double mu, double k1, double k2, double kappa, void *P, void *stream) {
    if (precision != COMMET_F64 && precision != COMMET_F32) return COMMET_ERR_INVALID_ARG;
    if (n_qp < 0 || n_fibres < 0 || n_fibres > kMaxFibres) return COMMET_ERR_INVALID_ARG;
    if (n_fibres > 0 && fibres == nullptr) return COMMET_ERR_INVALID_ARG;
    if (n_qp > 0 && (F == nullptr || P == nullptr)) return COMMET_ERR_INVALID_ARG;
    if (!(k2 > 0.0) || !std::isfinite(mu) || !std::isfinite(k1) || !std::isfinite(kappa))
        return COMMET_ERR_INVALID_ARG;
    if (n_qp == 0) return COMMET_OK;
    return launch_target_stress(precision, n_qp, F, n_fibres, fibres, mu, k1, k2, kappa, P,
                                reinterpret_cast<cudaStream_t>(stream));
}

// ------------------------------------------------------------------------ mesh

int commet_mesh_create(int64_t n_nodes, const double *X, int64_t n_el, const int32_t *conn, int32_t want_csr,
                       commet_mesh **out) {
    if (out == nullptr || n_nodes < 0 || n_el < 0) return COMMET_ERR_INVALID_ARG;
    if ((n_nodes > 0 && X == nullptr) || (n_el > 0 && conn == nullptr)) return COMMET_ERR_INVALID_ARG;
    if (n_nodes >= ((int64_t)1 << 31) / 3 || n_el >= ((int64_t)1 << 31) / 8) return COMMET_ERR_UNSUPPORTED;
    for (int64_t i = 0; i < 8 * n_el; ++i)
        if (conn[i] < 0 || conn[i] >= n_nodes) return COMMET_ERR_INVALID_ARG;
    for (int64_t i = 0; i < 3 * n_nodes; ++i)
        if (!std::isfinite(X[i])) return COMMET_ERR_INVALID_ARG;
    commet_mesh *mesh = new (std::nothrow) commet_mesh();
    if (!mesh) return COMMET_ERR_CUDA;
    mesh->n_nodes = n_nodes;
    mesh->n_el = n_el;
    cudaGetDevice(&mesh->device);
    int rc = COMMET_OK;
    if (cudaMalloc(&mesh->d_X, sizeof(double) * 3 * std::max<int64_t>(1, n_nodes)) != cudaSuccess ||
        cudaMalloc(&mesh->d_conn, sizeof(int32_t) * 8 * std::max<int64_t>(1, n_el)) != cudaSuccess)
        rc = COMMET_ERR_CUDA;
    if (rc == COMMET_OK && n_nodes > 0 &&
        cudaMemcpy(mesh->d_X, X, sizeof(double) * 3 * n_nodes, cudaMemcpyHostToDevice) != cudaSuccess)
        rc = COMMET_ERR_CUDA;
    if (rc == COMMET_OK && n_el > 0 &&
        cudaMemcpy(mesh->d_conn, conn, sizeof(int32_t) * 8 * n_el, cudaMemcpyHostToDevice) != cudaSuccess)
        rc = COMMET_ERR_CUDA;
    if (rc == COMMET_OK && want_csr) rc = build_csr_and_colouring(n_nodes, n_el, conn, mesh);
    if (rc == COMMET_OK && cudaMalloc(&mesh->d_red, sizeof(double) * kRedDoubles) != cudaSuccess) rc = COMMET_ERR_CUDA;
    if (rc == COMMET_OK && (cudaMalloc(&mesh->d_err, 64) != cudaSuccess || cudaMemset(mesh->d_err, 0, 64) != cudaSuccess))
        rc = COMMET_ERR_CUDA;
    if (rc != COMMET_OK) {
        commet_mesh_destroy(mesh);
        return rc;
    }
    *out = mesh;
    return COMMET_OK;
}

int commet_mesh_destroy(commet_mesh *mesh) {
    if (mesh == nullptr) return COMMET_ERR_INVALID_ARG;
    cudaFree(mesh->d_X);
    cudaFree(mesh->d_Xf);
    cudaFree(mesh->d_conn);
    cudaFree(mesh->d_rowptr);
    cudaFree(mesh->d_col);
    cudaFree(mesh->d_emap);
    cudaFree(mesh->d_rowlen);
    cudaFree(mesh->d_colour_el);
    cudaFree(mesh->d_fixed);
    cudaFree(mesh->d_fixed_dofs);
    cudaFree(mesh->d_fixed_vals);
    cudaFree(mesh->d_delta);
    cudaFree(mesh->d_red);
    cudaFree(mesh->d_err);
    delete[] mesh->h_rowptr;
    delete[] mesh->h_col;
    delete mesh;
    return COMMET_OK;
}

int commet_mesh_set_dirichlet(commet_mesh *mesh, int64_t n_fixed, const int64_t *dofs) {
    if (mesh == nullptr || n_fixed < 0 || (n_fixed > 0 && dofs == nullptr)) return COMMET_ERR_INVALID_ARG;
    const int64_t n = 3 * mesh->n_nodes;
    for (int64_t i = 0; i < n_fixed; ++i)
        if (dofs[i] < 0 || dofs[i] >= n || (i > 0 && dofs[i] <= dofs[i - 1])) return COMMET_ERR_INVALID_ARG;
    cudaFree(mesh->d_fixed);
    cudaFree(mesh->d_fixed_dofs);
    cudaFree(mesh->d_fixed_vals);
    cudaFree(mesh->d_delta);
    mesh->d_fixed = nullptr;
    mesh->d_fixed_dofs = nullptr;
    mesh->d_fixed_vals = nullptr;
    mesh->d_delta = nullptr;
    mesh->n_fixed = 0;
    if (n_fixed == 0) return COMMET_OK;
    std::vector<uint8_t> mask(n, 0);
    for (int64_t i = 0; i < n_fixed; ++i) mask[dofs[i]] = 1;
    COMMET_CUDA_TRY(cudaMalloc(&mesh->d_fixed, n));
    COMMET_CUDA_TRY(cudaMalloc(&mesh->d_fixed_dofs, sizeof(int64_t) * n_fixed));
    COMMET_CUDA_TRY(cudaMalloc(&mesh->d_fixed_vals, sizeof(double) * n_fixed));
    COMMET_CUDA_TRY(cudaMalloc(&mesh->d_delta, sizeof(double) * n));
    COMMET_CUDA_TRY(cudaMemcpy(mesh->d_fixed, mask.data(), n, cudaMemcpyHostToDevice));
    COMMET_CUDA_TRY(cudaMemcpy(mesh->d_fixed_dofs, dofs, sizeof(int64_t) * n_fixed, cudaMemcpyHostToDevice));
    mesh->n_fixed = n_fixed;
    return COMMET_OK;
}

int commet_set_dirichlet_values(const commet_mesh *mesh, int32_t precision, const double *values, void *u,
                                void *stream) {
    if (mesh == nullptr || (precision != COMMET_F64 && precision != COMMET_F32)) return COMMET_ERR_INVALID_ARG;
    if (mesh->n_fixed > 0 && (values == nullptr || u == nullptr)) return COMMET_ERR_INVALID_ARG;
    for (int64_t i = 0; i < mesh->n_fixed; ++i)
        if (!std::isfinite(values[i])) return COMMET_ERR_INVALID_ARG;
    if (!aligned16(u)) return COMMET_ERR_INVALID_ARG;
    return launch_set_dirichlet_values(mesh, precision, values, u, reinterpret_cast<cudaStream_t>(stream));
}

int commet_apply_dirichlet(const commet_mesh *mesh, int32_t precision, void *r, void *K_vals, const double *delta,
                           void *stream) {
    if (mesh == nullptr || (precision != COMMET_F64 && precision != COMMET_F32)) return COMMET_ERR_INVALID_ARG;
    if (mesh->h_rowptr == nullptr) return COMMET_ERR_NO_CSR;
    if (!aligned16(r) || !aligned16(K_vals)) return COMMET_ERR_INVALID_ARG;
    if (delta != nullptr) {
        if (r == nullptr || K_vals == nullptr) return COMMET_ERR_INVALID_ARG;
        for (int64_t i = 0; i < mesh->n_fixed; ++i)
            if (!std::isfinite(delta[i])) return COMMET_ERR_INVALID_ARG;
    }
    return launch_apply_dirichlet(mesh, precision, r, K_vals, delta, reinterpret_cast<cudaStream_t>(stream));
}

size_t commet_cg_workspace(const commet_mesh *mesh, int32_t precision) {
    if (mesh == nullptr || (precision != COMMET_F64 && precision != COMMET_F32)) return 0;
    return cg_workspace_bytes(mesh, precision);
}

int commet_cg_solve(const commet_mesh *mesh, int32_t precision, const void *K_vals, const void *b, void *x,
                    double rtol, int32_t max_iter, void *workspace, size_t ws_bytes, int32_t *iters, double *rel_res,
                    void *stream) {
    if (mesh == nullptr || (precision != COMMET_F64 && precision != COMMET_F32)) return COMMET_ERR_INVALID_ARG;
    if (mesh->h_rowptr == nullptr) return COMMET_ERR_NO_CSR;
    if (!(rtol >= 0.0) || max_iter < 1) return COMMET_ERR_INVALID_ARG;
    if (mesh->n_rows > 0 && (K_vals == nullptr || b == nullptr || x == nullptr || workspace == nullptr))
        return COMMET_ERR_INVALID_ARG;
    if (ws_bytes < cg_workspace_bytes(mesh, precision)) return COMMET_ERR_INVALID_ARG;
    if (!aligned16(K_vals) || !aligned16(b) || !aligned16(x) || (reinterpret_cast<uintptr_t>(workspace) & 255u) != 0)
        return COMMET_ERR_INVALID_ARG;
    if (mesh->n_rows == 0) {
        if (iters) *iters = 0;
        if (rel_res) *rel_res = 0.0;
        return COMMET_OK;
    }
    return launch_cg_solve(mesh, precision, K_vals, b, x, rtol, max_iter, workspace, iters, rel_res,
                           reinterpret_cast<cudaStream_t>(stream));
}

int commet_add_increment(const commet_mesh *mesh, int32_t precision, const void *du, double alpha, void *u,
                         void *stream) {
    if (mesh == nullptr || (precision != COMMET_F64 && precision != COMMET_F32)) return COMMET_ERR_INVALID_ARG;
    if (mesh->n_nodes > 0 && (du == nullptr || u == nullptr)) return COMMET_ERR_INVALID_ARG;
    if (!std::isfinite(alpha) || !aligned16(du) || !aligned16(u)) return COMMET_ERR_INVALID_ARG;
    return launch_add_increment(mesh, precision, du, alpha, u, reinterpret_cast<cudaStream_t>(stream));
}

int commet_norm2(const commet_mesh *mesh, int32_t precision, int64_t n, const void *x, double *out, void *stream) {
    if (mesh == nullptr || out == nullptr || n < 0 || (precision != COMMET_F64 && precision != COMMET_F32))
        return COMMET_ERR_INVALID_ARG;
    if (n > 0 && x == nullptr) return COMMET_ERR_INVALID_ARG;
    if (n == 0) {
        *out = 0.0;
        return COMMET_OK;
    }
    return launch_norm2(mesh, precision, n, x, out, reinterpret_cast<cudaStream_t>(stream));
}

int commet_mesh_info(const commet_mesh *mesh, int64_t *n_rows, int64_t *nnz, int32_t *n_colours) {
    if (mesh == nullptr) return COMMET_ERR_INVALID_ARG;
    if (n_rows) *n_rows = 3 * mesh->n_nodes;
    if (nnz) *nnz = mesh->nnz;
    if (n_colours) *n_colours = mesh->n_colours;
    return COMMET_OK;
}

int commet_mesh_csr(const commet_mesh *mesh, int64_t *rowptr, int32_t *col) {
    if (mesh == nullptr || rowptr == nullptr || col == nullptr) return COMMET_ERR_INVALID_ARG;
    if (mesh->h_rowptr == nullptr) return COMMET_ERR_NO_CSR;
    std::memcpy(rowptr, mesh->h_rowptr, sizeof(int64_t) * (mesh->n_rows + 1));
    std::memcpy(col, mesh->h_col, sizeof(int32_t) * mesh->nnz);
    return COMMET_OK;
}

int commet_compute_F(const commet_mesh *mesh, int32_t precision, const void *u, void *F, void *stream) {
    if (mesh == nullptr || (precision != COMMET_F64 && precision != COMMET_F32 && precision != COMMET_BF16_MLP))
        return COMMET_ERR_INVALID_ARG;
    if (mesh->n_el > 0 && (u == nullptr || F == nullptr)) return COMMET_ERR_INVALID_ARG;
    if (!aligned16(u) || !aligned16(F)) return COMMET_ERR_INVALID_ARG;
    return launch_compute_F(mesh, precision == COMMET_F64 ? COMMET_F64 : COMMET_F32, u, F,
                            reinterpret_cast<cudaStream_t>(stream));
}

int commet_elem_assemble(const commet_mesh *mesh, int32_t precision, const void *P, const void *A, void *f_e,
                         void *K_e, void *r, void *K_vals, void *stream) {
    if (mesh == nullptr || (precision != COMMET_F64 && precision != COMMET_F32 && precision != COMMET_BF16_MLP))
        return COMMET_ERR_INVALID_ARG;
    if (mesh->n_el > 0 && P == nullptr) return COMMET_ERR_INVALID_ARG;
    if (A == nullptr && (K_e != nullptr || K_vals != nullptr)) return COMMET_ERR_INVALID_ARG;
    if ((r != nullptr || K_vals != nullptr) && mesh->h_rowptr == nullptr) return COMMET_ERR_NO_CSR;
    if (!aligned16(P) || !aligned16(A) || !aligned16(f_e) || !aligned16(K_e) || !aligned16(r) || !aligned16(K_vals))
        return COMMET_ERR_INVALID_ARG;
    return launch_elem_assemble(mesh, precision == COMMET_F64 ? COMMET_F64 : COMMET_F32, P, A, f_e, K_e, r, K_vals,
                                reinterpret_cast<cudaStream_t>(stream));
}

int commet_elem_assemble_symmetric(const commet_mesh *mesh, int32_t precision, const void *P, const void *A,
                                   void *f_e, void *K_e, void *r, void *K_vals, void *stream) {
    if (mesh == nullptr || (precision != COMMET_F64 && precision != COMMET_F32 && precision != COMMET_BF16_MLP))
        return COMMET_ERR_INVALID_ARG;
    if (mesh->n_el > 0 && P == nullptr) return COMMET_ERR_INVALID_ARG;
    if (A == nullptr && (K_e != nullptr || K_vals != nullptr)) return COMMET_ERR_INVALID_ARG;
    if ((r != nullptr || K_vals != nullptr) && mesh->h_rowptr == nullptr) return COMMET_ERR_NO_CSR;
    if (!aligned16(P) || !aligned16(A) || !aligned16(f_e) || !aligned16(K_e) || !aligned16(r) || !aligned16(K_vals))
        return COMMET_ERR_INVALID_ARG;
    return launch_elem_assemble(mesh, precision == COMMET_F64 ? COMMET_F64 : COMMET_F32, P, A, f_e, K_e, r, K_vals,
                                reinterpret_cast<cudaStream_t>(stream), true);
}

int commet_elem_assemble_spatial(const commet_mesh *mesh, int32_t precision, const void *F, const void *tau,
                                 const void *c, void *f_e, void *K_e, void *r, void *K_vals, void *stream) {
    if (mesh == nullptr || (precision != COMMET_F64 && precision != COMMET_F32 && precision != COMMET_BF16_MLP))
        return COMMET_ERR_INVALID_ARG;
    if (mesh->n_el > 0 && (F == nullptr || tau == nullptr)) return COMMET_ERR_INVALID_ARG;
    if (c == nullptr && (K_e != nullptr || K_vals != nullptr)) return COMMET_ERR_INVALID_ARG;
    if ((r != nullptr || K_vals != nullptr) && mesh->h_rowptr == nullptr) return COMMET_ERR_NO_CSR;
    if (!aligned16(F) || !aligned16(tau) || !aligned16(c) || !aligned16(f_e) || !aligned16(K_e) || !aligned16(r) ||
        !aligned16(K_vals))
        return COMMET_ERR_INVALID_ARG;
    return launch_elem_assemble_spatial(mesh, precision == COMMET_F64 ? COMMET_F64 : COMMET_F32, F, tau, c, f_e, K_e,
                                        r, K_vals, reinterpret_cast<cudaStream_t>(stream));
}

int commet_residual_adjoint(const commet_mesh *mesh, int32_t precision, const void *lam, void *G, void *stream) {
    if (mesh == nullptr || (precision != COMMET_F64 && precision != COMMET_F32)) return COMMET_ERR_INVALID_ARG;
    if (mesh->n_el > 0 && (lam == nullptr || G == nullptr)) return COMMET_ERR_INVALID_ARG;
    if (!aligned16(lam) || !aligned16(G)) return COMMET_ERR_INVALID_ARG;
    return launch_assembly_adjoints(mesh, precision, lam, G, nullptr, nullptr, reinterpret_cast<cudaStream_t>(stream));
}

int commet_compute_F_adjoint(const commet_mesh *mesh, int32_t precision, const void *dF, void *du, void *stream) {
    if (mesh == nullptr || (precision != COMMET_F64 && precision != COMMET_F32)) return COMMET_ERR_INVALID_ARG;
    if (mesh->h_rowptr == nullptr) return COMMET_ERR_NO_CSR;
    if ((mesh->n_el > 0 && dF == nullptr) || (mesh->n_nodes > 0 && du == nullptr)) return COMMET_ERR_INVALID_ARG;
    if (!aligned16(dF) || !aligned16(du)) return COMMET_ERR_INVALID_ARG;
    return launch_assembly_adjoints(mesh, precision, nullptr, nullptr, dF, du, reinterpret_cast<cudaStream_t>(stream));
}

int commet_newton_assemble(const commet_model *m, const commet_mesh *mesh, const void *u, void *r, void *K_vals,
                           int32_t *status, void *stream) {
    if (m == nullptr || mesh == nullptr) return COMMET_ERR_INVALID_ARG;
    if (mesh->h_rowptr == nullptr) return COMMET_ERR_NO_CSR;
    if (mesh->n_el > 0 && (u == nullptr || r == nullptr || K_vals == nullptr)) return COMMET_ERR_INVALID_ARG;
    if (!aligned16(u) || !aligned16(r) || !aligned16(K_vals) || (reinterpret_cast<uintptr_t>(status) & 7u) != 0)
        return COMMET_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (status) {
        int rc = launch_status_init(status, s);
        if (rc != COMMET_OK) return rc;
    }
    return launch_newton_assemble(m, mesh, u, r, K_vals, status, s);
}

size_t commet_const_backward_workspace(const commet_model *m, int64_t n_qp) {
    if (m == nullptr || n_qp < 0) return 0;
    return backward_workspace_bytes(m, n_qp);
}

int commet_const_backward(const commet_model *m, int64_t n_qp, const void *F, const void *dL_dP, void *dL_dF,
                          void *dL_dtheta, void *workspace, size_t ws_bytes, void *stream) {
    if (m == nullptr || n_qp < 0) return COMMET_ERR_INVALID_ARG;
    // inner functions without a backward first: Gent-Thomas has no parameters (no dL_dtheta)
    if (m->inner != COMMET_INNER_MICNN && m->inner != COMMET_INNER_CANN) return COMMET_ERR_UNSUPPORTED;
    if (dL_dtheta == nullptr) return COMMET_ERR_INVALID_ARG;
    if (n_qp > 0 && (F == nullptr || dL_dP == nullptr)) return COMMET_ERR_INVALID_ARG;
    if (!aligned16(F) || !aligned16(dL_dP) || !aligned16(dL_dF) || !aligned16(dL_dtheta)) return COMMET_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(workspace) & 255u) != 0) return COMMET_ERR_INVALID_ARG;
    if (ws_bytes < backward_workspace_bytes(m, n_qp) || (workspace == nullptr && ws_bytes > 0))
        return COMMET_ERR_INVALID_ARG;
    if (m->kp.stress_free) return COMMET_ERR_UNSUPPORTED;
    return launch_const_backward(m, n_qp, F, dL_dP, dL_dF, dL_dtheta, workspace, ws_bytes,
                                 reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
