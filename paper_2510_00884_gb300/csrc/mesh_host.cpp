// Host-side graph work for a hex8 mesh: the CSR pattern of the global stiffness,
// the element -> CSR position map, and an element colouring for race-free scatter.
//
// Global dof numbering is node-major (3*node + i), as in the block layout of the
// global stiffness of Sec. 2.1. Every dof row of node n holds the columns of all
// nodes sharing an element with n (n included), three per node, in ascending order,
// so the entry (3*gI + i, 3*gK + k) sits at  pos(gI, gK) + i * rowlen(gI) + k  with
// pos(gI, gK) = rowptr[3*gI] + 3 * rank of gK among the neighbours of gI.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "internal.h"

namespace commet {

int build_csr_and_colouring(int64_t n_nodes, int64_t n_el, const int32_t *conn, commet_mesh *mesh) {
    // node -> elements incidence (CSR)
    std::vector<int64_t> ne_ptr(n_nodes + 1, 0);
    for (int64_t e = 0; e < n_el; ++e)
        for (int I = 0; I < 8; ++I) ne_ptr[conn[8 * e + I] + 1]++;
    for (int64_t n = 0; n < n_nodes; ++n) ne_ptr[n + 1] += ne_ptr[n];
    std::vector<int64_t> ne_idx(ne_ptr[n_nodes]);
    {
        std::vector<int64_t> fill(ne_ptr.begin(), ne_ptr.end() - 1);
        for (int64_t e = 0; e < n_el; ++e)
            for (int I = 0; I < 8; ++I) ne_idx[fill[conn[8 * e + I]]++] = e;
    }
    // node -> sorted unique neighbour nodes
    std::vector<int64_t> nb_ptr(n_nodes + 1, 0);
    std::vector<int32_t> nb_idx;
    nb_idx.reserve((size_t)n_nodes * 27);
    std::vector<int32_t> tmp;
    for (int64_t n = 0; n < n_nodes; ++n) {
        tmp.clear();
        for (int64_t p = ne_ptr[n]; p < ne_ptr[n + 1]; ++p) {
            const int64_t e = ne_idx[p];
            for (int I = 0; I < 8; ++I) tmp.push_back(conn[8 * e + I]);
        }
        std::sort(tmp.begin(), tmp.end());
        tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
        nb_idx.insert(nb_idx.end(), tmp.begin(), tmp.end());
        nb_ptr[n + 1] = (int64_t)nb_idx.size();
    }
    // CSR pattern
    const int64_t n_rows = 3 * n_nodes;
    std::vector<int64_t> rowptr(n_rows + 1, 0);
    for (int64_t n = 0; n < n_nodes; ++n) {
        const int64_t cnt = 3 * (nb_ptr[n + 1] - nb_ptr[n]);
        for (int i = 0; i < 3; ++i) rowptr[3 * n + i + 1] = rowptr[3 * n + i] + cnt;
    }
    const int64_t nnz = rowptr[n_rows];
    if (nnz >= ((int64_t)1 << 31)) return COMMET_ERR_UNSUPPORTED;
    int64_t *h_rowptr = new int64_t[n_rows + 1];
    int32_t *h_col = new int32_t[nnz > 0 ? nnz : 1];
    std::memcpy(h_rowptr, rowptr.data(), sizeof(int64_t) * (n_rows + 1));
    std::vector<int32_t> rowlen(n_nodes);
    for (int64_t n = 0; n < n_nodes; ++n) {
        const int64_t nn = nb_ptr[n + 1] - nb_ptr[n];
        rowlen[n] = (int32_t)(3 * nn);
        for (int i = 0; i < 3; ++i) {
            int64_t p = rowptr[3 * n + i];
            for (int64_t t = nb_ptr[n]; t < nb_ptr[n + 1]; ++t)
                for (int k = 0; k < 3; ++k) h_col[p++] = 3 * nb_idx[t] + k;
        }
    }
    // element -> CSR position of (3 gI, 3 gK)
    std::vector<uint32_t> emap((size_t)n_el * 64);
    for (int64_t e = 0; e < n_el; ++e)
        for (int I = 0; I < 8; ++I) {
            const int32_t gI = conn[8 * e + I];
            const int32_t *b = nb_idx.data() + nb_ptr[gI], *en = nb_idx.data() + nb_ptr[gI + 1];
            for (int K = 0; K < 8; ++K) {
                const int32_t gK = conn[8 * e + K];
                const int64_t rank = std::lower_bound(b, en, gK) - b;
                emap[(size_t)e * 64 + I * 8 + K] = (uint32_t)(rowptr[3 * (int64_t)gI] + 3 * rank);
            }
        }
    // greedy colouring in element order: smallest colour unused by node-sharing elements
    std::vector<int8_t> colour(n_el, -1);
    int n_col = 0;
    for (int64_t e = 0; e < n_el; ++e) {
        uint64_t used = 0;
        for (int I = 0; I < 8; ++I) {
            const int32_t n = conn[8 * e + I];
            for (int64_t p = ne_ptr[n]; p < ne_ptr[n + 1]; ++p) {
                const int8_t c = colour[ne_idx[p]];
                if (c >= 0) used |= (uint64_t)1 << c;
            }
        }
        int c = 0;
        while (c < 64 && ((used >> c) & 1)) ++c;
        if (c >= 64) {
            delete[] h_rowptr;
            delete[] h_col;
            return COMMET_ERR_UNSUPPORTED;
        }
        colour[e] = (int8_t)c;
        n_col = std::max(n_col, c + 1);
    }
    std::vector<int64_t> coff(n_col + 1, 0);
    for (int64_t e = 0; e < n_el; ++e) coff[colour[e] + 1]++;
    for (int c = 0; c < n_col; ++c) coff[c + 1] += coff[c];
    std::vector<int32_t> cel(n_el);
    {
        std::vector<int64_t> fill(coff.begin(), coff.end() - 1);
        for (int64_t e = 0; e < n_el; ++e) cel[fill[colour[e]]++] = (int32_t)e;
    }
    // device copies
    mesh->n_rows = n_rows;
    mesh->nnz = nnz;
    mesh->n_colours = n_col;
    for (int c = 0; c <= n_col; ++c) mesh->colour_off[c] = coff[c];
    mesh->h_rowptr = h_rowptr;
    mesh->h_col = h_col;
    COMMET_CUDA_TRY(cudaMalloc(&mesh->d_rowptr, sizeof(int64_t) * (n_rows + 1)));
    COMMET_CUDA_TRY(cudaMalloc(&mesh->d_col, sizeof(int32_t) * (nnz > 0 ? nnz : 1)));
    COMMET_CUDA_TRY(cudaMalloc(&mesh->d_emap, sizeof(uint32_t) * (size_t)std::max<int64_t>(1, n_el) * 64));
    COMMET_CUDA_TRY(cudaMalloc(&mesh->d_rowlen, sizeof(int32_t) * std::max<int64_t>(1, n_nodes)));
    COMMET_CUDA_TRY(cudaMalloc(&mesh->d_colour_el, sizeof(int32_t) * std::max<int64_t>(1, n_el)));
    COMMET_CUDA_TRY(cudaMemcpy(mesh->d_rowptr, h_rowptr, sizeof(int64_t) * (n_rows + 1), cudaMemcpyHostToDevice));
    if (nnz > 0) COMMET_CUDA_TRY(cudaMemcpy(mesh->d_col, h_col, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice));
    if (n_el > 0) {
        COMMET_CUDA_TRY(cudaMemcpy(mesh->d_emap, emap.data(), sizeof(uint32_t) * n_el * 64, cudaMemcpyHostToDevice));
        COMMET_CUDA_TRY(cudaMemcpy(mesh->d_colour_el, cel.data(), sizeof(int32_t) * n_el, cudaMemcpyHostToDevice));
    }
    if (n_nodes > 0)
        COMMET_CUDA_TRY(cudaMemcpy(mesh->d_rowlen, rowlen.data(), sizeof(int32_t) * n_nodes, cudaMemcpyHostToDevice));
    return COMMET_OK;
}

}  // namespace commet
