// Host-buffer form of the constitutive update and the element integrals (Algorithm 2 with
// the tables in host memory): the points, or the elements with their 8 points each, go
// through the GPU in chunks. Chunk c is copied in on one stream while chunk c - 1 is
// computed on the caller's stream and chunk c - 2 is copied out on a third, with two
// device buffers taking turns, so that the host-device copies hide behind the kernels
// (or the kernels behind the copies, whichever is longer).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>
#include <new>

#include "internal.h"

namespace commet {

namespace {

constexpr size_t kAlign = 256;

size_t round_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct ChunkBuf {
    size_t F, psi, P, A, fe, Ke, bytes;  // byte offsets within one buffer
};

// One buffer for npts points (and ne elements): F, psi, P, A, f_e, K_e of the chunk,
// each [rows][npts] (or [rows][ne]) contiguous.
ChunkBuf chunk_layout(size_t es, int64_t npts, int64_t ne, bool want_A) {
    ChunkBuf b{};
    size_t o = 0;
    b.F = o;
    o += round_up(es * 9 * npts);
    b.psi = o;
    o += round_up(es * npts);
    b.P = o;
    o += round_up(es * 9 * npts);
    b.A = o;
    o += want_A ? round_up(es * 81 * npts) : 0;
    b.fe = o;
    o += round_up(es * 24 * ne);
    b.Ke = o;
    o += want_A ? round_up(es * 576 * ne) : 0;
    b.bytes = o;
    return b;
}

size_t elem_size(const commet_model *m) { return m->precision == COMMET_F64 ? 8 : 4; }

// rows x width bytes from a [rows][pitch] table to a [rows][width] one, or back
int copy_rows(void *dst, size_t dpitch, const void *src, size_t spitch, size_t width, int rows, cudaMemcpyKind kind,
              cudaStream_t s) {
    if (width == 0) return COMMET_OK;
    return cudaMemcpy2DAsync(dst, dpitch, src, spitch, width, rows, kind, s) == cudaSuccess ? COMMET_OK
                                                                                          : COMMET_ERR_CUDA;
}

}  // namespace

int pipeline_res_create(commet_model *m) {
    PipelineRes *r = new (std::nothrow) PipelineRes();
    if (r == nullptr) return COMMET_ERR_CUDA;
    m->pipe = r;
    bool ok = cudaStreamCreateWithFlags(&r->in, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&r->out, cudaStreamNonBlocking) == cudaSuccess;
    cudaEvent_t *all[] = {&r->start, &r->end_in, &r->end_out, &r->ev_in[0], &r->ev_in[1],
                          &r->ev_done[0], &r->ev_done[1], &r->ev_free[0], &r->ev_free[1]};
    for (cudaEvent_t *e : all) ok = ok && cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess;
    return ok ? COMMET_OK : COMMET_ERR_CUDA;
}

// Streams and events are released once the work queued on them has completed.
void pipeline_res_destroy(commet_model *m) {
    PipelineRes *r = m->pipe;
    if (r == nullptr) return;
    cudaEvent_t all[] = {r->start, r->end_in, r->end_out, r->ev_in[0], r->ev_in[1],
                         r->ev_done[0], r->ev_done[1], r->ev_free[0], r->ev_free[1]};
    for (cudaEvent_t e : all)
        if (e) cudaEventDestroy(e);
    if (r->in) cudaStreamDestroy(r->in);
    if (r->out) cudaStreamDestroy(r->out);
    delete r;
    m->pipe = nullptr;
}

size_t host_pipeline_workspace(const commet_model *m, const commet_mesh *mesh, int64_t chunk, bool want_A) {
    const int64_t npts = mesh ? 8 * chunk : chunk, ne = mesh ? chunk : 0;
    return 2 * chunk_layout(elem_size(m), npts, ne, want_A).bytes;
}

// Stops the chunk loop with COMMET_ERR_CUDA when a runtime call fails; the join after the
// loop still runs.
#define PIPE_TRY(expr)                        \
    if ((expr) != cudaSuccess) {              \
        rc = COMMET_ERR_CUDA;                 \
        break;                                \
    }

int run_host_pipeline(const commet_model *m, const commet_mesh *mesh, int64_t n_qp, const void *F, void *psi, void *P,
                      void *A, void *f_e, void *K_e, void *ws, size_t ws_bytes, int64_t chunk, cudaStream_t s) {
    const bool want_A = A != nullptr;
    const size_t es = elem_size(m);
    const int64_t n_el = mesh ? mesh->n_el : 0;
    const int64_t npts_c = mesh ? 8 * chunk : chunk, ne_c = mesh ? chunk : 0;
    const ChunkBuf lay = chunk_layout(es, npts_c, ne_c, want_A);
    if (ws_bytes < 2 * lay.bytes) return COMMET_ERR_INVALID_ARG;
    const int64_t units = mesh ? n_el : n_qp;
    const int64_t n_chunks = (units + chunk - 1) / chunk;
    if (n_chunks == 0) return COMMET_OK;
    if (m->pipe == nullptr) return COMMET_ERR_CUDA;
    PipelineRes &st = *m->pipe;
    std::lock_guard<std::mutex> lock(st.mu);
    unsigned char *base = static_cast<unsigned char *>(ws);
    const int prec_elem = m->precision == COMMET_F64 ? COMMET_F64 : COMMET_F32;
    // the side streams start after the work already queued on the caller's stream (an
    // earlier call may still be using the workspace)
    COMMET_CUDA_TRY(cudaEventRecord(st.start, s));
    COMMET_CUDA_TRY(cudaStreamWaitEvent(st.in, st.start, 0));
    COMMET_CUDA_TRY(cudaStreamWaitEvent(st.out, st.start, 0));
    int rc = COMMET_OK;
    for (int64_t c = 0; c < n_chunks && rc == COMMET_OK; ++c) {
        const int b = (int)(c & 1);
        unsigned char *buf = base + b * lay.bytes;
        const int64_t u0 = c * chunk, nu = std::min<int64_t>(chunk, units - u0);
        const int64_t q0 = mesh ? 8 * u0 : u0, nq = mesh ? 8 * nu : nu;
        const size_t qpitch = es * n_qp, cw = es * nq;
        // in: F of the chunk, after chunk c - 2 has left this buffer
        if (c >= 2) PIPE_TRY(cudaStreamWaitEvent(st.in, st.ev_free[b], 0));
        rc = copy_rows(buf + lay.F, cw, static_cast<const unsigned char *>(F) + es * q0, qpitch, cw, 9,
                       cudaMemcpyHostToDevice, st.in);
        if (rc != COMMET_OK) break;
        PIPE_TRY(cudaEventRecord(st.ev_in[b], st.in));
        // kernels on the caller's stream
        PIPE_TRY(cudaStreamWaitEvent(s, st.ev_in[b], 0));
        rc = commet_const_update(m, nq, buf + lay.F, psi ? buf + lay.psi : nullptr, buf + lay.P,
                                 want_A ? buf + lay.A : nullptr, nullptr, s);
        if (rc != COMMET_OK) break;
        if (mesh && (f_e != nullptr || K_e != nullptr)) {
            commet_mesh view = *mesh;  // the chunk's elements: same nodes, a window of conn
            view.n_el = nu;
            view.d_conn = mesh->d_conn + 8 * u0;
            // A is the update's own tangent, the Hessian of an energy: major symmetric
            rc = launch_elem_assemble(&view, prec_elem, buf + lay.P, want_A ? buf + lay.A : nullptr,
                                      f_e ? buf + lay.fe : nullptr, K_e ? buf + lay.Ke : nullptr, nullptr, nullptr, s,
                                      true);
            if (rc != COMMET_OK) break;
        }
        PIPE_TRY(cudaEventRecord(st.ev_done[b], s));
        // out: the chunk's results
        PIPE_TRY(cudaStreamWaitEvent(st.out, st.ev_done[b], 0));
        if (psi)
            PIPE_TRY(cudaMemcpyAsync(static_cast<unsigned char *>(psi) + es * q0, buf + lay.psi, cw,
                                     cudaMemcpyDeviceToHost, st.out));
        rc = copy_rows(static_cast<unsigned char *>(P) + es * q0, qpitch, buf + lay.P, cw, cw, 9,
                       cudaMemcpyDeviceToHost, st.out);
        if (rc == COMMET_OK && want_A)
            rc = copy_rows(static_cast<unsigned char *>(A) + es * q0, qpitch, buf + lay.A, cw, cw, 81,
                           cudaMemcpyDeviceToHost, st.out);
        if (rc == COMMET_OK && mesh && f_e)
            rc = copy_rows(static_cast<unsigned char *>(f_e) + es * u0, es * n_el, buf + lay.fe, es * nu, es * nu, 24,
                           cudaMemcpyDeviceToHost, st.out);
        if (rc == COMMET_OK && mesh && K_e)
            rc = copy_rows(static_cast<unsigned char *>(K_e) + es * u0, es * n_el, buf + lay.Ke, es * nu, es * nu, 576,
                           cudaMemcpyDeviceToHost, st.out);
        if (rc != COMMET_OK) break;
        PIPE_TRY(cudaEventRecord(st.ev_free[b], st.out));
    }
    // Join, on every path: the caller's stream completes only when every copy queued on
    // either side stream has finished, so that on return (error or not) nothing still
    // reads the workspace or the host inputs, or writes the host outputs, behind the
    // caller's back.
    const bool j1 = cudaEventRecord(st.end_in, st.in) == cudaSuccess && cudaStreamWaitEvent(s, st.end_in, 0) == cudaSuccess;
    const bool j2 = cudaEventRecord(st.end_out, st.out) == cudaSuccess && cudaStreamWaitEvent(s, st.end_out, 0) == cudaSuccess;
    if (rc == COMMET_OK && !(j1 && j2)) rc = COMMET_ERR_CUDA;
    return rc;
}

#undef PIPE_TRY

}  // namespace commet
