// Streaming solves from host memory: two device slots, each with its own step graph,
// and three streams (upload, solve, download) so that the copies of neighbouring
// snapshots overlap the solve.  Built on the public C ABI only (pp_plan_info,
// pp_step_graph_*): the plan's internal workspace is shared by both graphs, so the
// solves themselves run one after the other on the solve stream.
//
// Ordering per snapshot k in slot s = k mod 2:
//   upload stream:   wait solved[s] (snapshot k-2 no longer reads slot s's inputs),
//                    copy u, v, chi, us_x, us_y, points, normals into slot s, record in[s];
//   solve stream:    wait in[s] and out[s] (snapshot k-2's results have left slot s),
//                    launch graph[s], record solved[s];
//   download stream: wait solved[s], copy P and forces to the host, record out[s].
#include <cuda_runtime.h>

#include <cstdint>
#include <new>

#include "../../include/pp.h"

struct pp_pipeline_s {
    pp_plan plan = nullptr;
    int n = 0, npts = 0;
    size_t field_bytes = 0;
    cudaStream_t up = nullptr, solve = nullptr, down = nullptr;
    struct Slot {
        void* f[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // u, v, chi, us_x, us_y
        double* pts = nullptr;
        double* nrm = nullptr;
        void* p = nullptr;
        double* forces = nullptr;
        pp_graph graph = nullptr;
        cudaEvent_t in = nullptr, solved = nullptr, out = nullptr;
    } slot[2];
    int64_t submitted = 0;
};

namespace {

void release(pp_pipeline_s* q) {
    if (q->up) cudaStreamSynchronize(q->up);
    if (q->solve) cudaStreamSynchronize(q->solve);
    if (q->down) cudaStreamSynchronize(q->down);
    for (auto& s : q->slot) {
        if (s.graph) pp_step_graph_destroy(s.graph);
        for (void* f : s.f)
            if (f) cudaFree(f);
        if (s.pts) cudaFree(s.pts);
        if (s.nrm) cudaFree(s.nrm);
        if (s.p) cudaFree(s.p);
        if (s.forces) cudaFree(s.forces);
        if (s.in) cudaEventDestroy(s.in);
        if (s.solved) cudaEventDestroy(s.solved);
        if (s.out) cudaEventDestroy(s.out);
    }
    if (q->up) cudaStreamDestroy(q->up);
    if (q->solve) cudaStreamDestroy(q->solve);
    if (q->down) cudaStreamDestroy(q->down);
    delete q;
}

}  // namespace

extern "C" int pp_pipeline_create(pp_plan plan, double lambda, int npts, const double* dS, double nu,
                                  pp_pipeline* out) {
    if (!out) return PP_ERR_ARG;
    *out = nullptr;
    if (!plan || npts < 0 || npts > (1 << 24)) return PP_ERR_ARG;
    pp_plan_info_t info;
    int st = pp_plan_info(plan, &info);
    if (st != PP_OK) return st;
    pp_pipeline_s* q = new (std::nothrow) pp_pipeline_s();
    if (!q) return PP_ERR_OOM;
    q->plan = plan;
    q->n = info.n;
    q->npts = npts;
    q->field_bytes = size_t(info.n) * info.n * (info.precision == PP_FP64 ? 8 : 4);
    bool ok = cudaStreamCreateWithFlags(&q->up, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&q->solve, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&q->down, cudaStreamNonBlocking) == cudaSuccess;
    const size_t pbytes = sizeof(double) * 2 * size_t(npts > 0 ? npts : 1);
    for (auto& s : q->slot) {
        for (void*& f : s.f) ok = ok && cudaMalloc(&f, q->field_bytes) == cudaSuccess;
        ok = ok && cudaMalloc(&s.pts, pbytes) == cudaSuccess && cudaMalloc(&s.nrm, pbytes) == cudaSuccess &&
             cudaMalloc(&s.p, q->field_bytes) == cudaSuccess &&
             cudaMalloc(&s.forces, sizeof(double) * 6) == cudaSuccess;
        ok = ok && cudaEventCreateWithFlags(&s.in, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&s.solved, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&s.out, cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        release(q);
        return PP_ERR_OOM;
    }
    for (auto& s : q->slot) {
        // the fields' contents do not matter for the capture; zero them so a replay
        // before the first upload reads defined values
        for (void* f : s.f) cudaMemsetAsync(f, 0, q->field_bytes, q->up);
        cudaMemsetAsync(s.pts, 0, pbytes, q->up);
        cudaMemsetAsync(s.nrm, 0, pbytes, q->up);
    }
    if (cudaStreamSynchronize(q->up) != cudaSuccess) {
        release(q);
        return PP_ERR_CUDA;
    }
    for (auto& s : q->slot) {
        st = pp_step_graph_create(plan, s.f[0], s.f[1], s.f[2], s.f[3], s.f[4], lambda, s.p, npts, s.pts, s.nrm, dS,
                                  nu, nullptr, npts > 0 ? s.forces : nullptr, &s.graph);
        if (st != PP_OK) {
            release(q);
            return st;
        }
    }
    *out = q;
    return PP_OK;
}

extern "C" int pp_pipeline_submit(pp_pipeline q, const void* u, const void* v, const void* chi, const void* us_x,
                                  const void* us_y, const double* points, const double* normals, void* p_out,
                                  double* forces) {
    if (!q || !u || !v || !chi || !us_x || !us_y) return PP_ERR_ARG;
    if (q->npts > 0 && (!points || !normals)) return PP_ERR_ARG;
    auto& s = q->slot[q->submitted & 1];
    const bool reuse = q->submitted >= 2;
    const void* src[5] = {u, v, chi, us_x, us_y};
    bool ok = !reuse || cudaStreamWaitEvent(q->up, s.solved, 0) == cudaSuccess;
    for (int i = 0; i < 5 && ok; ++i)
        ok = cudaMemcpyAsync(s.f[i], src[i], q->field_bytes, cudaMemcpyHostToDevice, q->up) == cudaSuccess;
    if (ok && q->npts > 0) {
        const size_t pb = sizeof(double) * 2 * size_t(q->npts);
        ok = cudaMemcpyAsync(s.pts, points, pb, cudaMemcpyHostToDevice, q->up) == cudaSuccess &&
             cudaMemcpyAsync(s.nrm, normals, pb, cudaMemcpyHostToDevice, q->up) == cudaSuccess;
    }
    ok = ok && cudaEventRecord(s.in, q->up) == cudaSuccess;
    ok = ok && cudaStreamWaitEvent(q->solve, s.in, 0) == cudaSuccess;
    ok = ok && (!reuse || cudaStreamWaitEvent(q->solve, s.out, 0) == cudaSuccess);
    if (!ok) {
        cudaGetLastError();
        return PP_ERR_CUDA;
    }
    int st = pp_step_graph_launch(s.graph, q->solve);
    if (st != PP_OK) return st;
    ok = cudaEventRecord(s.solved, q->solve) == cudaSuccess &&
         cudaStreamWaitEvent(q->down, s.solved, 0) == cudaSuccess;
    if (ok && p_out) ok = cudaMemcpyAsync(p_out, s.p, q->field_bytes, cudaMemcpyDeviceToHost, q->down) == cudaSuccess;
    if (ok && forces && q->npts > 0)
        ok = cudaMemcpyAsync(forces, s.forces, sizeof(double) * 6, cudaMemcpyDeviceToHost, q->down) == cudaSuccess;
    ok = ok && cudaEventRecord(s.out, q->down) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        return PP_ERR_CUDA;
    }
    ++q->submitted;
    return PP_OK;
}

extern "C" int pp_pipeline_wait(pp_pipeline q) {
    if (!q) return PP_ERR_ARG;
    if (cudaStreamSynchronize(q->down) != cudaSuccess || cudaStreamSynchronize(q->solve) != cudaSuccess ||
        cudaStreamSynchronize(q->up) != cudaSuccess) {
        cudaGetLastError();
        return PP_ERR_CUDA;
    }
    return PP_OK;
}

extern "C" int pp_pipeline_destroy(pp_pipeline q) {
    if (!q) return PP_OK;
    release(q);
    return PP_OK;
}
