// Batched tracking of many independent 2D fields of uneven size and length.
//
// Each field has its own plan (workspace sized for its shape, time chunking
// optionally chosen by the autotuner); all per-field run counters live in
// one device array so a single copy checks every field.  After a first,
// uncaptured run has settled every field's capacities, the whole batch --
// every field's pipeline, spread over a pool of forked streams so that
// independent fields overlap on the GPU -- is captured into one CUDA graph
// and each later execute is a single graph launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/ftk.h"
#include "ftk_internal.h"
#include "ftk_kernels.cuh"

using namespace ftk;

namespace {
constexpr int kMaxWorkers = 16;
}

struct ftk_batch {
    int n = 0;
    bool autotune = false;
    std::vector<ftk_plan *> plans;
    RunCounters *d_ctr = nullptr;
    RunCounters *h_ctr = nullptr;        // pinned, n entries
    std::vector<cudaStream_t> workers;
    cudaStream_t capture = nullptr;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<const float *> graph_src;   // inputs the graph was captured with
    bool warmed = false;
    cudaStream_t last = nullptr;
};

namespace {

void release(ftk_batch *b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (ftk_plan *p : b->plans)
        if (p) ftk_plan_destroy(p);
    for (cudaStream_t s : b->workers) cudaStreamDestroy(s);
    if (b->capture) cudaStreamDestroy(b->capture);
    if (b->fork) cudaEventDestroy(b->fork);
    for (cudaEvent_t e : b->join) cudaEventDestroy(e);
    cudaFree(b->d_ctr);
    if (b->h_ctr) cudaFreeHost(b->h_ctr);
    delete b;
}

// the device pointer a field's pipeline reads: the caller's, or the plan's
// aligned copy when the streaming kernel needs 16-byte aligned rows
ftk_status source_of(ftk_plan *pl, const float *f, cudaStream_t s, const float **src) {
    return plan_source(pl, f, false, s, src);
}

// launch every field on the worker pool, joined back into `origin`
ftk_status launch_all_fields(ftk_batch *b, const float *const *f, cudaStream_t origin) {
    cudaError_t e = cudaEventRecord(b->fork, origin);
    if (e != cudaSuccess) return cuda_fail(e, "fork event");
    const int K = (int)b->workers.size();
    for (int w = 0; w < K; ++w) {
        e = cudaStreamWaitEvent(b->workers[w], b->fork, 0);
        if (e != cudaSuccess) return cuda_fail(e, "fork wait");
    }
    for (int i = 0; i < b->n; ++i) {
        cudaStream_t ws = b->workers[i % K];
        const float *src = nullptr;
        ftk_status st = source_of(b->plans[i], f[i], ws, &src);
        if (st != FTK_OK) return st;
        st = plan_launch(b->plans[i], src, ws);
        if (st != FTK_OK) return st;
    }
    for (int w = 0; w < K; ++w) {
        e = cudaEventRecord(b->join[w], b->workers[w]);
        if (e != cudaSuccess) return cuda_fail(e, "join event");
        e = cudaStreamWaitEvent(origin, b->join[w], 0);
        if (e != cudaSuccess) return cuda_fail(e, "join wait");
    }
    return FTK_OK;
}

ftk_status capture_graph(ftk_batch *b, const float *const *f) {
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    cudaError_t e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    ftk_status st = launch_all_fields(b, f, b->capture);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->capture, &g);
    if (st != FTK_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    b->graph = g;
    e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    b->graph_src.assign(f, f + b->n);
    return FTK_OK;
}

// one copy of all counters, then per-field checks (overflow reruns are
// synchronous and invalidate the graph, whose buffers then changed)
ftk_status settle_all(ftk_batch *b) {
    cudaError_t e = cudaStreamSynchronize(b->last);
    if (e != cudaSuccess) return cuda_fail(e, "batch synchronise");
    e = cudaMemcpy(b->h_ctr, b->d_ctr, sizeof(RunCounters) * b->n, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "batch counters");
    for (int i = 0; i < b->n; ++i) {
        ftk_plan *pl = b->plans[i];
        const unsigned long long cap_before = (unsigned long long)pl->W.cap + (unsigned long long)pl->W.scap;
        *pl->h_ctr = b->h_ctr[i];
        pl->stream = b->workers[i % b->workers.size()];
        ftk_status st = plan_check(pl);
        if (st != FTK_OK) return st;
        if ((unsigned long long)pl->W.cap + (unsigned long long)pl->W.scap != cap_before) {
            b->graph_src.clear();     // buffers moved: capture again next time
        }
    }
    return FTK_OK;
}

}  // namespace

extern "C" {

ftk_status ftk_batch_create(int nfields, const int64_t (*dims)[3], const ftk_params *p, ftk_batch **out) {
    if (out) *out = nullptr;
    if (!out || !dims || nfields < 1) return fail(FTK_ERR_ARG, "need nfields >= 1, dims and out");
    for (int i = 0; i < nfields; ++i)
        if (dims[i][0] < 2 || dims[i][1] < 2 || dims[i][2] < 1)
            return fail(FTK_ERR_ARG, "every field needs nx, ny >= 2 and nt >= 1");
    ftk_params prm;
    if (p) prm = *p;
    else ftk_params_default(&prm);
    ftk_batch *b = new (std::nothrow) ftk_batch;
    if (!b) return fail(FTK_ERR_NOMEM, "host allocation failed");
    b->n = nfields;
    b->autotune = (prm.flags & FTK_FLAG_AUTOTUNE) != 0;
    prm.flags &= ~(FTK_FLAG_STAGE_TIMES | FTK_FLAG_AUTOTUNE);
    if (cudaMalloc(&b->d_ctr, sizeof(RunCounters) * nfields) != cudaSuccess ||
        cudaMallocHost(&b->h_ctr, sizeof(RunCounters) * nfields) != cudaSuccess) {
        cudaGetLastError();
        release(b);
        return fail(FTK_ERR_NOMEM, "device allocation failed");
    }
    b->plans.assign(nfields, nullptr);
    for (int i = 0; i < nfields; ++i) {
        ftk_status st = plan_create(2, dims[i][0], dims[i][1], 1, dims[i][2], &prm, b->d_ctr + i, &b->plans[i]);
        if (st != FTK_OK) {
            release(b);
            return st;
        }
    }
    const int K = std::min(kMaxWorkers, nfields);
    for (int w = 0; w < K; ++w) {
        cudaStream_t s;
        cudaEvent_t ev;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            release(b);
            return fail(FTK_ERR_CUDA, "stream creation failed");
        }
        b->workers.push_back(s);
        b->join.push_back(ev);
    }
    if (cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        release(b);
        return fail(FTK_ERR_CUDA, "stream creation failed");
    }
    *out = b;
    return FTK_OK;
}

ftk_status ftk_batch_execute(ftk_batch *b, const float *const *f, void *cuda_stream) {
    if (!b || !f) return fail(FTK_ERR_ARG, "batch and fields must be non-NULL");
    for (int i = 0; i < b->n; ++i)
        if (!f[i] || !is_device_pointer(f[i])) return fail(FTK_ERR_ARG, "batched fields must be device pointers");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    b->last = s;
    if (!b->warmed) {
        // first run: uncaptured, so capacities (and, on request, the time
        // chunking of every shape) settle before the graph is built
        if (b->autotune) {
            for (int i = 0; i < b->n; ++i) {
                const float *src = nullptr;
                ftk_status st = source_of(b->plans[i], f[i], s, &src);
                if (st != FTK_OK) return st;
                st = plan_autotune(b->plans[i], src, s);
                if (st != FTK_OK) return st;
            }
        }
        ftk_status st = launch_all_fields(b, f, s);
        if (st != FTK_OK) return st;
        st = settle_all(b);
        if (st != FTK_OK) return st;
        b->warmed = true;
        return FTK_OK;
    }
    const bool same = b->graph_src.size() == (size_t)b->n && std::equal(f, f + b->n, b->graph_src.begin());
    if (!b->exec || !same) {
        ftk_status st = capture_graph(b, f);
        if (st != FTK_OK) return st;
    }
    cudaError_t e = cudaGraphLaunch(b->exec, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    for (ftk_plan *pl : b->plans) pl->executed = true;
    return FTK_OK;
}

ftk_status ftk_batch_counts(ftk_batch *b, int64_t *counts) {
    if (!b || !counts) return fail(FTK_ERR_ARG, "batch and counts must be non-NULL");
    if (!b->last && !b->warmed) return fail(FTK_ERR_STATE, "batch has not been executed");
    ftk_status st = settle_all(b);
    if (st != FTK_OK) return st;
    for (int i = 0; i < b->n; ++i) counts[i] = b->plans[i]->h_ctr->punctures;
    return FTK_OK;
}

ftk_status ftk_batch_download(ftk_batch *b, ftk_result **outs) {
    if (!b || !outs) return fail(FTK_ERR_ARG, "batch and outs must be non-NULL");
    for (int i = 0; i < b->n; ++i) outs[i] = nullptr;
    ftk_status st = settle_all(b);
    if (st != FTK_OK) return st;
    for (int i = 0; i < b->n; ++i) {
        st = plan_result(b->plans[i], &outs[i]);
        if (st != FTK_OK) {
            for (int j = 0; j < i; ++j) { ftk_result_free(outs[j]); outs[j] = nullptr; }
            return st;
        }
    }
    return FTK_OK;
}

ftk_status ftk_batch_kernels(ftk_batch *b, int64_t *k) {
    if (!b || !k) return fail(FTK_ERR_ARG, "NULL argument");
    int64_t total = 0;
    for (ftk_plan *pl : b->plans) {
        ftk_plan_desc d;
        ftk_status st = ftk_plan_describe(pl, &d);
        if (st != FTK_OK) return st;
        total += d.kernels_per_execute;
    }
    *k = total;
    return FTK_OK;
}

ftk_status ftk_batch_destroy(ftk_batch *b) {
    if (!b) return FTK_OK;
    if (b->last) cudaStreamSynchronize(b->last);
    release(b);
    return FTK_OK;
}

ftk_status ftk_track_cp2d_batch(int nfields, const float *const *f, const int64_t (*dims)[3], const ftk_params *p,
                                ftk_result **outs, void *cuda_stream) {
    if (outs)
        for (int i = 0; i < nfields; ++i) outs[i] = nullptr;
    if (!outs || !f) return fail(FTK_ERR_ARG, "fields and outs must be non-NULL");
    ftk_batch *b = nullptr;
    ftk_status st = ftk_batch_create(nfields, dims, p, &b);
    if (st != FTK_OK) return st;
    st = ftk_batch_execute(b, f, cuda_stream);
    if (st == FTK_OK) st = ftk_batch_download(b, outs);
    const std::string keep = ftk_last_error();
    ftk_batch_destroy(b);
    set_last_error(keep.c_str());
    return st;
}

}  // extern "C"
