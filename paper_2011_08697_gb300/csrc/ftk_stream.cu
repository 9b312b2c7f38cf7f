// In-situ streams (the paper's push_field_data(), Sec. 8; ordinal/interval
// traversal with a two-slice window, Sec. 3.2) and a small serving layer that
// admits streams by device-memory footprint.
//
// Push k runs the pipeline on slices [k-1, k] (a one-slice run for k = 0).
// The run's faces that lie entirely in slice k-1 were reported by push k-1;
// they are merged into the stream's device-resident union-find over every
// puncture so far, which carries component minima.  The delta of push k is
// the ordinal faces of slice k and the interval faces of slab [k-1, k], with
// provisional labels (smallest face id connected so far); closing the stream
// returns every puncture with its final label, equal to the whole-field
// result.
//
// A steady-state push (k >= 2) of a device slice is one replay of a captured
// CUDA graph and one synchronisation: the slice's address is read by the copy
// kernel from mapped host memory, the stream's scalars live on the device,
// and the delta records and counts land directly in pinned, mapped host
// memory.  Host slices take the same kernels launched directly, after an
// ordinary host-to-device copy.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <climits>
#include <condition_variable>
#include <deque>
#include <unordered_set>
#include <vector>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "../../include/ftk.h"
#include "ftk_internal.h"
#include "ftk_kernels.cuh"

using namespace ftk;

struct ftk_server {
    size_t budget = 0;
    size_t used = 0;
    std::mutex mu;
    std::condition_variable cv;     // signalled whenever memory is returned or the queue moves
    std::deque<uint64_t> queue;     // tickets of the opens waiting for admission, oldest first
    uint64_t next_ticket = 0;
};

struct ftk_stream {
    int ndim = 2;
    int nx = 0, ny = 0, nz = 1;
    ftk_params p{};
    ftk_server *server = nullptr;
    size_t footprint = 0;
    ftk_plan *plan1 = nullptr, *plan2 = nullptr;
    float *d2 = nullptr;          // two slices, [previous | current], rows of the plans' pitch
    long long slice_verts = 0;    // grid vertices per slice
    long long slice_rows = 0;     // rows per slice (ny * nz)
    long long slice_elems = 0;    // floats per slice in d2 (slice_rows * pitch)
    int pitch = 0;
    int T = 12, tbit = 4;
    long long k = 0;              // pushes done (host copy)
    long long n = 0;              // global slots in use (host copy)
    bool failed = false;          // a push failed: the stream accepts no more
    cudaStream_t cs = nullptr;
    cudaEvent_t done = nullptr;   // end of a push (blocking sync)
    StreamDev *dS = nullptr;      // device-resident scalars
    StreamView *hV = nullptr;     // mapped host memory: host and device addresses
    StreamView *dV = nullptr;
    StreamSrc *hSrc = nullptr, *dSrc = nullptr;
    ftk_cp *h_delta = nullptr, *d_delta = nullptr;   // mapped delta records
    long long dcap = 0;
    // global union-find over all punctures so far
    long long acap = 0;
    long long *gfid = nullptr;
    int *gparent = nullptr;
    long long *gmin = nullptr;
    int *gshadow = nullptr;
    ftk_cp *grec = nullptr;
    long long *ord_fid[2] = {nullptr, nullptr};
    int *ord_gi[2] = {nullptr, nullptr};
    long long ocap = 0;
    long long lcap = 0;
    int *link_prev = nullptr, *old_root = nullptr;
    long long *blk = nullptr;     // per-block counts of the delta compaction
    long long bcap = 0;
    // incremental 2D detect: the last slice's cube-row words (committed, pending)
    uint32_t *st_in = nullptr, *st_out = nullptr;
    long long st_words = 0;
    // one captured push (k >= 2) replayed for every later push
    cudaGraphExec_t exec = nullptr;
    // the merge kernels' arguments for pushes with plan1 / plan2, in device
    // memory (reallocating the stream's arrays updates them, not the graph)
    StreamMerge *dM = nullptr;    // [2]
    bool merge_dirty = true;
};

namespace {

// capacity an array grows to when it must hold `need` entries
long long grow_cap(long long need) { return std::max<long long>(need + need / 2, 1 << 12); }

template <typename T>
ftk_status grow(T **ptr, long long cap, long long need, long long keep, cudaStream_t s, long long *newcap) {
    *newcap = cap;
    if (need <= cap) return FTK_OK;
    long long nc = grow_cap(need);
    T *np = nullptr;
    if (cudaMalloc(&np, sizeof(T) * nc) != cudaSuccess) {
        cudaGetLastError();
        return fail(FTK_ERR_NOMEM, "stream state allocation failed");
    }
    if (*ptr && keep > 0) {
        cudaError_t e = cudaMemcpyAsync(np, *ptr, sizeof(T) * keep, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) { cudaFree(np); return cuda_fail(e, "stream state copy"); }
        cudaStreamSynchronize(s);
    }
    cudaFree(*ptr);
    *ptr = np;
    *newcap = nc;
    return FTK_OK;
}

void drop_graph(ftk_stream *st) {
    if (st->exec) cudaGraphExecDestroy(st->exec);
    st->exec = nullptr;
}

// reserves `add` more bytes of device memory for the stream: within the
// server's budget (checked and charged under its mutex), else FTK_ERR_BUSY
ftk_status reserve(ftk_stream *st, size_t add) {
    if (st->server) {
        std::lock_guard<std::mutex> lock(st->server->mu);
        if (st->server->used + add > st->server->budget)
            return fail(FTK_ERR_BUSY, "the stream's device state would grow past the server's memory budget (" +
                                          std::to_string(add) + " more bytes)");
        st->server->used += add;
    }
    st->footprint += add;
    return FTK_OK;
}

void unreserve(ftk_stream *st, size_t sub) {
    if (st->server) {
        {
            std::lock_guard<std::mutex> lock(st->server->mu);
            st->server->used -= std::min(st->server->used, sub);
        }
        st->server->cv.notify_all();
    }
    st->footprint -= std::min(st->footprint, sub);
}

// every per-push array sized for a run of up to cap punctures on top of the
// n slots in use; a reallocation invalidates the captured push.  Growth is
// charged to the server's budget before any allocation (FTK_ERR_BUSY when it
// does not fit); slot indices are 32-bit, so n + cap must stay below 2^31.
ftk_status ensure_all(ftk_stream *st, long long cap) {
    ftk_status s;
    const long long need = st->n + cap;
    if (need > INT_MAX)
        return fail(FTK_ERR_RANGE, "the stream holds too many punctures for its 32-bit union-find slots");
    if (need > st->acap) {
        const size_t add = (size_t)(grow_cap(need) - st->acap) * (8 + 4 + 8 + 4 + sizeof(ftk_cp));
        if ((s = reserve(st, add)) != FTK_OK) return s;
        long long c0, c1, c2, c3, c4;
        if ((s = grow(&st->gfid, st->acap, need, st->n, st->cs, &c0)) != FTK_OK ||
            (s = grow(&st->gparent, st->acap, need, st->n, st->cs, &c1)) != FTK_OK ||
            (s = grow(&st->gmin, st->acap, need, st->n, st->cs, &c2)) != FTK_OK ||
            (s = grow(&st->gshadow, st->acap, need, st->n, st->cs, &c3)) != FTK_OK ||
            (s = grow(&st->grec, st->acap, need, st->n, st->cs, &c4)) != FTK_OK) {
            // arrays that did grow keep their new size; what was charged for
            // the rest is returned, and the next call grows them again
            unreserve(st, add);
            return s;
        }
        st->acap = c0;
        st->merge_dirty = true;
    }
    if (cap > st->lcap) {
        const size_t add = (size_t)(grow_cap(cap) - st->lcap) * 8;
        if ((s = reserve(st, add)) != FTK_OK) return s;
        long long a, b;
        if ((s = grow(&st->link_prev, st->lcap, cap, 0, st->cs, &a)) != FTK_OK ||
            (s = grow(&st->old_root, st->lcap, cap, 0, st->cs, &b)) != FTK_OK) {
            unreserve(st, add);
            return s;
        }
        st->lcap = a;
        st->merge_dirty = true;
    }
    const long long nblk = 4 * (cap / DELTA_BLOCK + 1);
    if (nblk > st->bcap) {
        const size_t add = (size_t)(grow_cap(nblk) - st->bcap) * 8;
        if ((s = reserve(st, add)) != FTK_OK) return s;
        long long a;
        if ((s = grow(&st->blk, st->bcap, nblk, 0, st->cs, &a)) != FTK_OK) {
            unreserve(st, add);
            return s;
        }
        st->bcap = a;
        st->merge_dirty = true;
    }
    if (cap > st->ocap) {
        // the buffer of the last push's parity keeps its ordinal faces
        const int keep = (int)((st->k - 1) & 1);
        long long nk = 0;
        if (st->k > 0) cudaMemcpy(&nk, &st->dS->n_ord[keep], sizeof(long long), cudaMemcpyDeviceToHost);
        const size_t add = (size_t)(grow_cap(cap) - st->ocap) * 24;
        if ((s = reserve(st, add)) != FTK_OK) return s;
        long long a = 0, b = 0;
        for (int q = 0; q < 2; ++q) {
            if ((s = grow(&st->ord_fid[q], st->ocap, cap, q == keep ? nk : 0, st->cs, &a)) != FTK_OK ||
                (s = grow(&st->ord_gi[q], st->ocap, cap, q == keep ? nk : 0, st->cs, &b)) != FTK_OK) {
                unreserve(st, add);
                return s;
            }
        }
        st->ocap = a;
        st->merge_dirty = true;
    }
    if (cap > st->dcap) {
        const long long nc = std::max<long long>(cap + cap / 2, 1 << 12);
        ftk_cp *h = nullptr;
        if (cudaHostAlloc(&h, sizeof(ftk_cp) * nc, cudaHostAllocMapped) != cudaSuccess) {
            cudaGetLastError();
            return fail(FTK_ERR_NOMEM, "pinned delta buffer allocation failed");
        }
        if (st->h_delta) cudaFreeHost(st->h_delta);
        st->h_delta = h;
        cudaHostGetDevicePointer((void **)&st->d_delta, h, 0);
        st->dcap = nc;
        st->merge_dirty = true;
    }
    return FTK_OK;
}

StreamMerge merge_args(ftk_stream *st, ftk_plan *pl) {
    StreamMerge M;
    std::memset(&M, 0, sizeof(M));
    M.face = pl->W.face;
    M.label = pl->W.label;
    M.packed = pl->W.packed;
    M.ctr = pl->W.ctr;
    M.slice_verts = st->slice_verts;
    M.T = st->T;
    M.tbit = st->tbit;
    M.S = st->dS;
    M.gfid = st->gfid; M.gparent = st->gparent; M.gmin = st->gmin; M.gshadow = st->gshadow; M.grec = st->grec;
    for (int q = 0; q < 2; ++q) { M.ord_fid[q] = st->ord_fid[q]; M.ord_gi[q] = st->ord_gi[q]; }
    M.link_prev = st->link_prev;
    M.old_root = st->old_root;
    M.blk = st->blk;
    M.st_in = st->st_in;
    M.st_out = st->st_out;
    M.st_words = st->st_words;
    M.delta = st->d_delta;
    M.view = st->dV;
    return M;
}

// refreshes the device copies of the merge arguments (before a push, on the
// stream's CUDA stream, so that the copy precedes the push's kernels)
ftk_status sync_merge(ftk_stream *st) {
    if (!st->merge_dirty) return FTK_OK;
    StreamMerge h[2] = {merge_args(st, st->plan1), merge_args(st, st->plan2)};
    const cudaError_t e = cudaMemcpyAsync(st->dM, h, sizeof(h), cudaMemcpyHostToDevice, st->cs);
    if (e != cudaSuccess) return cuda_fail(e, "merge arguments");
    // the source is pageable: the call returns once h has been staged
    st->merge_dirty = false;
    return FTK_OK;
}

// one push's device work: bring in the slice (host_slice: a host pointer to
// copy from; otherwise the device address in *dSrc), run the pipeline, merge
ftk_status enqueue_push(ftk_stream *st, ftk_plan *pl, long long k, const float *host_slice) {
    const size_t ebytes = sizeof(float) * (size_t)st->slice_elems;
    float *dst = k == 0 ? st->d2 : st->d2 + st->slice_elems;
    cudaError_t e;
    if (k >= 2 && (e = cudaMemcpyAsync(st->d2, st->d2 + st->slice_elems, ebytes, cudaMemcpyDeviceToDevice, st->cs)) !=
                      cudaSuccess)
        return cuda_fail(e, "slice shift");
    if (host_slice) {
        if (st->pitch == st->nx) {
            e = cudaMemcpyAsync(dst, host_slice, ebytes, cudaMemcpyHostToDevice, st->cs);
        } else {
            e = cudaMemcpy2DAsync(dst, (size_t)st->pitch * 4, host_slice, (size_t)st->nx * 4, (size_t)st->nx * 4,
                                  (size_t)st->slice_rows, cudaMemcpyHostToDevice, st->cs);
            if (e == cudaSuccess) e = launch_fill_pad(dst, st->nx, st->pitch, st->slice_rows, st->cs);
        }
    } else {
        e = launch_stream_copy(st->dSrc, dst, st->nx, st->pitch, st->slice_rows, st->cs);
    }
    if (e != cudaSuccess) return cuda_fail(e, "slice copy");
    ftk_status s = plan_launch(pl, st->d2, st->cs);
    if (s != FTK_OK) return s;
    if ((e = launch_stream_merge(st->dM + (pl == st->plan1 ? 0 : 1), merge_args(st, pl), pl->W.cap, st->cs)) !=
        cudaSuccess)
        return cuda_fail(e, "stream merge launch");
    return FTK_OK;
}

// captures the steady-state push (k >= 2) into a graph
void capture_push(ftk_stream *st) {
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(st->cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    const ftk_status s = enqueue_push(st, st->plan2, 2, nullptr);
    const cudaError_t e = cudaStreamEndCapture(st->cs, &g);
    if (s != FTK_OK || e != cudaSuccess || !g) {
        cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        return;
    }
    if (cudaGraphInstantiate(&st->exec, g, 0) != cudaSuccess) {
        cudaGetLastError();
        st->exec = nullptr;
    }
    cudaGraphDestroy(g);
}

void release(ftk_stream *st) {
    if (!st) return;
    if (st->cs) cudaStreamSynchronize(st->cs);
    drop_graph(st);
    if (st->plan1) ftk_plan_destroy(st->plan1);
    if (st->plan2) ftk_plan_destroy(st->plan2);
    cudaFree(st->d2);
    cudaFree(st->dS);
    cudaFree(st->dM);
    if (st->hV) cudaFreeHost(st->hV);
    if (st->hSrc) cudaFreeHost(st->hSrc);
    if (st->h_delta) cudaFreeHost(st->h_delta);
    cudaFree(st->gfid); cudaFree(st->gparent); cudaFree(st->gmin); cudaFree(st->gshadow); cudaFree(st->grec);
    for (int q = 0; q < 2; ++q) { cudaFree(st->ord_fid[q]); cudaFree(st->ord_gi[q]); }
    cudaFree(st->link_prev); cudaFree(st->old_root); cudaFree(st->blk);
    cudaFree(st->st_in); cudaFree(st->st_out);
    if (st->done) cudaEventDestroy(st->done);
    if (st->cs) cudaStreamDestroy(st->cs);
    if (st->server) {
        {
            std::lock_guard<std::mutex> lock(st->server->mu);
            st->server->used -= std::min(st->server->used, st->footprint);
        }
        st->server->cv.notify_all();
    }
    delete st;
}

// device bytes charged for a plan's workspace
size_t plan_bytes(long long cap, long long scap, long long nseg) {
    return (size_t)cap * (8 + 8 + 4 + 16 + 1 + 8 + sizeof(ftk_cp)) + (size_t)scap * (8 + 8 + 4 + 12) +
           (size_t)nseg * (4 + 8 + 8 + 4 + 8);
}
size_t plan_bytes(const ftk_plan *pl) { return plan_bytes(pl->W.cap, pl->W.scap, pl->W.nseg); }

// bytes ensure_all charges when it first sizes the per-push arrays for cap
size_t first_push_bytes(long long cap) {
    return (size_t)grow_cap(cap) * (8 + 4 + 8 + 4 + sizeof(ftk_cp)) + (size_t)grow_cap(cap) * 8 +
           (size_t)grow_cap(4 * (cap / DELTA_BLOCK + 1)) * 8 + (size_t)grow_cap(cap) * 24;
}

// the footprint open_stream charges for a stream of this shape, computed
// without allocating anything (the same sizes its plans and arrays get)
ftk_status stream_footprint(int ndim, int64_t nx, int64_t ny, int64_t nz, const ftk_params *p, size_t *fp) {
    ftk_params prm;
    if (p) prm = *p;
    else ftk_params_default(&prm);
    prm.flags &= ~FTK_FLAG_STAGE_TIMES;
    if (ndim == 2) nz = 1;
    PlanSizes a, b;
    ftk_status s;
    if ((s = plan_sizes(ndim, nx, ny, nz, 1, &prm, &a, true)) != FTK_OK ||
        (s = plan_sizes(ndim, nx, ny, nz, 2, &prm, &b, true)) != FTK_OK)
        return s;
    long long st_words = 0;
    if (ndim == 2 && a.variant != VAR_TILE && b.variant != VAR_TILE && a.B.nyb == b.B.nyb)
        st_words = stream2_state_words(b.F, b.B);
    const long long slice_elems = (long long)ny * nz * b.F.pitch;
    *fp = sizeof(float) * 2 * (size_t)slice_elems + plan_bytes(a.cap, a.scap, a.nseg) +
          plan_bytes(b.cap, b.scap, b.nseg) + sizeof(uint32_t) * 2 * (size_t)st_words +
          first_push_bytes(std::max(a.cap, b.cap));
    return FTK_OK;
}

// admission of a footprint by a server: immediately (timeout_ms = 0: only if
// no earlier open is waiting and it fits now) or after waiting in FIFO order
// for streams to close, for at most timeout_ms
ftk_status admit(ftk_server *srv, size_t fp, long long timeout_ms) {
    std::unique_lock<std::mutex> lock(srv->mu);
    if (fp > srv->budget)
        return fail(FTK_ERR_BUSY, "admission refused: the stream needs " + std::to_string(fp) +
                                      " bytes of device memory, more than the whole budget");
    if (srv->queue.empty() && srv->used + fp <= srv->budget) {
        srv->used += fp;
        return FTK_OK;
    }
    if (timeout_ms <= 0)
        return fail(FTK_ERR_BUSY, "admission refused: the stream needs " + std::to_string(fp) +
                                      " bytes of device memory beyond the budget");
    const uint64_t ticket = srv->next_ticket++;
    srv->queue.push_back(ticket);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
    const bool ok = srv->cv.wait_until(lock, deadline, [&] {
        return srv->queue.front() == ticket && srv->used + fp <= srv->budget;
    });
    srv->queue.erase(std::find(srv->queue.begin(), srv->queue.end(), ticket));
    if (ok) srv->used += fp;
    lock.unlock();
    srv->cv.notify_all();   // the next waiter may be at the head now
    if (!ok)
        return fail(FTK_ERR_BUSY, "admission refused: no room within " + std::to_string(timeout_ms) + " ms");
    return FTK_OK;
}

ftk_status open_stream(ftk_server *srv, int ndim, int64_t nx, int64_t ny, int64_t nz, const ftk_params *p,
                       long long timeout_ms, ftk_stream **out) {
    if (out) *out = nullptr;
    if (!out) return fail(FTK_ERR_ARG, "out is NULL");
    if (ndim != 2 && ndim != 3) return fail(FTK_ERR_ARG, "ndim must be 2 or 3");
    if (ndim == 2) nz = 1;
    if (nx < 2 || ny < 2 || (ndim == 3 && nz < 2)) return fail(FTK_ERR_ARG, "every spatial extent must be >= 2");
    // admission before any allocation: the footprint is known from the shape
    size_t fp = 0;
    ftk_status s = FTK_OK;
    if (srv) {
        if ((s = stream_footprint(ndim, nx, ny, nz, p, &fp)) != FTK_OK) return s;
        if ((s = admit(srv, fp, timeout_ms)) != FTK_OK) return s;
    }
    // returns the admitted bytes when the open fails below
    auto give_back = [&]() {
        if (!srv) return;
        {
            std::lock_guard<std::mutex> lock(srv->mu);
            srv->used -= std::min(srv->used, fp);
        }
        srv->cv.notify_all();
    };
    ftk_stream *st = new (std::nothrow) ftk_stream;
    if (!st) {
        give_back();
        return fail(FTK_ERR_NOMEM, "host allocation failed");
    }
    st->ndim = ndim;
    st->nx = (int)nx; st->ny = (int)ny; st->nz = (int)nz;
    if (p) st->p = *p;
    else ftk_params_default(&st->p);
    st->p.flags &= ~FTK_FLAG_STAGE_TIMES;
    st->slice_verts = (long long)nx * ny * nz;
    st->T = ndim == 2 ? 12 : 60;
    st->tbit = ndim == 2 ? 4 : 8;
    if ((s = plan_create(ndim, nx, ny, nz, 1, &st->p, nullptr, &st->plan1, true)) != FTK_OK ||
        (s = plan_create(ndim, nx, ny, nz, 2, &st->p, nullptr, &st->plan2, true)) != FTK_OK) {
        release(st);
        give_back();
        return s;
    }
    // incremental detect (2D streaming plans): push 0 stores slice 0's
    // cube-row words, every later push streams only its new slice
    if (ndim == 2 && st->plan1->variant != VAR_TILE && st->plan2->variant != VAR_TILE &&
        st->plan1->B.nyb == st->plan2->B.nyb) {
        st->st_words = stream2_state_words(st->plan2->F, st->plan2->B);
        if (cudaMalloc(&st->st_in, sizeof(uint32_t) * st->st_words) != cudaSuccess ||
            cudaMalloc(&st->st_out, sizeof(uint32_t) * st->st_words) != cudaSuccess) {
            cudaGetLastError();
            release(st);
            give_back();
            return fail(FTK_ERR_NOMEM, "stream allocation failed");
        }
        st->plan1->B.st_mode = 1;
        st->plan1->B.st_out = st->st_out;
        st->plan2->B.st_mode = 2;
        st->plan2->B.st_in = st->st_in;
        st->plan2->B.st_out = st->st_out;
        st->plan2->B.tc = 2;     // one unit per row block covers both slices
        st->plan2->B.ntc = 1;
    }
    st->pitch = st->plan2->F.pitch;
    st->slice_rows = (long long)ny * nz;
    st->slice_elems = st->slice_rows * st->pitch;
    if (cudaStreamCreateWithFlags(&st->cs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMalloc(&st->d2, sizeof(float) * 2 * st->slice_elems) != cudaSuccess ||
        cudaMalloc(&st->dS, sizeof(StreamDev)) != cudaSuccess ||
        cudaMalloc(&st->dM, 2 * sizeof(StreamMerge)) != cudaSuccess ||
        cudaMemset(st->dS, 0, sizeof(StreamDev)) != cudaSuccess ||
        cudaHostAlloc(&st->hV, sizeof(StreamView), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostAlloc(&st->hSrc, sizeof(StreamSrc), cudaHostAllocMapped) != cudaSuccess ||
        cudaEventCreateWithFlags(&st->done, cudaEventBlockingSync | cudaEventDisableTiming) != cudaSuccess ||
        cudaHostGetDevicePointer((void **)&st->dV, st->hV, 0) != cudaSuccess ||
        cudaHostGetDevicePointer((void **)&st->dSrc, st->hSrc, 0) != cudaSuccess) {
        cudaGetLastError();
        release(st);
        give_back();
        return fail(FTK_ERR_NOMEM, "stream allocation failed");
    }
    st->footprint = sizeof(float) * 2 * st->slice_elems + plan_bytes(st->plan1) + plan_bytes(st->plan2) +
                    sizeof(uint32_t) * 2 * (size_t)st->st_words;
    // the union-find and delta arrays for the first pushes are part of the
    // footprint admission checks (later growth is charged push by push)
    if ((s = ensure_all(st, std::max(st->plan1->W.cap, st->plan2->W.cap))) != FTK_OK) {
        release(st);
        give_back();
        return s;
    }
    if (srv) {
        // the admitted bytes become the stream's; they equal what it holds
        std::lock_guard<std::mutex> lock(srv->mu);
        srv->used = srv->used - std::min(srv->used, fp) + st->footprint;
        st->server = srv;
    }
    *out = st;
    return FTK_OK;
}

// the merge kernels' report, written by the device into mapped host memory
StreamView read_view(const ftk_stream *st) {
    const volatile StreamView *p = st->hV;
    StreamView v;
    v.run_status = p->run_status;
    v.status = p->status;
    v.punctures = p->punctures;
    v.delta = p->delta;
    return v;
}

// marks the stream failed; msg = nullptr keeps the message already set
ftk_status stream_error(ftk_stream *st, ftk_status s, const char *msg) {
    st->failed = true;
    if (!msg) return s;
    return fail(s, msg);
}

}  // namespace

extern "C" {

ftk_status ftk_server_create(uint64_t budget_bytes, ftk_server **out) {
    if (out) *out = nullptr;
    if (!out || budget_bytes == 0) return fail(FTK_ERR_ARG, "need a budget and out");
    ftk_server *s = new (std::nothrow) ftk_server;
    if (!s) return fail(FTK_ERR_NOMEM, "host allocation failed");
    s->budget = (size_t)budget_bytes;
    *out = s;
    return FTK_OK;
}

ftk_status ftk_server_used(ftk_server *s, uint64_t *used) {
    if (!s || !used) return fail(FTK_ERR_ARG, "NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    *used = s->used;
    return FTK_OK;
}

ftk_status ftk_server_destroy(ftk_server *s) {
    if (!s) return FTK_OK;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->used != 0) return fail(FTK_ERR_STATE, "streams are still open on this server");
    }
    delete s;
    return FTK_OK;
}

ftk_status ftk_stream_open(int ndim, int64_t nx, int64_t ny, int64_t nz, const ftk_params *p, ftk_stream **s) {
    return open_stream(nullptr, ndim, nx, ny, nz, p, 0, s);
}

ftk_status ftk_stream_open_in(ftk_server *srv, int ndim, int64_t nx, int64_t ny, int64_t nz, const ftk_params *p,
                              ftk_stream **s) {
    if (s) *s = nullptr;
    if (!srv) return fail(FTK_ERR_ARG, "server is NULL");
    return open_stream(srv, ndim, nx, ny, nz, p, 0, s);
}

ftk_status ftk_stream_open_wait(ftk_server *srv, int ndim, int64_t nx, int64_t ny, int64_t nz, const ftk_params *p,
                                int64_t timeout_ms, ftk_stream **s) {
    if (s) *s = nullptr;
    if (!srv) return fail(FTK_ERR_ARG, "server is NULL");
    if (timeout_ms < 0) return fail(FTK_ERR_ARG, "timeout_ms must be >= 0");
    return open_stream(srv, ndim, nx, ny, nz, p, (long long)timeout_ms, s);
}

ftk_status ftk_stream_footprint(int ndim, int64_t nx, int64_t ny, int64_t nz, const ftk_params *p, uint64_t *bytes) {
    if (!bytes) return fail(FTK_ERR_ARG, "bytes is NULL");
    if (ndim != 2 && ndim != 3) return fail(FTK_ERR_ARG, "ndim must be 2 or 3");
    size_t fp = 0;
    ftk_status st = stream_footprint(ndim, nx, ny, nz, p, &fp);
    if (st == FTK_OK) *bytes = fp;
    return st;
}

}  // extern "C"

namespace {

// first half of a push: queue the device work on the stream's CUDA stream
// (one graph replay for a steady-state device slice) without waiting
ftk_status push_begin(ftk_stream *st, const float *slice) {
    if (st->failed) return fail(FTK_ERR_STATE, "an earlier push of this stream failed");
    const long long k = st->k;
    ftk_plan *pl = k == 0 ? st->plan1 : st->plan2;
    // device slices: the copy kernel reads the address from mapped memory
    // (the captured push is replayed); host slices: an ordinary copy
    const bool on_dev = is_device_pointer(slice);
    if (on_dev) {
        st->hSrc->ptr = slice;
        std::atomic_thread_fence(std::memory_order_seq_cst);
    }
    ftk_status s = ensure_all(st, pl->W.cap);
    if (s != FTK_OK) return stream_error(st, s, nullptr);
    if ((s = sync_merge(st)) != FTK_OK) return stream_error(st, s, nullptr);
    cudaError_t e;
    if (on_dev && k >= 2 && !st->exec) capture_push(st);
    if (on_dev && k >= 2 && st->exec) {
        if ((e = cudaGraphLaunch(st->exec, st->cs)) != cudaSuccess) return stream_error(st, FTK_ERR_CUDA, cudaGetErrorString(e));
    } else if ((s = enqueue_push(st, pl, k, on_dev ? nullptr : slice)) != FTK_OK) {
        return stream_error(st, s, nullptr);
    }
    if ((e = cudaEventRecord(st->done, st->cs)) != cudaSuccess) return stream_error(st, FTK_ERR_CUDA, cudaGetErrorString(e));
    return FTK_OK;
}

// second half: wait for the push, repair an overflowed run, hand out the delta
ftk_status push_end(ftk_stream *st, ftk_result **delta) {
    ftk_plan *pl = st->k == 0 ? st->plan1 : st->plan2;
    ftk_status s;
    cudaError_t e;
    // a blocking-sync event: the waiting thread sleeps instead of spinning
    if ((e = cudaEventSynchronize(st->done)) != cudaSuccess) return stream_error(st, FTK_ERR_CUDA, cudaGetErrorString(e));
    StreamView v = read_view(st);
    if (v.run_status & (ST_OVERFLOW | ST_SOVERFLOW | ST_WIDE)) {
        // not merged: repair the run (larger capacity or exact rounding),
        // then merge it
        int64_t P = 0;
        if ((s = ftk_plan_count(pl, &P)) != FTK_OK) return stream_error(st, s, nullptr);
        if ((s = ensure_all(st, pl->W.cap)) != FTK_OK) return stream_error(st, s, nullptr);
        drop_graph(st);   // the run's capacity changed
        st->merge_dirty = true;   // the run's buffers changed with its capacity
        if ((s = sync_merge(st)) != FTK_OK) return stream_error(st, s, nullptr);
        if ((e = launch_stream_merge(st->dM + (pl == st->plan1 ? 0 : 1), merge_args(st, pl), pl->W.cap, st->cs)) !=
                cudaSuccess ||
            (e = cudaEventRecord(st->done, st->cs)) != cudaSuccess || (e = cudaEventSynchronize(st->done)) != cudaSuccess)
            return stream_error(st, FTK_ERR_CUDA, cudaGetErrorString(e));
        v = read_view(st);
    }
    if (v.run_status & ST_RANGE)
        return stream_error(st, FTK_ERR_RANGE, "a sample is non-finite or |f * 2^quant_shift| exceeds 2^28");
    if ((v.run_status | v.status) & ST_TIMEOUT) return stream_error(st, FTK_ERR_TIMEOUT, "a bounded device loop gave up");
    if ((v.run_status | v.status) & ST_PAIRING)
        return stream_error(st, FTK_ERR_INVARIANT, "the pairing invariant or a repeated face failed");
    const long long D = v.delta;
    ftk_result *r = new (std::nothrow) ftk_result;
    if (r) r->data = (ftk_cp *)std::malloc(std::max<size_t>(1, (size_t)D) * sizeof(ftk_cp));
    if (!r || !r->data) {
        delete r;
        return stream_error(st, FTK_ERR_NOMEM, "host allocation failed");
    }
    r->count = (size_t)D;
    if (D > 0) std::memcpy(r->data, st->h_delta, sizeof(ftk_cp) * (size_t)D);
    st->n += v.punctures;
    st->k += 1;
    *delta = r;
    return FTK_OK;
}

}  // namespace

extern "C" {

ftk_status ftk_stream_push(ftk_stream *st, const float *slice, ftk_result **delta) {
    if (delta) *delta = nullptr;
    if (!st || !slice || !delta) return fail(FTK_ERR_ARG, "stream, slice and delta must be non-NULL");
    ftk_status s = push_begin(st, slice);
    if (s != FTK_OK) return s;
    return push_end(st, delta);
}

ftk_status ftk_streams_push(int n, ftk_stream *const *streams, const float *const *slices, ftk_result **deltas) {
    if (n < 0 || (n > 0 && (!streams || !slices || !deltas))) return fail(FTK_ERR_ARG, "invalid argument");
    for (int i = 0; i < n; ++i) deltas[i] = nullptr;
    {
        std::unordered_set<const ftk_stream *> seen;
        for (int i = 0; i < n; ++i) {
            if (!streams[i] || !slices[i]) return fail(FTK_ERR_ARG, "NULL stream or slice");
            if (!seen.insert(streams[i]).second) return fail(FTK_ERR_ARG, "a stream appears twice in one call");
        }
    }
    // queue every push first (their device work overlaps on the streams' own
    // CUDA streams), then collect them in order
    ftk_status first = FTK_OK;
    std::string first_msg;
    std::vector<char> begun((size_t)n, 0);
    for (int i = 0; i < n; ++i) {
        const ftk_status s = push_begin(streams[i], slices[i]);
        if (s == FTK_OK) begun[(size_t)i] = 1;
        else if (first == FTK_OK) { first = s; first_msg = ftk_last_error(); }
    }
    for (int i = 0; i < n; ++i) {
        if (!begun[(size_t)i]) continue;
        const ftk_status s = push_end(streams[i], &deltas[i]);
        if (s != FTK_OK && first == FTK_OK) { first = s; first_msg = ftk_last_error(); }
    }
    if (first != FTK_OK) return fail(first, first_msg);
    return FTK_OK;
}

ftk_status ftk_stream_close(ftk_stream *st, ftk_result **final) {
    if (final) *final = nullptr;
    if (!st) return fail(FTK_ERR_ARG, "stream is NULL");
    ftk_status s = FTK_OK;
    if (final) {
        ftk_cp *d_out = nullptr;
        long long *d_cnt = nullptr;
        unsigned *d_st = nullptr;
        cudaError_t e = cudaSuccess;
        if (cudaMalloc(&d_out, sizeof(ftk_cp) * std::max<long long>(1, st->n)) != cudaSuccess ||
            cudaMalloc(&d_cnt, sizeof(long long)) != cudaSuccess ||
            cudaMalloc(&d_st, sizeof(unsigned)) != cudaSuccess) {
            cudaGetLastError();
            s = fail(FTK_ERR_NOMEM, "final result allocation failed");
        } else if ((e = cudaMemsetAsync(d_st, 0, sizeof(unsigned), st->cs)) != cudaSuccess ||
                   (e = launch_stream_final(st->n, st->gshadow, st->gparent, st->gmin, st->grec, d_out, d_cnt, d_st,
                                            st->cs)) != cudaSuccess ||
                   (e = cudaStreamSynchronize(st->cs)) != cudaSuccess) {
            s = cuda_fail(e, "final labels");
        } else {
            long long cnt = 0;
            cudaMemcpy(&cnt, d_cnt, sizeof(long long), cudaMemcpyDeviceToHost);
            ftk_result *r = new (std::nothrow) ftk_result;
            if (r) r->data = (ftk_cp *)std::malloc(std::max<size_t>(1, (size_t)cnt) * sizeof(ftk_cp));
            if (!r || !r->data) {
                delete r;
                s = fail(FTK_ERR_NOMEM, "host allocation failed");
            } else {
                r->count = (size_t)cnt;
                if (cnt > 0) cudaMemcpy(r->data, d_out, sizeof(ftk_cp) * cnt, cudaMemcpyDeviceToHost);
                // pushes interleave in face-id order (interval faces of slab
                // [k-1, k] arrive one push after the ordinal faces of slice k-1)
                std::sort(r->data, r->data + r->count,
                          [](const ftk_cp &a, const ftk_cp &b) { return a.face_id < b.face_id; });
                *final = r;
            }
        }
        cudaFree(d_out);
        cudaFree(d_cnt);
        cudaFree(d_st);
    }
    release(st);
    return s;
}

}  // extern "C"
