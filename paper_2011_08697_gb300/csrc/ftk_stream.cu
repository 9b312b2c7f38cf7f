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
#include <cuda_runtime.h>

#include <algorithm>
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
};

struct ftk_stream {
    int ndim = 2;
    int nx = 0, ny = 0, nz = 1;
    ftk_params p{};
    ftk_server *server = nullptr;
    size_t footprint = 0;
    ftk_plan *plan1 = nullptr, *plan2 = nullptr;
    float *d2 = nullptr;          // two slices, [previous | current]
    long long slice_verts = 0;
    int T = 12, tbit = 4;
    int k = 0;                    // pushes done
    cudaStream_t cs = nullptr;
    // global union-find over all punctures so far
    long long acap = 0, n = 0;
    long long *gfid = nullptr;
    int *gparent = nullptr;
    long long *gmin = nullptr;
    int *gshadow = nullptr;
    ftk_cp *grec = nullptr;
    // last-slice ordinal faces of the previous push (double-buffered)
    long long *ord_fid[2] = {nullptr, nullptr};
    int *ord_gi[2] = {nullptr, nullptr};
    long long ocap[2] = {0, 0};
    int n_ord = 0, cur = 0;
    // per-push scratch
    long long lcap = 0;
    int *link_prev = nullptr, *old_root = nullptr;
    ftk_cp *delta = nullptr;
    long long *d_small = nullptr;     // delta count, ordinal count
    unsigned *d_status = nullptr;
    long long *h_small = nullptr;     // pinned
    unsigned *h_status = nullptr;     // pinned
};

namespace {

template <typename T>
ftk_status grow(T **ptr, long long &cap, long long need, long long keep, cudaStream_t s) {
    if (need <= cap) return FTK_OK;
    long long nc = std::max<long long>(need + need / 2, 1 << 12);
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
    cap = nc;
    return FTK_OK;
}

ftk_status ensure_global(ftk_stream *st, long long need) {
    if (need <= st->acap) return FTK_OK;
    long long c0 = st->acap, c1 = st->acap, c2 = st->acap, c3 = st->acap, c4 = st->acap;
    ftk_status s;
    if ((s = grow(&st->gfid, c0, need, st->n, st->cs)) != FTK_OK) return s;
    if ((s = grow(&st->gparent, c1, need, st->n, st->cs)) != FTK_OK) return s;
    if ((s = grow(&st->gmin, c2, need, st->n, st->cs)) != FTK_OK) return s;
    if ((s = grow(&st->gshadow, c3, need, st->n, st->cs)) != FTK_OK) return s;
    if ((s = grow(&st->grec, c4, need, st->n, st->cs)) != FTK_OK) return s;
    if (st->server) {
        std::lock_guard<std::mutex> lock(st->server->mu);
        const size_t add = (size_t)(c0 - st->acap) * (8 + 4 + 8 + 4 + sizeof(ftk_cp));
        st->server->used += add;
        st->footprint += add;
    }
    st->acap = c0;
    return FTK_OK;
}

ftk_status ensure_scratch(ftk_stream *st, long long P) {
    if (P <= st->lcap && P <= st->ocap[0] && P <= st->ocap[1]) return FTK_OK;
    long long need = std::max<long long>(P, 1);
    long long a = st->lcap, b = st->lcap, c = st->lcap;
    ftk_status s;
    if ((s = grow(&st->link_prev, a, need, 0, st->cs)) != FTK_OK) return s;
    if ((s = grow(&st->old_root, b, need, 0, st->cs)) != FTK_OK) return s;
    if ((s = grow(&st->delta, c, need, 0, st->cs)) != FTK_OK) return s;
    st->lcap = a;
    // ordinal buffers: the current one keeps its contents
    for (int q = 0; q < 2; ++q) {
        long long oc = st->ocap[q];
        if ((s = grow(&st->ord_fid[q], oc, need, q == st->cur ? st->n_ord : 0, st->cs)) != FTK_OK) return s;
        long long oc2 = st->ocap[q];
        if ((s = grow(&st->ord_gi[q], oc2, need, q == st->cur ? st->n_ord : 0, st->cs)) != FTK_OK) return s;
        st->ocap[q] = oc;
    }
    return FTK_OK;
}

void release(ftk_stream *st) {
    if (!st) return;
    if (st->cs) cudaStreamSynchronize(st->cs);
    if (st->plan1) ftk_plan_destroy(st->plan1);
    if (st->plan2) ftk_plan_destroy(st->plan2);
    cudaFree(st->d2);
    cudaFree(st->gfid); cudaFree(st->gparent); cudaFree(st->gmin); cudaFree(st->gshadow); cudaFree(st->grec);
    for (int q = 0; q < 2; ++q) { cudaFree(st->ord_fid[q]); cudaFree(st->ord_gi[q]); }
    cudaFree(st->link_prev); cudaFree(st->old_root); cudaFree(st->delta);
    cudaFree(st->d_small); cudaFree(st->d_status);
    if (st->h_small) cudaFreeHost(st->h_small);
    if (st->h_status) cudaFreeHost(st->h_status);
    if (st->cs) cudaStreamDestroy(st->cs);
    if (st->server) {
        std::lock_guard<std::mutex> lock(st->server->mu);
        st->server->used -= std::min(st->server->used, st->footprint);
    }
    delete st;
}

size_t plan_bytes(const ftk_plan *pl) {
    const Workspace &W = pl->W;
    return (size_t)W.cap * (8 + 8 + 4 + 16 + 1 + 8 + sizeof(ftk_cp)) + (size_t)W.scap * (8 + 8 + 4) +
           (size_t)W.nseg * (4 + 8 + 8 + 4 + 8);
}

ftk_status open_stream(ftk_server *srv, int ndim, int64_t nx, int64_t ny, int64_t nz, const ftk_params *p,
                       ftk_stream **out) {
    if (out) *out = nullptr;
    if (!out) return fail(FTK_ERR_ARG, "out is NULL");
    if (ndim != 2 && ndim != 3) return fail(FTK_ERR_ARG, "ndim must be 2 or 3");
    if (ndim == 2) nz = 1;
    if (nx < 2 || ny < 2 || (ndim == 3 && nz < 2)) return fail(FTK_ERR_ARG, "every spatial extent must be >= 2");
    ftk_stream *st = new (std::nothrow) ftk_stream;
    if (!st) return fail(FTK_ERR_NOMEM, "host allocation failed");
    st->ndim = ndim;
    st->nx = (int)nx; st->ny = (int)ny; st->nz = (int)nz;
    if (p) st->p = *p;
    else ftk_params_default(&st->p);
    st->p.flags &= ~FTK_FLAG_STAGE_TIMES;
    st->slice_verts = (long long)nx * ny * nz;
    st->T = ndim == 2 ? 12 : 60;
    st->tbit = ndim == 2 ? 4 : 8;
    ftk_status s = FTK_OK;
    if ((s = plan_create(ndim, nx, ny, nz, 1, &st->p, nullptr, &st->plan1)) != FTK_OK ||
        (s = plan_create(ndim, nx, ny, nz, 2, &st->p, nullptr, &st->plan2)) != FTK_OK) {
        release(st);
        return s;
    }
    if (cudaStreamCreateWithFlags(&st->cs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMalloc(&st->d2, sizeof(float) * 2 * st->slice_verts) != cudaSuccess ||
        cudaMalloc(&st->d_small, sizeof(long long) * 2) != cudaSuccess ||
        cudaMalloc(&st->d_status, sizeof(unsigned)) != cudaSuccess ||
        cudaMallocHost(&st->h_small, sizeof(long long) * 2) != cudaSuccess ||
        cudaMallocHost(&st->h_status, sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        release(st);
        return fail(FTK_ERR_NOMEM, "stream allocation failed");
    }
    st->footprint = sizeof(float) * 2 * st->slice_verts + plan_bytes(st->plan1) + plan_bytes(st->plan2);
    if (srv) {
        std::lock_guard<std::mutex> lock(srv->mu);
        if (srv->used + st->footprint > srv->budget) {
            const std::string msg = "admission refused: the stream needs " + std::to_string(st->footprint) +
                                    " bytes of device memory beyond the budget";
            st->footprint = 0;
            st->server = nullptr;
            release(st);
            return fail(FTK_ERR_BUSY, msg);
        }
        srv->used += st->footprint;
        st->server = srv;
    }
    *out = st;
    return FTK_OK;
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
    return open_stream(nullptr, ndim, nx, ny, nz, p, s);
}

ftk_status ftk_stream_open_in(ftk_server *srv, int ndim, int64_t nx, int64_t ny, int64_t nz, const ftk_params *p,
                              ftk_stream **s) {
    if (!srv) return fail(FTK_ERR_ARG, "server is NULL");
    return open_stream(srv, ndim, nx, ny, nz, p, s);
}

ftk_status ftk_stream_push(ftk_stream *st, const float *slice, ftk_result **delta) {
    if (delta) *delta = nullptr;
    if (!st || !slice || !delta) return fail(FTK_ERR_ARG, "stream, slice and delta must be non-NULL");
    const size_t sbytes = sizeof(float) * (size_t)st->slice_verts;
    const cudaMemcpyKind kind = is_device_pointer(slice) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaError_t e;
    ftk_plan *pl = st->k == 0 ? st->plan1 : st->plan2;
    float *cur = st->k == 0 ? st->d2 : st->d2 + st->slice_verts;
    if (st->k >= 2) {
        e = cudaMemcpyAsync(st->d2, st->d2 + st->slice_verts, sbytes, cudaMemcpyDeviceToDevice, st->cs);
        if (e != cudaSuccess) return cuda_fail(e, "slice shift");
    }
    e = cudaMemcpyAsync(cur, slice, sbytes, kind, st->cs);
    if (e != cudaSuccess) return cuda_fail(e, "slice copy");
    ftk_status s = plan_launch(pl, st->d2, st->cs);
    if (s != FTK_OK) return s;
    int64_t P = 0;
    if ((s = ftk_plan_count(pl, &P)) != FTK_OK) return s;
    if ((s = ensure_global(st, st->n + P)) != FTK_OK) return s;
    if ((s = ensure_scratch(st, P)) != FTK_OK) return s;
    StreamMerge M;
    std::memset(&M, 0, sizeof(M));
    M.face = pl->W.face;
    M.label = pl->W.label;
    M.packed = pl->W.packed;
    M.ctr = pl->W.ctr;
    M.shift_t = st->k == 0 ? 0 : st->k - 1;
    M.shift_g = (long long)M.shift_t * st->slice_verts;
    M.first = st->k == 0 ? 1 : 0;
    M.slice_verts = st->slice_verts;
    M.T = st->T;
    M.tbit = st->tbit;
    M.n_base = st->n;
    M.gfid = st->gfid; M.gparent = st->gparent; M.gmin = st->gmin; M.gshadow = st->gshadow; M.grec = st->grec;
    M.ord_fid = st->ord_fid[st->cur];
    M.ord_gi = st->ord_gi[st->cur];
    M.n_ord = st->n_ord;
    M.link_prev = st->link_prev;
    M.old_root = st->old_root;
    M.delta = st->delta;
    M.delta_count = st->d_small;
    M.ord_fid_next = st->ord_fid[1 - st->cur];
    M.ord_gi_next = st->ord_gi[1 - st->cur];
    M.ord_count_next = st->d_small + 1;
    M.status = st->d_status;
    if ((e = cudaMemsetAsync(st->d_status, 0, sizeof(unsigned), st->cs)) != cudaSuccess) return cuda_fail(e, "status reset");
    if ((e = launch_stream_merge(M, st->cs)) != cudaSuccess) return cuda_fail(e, "stream merge launch");
    if ((e = cudaMemcpyAsync(st->h_small, st->d_small, sizeof(long long) * 2, cudaMemcpyDeviceToHost, st->cs)) != cudaSuccess ||
        (e = cudaMemcpyAsync(st->h_status, st->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, st->cs)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st->cs)) != cudaSuccess)
        return cuda_fail(e, "stream merge");
    if (*st->h_status & ST_TIMEOUT) return fail(FTK_ERR_TIMEOUT, "a bounded device loop gave up");
    if (*st->h_status & ST_PAIRING) return fail(FTK_ERR_INVARIANT, "a repeated face was not found in the previous push");
    const long long D = st->h_small[0];
    ftk_result *r = new (std::nothrow) ftk_result;
    if (!r) return fail(FTK_ERR_NOMEM, "host allocation failed");
    r->count = (size_t)D;
    r->data = (ftk_cp *)std::malloc(std::max<size_t>(1, (size_t)D) * sizeof(ftk_cp));
    if (!r->data) { delete r; return fail(FTK_ERR_NOMEM, "host allocation failed"); }
    if (D > 0 && (e = cudaMemcpy(r->data, st->delta, sizeof(ftk_cp) * D, cudaMemcpyDeviceToHost)) != cudaSuccess) {
        std::free(r->data);
        delete r;
        return cuda_fail(e, "delta download");
    }
    st->n += P;
    st->n_ord = (int)st->h_small[1];
    st->cur = 1 - st->cur;
    st->k += 1;
    *delta = r;
    return FTK_OK;
}

ftk_status ftk_stream_close(ftk_stream *st, ftk_result **final) {
    if (final) *final = nullptr;
    if (!st) return fail(FTK_ERR_ARG, "stream is NULL");
    ftk_status s = FTK_OK;
    if (final) {
        ftk_cp *d_out = nullptr;
        long long *d_cnt = nullptr;
        cudaError_t e = cudaSuccess;
        if (cudaMalloc(&d_out, sizeof(ftk_cp) * std::max<long long>(1, st->n)) != cudaSuccess ||
            cudaMalloc(&d_cnt, sizeof(long long)) != cudaSuccess) {
            cudaGetLastError();
            s = fail(FTK_ERR_NOMEM, "final result allocation failed");
        } else if ((e = cudaMemsetAsync(st->d_status, 0, sizeof(unsigned), st->cs)) != cudaSuccess ||
                   (e = launch_stream_final(st->n, st->gshadow, st->gparent, st->gmin, st->grec, d_out, d_cnt,
                                            st->d_status, st->cs)) != cudaSuccess ||
                   (e = cudaStreamSynchronize(st->cs)) != cudaSuccess) {
            s = cuda_fail(e, "final labels");
        } else {
            long long cnt = 0;
            cudaMemcpy(&cnt, d_cnt, sizeof(long long), cudaMemcpyDeviceToHost);
            ftk_result *r = new (std::nothrow) ftk_result;
            if (r) r->data = (ftk_cp *)std::malloc(std::max<size_t>(1, (size_t)cnt) * sizeof(ftk_cp));
            if (!r || !r->data) {
                delete r;
                cudaFree(d_out);
                cudaFree(d_cnt);
                release(st);
                return fail(FTK_ERR_NOMEM, "host allocation failed");
            }
            r->count = (size_t)cnt;
            if (cnt > 0) cudaMemcpy(r->data, d_out, sizeof(ftk_cp) * cnt, cudaMemcpyDeviceToHost);
            // pushes interleave in face-id order (interval faces of slab
            // [k-1, k] arrive one push after the ordinal faces of slice k-1)
            std::sort(r->data, r->data + r->count,
                      [](const ftk_cp &a, const ftk_cp &b) { return a.face_id < b.face_id; });
            *final = r;
        }
        cudaFree(d_out);
        cudaFree(d_cnt);
    }
    release(st);
    return s;
}

}  // extern "C"
