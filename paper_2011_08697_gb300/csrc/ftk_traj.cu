// Trajectories as ordered polylines and their slices at a time t (paper
// Sec. 4.1: a critical-point trajectory is a PL curve in spacetime that can be
// sliced at t = t0; Sec. 3.2), host side of the C ABI.  The kernels are in
// ftk_kernels.cu next to the linking they build on.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>

#include "../../include/ftk.h"
#include "ftk_internal.h"
#include "ftk_kernels.cuh"

using namespace ftk;

struct ftk_traj {
    int64_t n;
    int64_t *off;      // [n + 1]
    ftk_cp *pts;       // [off[n]]
    uint8_t *closed;   // [n]
};

struct ftk_slice {
    int64_t n;
    ftk_slice_point *pts;
};

void ftk::free_traj(ftk_plan *pl) {
    TrajBuffers &T = pl->traj;
    cudaFree(T.nbr); cudaFree(T.root); cudaFree(T.size); cudaFree(T.start); cudaFree(T.rsize);
    cudaFree(T.isroot); cudaFree(T.off); cudaFree(T.tidx); cudaFree(T.order); cudaFree(T.rec);
    cudaFree(T.toff); cudaFree(T.closed); cudaFree(T.tpt); cudaFree(T.nb2); cudaFree(T.rk[0]); cudaFree(T.rk[1]);
    cudaFree(T.maxlen); cudaFree(T.scan);
    std::memset(&T, 0, sizeof(T));
    pl->traj_cap = 0;
    pl->traj_valid = false;
}

namespace {

ftk_status alloc_traj(ftk_plan *pl, long long P) {
    if (P <= pl->traj_cap && pl->traj.nbr) return FTK_OK;
    free_traj(pl);
    const long long c = std::max<long long>(P, 1024);
    TrajBuffers &T = pl->traj;
    if (cudaMalloc(&T.nbr, sizeof(int) * 2 * c) != cudaSuccess || cudaMalloc(&T.root, sizeof(int) * c) != cudaSuccess ||
        cudaMalloc(&T.size, sizeof(int) * c) != cudaSuccess || cudaMalloc(&T.start, sizeof(int) * c) != cudaSuccess ||
        cudaMalloc(&T.rsize, sizeof(int) * c) != cudaSuccess || cudaMalloc(&T.isroot, sizeof(int) * c) != cudaSuccess ||
        cudaMalloc(&T.off, sizeof(long long) * (c + 1)) != cudaSuccess ||
        cudaMalloc(&T.tidx, sizeof(long long) * (c + 1)) != cudaSuccess ||
        cudaMalloc(&T.order, sizeof(int) * c) != cudaSuccess || cudaMalloc(&T.rec, sizeof(ftk_cp) * c) != cudaSuccess ||
        cudaMalloc(&T.toff, sizeof(long long) * (c + 1)) != cudaSuccess ||
        cudaMalloc(&T.closed, sizeof(uint8_t) * c) != cudaSuccess || cudaMalloc(&T.tpt, sizeof(int) * c) != cudaSuccess ||
        cudaMalloc(&T.nb2, sizeof(int) * 2 * c) != cudaSuccess || cudaMalloc(&T.rk[0], sizeof(int4) * 2 * c) != cudaSuccess ||
        cudaMalloc(&T.rk[1], sizeof(int4) * 2 * c) != cudaSuccess || cudaMalloc(&T.maxlen, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&T.scan, sizeof(long long) * 1025) != cudaSuccess) {
        cudaGetLastError();
        free_traj(pl);
        return fail(FTK_ERR_NOMEM, "device allocation of the trajectory buffers failed");
    }
    pl->traj_cap = c;
    return FTK_OK;
}

// builds the trajectories of the plan's last execute on the device
ftk_status build_traj(ftk_plan *pl, long long *P_out) {
    int64_t P = 0;
    ftk_status s = ftk_plan_count(pl, &P);      // settles the run
    if (s != FTK_OK) return s;
    *P_out = P;
    if (pl->traj_valid) return FTK_OK;
    if (P > INT_MAX) return fail(FTK_ERR_RANGE, "too many punctures for the trajectory walk's 32-bit indices");
    if ((s = alloc_traj(pl, P)) != FTK_OK) return s;
    if (P == 0) {
        pl->traj_n = 0;
        pl->traj_valid = true;
        return FTK_OK;
    }
    cudaStream_t st = pl->stream;
    long long *h_n = nullptr;   // [0] trajectories, [1] points of the longest (as an int)
    if (cudaMallocHost(&h_n, 2 * sizeof(long long)) != cudaSuccess) {
        cudaGetLastError();
        return fail(FTK_ERR_NOMEM, "pinned allocation failed");
    }
    h_n[1] = 0;
    cudaError_t e = launch_trajectories(pl->ndim, pl->F, pl->W, P, pl->traj, st, h_n, reinterpret_cast<int *>(h_n + 1));
    const long long ntraj = h_n[0];
    const long long maxlen = *reinterpret_cast<int *>(h_n + 1);
    cudaFreeHost(h_n);
    if (e != cudaSuccess) return cuda_fail(e, "trajectory kernels");
    if ((e = launch_traj_walk(pl->W, P, ntraj, maxlen, pl->traj, st)) != cudaSuccess)
        return cuda_fail(e, "trajectory walk");
    unsigned status = 0;
    if ((e = cudaMemcpyAsync(&status, &pl->W.ctr->status, sizeof(unsigned), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_fail(e, "trajectory walk");
    if (status & ST_PAIRING) return fail(FTK_ERR_INVARIANT, "a trajectory is not a single path or loop");
    pl->traj_n = ntraj;
    pl->traj_valid = true;
    return FTK_OK;
}

}  // namespace

extern "C" {

ftk_status ftk_plan_trajectories(ftk_plan *pl, ftk_traj **out) {
    if (out) *out = nullptr;
    if (!pl || !out) return fail(FTK_ERR_ARG, "plan and out must be non-NULL");
    long long P = 0;
    ftk_status s = build_traj(pl, &P);
    if (s != FTK_OK) return s;
    const long long n = pl->traj_n;
    ftk_traj *tr = new (std::nothrow) ftk_traj;
    if (!tr) return fail(FTK_ERR_NOMEM, "host allocation failed");
    tr->n = n;
    tr->off = (int64_t *)std::malloc(sizeof(int64_t) * (size_t)(n + 1));
    tr->pts = (ftk_cp *)std::malloc(sizeof(ftk_cp) * (size_t)std::max<long long>(1, P));
    tr->closed = (uint8_t *)std::malloc((size_t)std::max<long long>(1, n));
    if (!tr->off || !tr->pts || !tr->closed) {
        ftk_traj_free(tr);
        return fail(FTK_ERR_NOMEM, "host allocation failed");
    }
    tr->off[0] = 0;
    if (n > 0) {
        cudaError_t e;
        if ((e = cudaMemcpy(tr->off, pl->traj.toff, sizeof(int64_t) * (size_t)(n + 1), cudaMemcpyDeviceToHost)) !=
                cudaSuccess ||
            (e = cudaMemcpy(tr->pts, pl->traj.rec, sizeof(ftk_cp) * (size_t)P, cudaMemcpyDeviceToHost)) != cudaSuccess ||
            (e = cudaMemcpy(tr->closed, pl->traj.closed, (size_t)n, cudaMemcpyDeviceToHost)) != cudaSuccess) {
            ftk_traj_free(tr);
            return cuda_fail(e, "trajectory download");
        }
    }
    *out = tr;
    return FTK_OK;
}

ftk_status ftk_plan_trajectories_filtered(ftk_plan *pl, const ftk_traj_filter *flt, ftk_traj **out) {
    if (out) *out = nullptr;
    if (!pl || !flt || !out) return fail(FTK_ERR_ARG, "plan, filter and out must be non-NULL");
    if (flt->smooth_half_window < 0 || flt->min_points < 0 || !(flt->min_duration == flt->min_duration))
        return fail(FTK_ERR_ARG, "invalid filter");
    long long P = 0;
    ftk_status s = build_traj(pl, &P);
    if (s != FTK_OK) return s;
    const long long n = pl->traj_n;
    ftk_traj *tr = new (std::nothrow) ftk_traj;
    if (!tr) return fail(FTK_ERR_NOMEM, "host allocation failed");
    tr->n = 0;
    tr->off = nullptr;
    tr->pts = nullptr;
    tr->closed = nullptr;
    int *ksize = nullptr, *kone = nullptr;
    unsigned long long *ext = nullptr;
    long long *noff = nullptr, *nidx = nullptr, *d_off = nullptr;
    ftk_cp *d_pts = nullptr;
    uint8_t *d_closed = nullptr;
    long long tot[2] = {0, 0};
    cudaError_t e = cudaSuccess;
    cudaStream_t st = pl->stream;
    const size_t nn = (size_t)std::max<long long>(1, n);
    if (cudaMalloc(&ksize, sizeof(int) * nn) != cudaSuccess || cudaMalloc(&kone, sizeof(int) * nn) != cudaSuccess ||
        cudaMalloc(&ext, sizeof(unsigned long long) * 2 * nn) != cudaSuccess ||
        cudaMalloc(&noff, sizeof(long long) * (nn + 1)) != cudaSuccess ||
        cudaMalloc(&nidx, sizeof(long long) * (nn + 1)) != cudaSuccess) {
        cudaGetLastError();
        s = fail(FTK_ERR_NOMEM, "device allocation failed");
    } else if (n > 0) {
        if ((e = launch_traj_filter(pl->traj, P, n, flt->min_duration, flt->min_points, flt->drop_loops,
                                    flt->smooth_half_window, ext, ksize, kone, noff, nidx, st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(&tot[0], noff + n, sizeof(long long), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(&tot[1], nidx + n, sizeof(long long), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess) {
            s = cuda_fail(e, "trajectory filter");
        } else if (cudaMalloc(&d_pts, sizeof(ftk_cp) * (size_t)std::max<long long>(1, tot[0])) != cudaSuccess ||
                   cudaMalloc(&d_off, sizeof(long long) * (size_t)(tot[1] + 1)) != cudaSuccess ||
                   cudaMalloc(&d_closed, (size_t)std::max<long long>(1, tot[1])) != cudaSuccess) {
            cudaGetLastError();
            s = fail(FTK_ERR_NOMEM, "device allocation failed");
        } else if ((e = launch_traj_compact(pl->traj, P, flt->smooth_half_window, noff, nidx, kone, d_pts, d_off,
                                            d_closed, st)) != cudaSuccess ||
                   (e = cudaStreamSynchronize(st)) != cudaSuccess) {
            s = cuda_fail(e, "trajectory compaction");
        }
    }
    if (s == FTK_OK) {
        const long long nk = tot[1], pk = tot[0];
        tr->n = nk;
        tr->off = (int64_t *)std::malloc(sizeof(int64_t) * (size_t)(nk + 1));
        tr->pts = (ftk_cp *)std::malloc(sizeof(ftk_cp) * (size_t)std::max<long long>(1, pk));
        tr->closed = (uint8_t *)std::malloc((size_t)std::max<long long>(1, nk));
        if (!tr->off || !tr->pts || !tr->closed) {
            s = fail(FTK_ERR_NOMEM, "host allocation failed");
        } else {
            tr->off[nk] = pk;
            if (nk > 0 &&
                ((e = cudaMemcpy(tr->off, d_off, sizeof(int64_t) * (size_t)nk, cudaMemcpyDeviceToHost)) != cudaSuccess ||
                 (e = cudaMemcpy(tr->pts, d_pts, sizeof(ftk_cp) * (size_t)pk, cudaMemcpyDeviceToHost)) != cudaSuccess ||
                 (e = cudaMemcpy(tr->closed, d_closed, (size_t)nk, cudaMemcpyDeviceToHost)) != cudaSuccess))
                s = cuda_fail(e, "filtered trajectory download");
        }
    }
    cudaFree(ksize); cudaFree(kone); cudaFree(ext); cudaFree(noff); cudaFree(nidx);
    cudaFree(d_pts); cudaFree(d_off); cudaFree(d_closed);
    if (s != FTK_OK) {
        ftk_traj_free(tr);
        return s;
    }
    *out = tr;
    return FTK_OK;
}

int64_t ftk_traj_count(const ftk_traj *tr) { return tr ? tr->n : 0; }
const int64_t *ftk_traj_offsets(const ftk_traj *tr) { return tr ? tr->off : nullptr; }
const ftk_cp *ftk_traj_points(const ftk_traj *tr) { return tr ? tr->pts : nullptr; }
const uint8_t *ftk_traj_closed(const ftk_traj *tr) { return tr ? tr->closed : nullptr; }
void ftk_traj_free(ftk_traj *tr) {
    if (!tr) return;
    std::free(tr->off);
    std::free(tr->pts);
    std::free(tr->closed);
    delete tr;
}

ftk_status ftk_plan_slice(ftk_plan *pl, double t, ftk_slice **out) {
    if (out) *out = nullptr;
    if (!pl || !out) return fail(FTK_ERR_ARG, "plan and out must be non-NULL");
    if (!(t == t)) return fail(FTK_ERR_ARG, "t is NaN");
    long long P = 0;
    ftk_status s = build_traj(pl, &P);
    if (s != FTK_OK) return s;
    const long long n = pl->traj_n;
    ftk_slice *sl = new (std::nothrow) ftk_slice;
    if (!sl) return fail(FTK_ERR_NOMEM, "host allocation failed");
    sl->n = 0;
    sl->pts = nullptr;
    long long total = 0;
    int *cnt = nullptr;
    long long *soff = nullptr;
    ftk_slice_point *d_pts = nullptr;
    cudaError_t e = cudaSuccess;
    cudaStream_t st = pl->stream;
    if (n > 0) {
        // one crossing flag per segment, named by its first point
        if (cudaMalloc(&cnt, sizeof(int) * (size_t)P) != cudaSuccess ||
            cudaMalloc(&soff, sizeof(long long) * (size_t)(P + 1)) != cudaSuccess) {
            cudaGetLastError();
            s = fail(FTK_ERR_NOMEM, "device allocation failed");
        } else if ((e = launch_traj_slice(pl->traj, P, t, cnt, soff, nullptr, st)) != cudaSuccess ||
                   (e = cudaMemcpyAsync(&total, soff + P, sizeof(long long), cudaMemcpyDeviceToHost, st)) !=
                       cudaSuccess ||
                   (e = cudaStreamSynchronize(st)) != cudaSuccess) {
            s = cuda_fail(e, "slice count");
        } else if (total > 0) {
            if (cudaMalloc(&d_pts, sizeof(ftk_slice_point) * (size_t)total) != cudaSuccess) {
                cudaGetLastError();
                s = fail(FTK_ERR_NOMEM, "device allocation failed");
            } else if ((e = launch_traj_slice(pl->traj, P, t, cnt, soff, d_pts, st)) != cudaSuccess ||
                       (e = cudaStreamSynchronize(st)) != cudaSuccess) {
                s = cuda_fail(e, "slice points");
            }
        }
    }
    if (s == FTK_OK) {
        sl->pts = (ftk_slice_point *)std::malloc(sizeof(ftk_slice_point) * (size_t)std::max<long long>(1, total));
        if (!sl->pts) s = fail(FTK_ERR_NOMEM, "host allocation failed");
        else if (total > 0 &&
                 (e = cudaMemcpy(sl->pts, d_pts, sizeof(ftk_slice_point) * (size_t)total, cudaMemcpyDeviceToHost)) !=
                     cudaSuccess)
            s = cuda_fail(e, "slice download");
        sl->n = total;
    }
    cudaFree(cnt);
    cudaFree(soff);
    cudaFree(d_pts);
    if (s != FTK_OK) {
        ftk_slice_free(sl);
        return s;
    }
    *out = sl;
    return FTK_OK;
}

int64_t ftk_slice_count(const ftk_slice *sl) { return sl ? sl->n : 0; }
const ftk_slice_point *ftk_slice_data(const ftk_slice *sl) { return sl ? sl->pts : nullptr; }
void ftk_slice_free(ftk_slice *sl) {
    if (!sl) return;
    std::free(sl->pts);
    delete sl;
}

}  // extern "C"
