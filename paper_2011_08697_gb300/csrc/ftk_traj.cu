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
    cudaFree(T.toff); cudaFree(T.closed);
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
        cudaMalloc(&T.closed, sizeof(uint8_t) * c) != cudaSuccess) {
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
    long long *h_n = nullptr;
    if (cudaMallocHost(&h_n, sizeof(long long)) != cudaSuccess) {
        cudaGetLastError();
        return fail(FTK_ERR_NOMEM, "pinned allocation failed");
    }
    cudaError_t e = launch_trajectories(pl->ndim, pl->F, pl->W, P, pl->traj, st, h_n);
    const long long ntraj = *h_n;
    cudaFreeHost(h_n);
    if (e != cudaSuccess) return cuda_fail(e, "trajectory kernels");
    if ((e = launch_traj_walk(pl->W, P, ntraj, pl->traj, st)) != cudaSuccess) return cuda_fail(e, "trajectory walk");
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
        if (cudaMalloc(&cnt, sizeof(int) * (size_t)n) != cudaSuccess ||
            cudaMalloc(&soff, sizeof(long long) * (size_t)(n + 1)) != cudaSuccess) {
            cudaGetLastError();
            s = fail(FTK_ERR_NOMEM, "device allocation failed");
        } else if ((e = launch_traj_slice(pl->traj, n, t, cnt, soff, nullptr, st)) != cudaSuccess ||
                   (e = cudaMemcpyAsync(&total, soff + n, sizeof(long long), cudaMemcpyDeviceToHost, st)) !=
                       cudaSuccess ||
                   (e = cudaStreamSynchronize(st)) != cudaSuccess) {
            s = cuda_fail(e, "slice count");
        } else if (total > 0) {
            if (cudaMalloc(&d_pts, sizeof(ftk_slice_point) * (size_t)total) != cudaSuccess) {
                cudaGetLastError();
                s = fail(FTK_ERR_NOMEM, "device allocation failed");
            } else if ((e = launch_traj_slice(pl->traj, n, t, cnt, soff, d_pts, st)) != cudaSuccess ||
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
