// Host side of the C ABI declared in include/ftk.h: argument checking,
// blocking choice, device workspace (plans), result download, error codes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/ftk.h"
#include "ftk_kernels.cuh"
#include "ftk_internal.h"

using namespace ftk;

namespace {
thread_local std::string g_err;
}  // namespace

ftk_status ftk::fail(ftk_status s, const std::string &msg) {
    g_err = msg;
    return s;
}

ftk_status ftk::cuda_fail(cudaError_t e, const char *what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return FTK_ERR_CUDA;
}

namespace {

#define FTK_CUDA(call)                                   \
    do {                                                 \
        cudaError_t e__ = (call);                        \
        if (e__ != cudaSuccess) return cuda_fail(e__, #call); \
    } while (0)

constexpr size_t kSmemBudget = 110 * 1024;   // two detect CTAs per SM

}  // namespace

bool ftk::is_device_pointer(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void ftk::set_last_error(const char *msg) { g_err = msg ? msg : ""; }

namespace {

void free_workspace(Workspace &W) {
    cudaFree(W.ctr);
    cudaFree(W.seg_cnt);
    cudaFree(W.seg_stage);
    cudaFree(W.seg_off);
    cudaFree(W.staging);
    cudaFree(W.face);
    cudaFree(W.parent);
    cudaFree(W.off);
    cudaFree(W.morse);
    cudaFree(W.label);
    cudaFree(W.packed);
    cudaFree(W.surv);
    cudaFree(W.surv_mask);
    cudaFree(W.surv_off);
    cudaFree(W.litem);
    cudaFree(W.seg_scnt);
    cudaFree(W.seg_sstage);
    cudaFree(W.tile);
    cudaFree(W.seg_tile);
    std::memset(&W, 0, sizeof(W));
}

ftk_status alloc_survivors(Workspace &W, long long scap) {
    cudaFree(W.surv); W.surv = nullptr;
    cudaFree(W.surv_mask); W.surv_mask = nullptr;
    cudaFree(W.surv_off); W.surv_off = nullptr;
    cudaFree(W.litem); W.litem = nullptr;
    cudaFree(W.tile); W.tile = nullptr;
    W.scap = 0;
    const long long ntile = (scap + LB_TILE - 1) / LB_TILE;
    if (cudaMalloc(&W.surv, scap * sizeof(long long)) != cudaSuccess ||
        cudaMalloc(&W.surv_mask, scap * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&W.surv_off, scap * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&W.litem, 3 * scap * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&W.tile, ntile * sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        return fail(FTK_ERR_NOMEM, "device allocation of the survivor arrays failed");
    }
    W.scap = scap;
    return FTK_OK;
}

ftk_status alloc_capacity(Workspace &W, long long cap) {
    cudaFree(W.staging); W.staging = nullptr;
    cudaFree(W.face); W.face = nullptr;
    cudaFree(W.parent); W.parent = nullptr;
    cudaFree(W.off); W.off = nullptr;
    cudaFree(W.morse); W.morse = nullptr;
    cudaFree(W.label); W.label = nullptr;
    cudaFree(W.packed); W.packed = nullptr;
    W.cap = 0;
    if (cudaMalloc(&W.staging, cap * sizeof(long long)) != cudaSuccess ||
        cudaMalloc(&W.face, cap * sizeof(long long)) != cudaSuccess ||
        cudaMalloc(&W.parent, cap * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&W.off, cap * sizeof(float4)) != cudaSuccess ||
        cudaMalloc(&W.morse, cap * sizeof(int8_t)) != cudaSuccess ||
        cudaMalloc(&W.label, cap * sizeof(long long)) != cudaSuccess ||
        cudaMalloc(&W.packed, cap * sizeof(ftk_cp)) != cudaSuccess) {
        cudaGetLastError();
        return fail(FTK_ERR_NOMEM, "device allocation of the puncture arrays failed");
    }
    W.cap = cap;
    return FTK_OK;
}

int sm_count() {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 148;
}

// time chunks: split each spatial block's time range so that the units fill
// whole waves of resident CTAs as closely as possible
void choose_time_chunks(const Field &F, Blocking &B, long long spatial, long long wave) {
    long long best_ntc = 1;
    double best = -1.0;
    for (long long k = 1; k <= 6; ++k) {
        long long ntc = std::max<long long>(1, (k * wave) / std::max<long long>(1, spatial));
        ntc = std::min<long long>(ntc, F.nt);
        const int tc = (int)((F.nt + ntc - 1) / ntc);
        ntc = (F.nt + tc - 1) / tc;
        const long long units = ntc * spatial;
        const double waves = (double)units / (double)wave;
        const double fill = waves / std::ceil(waves);        // occupancy of the last wave
        const double over = 1.0 / tc;                         // re-read slice per chunk
        const double score = fill - over;
        if (score > best) { best = score; best_ntc = ntc; }
    }
    B.tc = (int)((F.nt + best_ntc - 1) / best_ntc);
    B.ntc = (F.nt + B.tc - 1) / B.tc;
}

// row pitch of the field the kernels read: the width rounded up to 4 floats
// when a streaming kernel takes the shape, else the width itself (the tiled
// kernel reads any width in place)
int stream_pitch(int ndim, int nx) {
    const int p = (nx + 3) & ~3;
    return p <= (ndim == 2 ? STREAM2_MAX_NX : STREAM3_MAX_NX) ? p : nx;
}

ftk_status choose_blocking(int ndim, const Field &F, Blocking &B, int &variant) {
    static const int cand2[] = {16, 8, 4, 2, 1};
    static const int cand3[][2] = {{8, 4}, {8, 2}, {4, 4}, {4, 2}, {2, 2}, {2, 1}, {1, 1}};
    const int sms = sm_count();
    B.nxb = 1;
    B.wx = F.nx;
    // the streaming kernels read rows padded to a multiple of 4 floats
    // (F.pitch, chosen by stream_pitch)
    if (ndim == 2 && F.pitch % 4 == 0 && F.pitch <= (F.comps == 2 ? STREAM2_VEC_MAX_NX : STREAM2_MAX_NX)) {
        variant = VAR_STREAM2;
        B.ry = STREAM2_ROWS; B.rz = 1;
        B.nyb = (F.ny + B.ry - 1) / B.ry;
        B.nzb = 1;
        choose_time_chunks(F, B, B.nyb, (long long)sms * stream2_ctas_per_sm(F.pitch, F.comps));
        return FTK_OK;
    }
    if (ndim == 3 && F.pitch % 4 == 0 && F.pitch <= STREAM3_MAX_NX) {
        variant = VAR_STREAM3;
        // the kernel's consumer warps fix the rows per unit; two cube planes
        // per unit measured fastest on 128^3 x 16 (against 4 and 8: more,
        // shorter units balance better than they lose to the z halo)
        B.ry = stream3_ry(F.pitch);
        B.rz = std::min(2, F.nz);
        B.nyb = (F.ny + B.ry - 1) / B.ry;
        B.nzb = (F.nz + B.rz - 1) / B.rz;
        choose_time_chunks(F, B, (long long)B.nyb * B.nzb, (long long)sms * stream3_ctas_per_sm(F.pitch, B));
        return FTK_OK;
    }
    variant = VAR_TILE;
    bool ok = false;
    if (ndim == 2) {
        for (int ry : cand2) {
            B.ry = ry; B.rz = 1;
            if (detect_smem_bytes(2, F, B) <= kSmemBudget) { ok = true; break; }
        }
    } else {
        for (auto &c : cand3) {
            B.ry = c[0]; B.rz = c[1];
            if (detect_smem_bytes(3, F, B) <= kSmemBudget) { ok = true; break; }
        }
    }
    if (!ok) {
        // rows too wide for one tile: one row (and plane) per unit, the row
        // cut into windows of wx cube columns, the widest multiple of 32
        // that fits; segments become (t, z, y, window), still in face-id order
        B.ry = 1; B.rz = 1;
        B.nxb = 2;
        B.wx = std::min(F.nx, 1 << 16) & ~31;
        while (B.wx >= 32 && detect_smem_bytes(ndim, F, B) > kSmemBudget) B.wx -= 32;
        if (B.wx < 32) return fail(FTK_ERR_ARG, "no x window of the detect tile fits shared memory");
        B.nxb = (F.nx + B.wx - 1) / B.wx;
    }
    B.nyb = (F.ny + B.ry - 1) / B.ry;
    B.nzb = ndim == 3 ? (F.nz + B.rz - 1) / B.rz : 1;
    // enough units to fill the GPU: split time into chunks if the spatial
    // blocks alone are too few
    const long long spatial = (long long)B.nyb * B.nzb * B.nxb;
    const long long want = 4LL * sms;
    long long chunks = spatial >= want ? 1 : (want + spatial - 1) / spatial;
    chunks = std::min<long long>(chunks, F.nt);
    B.tc = (int)((F.nt + chunks - 1) / chunks);
    B.ntc = (F.nt + B.tc - 1) / B.tc;
    return FTK_OK;
}

ftk_status check_params(const ftk_params *p) {
    if (p && (p->quant_shift < 0 || p->quant_shift > 40))
        return fail(FTK_ERR_ARG, "quant_shift must lie in [0, 40]");
    if (p && p->flags & ~(FTK_FLAG_STAGE_TIMES | FTK_FLAG_AUTOTUNE)) return fail(FTK_ERR_ARG, "unknown flag bits");
    if (p && p->max_punctures < 0) return fail(FTK_ERR_ARG, "max_punctures must be >= 0");
    return FTK_OK;
}

ftk_status read_counters(ftk_plan *pl) {
    FTK_CUDA(cudaStreamSynchronize(pl->stream));
    FTK_CUDA(cudaMemcpy(pl->h_ctr, pl->W.ctr, sizeof(RunCounters), cudaMemcpyDeviceToHost));
    return FTK_OK;
}

ftk_status status_of(unsigned st) {
    if (st & ST_RANGE) return fail(FTK_ERR_RANGE, "a sample is non-finite or |f * 2^quant_shift| exceeds 2^28");
    if (st & ST_TIMEOUT) return fail(FTK_ERR_TIMEOUT, "a bounded device loop gave up");
    if (st & ST_PAIRING) return fail(FTK_ERR_INVARIANT, "a spacetime cell had other than 0 or 2 punctured sides");
    return FTK_OK;
}

ftk_status launch(ftk_plan *pl, const float *dev_f, cudaStream_t s, int variant) {
    pl->F.f = dev_f;
    pl->traj_valid = false;
    cudaError_t e = launch_pipeline(pl->ndim, variant, pl->F, pl->B, pl->W, s, pl->timing ? pl->ev : nullptr);
    if (e != cudaSuccess) return cuda_fail(e, (std::string("pipeline launch (") + last_launch_stage() + ")").c_str());
    pl->stream = s;
    pl->executed = true;
    return FTK_OK;
}

// grow and re-run on overflow (synchronously), check device status; the
// counters of the last run are in pl->h_ctr when have_counters is set
ftk_status settle_from(ftk_plan *pl, bool have_counters) {
    if (!pl->executed) return fail(FTK_ERR_STATE, "plan has not been executed");
    int variant = pl->variant;
    for (int attempt = 0; attempt < 6; ++attempt) {
        ftk_status s = FTK_OK;
        if (!have_counters || attempt > 0) {
            s = read_counters(pl);
            if (s != FTK_OK) return s;
        }
        const unsigned st = pl->h_ctr->status;
        if (st & ST_RANGE) return status_of(st);
        if (st & ST_WIDE) {
            // a sample beyond the fast rounding range: redo with exact rounding
            variant = exact_variant(pl->variant);
            s = launch(pl, pl->last_dev, pl->stream, variant);
            if (s != FTK_OK) return s;
            continue;
        }
        if (!(st & (ST_OVERFLOW | ST_SOVERFLOW))) {
            if (pl->timing) {
                pl->nstage = 5;
                for (int i = 0; i < 5; ++i) cudaEventElapsedTime(&pl->stage_ms[i], pl->ev[i], pl->ev[i + 1]);
            }
            return status_of(st);
        }
        if (st & ST_SOVERFLOW) {
            const long long need = (long long)pl->h_ctr->survivors;
            s = alloc_survivors(pl->W, std::max<long long>(need + need / 4 + 1024, 2 * pl->W.scap));
            if (s != FTK_OK) return s;
        } else {
            const long long need = (long long)pl->h_ctr->staged;
            s = alloc_capacity(pl->W, std::max<long long>(need + need / 4 + 1024, 2 * pl->W.cap));
            if (s != FTK_OK) return s;
        }
        s = launch(pl, pl->last_dev, pl->stream, variant);
        if (s != FTK_OK) return s;
    }
    return fail(FTK_ERR_NOMEM, "puncture capacity did not converge");
}

ftk_status settle(ftk_plan *pl) { return settle_from(pl, false); }

ftk_status make_result(ftk_plan *pl, ftk_result **out) {
    const long long P = pl->h_ctr->punctures;
    ftk_result *r = new (std::nothrow) ftk_result;
    if (!r) return fail(FTK_ERR_NOMEM, "host allocation failed");
    r->count = (size_t)P;
    r->data = (ftk_cp *)std::malloc(std::max<size_t>(1, (size_t)P) * sizeof(ftk_cp));
    if (!r->data) {
        delete r;
        return fail(FTK_ERR_NOMEM, "host allocation failed");
    }
    if (P > 0) {
        cudaError_t e = cudaMemcpy(r->data, pl->W.packed, (size_t)P * sizeof(ftk_cp), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            std::free(r->data);
            delete r;
            return cuda_fail(e, "result download");
        }
    }
    *out = r;
    return FTK_OK;
}

// ---------------------------------------------------------------------------
// Autotuner: measured time chunking per (shape, variant, SM count)
// ---------------------------------------------------------------------------
struct TuneKey {
    int ndim, comps, nx, ny, nz, nt, variant, sms;
    bool operator<(const TuneKey &o) const {
        return std::tie(ndim, comps, nx, ny, nz, nt, variant, sms) <
               std::tie(o.ndim, o.comps, o.nx, o.ny, o.nz, o.nt, o.variant, o.sms);
    }
};
std::mutex g_tune_mu;
// a tuned launch shape: time chunks, and (3D streaming) cube planes per unit
struct Tuned {
    int ntc;
    int rz;
};
std::map<TuneKey, Tuned> g_tuned;

TuneKey tune_key(const ftk_plan *pl) {
    return TuneKey{pl->ndim, pl->F.comps, pl->F.nx, pl->F.ny, pl->F.nz, pl->F.nt, pl->variant, sm_count()};
}

void set_chunks(ftk_plan *pl, int ntc) {
    pl->B.tc = (pl->F.nt + ntc - 1) / ntc;
    pl->B.ntc = (pl->F.nt + pl->B.tc - 1) / pl->B.tc;
}

// cube planes per unit (segments are per z plane, so nothing else changes)
void set_rz(ftk_plan *pl, int rz) {
    pl->B.rz = std::max(1, std::min(rz, pl->F.nz));
    pl->B.nzb = (pl->F.nz + pl->B.rz - 1) / pl->B.rz;
}

void set_tuned(ftk_plan *pl, const Tuned &t) {
    if (pl->ndim == 3 && pl->variant != VAR_TILE) set_rz(pl, t.rz);
    set_chunks(pl, t.ntc);
}

void apply_tuned(ftk_plan *pl) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tuned.find(tune_key(pl));
    if (it != g_tuned.end()) set_tuned(pl, it->second);
}

}  // namespace

// the device field the kernels read: f itself when they can read it in
// place, else the plan's own copy (host input, a padded row pitch, or a
// start that is not 16-byte aligned for the bulk copies), queued on s
ftk_status ftk::plan_source(ftk_plan *pl, const float *f, bool host, cudaStream_t s, const float **src) {
    const Field &F = pl->F;
    const long long rows = (long long)F.nt * F.nz * F.ny;
    const bool padded = F.pitch != F.nx;
    const bool misaligned = pl->variant != VAR_TILE && ((uintptr_t)f & 15u) != 0;
    *src = f;
    if (!host && !padded && !misaligned) return FTK_OK;
    const size_t bytes = (size_t)rows * F.pitch * sizeof(float) * (F.comps == 2 ? 2 : 1);
    if (!pl->d_input && cudaMalloc(&pl->d_input, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(FTK_ERR_NOMEM, "device input buffer allocation failed");
    }
    cudaError_t e;
    if (!padded) {
        e = cudaMemcpyAsync(pl->d_input, f, bytes, host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s);
    } else if (host) {
        e = cudaMemcpy2DAsync(pl->d_input, (size_t)F.pitch * 4, f, (size_t)F.nx * 4, (size_t)F.nx * 4, (size_t)rows,
                              cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = launch_fill_pad(pl->d_input, F.nx, F.pitch, rows, s);
    } else {
        e = launch_pad_rows(f, pl->d_input, F.nx, F.pitch, rows, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "input copy");
    *src = pl->d_input;
    return FTK_OK;
}

ftk_status ftk::plan_launch(ftk_plan *pl, const float *f, cudaStream_t s) {
    pl->last_f = f;
    pl->last_dev = f;
    pl->last_host = false;
    return launch(pl, f, s, pl->variant);
}

ftk_status ftk::plan_check(ftk_plan *pl) { return settle_from(pl, true); }

ftk_status ftk::plan_result(ftk_plan *pl, ftk_result **out) { return make_result(pl, out); }

ftk_status ftk::plan_autotune(ftk_plan *pl, const float *f, cudaStream_t s) {
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tuned.find(tune_key(pl));
        if (it != g_tuned.end()) {
            set_tuned(pl, it->second);
            return FTK_OK;
        }
    }
    // candidates: the heuristic time chunking and powers of two around it;
    // for the 3D streaming kernel also 2, 4 and 8 cube planes per unit (each
    // with the chunkings that give about one and two waves)
    const int heur = pl->B.ntc;
    const int rz0 = pl->B.rz;
    std::vector<Tuned> cand = {{heur, rz0}};
    for (int c = 1; c <= pl->F.nt; c *= 2)
        if (c != heur && c <= 4 * heur + 4 && 4 * c + 4 >= heur) cand.push_back({c, rz0});
    if (pl->ndim == 3 && pl->variant != VAR_TILE) {
        for (int rz : {2, 4, 8}) {
            if (rz == rz0 || rz > pl->F.nz) continue;
            for (int c = 1; c <= pl->F.nt && c <= 8; c *= 2) cand.push_back({c, rz});
        }
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    Tuned bt = cand[0];
    for (const Tuned &c : cand) {
        set_tuned(pl, c);
        float tot = 0.0f;
        for (int rep = 0; rep < 3; ++rep) {
            ftk_status st = launch(pl, f, s, pl->variant);      // first run warms up
            if (st != FTK_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); return st; }
            if (rep == 0) continue;
            cudaEventRecord(e0, s);
            st = launch(pl, f, s, pl->variant);
            cudaEventRecord(e1, s);
            if (st != FTK_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); return st; }
            cudaEventSynchronize(e1);
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            tot += ms;
        }
        if (tot < best) { best = tot; bt = c; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    set_tuned(pl, bt);
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tuned[tune_key(pl)] = bt;
    return FTK_OK;
}

extern "C" {

void ftk_params_default(ftk_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    for (int a = 0; a < 3; ++a) p->spacing[a] = 1.0;
    p->dt = 1.0;
    p->quant_shift = 20;
}

const char *ftk_status_string(ftk_status s) {
    switch (s) {
        case FTK_OK: return "ok";
        case FTK_ERR_ARG: return "invalid argument";
        case FTK_ERR_RANGE: return "sample out of fixed-point range";
        case FTK_ERR_NOMEM: return "out of memory";
        case FTK_ERR_CUDA: return "CUDA error";
        case FTK_ERR_TIMEOUT: return "device wait timed out";
        case FTK_ERR_BUSY: return "admission refused";
        case FTK_ERR_INVARIANT: return "pairing invariant violated";
        case FTK_ERR_STATE: return "invalid state";
    }
    return "unknown status";
}

const char *ftk_last_error(void) { return g_err.c_str(); }

const char *ftk_version(void) { return "ftk-gb300 0.1 sm_103a"; }

ftk_status ftk_debug_set_wait_limits(int64_t uf_steps, int64_t lookback_cycles) {
    const cudaError_t e = set_wait_limits(uf_steps, lookback_cycles);
    if (e != cudaSuccess) return cuda_fail(e, "setting the wait limits");
    return FTK_OK;
}

}  // extern "C"

// initial puncture and survivor capacities of a plan (grow on demand); the
// compact form (in-situ stream slabs, which are small and many) starts
// smaller, so that the grid-stride kernels sized by the capacities launch
// few blocks
static long long initial_cap(const ftk_params &p, long long nverts, bool compact = false) {
    if (p.max_punctures > 0) return p.max_punctures;
    return compact ? std::max<long long>(1 << 12, std::min<long long>(nverts / 128, 1LL << 26))
                   : std::max<long long>(1 << 16, std::min<long long>(nverts / 32, 1LL << 26));
}
static long long initial_scap(long long nverts, bool compact = false) {
    return compact ? std::max<long long>(1 << 12, std::min<long long>(nverts / 64, 1LL << 26))
                   : std::max<long long>(1 << 16, std::min<long long>(nverts / 32, 1LL << 26));
}

ftk_status ftk::plan_sizes(int ndim, int64_t nx, int64_t ny, int64_t nz, int64_t nt, const ftk_params *p,
                           PlanSizes *out, bool compact) {
    if (ndim != 2 && ndim != 3) return fail(FTK_ERR_ARG, "ndim must be 2 or 3");
    if (ndim == 2) nz = 1;
    if (nx < 2 || ny < 2 || (ndim == 3 && nz < 2) || nt < 1)
        return fail(FTK_ERR_ARG, "every spatial extent must be >= 2 and nt >= 1");
    if (nx > (1 << 30) || ny > (1 << 30) || nz > (1 << 30) || nt > (1 << 30))
        return fail(FTK_ERR_ARG, "extent too large");
    ftk_status s = check_params(p);
    if (s != FTK_OK) return s;
    ftk_params prm;
    if (p) prm = *p;
    else ftk_params_default(&prm);
    std::memset(out, 0, sizeof(*out));
    out->F.nx = (int)nx; out->F.ny = (int)ny; out->F.nz = (int)nz; out->F.nt = (int)nt;
    out->F.pitch = stream_pitch(ndim, (int)nx);
    s = choose_blocking(ndim, out->F, out->B, out->variant);
    if (s != FTK_OK) return s;
    const long long nverts = (long long)nx * ny * nz * nt;
    out->nseg = segment_count(out->F, out->B);
    out->cap = initial_cap(prm, nverts, compact);
    out->scap = out->variant != VAR_TILE ? initial_scap(nverts, compact) : 0;
    return FTK_OK;
}

ftk_status ftk::plan_create(int ndim, int64_t nx, int64_t ny, int64_t nz, int64_t nt, const ftk_params *p,
                            RunCounters *ctr, ftk_plan **plan, bool compact, int comps) {
    if (plan) *plan = nullptr;
    if (!plan) return fail(FTK_ERR_ARG, "plan is NULL");
    if (ndim != 2 && ndim != 3) return fail(FTK_ERR_ARG, "ndim must be 2 or 3");
    if (ndim == 2) nz = 1;
    if (nx < 2 || ny < 2 || (ndim == 3 && nz < 2) || nt < 1)
        return fail(FTK_ERR_ARG, "every spatial extent must be >= 2 and nt >= 1");
    if (nx > (1 << 30) || ny > (1 << 30) || nz > (1 << 30) || nt > (1 << 30))
        return fail(FTK_ERR_ARG, "extent too large");
    const long long T = ndim == 2 ? 12 : 60;
    const double nv = (double)nx * ny * nz * nt;
    if (nv * T > 9.0e18) return fail(FTK_ERR_ARG, "face ids would overflow int64");
    ftk_status s = check_params(p);
    if (s != FTK_OK) return s;

    ftk_plan *pl = new (std::nothrow) ftk_plan;
    if (!pl) return fail(FTK_ERR_NOMEM, "host allocation failed");
    std::memset(pl, 0, sizeof(*pl));
    if (p) pl->p = *p;
    else ftk_params_default(&pl->p);
    pl->ndim = ndim;
    cudaGetDevice(&pl->device);
    pl->F.nx = (int)nx; pl->F.ny = (int)ny; pl->F.nz = (int)nz; pl->F.nt = (int)nt;
    pl->F.comps = comps == 2 ? 2 : 1;
    pl->F.pitch = pl->F.comps == 2 ? (int)nx : stream_pitch(ndim, (int)nx);
    pl->F.scale = (float)std::ldexp(1.0, pl->p.quant_shift);
    field_divisors(pl->F);
    pl->nverts = (long long)nx * ny * nz * nt;
    s = choose_blocking(ndim, pl->F, pl->B, pl->variant);
    if (s != FTK_OK) { delete pl; return s; }
    pl->W.nseg = segment_count(pl->F, pl->B);   // segments (t, z, y-block[, x-window])
    pl->timing = (pl->p.flags & 1u) != 0;

    Workspace &W = pl->W;
    pl->external_ctr = ctr != nullptr;
    if (ctr) W.ctr = ctr;
    if ((!ctr && cudaMalloc(&W.ctr, sizeof(RunCounters)) != cudaSuccess) ||
        cudaMalloc(&W.seg_cnt, W.nseg * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&W.seg_stage, W.nseg * sizeof(long long)) != cudaSuccess ||
        cudaMalloc(&W.seg_off, W.nseg * sizeof(long long)) != cudaSuccess ||
        cudaMallocHost(&pl->h_ctr, sizeof(RunCounters)) != cudaSuccess) {
        cudaGetLastError();
        if (pl->external_ctr) W.ctr = nullptr;
        free_workspace(W);
        if (pl->h_ctr) cudaFreeHost(pl->h_ctr);
        delete pl;
        return fail(FTK_ERR_NOMEM, "device allocation failed");
    }
    s = alloc_capacity(W, initial_cap(pl->p, pl->nverts, compact));
    if (s == FTK_OK && pl->variant != VAR_TILE) {
        const long long nst = (W.nseg + SEG_TILE - 1) / SEG_TILE;
        if (cudaMalloc(&W.seg_scnt, W.nseg * sizeof(int)) != cudaSuccess ||
            cudaMalloc(&W.seg_sstage, W.nseg * sizeof(long long)) != cudaSuccess ||
            cudaMalloc(&W.seg_tile, nst * sizeof(unsigned long long)) != cudaSuccess) {
            cudaGetLastError();
            s = fail(FTK_ERR_NOMEM, "device allocation failed");
        } else {
            s = alloc_survivors(W, initial_scap(pl->nverts, compact));
        }
    }
    if (s != FTK_OK) {
        if (pl->external_ctr) W.ctr = nullptr;
        free_workspace(W);
        cudaFreeHost(pl->h_ctr);
        delete pl;
        return s;
    }
    apply_tuned(pl);
    if (pl->timing)
        for (int i = 0; i < 6; ++i) cudaEventCreate(&pl->ev[i]);
    *plan = pl;
    return FTK_OK;
}

extern "C" {

ftk_status ftk_plan_create(int ndim, int64_t nx, int64_t ny, int64_t nz, int64_t nt,
                           const ftk_params *p, ftk_plan **plan) {
    return plan_create(ndim, nx, ny, nz, nt, p, nullptr, plan);
}

ftk_status ftk_plan_execute(ftk_plan *pl, const float *f, void *cuda_stream) {
    if (!pl || !f) return fail(FTK_ERR_ARG, "plan and field must be non-NULL");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const bool host = !is_device_pointer(f);
    const float *src = f;
    ftk_status st = ftk::plan_source(pl, f, host, s, &src);
    if (st != FTK_OK) return st;
    pl->last_f = f;
    pl->last_dev = src;
    pl->last_host = host;
    if ((pl->p.flags & FTK_FLAG_AUTOTUNE) && !pl->tuned) {
        // first execute of an autotuned plan: measure the candidate launch
        // shapes on this field (the result is cached per shape)
        st = ftk::plan_autotune(pl, src, s);
        if (st != FTK_OK) return st;
        pl->tuned = true;
    }
    cudaEvent_t copied = nullptr;
    if (host) {
        // the host buffer may be reused as soon as this call returns: wait for
        // the copy (not for the pipeline queued behind it)
        if (!pl->copy_ev) {
            cudaError_t e = cudaEventCreateWithFlags(&pl->copy_ev, cudaEventDisableTiming);
            if (e != cudaSuccess) return cuda_fail(e, "event creation");
        }
        copied = pl->copy_ev;
        cudaError_t e = cudaEventRecord(copied, s);
        if (e != cudaSuccess) return cuda_fail(e, "event record");
    }
    st = launch(pl, src, s, pl->variant);
    if (copied) {
        cudaError_t e = cudaEventSynchronize(copied);
        if (e != cudaSuccess && st == FTK_OK) st = cuda_fail(e, "input copy");
    }
    return st;
}

ftk_status ftk_plan_count(ftk_plan *pl, int64_t *count) {
    if (!pl || !count) return fail(FTK_ERR_ARG, "plan and count must be non-NULL");
    ftk_status s = settle(pl);
    if (s != FTK_OK) return s;
    *count = pl->h_ctr->punctures;
    return FTK_OK;
}

ftk_status ftk_plan_download(ftk_plan *pl, ftk_result **out) {
    if (out) *out = nullptr;
    if (!pl || !out) return fail(FTK_ERR_ARG, "plan and out must be non-NULL");
    ftk_status s = settle(pl);
    if (s != FTK_OK) return s;
    return make_result(pl, out);
}

ftk_status ftk_plan_download_into(ftk_plan *pl, ftk_cp *dst, int64_t cap, int64_t *count) {
    if (!pl || !count || (cap > 0 && !dst) || cap < 0) return fail(FTK_ERR_ARG, "invalid argument");
    *count = 0;
    ftk_status s = settle(pl);
    if (s != FTK_OK) return s;
    const long long P = pl->h_ctr->punctures;
    *count = P;
    if (P > cap) return fail(FTK_ERR_NOMEM, "the output buffer holds fewer records than there are punctures");
    if (P > 0) {
        cudaError_t e = cudaMemcpyAsync(dst, pl->W.packed, (size_t)P * sizeof(ftk_cp), cudaMemcpyDeviceToHost, pl->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(pl->stream);
        if (e != cudaSuccess) return cuda_fail(e, "result download");
    }
    return FTK_OK;
}

ftk_status ftk_plan_device_view(ftk_plan *pl, ftk_device_view *v) {
    if (!pl || !v) return fail(FTK_ERR_ARG, "plan and view must be non-NULL");
    ftk_status s = settle(pl);
    if (s != FTK_OK) return s;
    v->count = pl->h_ctr->punctures;
    v->face_id = (const int64_t *)pl->W.face;
    v->label = (const int64_t *)pl->W.label;
    v->off = (const float *)pl->W.off;
    v->morse = pl->W.morse;
    return FTK_OK;
}

ftk_status ftk_plan_stage_times(ftk_plan *pl, float *ms, int cap, int *n) {
    if (!pl || !ms || !n) return fail(FTK_ERR_ARG, "NULL argument");
    if (!pl->timing) return fail(FTK_ERR_STATE, "plan created without the stage-timing flag");
    *n = std::min(cap, pl->nstage);
    for (int i = 0; i < *n; ++i) ms[i] = pl->stage_ms[i];
    return FTK_OK;
}

ftk_status ftk_plan_describe(ftk_plan *pl, ftk_plan_desc *d) {
    if (!pl || !d) return fail(FTK_ERR_ARG, "NULL argument");
    std::memset(d, 0, sizeof(*d));
    d->detect_variant = pl->variant;
    d->kernels_per_execute = pl->variant == VAR_TILE ? 5 : pl->ndim == 3 ? 9 : 8;
    d->rows_per_unit = pl->B.ry;
    d->slices_per_unit = pl->B.tc;
    d->detect_units = (int64_t)pl->B.ntc * pl->B.nyb * pl->B.nzb * std::max(1, pl->B.nxb);
    d->capacity = pl->W.cap;
    return FTK_OK;
}

ftk_status ftk_plan_destroy(ftk_plan *pl) {
    if (!pl) return FTK_OK;
    if (pl->executed) cudaStreamSynchronize(pl->stream);
    if (pl->external_ctr) pl->W.ctr = nullptr;
    free_workspace(pl->W);
    cudaFree(pl->d_input);
    if (pl->h_ctr) cudaFreeHost(pl->h_ctr);
    if (pl->timing)
        for (int i = 0; i < 6; ++i) cudaEventDestroy(pl->ev[i]);
    if (pl->copy_ev) cudaEventDestroy(pl->copy_ev);
    free_traj(pl);
    delete pl;
    return FTK_OK;
}

static ftk_status track_once(int ndim, const float *f, int64_t nx, int64_t ny, int64_t nz, int64_t nt,
                             const ftk_params *p, ftk_result **out, void *stream, int comps = 1) {
    if (out) *out = nullptr;
    if (!f || !out) return fail(FTK_ERR_ARG, "field and out must be non-NULL");
    ftk_plan *pl = nullptr;
    ftk_status s = plan_create(ndim, nx, ny, nz, nt, p, nullptr, &pl, false, comps);
    if (s != FTK_OK) return s;
    s = ftk_plan_execute(pl, f, stream);
    if (s == FTK_OK) s = ftk_plan_download(pl, out);
    std::string keep = g_err;
    ftk_plan_destroy(pl);
    g_err = keep;
    return s;
}

ftk_status ftk_track_cp2d(const float *f, int64_t nx, int64_t ny, int64_t nt, const ftk_params *p,
                          ftk_result **out, void *stream) {
    return track_once(2, f, nx, ny, 1, nt, p, out, stream);
}

ftk_status ftk_track_cp3d(const float *f, int64_t nx, int64_t ny, int64_t nz, int64_t nt,
                          const ftk_params *p, ftk_result **out, void *stream) {
    return track_once(3, f, nx, ny, nz, nt, p, out, stream);
}

ftk_status ftk_track_vec2d(const float *v, int64_t nx, int64_t ny, int64_t nt, const ftk_params *p,
                           ftk_result **out, void *stream) {
    return track_once(2, v, nx, ny, 1, nt, p, out, stream, 2);
}

ftk_status ftk_plan_create_vec2d(int64_t nx, int64_t ny, int64_t nt, const ftk_params *p, ftk_plan **plan) {
    return plan_create(2, nx, ny, 1, nt, p, nullptr, plan, false, 2);
}

size_t ftk_result_count(const ftk_result *r) { return r ? r->count : 0; }
const ftk_cp *ftk_result_data(const ftk_result *r) { return r ? r->data : nullptr; }
void ftk_result_free(ftk_result *r) {
    if (!r) return;
    std::free(r->data);
    delete r;
}

}  // extern "C"
