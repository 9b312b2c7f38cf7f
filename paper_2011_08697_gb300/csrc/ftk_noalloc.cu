// ftk_track_cp2d_noalloc: the 2D tracking pipeline with every scratch array
// carved out of one file-scope device array, for callers that cannot
// allocate device memory.  The paper has no counterpart.
//
// The array below is a device symbol: in host code its name is only a
// host-side stand-in, never a device address.  The device address is looked
// up once per device with cudaGetSymbolAddress (that device current) and
// passed to the kernels as ordinary pointers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/ftk.h"
#include "ftk_kernels.cuh"

using namespace ftk;

static __device__ __align__(256) unsigned char g_noalloc_scratch[FTK_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
constexpr size_t kSmemBudget = 110 * 1024;
std::mutex g_setup_mu;
unsigned char *g_scratch_dev[kMaxDevices] = {};

ftk_status err(ftk_status s, const std::string &msg) {
    set_last_error(msg.c_str());
    return s;
}

ftk_status cuda_err(cudaError_t e, const char *what) {
    return err(FTK_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// device memory of the current device (whose scratch array and kernels the
// call uses), or managed memory
bool on_device(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

// one-time set-up per device: the scratch array's device address
ftk_status scratch_base(unsigned char **base) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_err(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return err(FTK_ERR_ARG, "device index out of range");
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_dev[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_err(e, "cudaGetSymbolAddress(scratch)");
        g_scratch_dev[dev] = static_cast<unsigned char *>(p);
    }
    *base = g_scratch_dev[dev];
    return FTK_OK;
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

}  // namespace

extern "C" ftk_status ftk_track_cp2d_noalloc(const float *f_dev, int64_t nx, int64_t ny, int64_t nt,
                                             const ftk_params *p, ftk_cp *out_dev, int64_t out_cap,
                                             int64_t *count, void *cuda_stream) {
    if (count) *count = 0;
    if (!f_dev || !out_dev || !count) return err(FTK_ERR_ARG, "f_dev, out_dev and count must be non-NULL");
    if (nx < 2 || ny < 2 || nt < 1) return err(FTK_ERR_ARG, "every spatial extent must be >= 2 and nt >= 1");
    if (nx > (1 << 30) || ny > (1 << 30) || nt > (1 << 30)) return err(FTK_ERR_ARG, "extent too large");
    if (out_cap < 0) return err(FTK_ERR_ARG, "out_cap must be >= 0");
    ftk_params prm;
    if (p) prm = *p;
    else ftk_params_default(&prm);
    if (prm.quant_shift < 0 || prm.quant_shift > 40) return err(FTK_ERR_ARG, "quant_shift must lie in [0, 40]");
    if (prm.flags != 0) return err(FTK_ERR_ARG, "no flags are supported by the no-alloc entry point");
    if (!on_device(f_dev) || !on_device(out_dev))
        return err(FTK_ERR_ARG, "f_dev and out_dev must be device pointers on the current device");

    unsigned char *base = nullptr;
    ftk_status s = scratch_base(&base);
    if (s != FTK_OK) return s;

    Field F;
    F.f = f_dev;
    F.nx = (int)nx; F.ny = (int)ny; F.nz = 1; F.nt = (int)nt;
    F.pitch = (int)nx;   // the tiled kernel reads the field in place
    F.scale = (float)std::ldexp(1.0, prm.quant_shift);
    field_divisors(F);

    Blocking B{};
    static const int cand[] = {16, 8, 4, 2, 1};
    bool ok = false;
    for (int ry : cand) {
        B.ry = ry; B.rz = 1;
        if (detect_smem_bytes(2, F, B) <= kSmemBudget) { ok = true; break; }
    }
    if (!ok) return err(FTK_ERR_ARG, "grid rows too wide for the detect tile (nx too large)");
    B.nyb = (F.ny + B.ry - 1) / B.ry;
    B.nzb = 1;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long want = 4LL * sms;
    long long chunks = B.nyb >= want ? 1 : (want + B.nyb - 1) / B.nyb;
    chunks = std::min<long long>(chunks, F.nt);
    B.tc = (int)((F.nt + chunks - 1) / chunks);
    B.ntc = (F.nt + B.tc - 1) / B.tc;

    const long long nseg = (long long)F.nt * B.nyb;
    if (nseg > FTK_NOALLOC_MAX_SEGMENTS)
        return err(FTK_ERR_ARG, "grid exceeds the no-alloc segment limit (FTK_NOALLOC_MAX_SEGMENTS)");

    // carve the workspace out of the scratch array
    Workspace W;
    std::memset(&W, 0, sizeof(W));
    size_t off = 0;
    W.ctr = reinterpret_cast<RunCounters *>(base + off);
    off = align256(off + sizeof(RunCounters));
    W.seg_cnt = reinterpret_cast<int *>(base + off);
    off = align256(off + sizeof(int) * nseg);
    W.seg_stage = reinterpret_cast<long long *>(base + off);
    off = align256(off + sizeof(long long) * nseg);
    W.seg_off = reinterpret_cast<long long *>(base + off);
    off = align256(off + sizeof(long long) * nseg);
    const long long cap = std::min<long long>(out_cap, FTK_NOALLOC_MAX_PUNCTURES);
    W.staging = reinterpret_cast<long long *>(base + off);
    off = align256(off + sizeof(long long) * FTK_NOALLOC_MAX_PUNCTURES);
    W.face = reinterpret_cast<long long *>(base + off);
    off = align256(off + sizeof(long long) * FTK_NOALLOC_MAX_PUNCTURES);
    W.label = reinterpret_cast<long long *>(base + off);
    off = align256(off + sizeof(long long) * FTK_NOALLOC_MAX_PUNCTURES);
    W.off = reinterpret_cast<float4 *>(base + off);
    off = align256(off + sizeof(float4) * FTK_NOALLOC_MAX_PUNCTURES);
    W.parent = reinterpret_cast<int *>(base + off);
    off = align256(off + sizeof(int) * FTK_NOALLOC_MAX_PUNCTURES);
    W.morse = reinterpret_cast<int8_t *>(base + off);
    off = align256(off + sizeof(int8_t) * FTK_NOALLOC_MAX_PUNCTURES);
    if (off > FTK_NOALLOC_SCRATCH_BYTES) return err(FTK_ERR_ARG, "internal: scratch layout exceeds the array");
    W.packed = out_dev;
    W.cap = cap;
    W.nseg = nseg;

    cudaStream_t st = (cudaStream_t)cuda_stream;
    cudaError_t e = launch_pipeline(2, VAR_TILE, F, B, W, st, nullptr);
    if (e != cudaSuccess) return cuda_err(e, "pipeline launch");
    // counters read back on the caller's stream (no legacy-stream copy, which
    // would wait for every blocking stream of the context)
    RunCounters h;
    e = cudaMemcpyAsync(&h, W.ctr, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_err(e, "counter read-back");
    *count = h.punctures;
    if (h.status & ST_RANGE)
        return err(FTK_ERR_RANGE, "a sample is non-finite or |f * 2^quant_shift| exceeds 2^28");
    if (h.status & ST_OVERFLOW)
        return err(FTK_ERR_NOMEM, "more punctured faces than out_cap or FTK_NOALLOC_MAX_PUNCTURES");
    if (h.status & ST_TIMEOUT) return err(FTK_ERR_TIMEOUT, "a bounded device loop gave up");
    if (h.status & ST_PAIRING)
        return err(FTK_ERR_INVARIANT, "a spacetime cell had other than 0 or 2 punctured sides");
    return FTK_OK;
}
