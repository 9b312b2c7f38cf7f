// Kernel declarations and launch parameter blocks shared by the host code.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/ftk.h"

namespace ftk {

enum : unsigned {
    ST_RANGE = 1u,      // a sample is non-finite or |f 2^S| > 2^28
    ST_OVERFLOW = 2u,   // staging capacity exceeded (count is still exact)
    ST_PAIRING = 4u,    // a cell with a punctured-side count other than 0 or 2
    ST_TIMEOUT = 8u,    // bounded device loop gave up
};

// Device-resident counters of one pipeline run (one memset clears them).
struct RunCounters {
    unsigned status;
    unsigned pad;
    unsigned long long staged;   // punctures written (or attempted) to staging
    long long punctures;         // final count P (set by the scan kernel)
};

struct Field {
    const float *f;      // C-contiguous f[t][z][y][x]
    int nx, ny, nz, nt;  // nz = 1 in 2D
    float scale;         // 2^quant_shift
};

struct Blocking {
    int ry, rz;          // rows / planes of base vertices per unit
    int nyb, nzb;        // y and z blocks
    int tc, ntc;         // slices per time chunk, number of time chunks
};

struct Workspace {
    RunCounters *ctr;
    int *seg_cnt;            // [nseg] punctures per segment
    long long *seg_stage;    // [nseg] offset of the segment's run in staging
    long long *seg_off;      // [nseg] exclusive scan of seg_cnt
    long long *staging;      // [cap] face ids, per-segment runs
    long long *face;         // [cap] face ids sorted
    int *parent;             // [cap] union-find
    float4 *off;             // [cap] in-cell offsets x, y, z, t
    int8_t *morse;           // [cap]
    long long *label;        // [cap]
    ftk_cp *packed;          // [cap] host-layout records
    long long cap;
    long long nseg;
};

// segment = (t, z, y-block): a contiguous run of face ids
__host__ __device__ inline long long segment_of(long long g, const Field &F, const Blocking &B) {
    const long long row = g / F.nx;             // (t*nz + z)*ny + y
    const long long y = row % F.ny;
    const long long tz = row / F.ny;            // t*nz + z
    return tz * B.nyb + y / B.ry;
}

size_t detect_smem_bytes(int ndim, const Field &F, const Blocking &B);
cudaError_t launch_pipeline(int ndim, const Field &F, const Blocking &B, const Workspace &W,
                            cudaStream_t s, cudaEvent_t *ev /* 6 events or null */);

// sets the thread-local message returned by ftk_last_error()
void set_last_error(const char *msg);

}  // namespace ftk
