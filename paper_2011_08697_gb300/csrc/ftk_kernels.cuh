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
    ST_WIDE = 16u,      // a value outside the fast rounding range: rerun exactly
    ST_SOVERFLOW = 32u, // survivor capacity exceeded (count is still exact)
};

// Device-resident counters of one pipeline run (one memset clears them).
struct RunCounters {
    unsigned status;
    unsigned pad;
    unsigned long long staged;     // punctures written (or attempted) to staging
    long long punctures;           // final count P (set by the scan kernel)
    unsigned long long survivors;  // spacetime cubes that survived the sign cull
    unsigned long long pending;    // 3D punctures left to the exact classification
    unsigned long long tiles;      // survivor tiles handed out (survivor scan)
    unsigned long long seg_tiles;  // segment tiles handed out (segment scan)
    long long surv_total;          // punctures over every surviving cube
    unsigned long long pairs;      // cells linked (two punctured sides)
    unsigned long long incid;      // sum over punctured faces of their cell count
    unsigned long long nlink[3];   // 2D link items per first-step axis (streaming variant)
};

// Division by a fixed divisor d for numerators n < 2^31: with
// l = ceil(log2 d) and m = ceil(2^(31+l) / d), floor(n / d) = (n m) >> (31+l),
// because n m / 2^(31+l) exceeds n / d by less than n / 2^(31+l) < 2^-l <= 1/d,
// which cannot carry the fractional part (at most (d-1)/d) past an integer.
struct FastDiv {
    unsigned long long m;
    int shift;
};
inline FastDiv make_fastdiv(unsigned d) {
    int l = 0;
    while ((1ull << l) < d) ++l;
    FastDiv f;
    const unsigned long long num = 1ull << (31 + l);
    f.m = (num + d - 1) / d;
    f.shift = 31 + l;
    return f;
}
__host__ __device__ inline unsigned fdiv(unsigned n, const FastDiv &f) {
    return (unsigned)(((unsigned long long)n * f.m) >> f.shift);
}

struct Field {
    const float *f;      // f[t][z][y][x], rows of `pitch` floats (the first nx are the grid's)
    int nx, ny, nz, nt;  // nz = 1 in 2D
    int pitch;           // floats from one grid row to the next (>= nx)
    float scale;         // 2^quant_shift
    int small;           // nx*ny*nz*nt < 2^31: vertex ids decode with FastDiv
    FastDiv dx, dy, dz;  // division by nx, ny, nz
    int comps = 1;       // 2: a 2D vector field, components interleaved per vertex
                         // (pitch = nx); otherwise a scalar field
};

// fills the FastDiv fields of a Field whose extents are set
inline void field_divisors(Field &F) {
    F.dx = make_fastdiv((unsigned)F.nx);
    F.dy = make_fastdiv((unsigned)F.ny);
    F.dz = make_fastdiv((unsigned)F.nz);
    const double nv = (double)F.nx * F.ny * F.nz * F.nt;
    F.small = nv < 2147483648.0 ? 1 : 0;
}

struct Blocking {
    int ry, rz;          // rows / planes of base vertices per unit
    int nyb, nzb;        // y and z blocks
    int tc, ntc;         // slices per time chunk, number of time chunks
    // tiled kernel on rows too wide for its tile: nxb windows of wx cube
    // columns, one row per unit (ry = rz = 1); nxb <= 1 means whole rows
    int nxb, wx;
    // incremental mode of the 2D streaming kernel for in-situ streams: 0 off;
    // 1 store the last slice's cube-row words to st_out; 2 take slice 0's
    // words from st_in (only slice 1 is streamed) and store slice 1's to st_out
    int st_mode;
    const uint32_t *st_in;
    uint32_t *st_out;
};

struct Workspace {
    RunCounters *ctr;
    int *seg_cnt;            // [nseg] punctures per segment
    long long *seg_stage;    // [nseg] offset of the segment's run in staging
    long long *seg_off;      // [nseg] exclusive scan of seg_cnt
    long long *staging;      // [cap] tiled variant: face ids, per-segment runs
    long long *face;         // [cap] face ids sorted
    int *parent;             // [cap] union-find
    float4 *off;             // [cap] in-cell offsets x, y, z, t
    int8_t *morse;           // [cap]
    long long *label;        // [cap]
    ftk_cp *packed;          // [cap] host-layout records
    long long cap;
    long long nseg;
    // streaming variant: surviving cubes, evaluated after the dense pass
    long long *surv;                // [scap] vertex id of each surviving cube, per-segment runs
    unsigned long long *surv_mask;  // [scap] punctured face types of the cube
    int *surv_off;                  // [scap] punctures of the survivors before it in list order
    int *seg_scnt;                  // [nseg] survivors per segment
    long long *seg_sstage;          // [nseg] start of the segment's run in surv
    unsigned long long *tile;       // [scap / LB_TILE] look-back state of the survivor scan
    unsigned long long *seg_tile;   // [nseg / SEG_TILE] look-back state of the segment scan
    int *litem;                     // [3 scap] 2D link items: list a (at a scap) holds the survivors
                                    // with cells of first-step axis a (axis 0: every punctured one)
    long long scap;
    int uf_limit;                   // union-find bound of the label pass (set at launch; below the
                                    // default only in tests)
};

constexpr int LB_TILE = 2048;       // survivors per tile of the survivor scan
constexpr int SEG_TILE = 2048;      // segments per tile of the segment scan

// segment = (t, z, y-block), or (t, z, y, x-window) for windowed rows: a
// contiguous run of face ids
__host__ __device__ inline long long segment_of_coords(int x, int y, int z, int t, const Field &F, const Blocking &B) {
    const long long s = ((long long)t * F.nz + z) * B.nyb + y / B.ry;
    return B.nxb > 1 ? s * B.nxb + x / B.wx : s;
}
__host__ __device__ inline long long segment_of(long long g, const Field &F, const Blocking &B) {
    long long s, row;
    if (F.small) {
        const unsigned r = fdiv((unsigned)g, F.dx);              // (t*nz + z)*ny + y
        const unsigned tz = fdiv(r, F.dy);
        const unsigned y = r - tz * (unsigned)F.ny;
        s = (long long)tz * B.nyb + y / B.ry;
        row = r;
    } else {
        row = g / F.nx;                          // (t*nz + z)*ny + y
        const long long y = row % F.ny;
        const long long tz = row / F.ny;         // t*nz + z
        s = tz * B.nyb + y / B.ry;
    }
    return B.nxb > 1 ? s * B.nxb + (g - row * F.nx) / B.wx : s;
}
// segments of a field: (t, z, y-block[, x-window])
inline long long segment_count(const Field &F, const Blocking &B) {
    return (long long)F.nt * F.nz * B.nyb * (B.nxb > 1 ? B.nxb : 1);
}

// detect-kernel variants
enum : int {
    VAR_TILE = 0,           // smem-tile kernel: any 2D/3D shape
    VAR_STREAM2 = 1,        // streaming 2D kernel (nx % 4 == 0, 16-byte aligned rows)
    VAR_STREAM2_EXACT = 2,  // same, exact rounding for |f 2^S| > 2^22
    VAR_STREAM3 = 3,        // streaming 3D kernel (pitch % 4 == 0, pitch <= 1024, 16-byte aligned)
    VAR_STREAM3_EXACT = 4,  // same, exact rounding
};
constexpr int STREAM3_MAX_NX = 1024;  // widest row the 3D streaming kernel takes
inline int exact_variant(int v) {
    return v == VAR_STREAM2 ? VAR_STREAM2_EXACT : v == VAR_STREAM3 ? VAR_STREAM3_EXACT : v;
}
constexpr float RANGE_LIMIT = 268435456.0f;   // 2^28: the exact quantisation's range of |f 2^S|
constexpr int STREAM2_ROWS = 16;      // cube rows per unit of the streaming kernel
constexpr int STREAM2_MAX_NX = 4096;  // widest row the streaming kernel takes
constexpr int STREAM2_VEC_MAX_NX = 2048;   // widest row of vectors it takes

size_t detect_smem_bytes(int ndim, const Field &F, const Blocking &B);
size_t stream2_smem_bytes(int nx, int comps = 1);
int stream2_threads(int nx);
int stream2_ctas_per_sm(int nx, int comps = 1);
// words of incremental detect state of a 2D streaming plan (0 if it has none)
long long stream2_state_words(const Field &F, const Blocking &B);
// 3D streaming kernel: smem per CTA for B.ry, B.rz, B.ns; threads; resident
// CTAs per SM; launch (the smem attribute is set outside graph capture)
size_t stream3_smem_bytes(int nx, const Blocking &B);
int stream3_threads(int nx);
int stream3_ctas_per_sm(int nx, const Blocking &B);
// cube rows per unit of the 3D streaming kernel for a row pitch
int stream3_ry(int nx);
cudaError_t launch_detect3(int variant, const Field &F, const Blocking &B, const Workspace &W, cudaStream_t s,
                           bool capturing);
// Raises a kernel's dynamic shared-memory cap to at least `smem` bytes and
// never lowers it (thread-safe: plans on several host threads share the
// kernels).  Inside a stream capture a needed raise is an error instead:
// the first, uncaptured launch of each shape configures it.
cudaError_t raise_smem_cap(const void *kernel, size_t smem, bool capturing);
// 2D streaming kernel launch (ftk_detect2.cu; same attribute rule)
cudaError_t launch_detect2(int variant, const Field &F, const Blocking &B, const Workspace &W, cudaStream_t s,
                           bool capturing);
// rows of nx floats at src (any alignment) -> rows of pitch floats at dst,
// columns nx..pitch-1 repeating column nx-1
cudaError_t launch_pad_rows(const float *src, float *dst, int nx, int pitch, long long rows, cudaStream_t s);
// columns nx..pitch-1 of every row of dst := column nx-1
cudaError_t launch_fill_pad(float *dst, int nx, int pitch, long long rows, cudaStream_t s);
cudaError_t launch_pipeline(int ndim, int variant, const Field &F, const Blocking &B, const Workspace &W,
                            cudaStream_t s, cudaEvent_t *ev /* 6 events or null */);

// Device-resident scalars of an in-situ stream, advanced by the merge
// kernels themselves so that one captured push can be replayed unchanged.
struct StreamDev {
    long long n;          // global union-find slots in use
    long long k;          // pushes merged
    long long n_ord[2];   // last-slice ordinal faces of push k, stored at parity k & 1
    unsigned status;      // merge status bits of the current push
    unsigned pad;
};
// Written by the merge kernels into pinned, mapped host memory.
struct StreamView {
    unsigned run_status;  // status bits of the push's pipeline run
    unsigned status;      // merge status bits
    long long punctures;  // P of the run
    long long delta;      // delta records written
};
// Holder of the next slice's address (pinned, mapped host memory).
struct StreamSrc {
    const float *ptr;
};

struct StreamMerge {
    // run (plan workspace, sorted by local face id)
    const long long *face;      // [P] local face ids
    const long long *label;     // [P] local labels (smallest local face id of the run's component)
    const ftk_cp *packed;       // [P] records of the run
    const RunCounters *ctr;     // run counters (P, status)
    long long slice_verts;      // vertices per slice
    int T;                      // face types
    int tbit;                   // time bit of a chain
    StreamDev *S;
    // stream state
    long long *gfid;            // [acap] global face id per slot
    int *gparent;               // [acap]
    long long *gmin;            // [acap] component minimum (valid at roots)
    int *gshadow;               // [acap] 1 if the slot repeats an earlier slot
    ftk_cp *grec;               // [acap] global records
    long long *ord_fid[2];      // last-slice ordinal faces of a push (global ids, sorted), by parity
    int *ord_gi[2];             // their slots
    int *link_prev;             // [P] earlier slot of a shadow, -1 otherwise
    int *old_root;              // [P] root of that earlier slot before this push's unions
    long long *blk;             // [4 * (P / DELTA_BLOCK + 1)] per-block counts and offsets
    uint32_t *st_in;            // incremental detect state: committed after a good push
    const uint32_t *st_out;
    long long st_words;
    ftk_cp *delta;              // [P] delta records (mapped host memory)
    StreamView *view;           // (mapped host memory)
};
constexpr int DELTA_BLOCK = 1024;     // punctures per block of the delta compaction

// the merge kernels read their arguments from dM (device memory, a copy of
// M), so that the stream's arrays can be reallocated without recapturing a
// graph that holds them; cap bounds the run's punctures
cudaError_t launch_stream_merge(const StreamMerge *dM, const StreamMerge &M, long long cap, cudaStream_t s);
// copies `rows` rows of nx floats from the address in *src (device memory)
// to dst with row pitch `pitch` (padding as launch_pad_rows)
cudaError_t launch_stream_copy(const StreamSrc *src, float *dst, int nx, int pitch, long long rows, cudaStream_t s);
cudaError_t launch_stream_final(long long n, const int *gshadow, int *gparent, const long long *gmin,
                                const ftk_cp *grec, ftk_cp *out, long long *count, unsigned *status,
                                cudaStream_t s);

// Trajectories of a run (ordered polylines) and their slices at a time.
struct TrajBuffers {
    int *nbr;            // [2P] punctured partners in the face's cells
    int *root, *size, *start, *rsize, *isroot;   // [P]
    long long *off;      // [P + 1] first point of each root's trajectory
    long long *tidx;     // [P + 1] trajectory number of each root
    int *order;          // [P] punctures in trajectory, then path order
    ftk_cp *rec;         // [P] their records
    long long *toff;     // [ntraj + 1] first point of each trajectory
    uint8_t *closed;     // [ntraj] 1 for a loop
    int *tpt;            // [P] trajectory of each point (record order)
    int *nb2;            // [2P] partners with every loop cut open at its root
    int4 *rk[2];         // [2P] ranking states (node, prev, dist, ended) per point and direction
    int *maxlen;         // [1] points of the longest trajectory
    long long *scan;     // [1025] block sums of the scans
};
// edges, roots, sizes and the scans; *ntraj and *maxlen (the longest
// trajectory; host, pinned) after a synchronisation
cudaError_t launch_trajectories(int ndim, const Field &F, const Workspace &W, long long P, const TrajBuffers &T,
                                cudaStream_t s, long long *ntraj, int *maxlen);
// the path order (ranking rounds for trajectories of up to maxlen points),
// trajectory of each point, records, toff, closed
cudaError_t launch_traj_walk(const Workspace &W, long long P, long long ntraj, long long maxlen, const TrajBuffers &T,
                             cudaStream_t s);
// pts == nullptr: crossing flags per segment (named by its first point) into
// cnt[P] and their scan into soff (soff[P] = total); else the crossing
// points at soff
cudaError_t launch_traj_slice(const TrajBuffers &T, long long P, double t0, int *cnt, long long *soff,
                              ftk_slice_point *pts, cudaStream_t s);

// bounds of the union-find loops and the look-back waits on the current
// device (<= 0: the defaults)
cudaError_t set_wait_limits(long long uf_steps, long long lookback_cycles);
// the union-find bound in force (handed to every launch)
int uf_limit();

// filtering: kept sizes / flags per trajectory and their scans (noff[ntraj],
// nidx[ntraj] = totals); compaction of the kept trajectories with type
// smoothing of half-window h
// (ext: [2 ntraj] scratch for the time extents)
cudaError_t launch_traj_filter(const TrajBuffers &T, long long P, long long ntraj, double min_duration,
                               long long min_points, int drop_loops, int h, unsigned long long *ext, int *kept_size,
                               int *kept_one, long long *noff, long long *nidx, cudaStream_t s);
cudaError_t launch_traj_compact(const TrajBuffers &T, long long P, int h, const long long *noff,
                                const long long *nidx, const int *kept_one, ftk_cp *out, long long *out_off,
                                uint8_t *out_closed, cudaStream_t s);

// name of the step whose CUDA call failed in the last launch_pipeline
const char *last_launch_stage();

// sets the thread-local message returned by ftk_last_error()
void set_last_error(const char *msg);

}  // namespace ftk
