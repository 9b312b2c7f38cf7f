/*
 * ftk.h -- C ABI of the GB300 critical-point tracker.
 *
 * The library tracks critical points of a time-varying scalar field on a
 * regular grid (2D + time or 3D + time) exactly, following the method of
 * "FTK: A Simplicial Spacetime Meshing Framework for Robust and Scalable
 * Feature Tracking" (arXiv 2011.08697):
 *
 *   1. every time slice is quantised to fixed point, F = rint(f * 2^S), and
 *      differentiated with integer central differences (Sec. 4.3: gradients
 *      of integer or central-difference data are the degenerate case SoS
 *      must handle; one-sided differences at the domain boundary);
 *   2. the spacetime grid is subdivided implicitly into simplices (Sec. 3.3,
 *      each unit (n+1)-cube split into (n+1)! simplices); every n-simplex
 *      ("face") is tested for a puncture by the critical-point trajectory
 *      with the exact point-in-simplex predicate of Sec. 4.3 / Eq. (1),
 *      with Simulation of Simplicity breaking ties by global vertex index;
 *   3. each punctured face is located (barycentric coordinates of Eq. (1))
 *      and classified (Morse index of the interpolated Hessian, Sec. 4.1);
 *   4. punctured faces that share a spacetime cell ((n+1)-simplex) are
 *      linked into trajectories (Algorithm 1, left column), each labelled by
 *      the smallest face id it contains.
 *
 * Conventions
 *   Field layout: C-contiguous float32, f[t][y][x] (2D) or f[t][z][y][x]
 *   (3D), x fastest.  Every spatial extent must be >= 2.
 *   Global vertex id g = ((t*nz + z)*ny + y)*nx + x   (nz = 1 in 2D).
 *   Face id = g * T + type, T = 12 (2D) or 60 (3D); the type is the rank of
 *   the face's chain of axis bitmasks in lexicographic order (axis bit 0 = x,
 *   1 = y, 2 = z in 3D, and the last bit = t).
 *
 * Errors: every call returns an ftk_status; nothing is thrown or aborted
 * across the ABI.  On error every output pointer is set to NULL, and
 * ftk_last_error() describes the failure (thread-local string).
 *
 * Memory: input pointers are borrowed.  A device pointer must stay valid
 * until the work queued on the given CUDA stream has completed; a host
 * pointer is copied before the call returns.  Results (ftk_result) are
 * library-owned host arrays released with ftk_result_free().
 */
#ifndef FTK_GB300_H
#define FTK_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FTK_OK = 0,
    FTK_ERR_ARG = 1,        /* invalid argument (null pointer, extent < 2, ...) */
    FTK_ERR_RANGE = 2,      /* a sample is non-finite or |f * 2^S| > 2^28 */
    FTK_ERR_NOMEM = 3,      /* device or host allocation failed */
    FTK_ERR_CUDA = 4,       /* a CUDA runtime call failed */
    FTK_ERR_TIMEOUT = 5,    /* a bounded device-side wait gave up */
    FTK_ERR_BUSY = 6,       /* admission refused (device memory budget) */
    FTK_ERR_INVARIANT = 7,  /* a spacetime cell had a punctured-side count other than 0 or 2 */
    FTK_ERR_STATE = 8       /* call not valid in the object's current state */
} ftk_status;

#define FTK_FLAG_STAGE_TIMES 1u   /* record per-stage device times (plans) */
#define FTK_FLAG_AUTOTUNE 2u      /* choose each shape's launch shape (time chunking; cube planes
                                     per unit of the 3D streaming kernel) by measurement on the
                                     first execute of a plan or batch, cached per shape */

/* Tracking parameters.  ftk_params_default() fills the defaults. */
typedef struct {
    double   origin[3];      /* physical coordinate of grid index 0 (x, y, z) */
    double   spacing[3];     /* physical grid spacing (x, y, z) */
    double   t0, dt;         /* physical time of slice 0 and slice spacing */
    int32_t  quant_shift;    /* fixed-point scale 2^quant_shift; default 20 */
    uint32_t flags;          /* FTK_FLAG_* bits; other bits reserved, must be 0 */
    int64_t  max_punctures;  /* initial device capacity; 0 = automatic (grows on demand) */
} ftk_params;

/* One punctured face (one point of a critical-point trajectory). */
typedef struct {
    int64_t face_id;      /* g * T + type */
    int64_t label;        /* trajectory label: smallest face id of its component */
    int32_t base[4];      /* grid indices x, y, z, t of the face's base vertex (z = 0 in 2D) */
    float   off[4];       /* in-cell offsets along x, y, z, t (position = base + off) */
    int8_t  morse_index;  /* number of negative Hessian eigenvalues: 0 = minimum,
                             n = maximum, else saddle; -1 = degenerate Hessian */
    uint8_t ordinal;      /* 1 if all vertices of the face lie in one time slice */
    uint8_t ndim;         /* 2 or 3 */
    uint8_t reserved[5];
} ftk_cp;                 /* 56 bytes */

/* Device-side view of a plan's results (structure of arrays, valid until the
 * next execute or destroy).  Arrays are ordered by increasing face id. */
typedef struct {
    int64_t        count;
    const int64_t *face_id;   /* [count] */
    const int64_t *label;     /* [count] */
    const float   *off;       /* [count][4] */
    const int8_t  *morse;     /* [count] */
} ftk_device_view;

/* A point where a trajectory crosses the time slice t = t0 (grid units). */
typedef struct {
    int64_t label;           /* the trajectory's label */
    int64_t face_a, face_b;  /* punctured faces at the ends of the crossing segment, face_a < face_b */
    double  pos[3];          /* grid coordinates x, y, z of the crossing (z = 0 in 2D) */
} ftk_slice_point;           /* 48 bytes */

typedef struct ftk_result ftk_result;
typedef struct ftk_traj ftk_traj;
typedef struct ftk_slice ftk_slice;
typedef struct ftk_plan ftk_plan;
typedef struct ftk_stream ftk_stream;
typedef struct ftk_batch ftk_batch;
typedef struct ftk_server ftk_server;

void        ftk_params_default(ftk_params *p);
const char *ftk_status_string(ftk_status s);
const char *ftk_last_error(void);
/* Library version string, e.g. "ftk-gb300 0.1 sm_103a". */
const char *ftk_version(void);
/* Test hook (the paper has no counterpart): bounds of the union-find path
 * walks of the label pass (steps per find; later launches in this process)
 * and of the decoupled look-back waits of the scans (clock cycles; on the
 * current device).  A loop that runs out gives up and the run reports
 * FTK_ERR_TIMEOUT; the device stays usable.  Values <= 0 restore the
 * defaults (2^22 steps, 4e9 cycles).  The linking, stream merges and the
 * detect kernels' waits on their bulk copies keep their own fixed bounds.
 * Not for concurrent use with other calls. */
ftk_status ftk_debug_set_wait_limits(int64_t uf_steps, int64_t lookback_cycles);

/* ---------------------------------------------------------------------
 * One-shot tracking (paper Sec. 8, post hoc analysis of a whole field).
 * f: device or host pointer to nt slices of ny*nx (2D) or nz*ny*nx (3D)
 * floats.  *out receives all punctured faces sorted by face_id.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream).  The call
 * returns after the results are on the host.
 * ------------------------------------------------------------------- */
ftk_status ftk_track_cp2d(const float *f, int64_t nx, int64_t ny, int64_t nt,
                          const ftk_params *p, ftk_result **out, void *cuda_stream);
ftk_status ftk_track_cp3d(const float *f, int64_t nx, int64_t ny, int64_t nz, int64_t nt,
                          const ftk_params *p, ftk_result **out, void *cuda_stream);

/* ---------------------------------------------------------------------
 * Zeros of a time-varying 2D vector field (paper Sec. 4.1: critical points
 * of a vector field are the points where v = 0; sources, sinks and saddles
 * are told apart by the eigenvalues of the Jacobian).  v: device or host
 * pointer to nt slices of ny*nx vertices with the two components
 * interleaved, v[t][y][x][c] (c = 0: x, c = 1: y).  Each component is
 * quantised like a scalar sample (F = rint(v * 2^quant_shift)) and takes
 * the place of the gradient; the mesh, the SoS predicate, the location and
 * the linking are those of ftk_track_cp2d.  morse_index holds the number
 * of Jacobian eigenvalues with negative real part (0 source, 1 saddle,
 * 2 sink), taken exactly from the integer central-difference Jacobian of v
 * at the face's vertices, weighted by the Cramer numerators; -1 where the
 * weighted Jacobian has determinant zero, or trace zero with a positive
 * determinant (a centre: no real-part sign).  Records sorted by face_id.
 * ftk_plan_create_vec2d makes a plan for such fields: execute, count,
 * download, trajectories and slices behave as for a scalar plan, with v in
 * place of f.  Errors as ftk_track_cp2d (FTK_ERR_RANGE when a component
 * is non-finite or beyond 2^28 after scaling).
 * ------------------------------------------------------------------- */
ftk_status ftk_track_vec2d(const float *v, int64_t nx, int64_t ny, int64_t nt,
                           const ftk_params *p, ftk_result **out, void *cuda_stream);
ftk_status ftk_plan_create_vec2d(int64_t nx, int64_t ny, int64_t nt, const ftk_params *p, ftk_plan **plan);

/* Result access.  ftk_result_data() entries are sorted by face_id. */
size_t        ftk_result_count(const ftk_result *r);
const ftk_cp *ftk_result_data(const ftk_result *r);
void          ftk_result_free(ftk_result *r);

/* ---------------------------------------------------------------------
 * Plans: device workspace for repeated tracking of fields of one shape.
 * ftk_plan_execute queues the whole pipeline on cuda_stream and returns
 * without synchronising; results stay in device memory.  f may be a device
 * pointer or a host pointer (copied to a plan-owned device buffer on the
 * same stream).  ftk_plan_count / ftk_plan_download synchronise the plan's
 * last stream, re-run the pipeline with a larger capacity if the punctures
 * outgrew it, and report device-side errors.  With a host pointer f,
 * ftk_plan_execute returns once the copy of f has completed (the caller may
 * then overwrite f); the pipeline itself may still be running.
 * ------------------------------------------------------------------- */
ftk_status ftk_plan_create(int ndim, int64_t nx, int64_t ny, int64_t nz, int64_t nt,
                           const ftk_params *p, ftk_plan **plan);
ftk_status ftk_plan_execute(ftk_plan *plan, const float *f, void *cuda_stream);
ftk_status ftk_plan_count(ftk_plan *plan, int64_t *count);
ftk_status ftk_plan_download(ftk_plan *plan, ftk_result **out);
/* Copies the last execute's records (sorted by face_id) into a caller-owned
 * host buffer of cap records (pinned memory gives the full link speed);
 * *count receives the number of punctures.  More punctures than cap:
 * FTK_ERR_NOMEM with *count set and nothing copied.  Synchronises. */
ftk_status ftk_plan_download_into(ftk_plan *plan, ftk_cp *dst, int64_t cap, int64_t *count);
ftk_status ftk_plan_device_view(ftk_plan *plan, ftk_device_view *view);
/* Trajectories of the last execute as ordered polylines (paper Sec. 4.1: a
 * trajectory is a PL curve through spacetime).  Two punctured sides of one
 * spacetime cell are consecutive points (the interpolated field is linear
 * in the cell, so its zero set there is the segment between them); every
 * face lies in at most two cells, so a trajectory is a path or a loop.
 * Trajectories come in increasing label order; trajectory i holds the
 * records points[offsets[i] .. offsets[i+1]) in path order, starting at
 * the end with the smaller record index (= smaller face id) -- a loop
 * starts at its smallest face id and continues to its smaller neighbour,
 * and closed[i] = 1.  Synchronises; results are library-owned host arrays
 * released with ftk_traj_free. */
ftk_status     ftk_plan_trajectories(ftk_plan *plan, ftk_traj **out);
int64_t        ftk_traj_count(const ftk_traj *tr);
const int64_t *ftk_traj_offsets(const ftk_traj *tr);    /* [count + 1] */
const ftk_cp  *ftk_traj_points(const ftk_traj *tr);     /* [offsets[count]] */
const uint8_t *ftk_traj_closed(const ftk_traj *tr);     /* [count] */
void           ftk_traj_free(ftk_traj *tr);
/* Post-processing of the trajectories (paper Sec. 4.2: filtering by
 * attributes, and smoothing of the critical-point types along a trajectory
 * with a shifting window).  A trajectory is kept iff its time extent
 * (largest minus smallest point time base[3] + off[3]) is >= min_duration,
 * it has >= min_points points, and it is not a loop when drop_loops is set.
 * With smooth_half_window = h > 0, a point's morse_index becomes the common
 * index of the h points before and the h points after it along the path
 * when those 2h points agree and it differs (a loop wraps around; a point
 * of a path with fewer than h points on a side keeps its index); every
 * decision reads the unsmoothed indices.  Same layout as
 * ftk_plan_trajectories. */
typedef struct {
    double  min_duration;
    int64_t min_points;
    int32_t drop_loops;
    int32_t smooth_half_window;
} ftk_traj_filter;
ftk_status ftk_plan_trajectories_filtered(ftk_plan *plan, const ftk_traj_filter *filter, ftk_traj **out);
/* The crossings of every trajectory of the last execute with the time
 * slice t (grid units: slice k is at t = k; paper Sec. 4.1, slicing the PL
 * curve at t = t0): one point per segment (consecutive points a, b of a
 * trajectory, and the closing segment of a loop) with t_a <= t < t_b or
 * t_b <= t < t_a, where t of a point is base[3] + off[3], interpolated
 * linearly in time along the segment (in double precision).  At an integer
 * t = k every crossing is an ordinal puncture of slice k.  Points come
 * grouped by trajectory (label order), in path order.  Synchronises. */
ftk_status             ftk_plan_slice(ftk_plan *plan, double t, ftk_slice **out);
int64_t                ftk_slice_count(const ftk_slice *s);
const ftk_slice_point *ftk_slice_data(const ftk_slice *s);
void                   ftk_slice_free(ftk_slice *s);
/* Per-stage device times (ms) of the last synchronised execute (plan created
 * with FTK_FLAG_STAGE_TIMES), five entries: dense detect; survivor
 * evaluation and the scans (tiled variant: the segment scan); placement,
 * location and classification (tiled: finalize); linking; labels and
 * records.  n = number of entries written. */
ftk_status ftk_plan_stage_times(ftk_plan *plan, float *ms, int cap, int *n);
ftk_status ftk_plan_destroy(ftk_plan *plan);

/* Launch configuration a plan chose (for reports and benchmarks). */
typedef struct {
    int32_t detect_variant;       /* 0 = tiled detect, 1 = streaming 2D detect,
                                     2 = streaming 2D detect with exact rounding */
    int32_t kernels_per_execute;  /* kernel launches one execute queues
                                     (an overflow or exact-rounding re-run adds more) */
    int32_t rows_per_unit;        /* grid rows (y) of base vertices per detect unit */
    int32_t slices_per_unit;      /* time slices of base vertices per detect unit */
    int64_t detect_units;         /* CTAs of the detect launch */
    int64_t capacity;             /* current puncture capacity */
} ftk_plan_desc;
ftk_status ftk_plan_describe(ftk_plan *plan, ftk_plan_desc *desc);

/* ---------------------------------------------------------------------
 * Batches: many independent 2D fields of uneven size and length (the paper's
 * method applied field by field; the batching itself has no counterpart in
 * the paper).  dims[i] = {nx, ny, nt} of field i.  ftk_batch_execute takes
 * device pointers; the first execute runs uncaptured and synchronously
 * (capacities settle, and with FTK_FLAG_AUTOTUNE every shape's time
 * chunking is chosen by measurement and cached per shape); later executes
 * replay one CUDA graph holding every field's pipeline, spread over a pool of
 * streams, and return without synchronising.  ftk_batch_counts /
 * ftk_batch_download synchronise, check all fields with one counter copy and
 * re-run any field whose punctures outgrew its capacity.
 * ------------------------------------------------------------------- */
ftk_status ftk_batch_create(int nfields, const int64_t (*dims)[3], const ftk_params *p, ftk_batch **batch);
ftk_status ftk_batch_execute(ftk_batch *batch, const float *const *f_dev, void *cuda_stream);
ftk_status ftk_batch_counts(ftk_batch *batch, int64_t *counts /* [nfields] */);
ftk_status ftk_batch_download(ftk_batch *batch, ftk_result **outs /* [nfields] */);
ftk_status ftk_batch_destroy(ftk_batch *batch);
/* Kernel launches one execute queues over all fields (re-runs excluded). */
ftk_status ftk_batch_kernels(ftk_batch *batch, int64_t *kernels_per_execute);
/* One-shot batch: outs[i] receives field i's punctured faces, sorted by face_id. */
ftk_status ftk_track_cp2d_batch(int nfields, const float *const *f_dev, const int64_t (*dims)[3],
                                const ftk_params *p, ftk_result **outs, void *cuda_stream);

/* ---------------------------------------------------------------------
 * In-situ streams (paper Sec. 8, push_field_data(); Sec. 3.2, traversal
 * of ordinal then interval elements with a sliding window of two slices).
 * A stream keeps the previous slice and a union-find over every puncture so
 * far resident on the device.  Push k (slice k, host or device pointer of
 * nz*ny*nx floats) returns the delta: the punctured ordinal faces of slice k
 * and interval faces of slab [k-1, k], face ids and base t global to the
 * stream, labels provisional (smallest face id connected so far).  Close
 * returns every puncture with its final label (the whole-field result,
 * sorted by face_id) and releases the stream; final may be NULL.  A stream
 * owns its CUDA stream; one handle must not be used by two threads at once,
 * but different streams may push concurrently from different threads and
 * their work overlaps on the device.
 * ------------------------------------------------------------------- */
ftk_status ftk_stream_open(int ndim, int64_t nx, int64_t ny, int64_t nz, const ftk_params *p, ftk_stream **s);
ftk_status ftk_stream_push(ftk_stream *s, const float *slice, ftk_result **delta);
ftk_status ftk_stream_close(ftk_stream *s, ftk_result **final);

/* Pushes one slice into each of n distinct streams in one call (continuous
 * batching: a serving loop passes every slice that has arrived since its
 * last call).  All n pushes are queued before any is waited for, so their
 * device work overlaps; deltas[i] receives stream i's delta as from
 * ftk_stream_push.  On an error the first failing status is returned, the
 * failing streams' deltas are NULL (and those streams accept no more
 * pushes) and the other streams' deltas are valid and must be freed. */
ftk_status ftk_streams_push(int n, ftk_stream *const *streams, const float *const *slices, ftk_result **deltas);

/* Serving: streams opened in a server are admitted only while the sum of
 * their device-memory footprints stays within budget_bytes.  The footprint
 * (ftk_stream_footprint: the stream's plans, two-slice window and the
 * union-find and delta arrays of its first pushes) is known from the shape
 * and checked before anything is allocated.  ftk_stream_open_in refuses
 * with FTK_ERR_BUSY when it does not fit now (or earlier opens are
 * waiting); ftk_stream_open_wait queues first-come first-served and admits
 * the stream as soon as closing streams have freed enough of the budget,
 * or refuses with FTK_ERR_BUSY after timeout_ms.  A stream whose state
 * later grows charges the growth to the budget before allocating it; growth
 * past the budget fails that push with FTK_ERR_BUSY. */
ftk_status ftk_server_create(uint64_t budget_bytes, ftk_server **server);
ftk_status ftk_server_used(ftk_server *server, uint64_t *used_bytes);
ftk_status ftk_server_destroy(ftk_server *server);   /* FTK_ERR_STATE while streams are open */
ftk_status ftk_stream_open_in(ftk_server *server, int ndim, int64_t nx, int64_t ny, int64_t nz,
                              const ftk_params *p, ftk_stream **s);
ftk_status ftk_stream_open_wait(ftk_server *server, int ndim, int64_t nx, int64_t ny, int64_t nz,
                                const ftk_params *p, int64_t timeout_ms, ftk_stream **s);
ftk_status ftk_stream_footprint(int ndim, int64_t nx, int64_t ny, int64_t nz, const ftk_params *p,
                                uint64_t *bytes);

/* ---------------------------------------------------------------------
 * Isovolume tracking (paper Sec. 6.1; Algorithm 1, right column): the level
 * set f = c of a time-varying scalar field, reconstructed on the same
 * simplicial spacetime mesh as an (n-1)-dimensional object in n + 1
 * dimensions (a surface swept through time in 3D + time).
 *
 *   1. edge pass: every 1-simplex (v, v + bits(m)) of the mesh -- base
 *      vertex v, nonempty axis mask m -- is tested.  The test is the 1-D
 *      case of the critical-point predicate on w = f - c (Sec. 6.1), whose
 *      symbolic perturbation is a positive infinitesimal: a vertex is above
 *      iff f >= c, and an edge is intersected iff its vertices disagree.
 *      The comparison of a float32 sample with the double isovalue is
 *      exact.
 *   2. location: mu = w(v) / (w(v) - w(v + m)), the crossing of the
 *      linear interpolant, in FP32 with w formed by an exact two-sum
 *      against the isovalue split into two floats (|error| < 1e-6 of the
 *      edge length).
 *   3. cell pass: every (n+1)-simplex (a pentachoron in 3D + time, a
 *      tetrahedron in 2D + time) unites its intersected edges -- 4 or 6,
 *      3 or 4 (Sec. 6.1 cases I and II); each connected piece of the
 *      isovolume is labelled by the smallest edge id it contains.  With
 *      nt = 1 there are no cells and every edge is its own piece.
 *
 * Edge id = g * (2^(n+1) - 1) + (m - 1), g the base vertex's global id
 * (as for faces), m's bits: 0 = x, 1 = y, 2 = z (3D), last = t.  Records
 * are sorted by edge id.  Non-finite samples -> FTK_ERR_RANGE; more than
 * 2^31 - 1 intersected edges -> FTK_ERR_RANGE.  Layout, ownership and
 * errors as for the critical-point calls; the isovalue must not be NaN.
 * ------------------------------------------------------------------- */
typedef struct {
    int64_t edge_id;
    int64_t label;       /* smallest edge id of the connected piece */
    int32_t base[4];     /* x, y, z, t of the edge's lower vertex (z = 0 in 2D) */
    float off[4];        /* intersection point minus base (x, y, z, t) */
    uint8_t ordinal;     /* 1: the edge lies inside one time slice */
    uint8_t ndim;        /* 2 or 3 */
    uint8_t reserved[6];
} ftk_iso_point;         /* 56 bytes */

typedef struct ftk_iso_result ftk_iso_result;
typedef struct ftk_iso_plan ftk_iso_plan;

ftk_status ftk_track_iso2d(const float *f, int64_t nx, int64_t ny, int64_t nt, double isovalue,
                           ftk_iso_result **out, void *cuda_stream);
ftk_status ftk_track_iso3d(const float *f, int64_t nx, int64_t ny, int64_t nz, int64_t nt, double isovalue,
                           ftk_iso_result **out, void *cuda_stream);
size_t ftk_iso_result_count(const ftk_iso_result *r);
const ftk_iso_point *ftk_iso_result_data(const ftk_iso_result *r);
void ftk_iso_result_free(ftk_iso_result *r);

/* Plans keep the device workspace of one shape (nz = 1 for ndim = 2) and
 * the last run's records in device memory.  execute queues the pipeline on
 * cuda_stream (a host field is copied before it returns); count waits for
 * it, grows the capacities and runs again if the records did not fit, and
 * checks the run's status; download / download_into copy the records
 * (download_into: into a caller buffer of cap records, FTK_ERR_NOMEM if it
 * is too small, *n set either way); device_records gives their device
 * address (valid until the next execute). */
ftk_status ftk_iso_plan_create(int ndim, int64_t nx, int64_t ny, int64_t nz, int64_t nt, ftk_iso_plan **plan);
ftk_status ftk_iso_plan_execute(ftk_iso_plan *plan, const float *f, double isovalue, void *cuda_stream);
ftk_status ftk_iso_plan_count(ftk_iso_plan *plan, int64_t *n);
ftk_status ftk_iso_plan_download(ftk_iso_plan *plan, ftk_iso_result **out);
ftk_status ftk_iso_plan_download_into(ftk_iso_plan *plan, ftk_iso_point *dst, int64_t cap, int64_t *n);
ftk_status ftk_iso_plan_device_records(ftk_iso_plan *plan, const ftk_iso_point **records, int64_t *n);
/* device times (ms) of the last run's four stages -- edge bits (the dense
 * pass), edge emission, cell pass, labels -- into ms[0..min(cap, 4)) */
ftk_status ftk_iso_plan_stage_times(ftk_iso_plan *plan, float *ms, int cap, int *n);
ftk_status ftk_iso_plan_destroy(ftk_iso_plan *plan);

/* ---------------------------------------------------------------------
 * Tracking without device allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc -- code that
 * runs inside a host application which has already reserved the device's
 * memory for its own pool (an in situ coupling inside a simulation), code
 * that must not trigger the implicit device synchronisation that
 * cudaMalloc/cudaFree may cause, or loops that cannot afford allocation
 * latency.  It runs the same 2D pipeline as ftk_track_cp2d, but every
 * scratch array lives in one file-scope device array of
 * FTK_NOALLOC_SCRATCH_BYTES (64 MiB) that every GPU loading the library
 * holds until the process exits.
 *
 *   f_dev    device pointer, nt x ny x nx float32 (host pointers are rejected)
 *   out_dev  device buffer of out_cap ftk_cp records; receives the punctured
 *            faces sorted by face_id (same records as ftk_track_cp2d)
 *   count    host pointer; receives the number of punctured faces, also when
 *            the call fails with FTK_ERR_NOMEM because they did not fit
 *
 * Limits: at most FTK_NOALLOC_MAX_SEGMENTS segments (nt * ceil(ny / rows per
 * tile)) and FTK_NOALLOC_MAX_PUNCTURES punctured faces per call; larger
 * grids are rejected with FTK_ERR_ARG, more punctures (or more than out_cap)
 * with FTK_ERR_NOMEM.  The call allocates nothing (no cudaMalloc, cudaFree
 * or allocating library routine); it synchronises cuda_stream before it
 * returns.  The first call on each device looks up the scratch array's
 * device address (with that device current); make that first call before
 * any stream capture.  All calls share the one scratch array and it keeps
 * the previous call's contents (the pipeline clears what must start at
 * zero), so calls that overlap on the GPU -- from several host threads or
 * streams at once -- race and must be serialised by the caller.
 * ------------------------------------------------------------------- */
#define FTK_NOALLOC_SCRATCH_BYTES (64u << 20)
#define FTK_NOALLOC_MAX_SEGMENTS 262144
#define FTK_NOALLOC_MAX_PUNCTURES 1310720
ftk_status ftk_track_cp2d_noalloc(const float *f_dev, int64_t nx, int64_t ny, int64_t nt,
                                  const ftk_params *p, ftk_cp *out_dev, int64_t out_cap,
                                  int64_t *count, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* FTK_GB300_H */
