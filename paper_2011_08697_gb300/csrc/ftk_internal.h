// Internal host-side definitions shared by the C-ABI translation units
// (plans, batches, streams).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "../../include/ftk.h"
#include "ftk_kernels.cuh"

struct ftk_result {
    ftk_cp *data;
    size_t count;
};

struct ftk_plan {
    bool external_ctr;         // counters live in a batch-owned array
    int ndim;
    int variant;               // detect kernel (VAR_*)
    int device;
    ftk::Field F;
    ftk::Blocking B;
    ftk_params p;
    long long nverts;
    ftk::Workspace W;
    float *d_input;
    ftk::RunCounters *h_ctr;        // pinned mirror of the device counters
    cudaStream_t stream;
    const float *last_f;
    const float *last_dev;     // device copy the last run read
    bool last_host;
    bool executed;
    bool timing;
    cudaEvent_t ev[6];
    cudaEvent_t copy_ev;       // end of the host-input copy of the last execute
    ftk::TrajBuffers traj;     // trajectory buffers (allocated on first use)
    long long traj_cap;        // punctures they hold
    long long traj_n;          // trajectories of the last execute (valid if traj_valid)
    bool traj_valid;
    bool tuned;                // FTK_FLAG_AUTOTUNE: launch shape measured
    float stage_ms[5];
    int nstage;
};


namespace ftk {

// what a plan of a shape would allocate, computed without allocating
struct PlanSizes {
    int variant;
    Field F;
    Blocking B;
    long long nseg, cap, scap;
};
ftk_status plan_sizes(int ndim, int64_t nx, int64_t ny, int64_t nz, int64_t nt, const ftk_params *p,
                      PlanSizes *out, bool compact = false);

ftk_status fail(ftk_status s, const std::string &msg);
ftk_status cuda_fail(cudaError_t e, const char *what);
bool is_device_pointer(const void *p);
// plan with its counters at ctr (nullptr: the plan allocates them)
ftk_status plan_create(int ndim, int64_t nx, int64_t ny, int64_t nz, int64_t nt, const ftk_params *p,
                       RunCounters *ctr, ftk_plan **plan, bool compact = false, int comps = 1);
// the device field the kernels read (f, or the plan's copy of it queued on s)
ftk_status plan_source(ftk_plan *pl, const float *f, bool host, cudaStream_t s, const float **src);
// queue the pipeline on s, reading device field f (no host copies)
ftk_status plan_launch(ftk_plan *pl, const float *f, cudaStream_t s);
// after the counters have been copied to pl->h_ctr: grow and re-run on
// overflow (synchronously), check the device status
ftk_status plan_check(ftk_plan *pl);
ftk_status plan_result(ftk_plan *pl, ftk_result **out);
// measured choice of the time chunking for the plan's shape (cached per shape)
ftk_status plan_autotune(ftk_plan *pl, const float *f, cudaStream_t s);
// releases the plan's trajectory buffers
void free_traj(ftk_plan *pl);

}  // namespace ftk
