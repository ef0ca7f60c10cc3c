// Chebyshev refinements of several scenes batched into one persistent
// kernel (the serving loop's batched passes over K across requests).
//
// A scene whose solve reaches a Chebyshev refinement hands it to the batcher
// as a job: its graph and vectors, its own number of steps and its own
// coefficients (each request keeps its own schedule, so the requests'
// convergence is not tied together).  The batcher's thread gathers the jobs
// that are waiting, and one cooperative launch then runs every job's row
// groups ("tiles") step after step, with a grid-wide barrier between steps;
// a job simply has no work in the steps past its own count.  Each group is
// computed by the same device code as the scene's own Chebyshev pass
// (tile_group with OpCheb), so a result does not depend on what it was
// batched with.
#pragma once

#include <cuda_runtime.h>

#include "batcher.h"
#include "kern.h"

namespace tk {

constexpr int kChebMaxSteps = 64;  // steps a batched refinement may take
constexpr int kChebMaxJobs = 64;   // jobs in one launch
constexpr int kBatchLanes = 2;     // launches that may run at once (each on at most 1 / kBatchLanes of the GPU)
// Refinements of at most this many row groups are batched; larger ones fill
// the GPU by themselves and run on their own stream.
constexpr int kBatchMaxTiles = 640;

struct __align__(16) ChebJob {
    GridC g;
    GraphP gp;
    const float *val;
    float *r, *d;
    float *p[2];             // step k reads p[k & 1] and writes p[(k + 1) & 1]
    double *x64;             // x += d after the last step (with its FP32-pair split xh, xl, if set)
    float *xh, *xl;
    int nsteps, tile0, W, pad;
    float c1[kChebMaxSteps], c2[kChebMaxSteps];
};


// Hand one refinement to the batcher and block until its batch has been
// launched: the batch waits for `ready` (recorded on the scene's stream once
// the job's inputs are there) and records `done` when it has finished.
// False (nothing launched) when the job cannot be batched; the caller then
// runs the refinement itself.
bool batcher_run(ChebBatcher *b, const ChebJob &job, cudaEvent_t ready, cudaEvent_t done);


// A job can be batched: FP32 scene, the gathered vector's tile fits, no
// streamed passes, at most kChebMaxSteps steps and kBatchMaxTiles groups.
bool batch_eligible(const GridC &g, int nsteps);

// Device side (kernels_solve.cu).  The grid barrier's state; count and gen
// must be zero before the first launch that uses it, abort and status too.
struct BatchBarrier {
    unsigned count, gen;
    int abort, status;
};
// One cooperative launch over the jobs d_jobs[0 .. njobs) (their host copy
// h_jobs gives tile counts and tile sizes), all with the given W.
// The grid is at most 1 / share of the blocks the GPU holds at once, so that
// `share` such launches fit side by side.
cudaError_t launch_cheb_batch(cudaStream_t st, const ChebJob *d_jobs, const ChebJob *h_jobs, int njobs, int W,
                              BatchBarrier *bar, int share);
// tiles (groups of kGroup rows) of a job's pass
int batch_tiles(const GridC &g);

// Self-test of the batch kernels' bounded grid barrier: `blocks` blocks of
// one cooperative launch meet at a barrier that expects blocks + (arrive ? 0
// : 1) arrivals.  Returns 0 when the barrier completed, STATUS_TIMEOUT when
// it gave up (every block then returns), -1 on a CUDA error.  Synchronises
// the stream; allocates and frees 16 bytes of device memory.
int batch_barrier_selftest(cudaStream_t st, int blocks, int arrive);


}  // namespace tk
