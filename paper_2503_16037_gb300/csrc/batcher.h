// Host interface of the batcher of Chebyshev refinements (the serving loop's
// batched passes over K), for host-only code; the device side and the job
// layout are in batch.h.
#pragma once

#include "tursca.h"

namespace tk {

class ChebBatcher;

// A batcher on the current device (its own stream and thread), or null.
ChebBatcher *batcher_create();
void batcher_destroy(ChebBatcher *b);

// launches, jobs run in them, and the largest launch (jobs)
void batcher_stats(ChebBatcher *b, long long *batches, long long *jobs, int *max_jobs);

// Route a scene's Chebyshev refinements through b (null: its own passes);
// FP32 + refinement scenes only.
void scene_attach_batcher(tursca_scene *sc, ChebBatcher *b);

}  // namespace tk
