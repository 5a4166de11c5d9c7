// batch_engine.h -- internal: a batch object (svd_batch_*) reused for
// successive groups of plans, as the serving loop does with its slots.
#pragma once

#include <cstddef>

#include <cuda_runtime.h>

#include "../../include/ranky.h"

// Worker streams, events and a device work list with room for item_capacity
// block/merge eigensolves; no plans yet.
svd_status batch_engine_create(int nstreams, size_t item_capacity, svd_batch_t* out);
// Point the batch at n plans (each alive until batch_engine_detach, after
// the pass on them has finished).  The work lists are uploaded on `stream` from page-locked
// staging (synchronously when stream is null); the previous pass of this
// batch must have finished.  SVD_ERR_INVALID_ARG when the lists exceed the
// capacity.
svd_status batch_engine_assign(svd_batch_t b, int n, const svd_plan_t* plans, cudaStream_t stream);
// Forget the current plans (still alive; their pass has finished): they
// keep no stream of the batch.  Call before the plans are freed.
void batch_engine_detach(svd_batch_t b);
