// Lock-step batches of frame solves (batch.cu): the host interface used by
// the C ABI (fsim_solve_batch) and the request server's batch workers.
#pragma once
#include <cstddef>
#include <functional>

#include "runtime.h"

namespace fsim {

class Batch;

// One request handed to a batch: the request itself, an opaque tag returned
// with its result, and a host buffer (3n, or NULL) for its positions.
struct BatchReq {
  fsim_request req{};
  void* user = nullptr;
  double* x_host = nullptr;
};
// Asked at every iteration boundary for a request for a free slot (false:
// none now).  Called on the batch's host thread.
using BatchPull = std::function<bool(BatchReq*)>;
// A finished request: its tag, status and statistics (positions delivered).
using BatchDone = std::function<void(void* user, int status, const fsim_frame_stats& st)>;

// A batch of up to cap frames of mesh ms running on `stream` (NULL on error,
// with the status in *status: FSIM_EINVAL when the mesh cannot be batched,
// FSIM_ENOMEM, FSIM_ECUDA).
Batch* batch_create(fsim_ctx_t ctx, MeshState& ms, int cap, cudaStream_t stream, int* status);
void batch_destroy(Batch* b);
// Device bytes the batch holds.
size_t batch_bytes(const Batch* b);
// Run until `pull` has nothing and every slot is free.
int batch_run(Batch* b, const BatchPull& pull, const BatchDone& done);
// Whether a request can run in a batch (mixed precision, Woodbury global
// step, a mesh whose supernodes fit the batched solves).
bool batch_servable(const MeshState& ms, const fsim_request& q);

}  // namespace fsim
