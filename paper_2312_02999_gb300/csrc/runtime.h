// Host runtime types shared by the C ABI (capi.cu) and the request server
// (serve.cpp).  Not part of the public C ABI.
#pragma once
#include <cstddef>
#include <cstdint>
#include <memory>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/fsim.h"
#include "kernels.h"

namespace fsim {

constexpr int kCounters = 16;   // device counter words of a workspace
constexpr int kScal = 8;        // device float64 scalars of a workspace

// One uploaded mesh: constant device data (topology, factor, Sigma^-1) plus
// its default workspace, all reachable through d.
struct MeshState {
  DevMesh d;
  bool prefactored = false, actuated = false;
  fsim_params p{};
  double kappa = 0.0;
  int64_t factor_nnz = 0;
  std::vector<void*> allocs;     // device buffers owned by this mesh
  size_t ws_bytes = 0;           // bytes of one per-solve workspace
  double mean_edge = 0.0;        // mean proxy edge length at rest
  // host copies kept for the prefactor
  std::vector<double> rest;
  std::vector<int32_t> tets;
  std::vector<uint8_t> pinned;
  std::vector<uint8_t> x2mask;
  // scratch for the step entry points
  double* gtmp = nullptr;
  double* proj = nullptr;
  double* dxtmp = nullptr;
  bool has_x = false;
  // TMA descriptors of the tensor-core Sigma^-1 product (DevMesh::tc_maps)
  std::vector<uint64_t> tc_maps;
};

// Where a solve runs: its stream, its pinned read-back words, the CTA count
// of cooperative launches, and the list that owns buffers it grows.
struct Exec {
  cudaStream_t stream = nullptr;
  int* h_counters = nullptr;     // kCounters pinned ints
  double* h_scal = nullptr;      // kScal pinned doubles
  int coop_ctas = 1;
  bool alone = true;             // no other solve shares the GPU
  std::vector<void*>* allocs = nullptr;
  size_t* bytes = nullptr;
  // asked before the reduced-system buffers grow by `delta` bytes; nonzero
  // refuses (the solve then returns FSIM_ENOMEM).  NULL: no budget.
  int (*grow)(void* user, size_t delta) = nullptr;
  void* grow_user = nullptr;
};

// Allocate the per-solve buffers of workspace m (a copy of a prefactored
// mesh's DevMesh whose constant pointers stay shared).
int rt_alloc_workspace(const MeshState& ms, DevMesh& m, std::vector<void*>& allocs, size_t* bytes);
// Grow the reduced-system buffers of workspace m to hold nc (synchronises ex.stream).
int rt_ensure_reduced(const Exec& ex, DevMesh& m, int nc);
// Device bytes of the reduced-system buffers sized for nc_cap.
size_t rt_reduced_bytes(int nc_cap);
// Algorithm 1 for one frame on workspace m; actuation must already be in m.act.
int rt_solve_frame(const Exec& ex, const MeshState& ms, DevMesh& m, const double* x_init,
                   bool init_is_dev, int precision, fsim_frame_stats* stats);
void rt_free_list(std::vector<void*>& allocs);
void rt_destroy_graphs(DevMesh& m);
// Bytes a new workspace of this mesh takes (per-solve buffers plus the
// reduced-system buffers at their initial size).
size_t rt_slot_bytes(const MeshState& ms);

}  // namespace fsim

struct fsim_ctx_s {
  int device = 0;
  int num_sms = 0;
  cudaStream_t stream = nullptr;
  std::vector<std::unique_ptr<fsim::MeshState>> meshes;
  // pinned host readback area
  int* h_counters = nullptr;   // kCounters ints
  double* h_scal = nullptr;    // kScal doubles
};

namespace fsim {
MeshState* rt_mesh(fsim_ctx_t ctx, int mesh_id);
}
