// Admission policy of the request server (serve.cpp): which queued frame
// solve may start now, and on which workspace slot.  Pure host logic with
// no CUDA calls, so it is unit-tested on the CPU.
//
// A slot is one per-solve workspace bound to a mesh.  Slots are reused by
// later requests for the same mesh; a new slot is created while the memory
// budget allows; idle slots of other meshes are evicted (oldest first) when
// that makes room.  Requests are scanned in arrival order.  When the oldest
// request cannot be admitted for lack of memory, later requests may still
// start on idle slots of their own mesh but may not create slots, so that
// the blocked request gets the next memory that frees up (no starvation).
#pragma once
#include <cstddef>
#include <cstdint>
#include <vector>

namespace fsim {

struct SlotView {
  int mesh = -1;
  bool busy = false;
  size_t bytes = 0;
  int64_t last_used = 0;   // logical time of the last release (eviction order)
};

struct Admission {
  int job = -1;            // index into the queue, -1 = nothing can start
  int slot = -1;           // slot to reuse, -1 = create a new slot
  std::vector<int> evict;  // idle slots to free before creating
};

// queue_mesh[i]: mesh of the i-th queued request (arrival order);
// need[mesh]: bytes of a new slot for that mesh; used: bytes of all slots;
// budget <= 0: unlimited; max_slots: cap on the number of live slots.
inline Admission admit(const std::vector<int>& queue_mesh, const std::vector<SlotView>& slots,
                       const std::vector<size_t>& need, size_t used, int64_t budget,
                       int max_slots) {
  Admission a;
  bool may_create = true;
  int live = (int)slots.size();
  for (int i = 0; i < (int)queue_mesh.size(); ++i) {
    const int mesh = queue_mesh[i];
    // 1. an idle slot of the same mesh
    for (int k = 0; k < (int)slots.size(); ++k) {
      if (!slots[k].busy && slots[k].mesh == mesh) {
        a.job = i;
        a.slot = k;
        return a;
      }
    }
    if (!may_create) continue;
    const size_t nb = (mesh >= 0 && mesh < (int)need.size()) ? need[mesh] : 0;
    // 2. a new slot within the budget and the slot cap
    if ((budget <= 0 || used + nb <= (size_t)budget) && live < max_slots) {
      a.job = i;
      a.slot = -1;
      return a;
    }
    // 3. evict idle slots of other meshes, least recently used first
    std::vector<int> idle;
    for (int k = 0; k < (int)slots.size(); ++k)
      if (!slots[k].busy && slots[k].mesh != mesh) idle.push_back(k);
    for (size_t x = 1; x < idle.size(); ++x)       // insertion sort by last_used
      for (size_t y = x; y > 0 && slots[idle[y]].last_used < slots[idle[y - 1]].last_used; --y) {
        const int t = idle[y];
        idle[y] = idle[y - 1];
        idle[y - 1] = t;
      }
    size_t freed = 0;
    int nfree = 0;
    std::vector<int> ev;
    for (int k : idle) {
      const bool mem_ok = budget <= 0 || used - freed + nb <= (size_t)budget;
      const bool cap_ok = live - nfree < max_slots;
      if (mem_ok && cap_ok) break;
      ev.push_back(k);
      freed += slots[k].bytes;
      ++nfree;
    }
    const bool mem_ok = budget <= 0 || used - freed + nb <= (size_t)budget;
    const bool cap_ok = live - nfree < max_slots;
    if (mem_ok && cap_ok) {
      a.job = i;
      a.slot = -1;
      a.evict = ev;
      return a;
    }
    // the oldest blocked request keeps the next free memory
    may_create = false;
  }
  return a;
}

// Growth of a running slot's reduced-system buffers (n_c rose above their
// size): allowed when the bytes of all slots plus the growth stay within the
// budget (budget <= 0: unlimited).  Running slots are never evicted, so a
// growth that does not fit fails its solve with FSIM_ENOMEM.
inline bool admit_growth(size_t used, size_t delta, int64_t budget) {
  return budget <= 0 || used + delta <= (size_t)budget;
}

}  // namespace fsim
