"""Admission policy of the request server (host logic, CPU only).

The policy header is compiled into a small shared library with the host
compiler and driven through ctypes: slot reuse, creation under the memory
budget, least-recently-used eviction, the slot cap, and that a request
blocked for memory is not overtaken by later requests that would need new
slots.
"""
import ctypes as C
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2312_02999_gb300", "csrc")

_SRC = r'''
#include "admission.h"
extern "C" int admit_c(int nq, const int* qmesh, int ns, const int* smesh, const int* sbusy,
                       const long long* sbytes, const long long* slast, int nm,
                       const long long* need, long long used, long long budget, int max_slots,
                       int* slot_out, int* evict_out, int* n_evict) {
  std::vector<int> q(qmesh, qmesh + nq);
  std::vector<fsim::SlotView> s(ns);
  for (int k = 0; k < ns; ++k) s[k] = {smesh[k], sbusy[k] != 0, (size_t)sbytes[k], slast[k]};
  std::vector<size_t> nd(need, need + nm);
  fsim::Admission a = fsim::admit(q, s, nd, (size_t)used, budget, max_slots);
  *slot_out = a.slot;
  *n_evict = (int)a.evict.size();
  for (size_t i = 0; i < a.evict.size(); ++i) evict_out[i] = a.evict[i];
  return a.job;
}
extern "C" int growth_c(long long used, long long delta, long long budget) {
  return fsim::admit_growth((size_t)used, (size_t)delta, budget) ? 1 : 0;
}
'''


@pytest.fixture(scope="module")
def admit(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("admission")
    src = d / "admit.cpp"
    src.write_text(_SRC)
    so = d / "libadmit.so"
    subprocess.run([cxx, "-std=c++17", "-O1", "-shared", "-fPIC", "-I", CSRC, str(src), "-o", str(so)],
                   check=True, capture_output=True)
    lib = C.CDLL(str(so))

    def call(queue, slots, need, used, budget, max_slots=16):
        I = C.c_int
        L = C.c_longlong
        nq, ns = len(queue), len(slots)
        q = (I * max(nq, 1))(*queue)
        sm = (I * max(ns, 1))(*[s[0] for s in slots])
        sb = (I * max(ns, 1))(*[int(s[1]) for s in slots])
        sy = (L * max(ns, 1))(*[s[2] for s in slots])
        sl = (L * max(ns, 1))(*[s[3] for s in slots])
        nd = (L * max(len(need), 1))(*need)
        slot, nev = I(), I()
        ev = (I * max(ns, 1))()
        job = lib.admit_c(nq, q, ns, sm, sb, sy, sl, len(need), nd, L(used), L(budget), max_slots,
                          C.byref(slot), ev, C.byref(nev))
        return job, slot.value, [ev[i] for i in range(nev.value)]
    call.growth = lambda used, delta, budget: bool(lib.growth_c(C.c_longlong(used),
                                                                C.c_longlong(delta),
                                                                C.c_longlong(budget)))
    return call


def test_empty_queue_admits_nothing(admit):
    assert admit([], [], [10], 0, 100)[0] == -1


def test_idle_slot_of_same_mesh_is_reused(admit):
    # slots: (mesh, busy, bytes, last_used)
    job, slot, ev = admit([1], [(0, False, 10, 1), (1, False, 10, 2)], [10, 10], 20, 20)
    assert (job, slot, ev) == (0, 1, [])


def test_new_slot_within_budget(admit):
    job, slot, ev = admit([0], [(0, True, 10, 1)], [10], 10, 25)
    assert (job, slot, ev) == (0, -1, [])
    # no budget means no cap
    assert admit([0], [(0, True, 10, 1)] * 3, [10], 30, 0)[:2] == (0, -1)


def test_lru_eviction_makes_room(admit):
    slots = [(1, False, 10, 5), (2, False, 10, 3), (0, True, 10, 9)]
    job, slot, ev = admit([0], slots, [10, 10, 10], 30, 30)
    assert (job, slot) == (0, -1)
    assert ev == [1]            # mesh 2's slot was used least recently
    job, slot, ev = admit([0], slots, [20, 10, 10], 30, 30)
    assert sorted(ev) == [0, 1]


def test_blocked_request_is_not_overtaken_by_slot_creation(admit):
    # mesh 0 needs 50 bytes and only busy slots hold memory: it must wait;
    # the later request for mesh 1 may reuse its idle slot but may not create
    slots = [(2, True, 40, 1), (1, False, 10, 2)]
    job, slot, ev = admit([0, 1], slots, [50, 10, 40], 50, 60)
    assert (job, slot, ev) == (1, 1, [])
    slots = [(2, True, 40, 1)]
    assert admit([0, 1], slots, [50, 10, 40], 40, 60)[0] == -1


def test_slot_cap(admit):
    slots = [(0, True, 1, 1), (1, True, 1, 2)]
    assert admit([2], slots, [1, 1, 1], 2, 0, max_slots=2)[0] == -1
    slots = [(0, True, 1, 1), (1, False, 1, 2)]
    job, slot, ev = admit([2], slots, [1, 1, 1], 2, 0, max_slots=2)
    assert (job, slot, ev) == (0, -1, [1])


def test_running_slot_growth_respects_the_budget(admit):
    # a running slot's reduced-system buffers may grow only while all slots
    # together stay within the budget (the solve fails with ENOMEM otherwise)
    assert admit.growth(90, 10, 100)
    assert not admit.growth(90, 11, 100)
    assert admit.growth(10 ** 12, 10 ** 12, 0)          # no budget
