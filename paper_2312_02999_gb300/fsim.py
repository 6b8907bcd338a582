"""Thin ctypes binding of the fsim C ABI (include/fsim.h).

Argument marshalling only: every numerical step runs in the CUDA library
``libfsim.so`` (built in-tree by ``paper_2312_02999_gb300.build``).  There is
no CPU fallback: importing this module without the library raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfsim.so")

FSIM_OK = 0
FSIM_EINVAL = -1
FSIM_ENOMEM = -2
FSIM_ECUDA = -3
FSIM_ENOT_SPD = -4
FSIM_ENOT_CONVERGED = -5
FSIM_ELS_FAIL = -6
FSIM_ECONTACT_OVERFLOW = -7
FSIM_ENONFINITE = -8
FSIM_EINTERSECTING = -9
FSIM_ENOT_READY = -10
FP64 = 0
MIXED = 1
REDUCED_UNUSED = -1
REDUCED_COOPERATIVE = 0
REDUCED_NONE = 1
REDUCED_ONE_CTA = 2
REDUCED_CLUSTER = 3

STATUS_NAMES = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ENOT_SPD",
                -5: "ENOT_CONVERGED", -6: "ELS_FAIL", -7: "ECONTACT_OVERFLOW",
                -8: "ENONFINITE", -9: "EINTERSECTING", -10: "ENOT_READY"}


class FsimError(RuntimeError):
    def __init__(self, status, what):
        super().__init__(f"{what} failed: {STATUS_NAMES.get(status, status)}")
        self.status = status


class Params(C.Structure):
    _fields_ = [("weight_scale", C.c_double), ("dhat", C.c_double), ("kappa", C.c_double),
                ("tol_abs", C.c_double), ("tol_rel", C.c_double), ("max_iters", C.c_int32),
                ("max_ls", C.c_int32), ("ccd_s", C.c_double), ("accd_max_iters", C.c_int32),
                ("coop_ctas", C.c_int32), ("contact_capacity", C.c_int64),
                ("active_capacity", C.c_int64), ("skin", C.c_double), ("solver", C.c_int32),
                ("cg_max_iters", C.c_int32), ("cg_tol", C.c_double), ("adaptive_kappa", C.c_int32),
                ("ee_mollifier", C.c_int32), ("reduced_one_cta_max", C.c_int32),
                ("sigma_product_simt", C.c_int32), ("barrier_lane_per_pair", C.c_int32)]


class FrameStats(C.Structure):
    _fields_ = [("status", C.c_int32), ("iterations", C.c_int32), ("ls_trials", C.c_int32),
                ("n_c", C.c_int32), ("n_c_max", C.c_int32), ("kappa_doublings", C.c_int32),
                ("contacts", C.c_int64), ("grad_norm", C.c_double), ("grad_norm0", C.c_double),
                ("energy", C.c_double), ("alpha_min", C.c_double), ("sum_nc3", C.c_double),
                ("cg_iterations", C.c_int64), ("reduced_steps", C.c_int32 * 4),
                ("fp64_steps", C.c_int32)]

    def as_dict(self):
        out = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            out[k] = list(v) if k == "reduced_steps" else v
        return out


class MeshInfo(C.Structure):
    _fields_ = [(k, C.c_int64) for k in ("n", "T", "Ns", "Nt", "Ne", "n_free", "n1", "n2",
                                         "factor_nnz", "n_supernodes", "n_levels",
                                         "workspace_bytes")] + \
               [("kappa", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


FSIM_REQ_DEVICE = 1


class Request(C.Structure):
    _fields_ = [("mesh_id", C.c_int32), ("precision", C.c_int32),
                ("fiber", C.POINTER(C.c_double)), ("stretch", C.POINTER(C.c_double)),
                ("x_init", C.POINTER(C.c_double)), ("flags", C.c_int32), ("reserved0", C.c_int32),
                ("x_out_dev", C.POINTER(C.c_double))]


class ServerConfig(C.Structure):
    _fields_ = [("workers", C.c_int32), ("batch_frames", C.c_int32), ("mem_budget_bytes", C.c_int64)]


class ServerInfo(C.Structure):
    _fields_ = [("workers", C.c_int32), ("slots", C.c_int32), ("peak_slots", C.c_int32),
                ("peak_running", C.c_int32), ("queued", C.c_int64), ("completed", C.c_int64),
                ("bytes_in_use", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = C.c_void_p
_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_I64 = C.POINTER(C.c_int64)
_U8 = C.POINTER(C.c_uint8)

_SIGS = {
    "fsim_default_params": [C.POINTER(Params)],
    "fsim_create": [C.POINTER(_P), C.c_int],
    "fsim_destroy": [_P],
    "fsim_launch_count": [_P, _I64],
    "fsim_mesh_upload": [_P, C.POINTER(C.c_int), _D, C.c_int64, _I32, C.c_int64, _U8, _I32,
                         C.c_int64, _I64, _I32, _D, C.c_int64, _U8],
    "fsim_prefactor": [_P, C.c_int, C.POINTER(Params)],
    "fsim_set_actuation": [_P, C.c_int, _D, _D],
    "fsim_solve_frame": [_P, C.c_int, _D, C.c_int, C.POINTER(FrameStats)],
    "fsim_solve_frame_dev": [_P, C.c_int, C.c_void_p, C.c_int, C.POINTER(FrameStats)],
    "fsim_read_positions": [_P, C.c_int, _D],
    "fsim_read_positions_dev": [_P, C.c_int, C.c_void_p],
    "fsim_read_contacts": [_P, C.c_int, _I32, C.c_int64, _I64],
    "fsim_eval_elastic": [_P, C.c_int, _D, C.c_int, _D, _D, _D],
    "fsim_eval_proxy": [_P, C.c_int, _D, _D],
    "fsim_eval_contacts": [_P, C.c_int, _D, _I32, C.c_int64, _I64, _D],
    "fsim_eval_barrier": [_P, C.c_int, _D, _D, _I32, _I32, _D, C.c_int64],
    "fsim_eval_global_step": [_P, C.c_int, _D, C.c_int, _D, _I32],
    "fsim_eval_sigma_inv_mr": [_P, C.c_int, _D, C.c_int32, C.c_int32, _D],
    "fsim_check_status": [_P, _I32, C.POINTER(C.c_uint64)],
    "fsim_eval_ccd": [_P, C.c_int, _D, _D, _D],
    "fsim_eval_energy": [_P, C.c_int, _D, C.c_int, _D, _D],
    "fsim_mesh_info_get": [_P, C.c_int, C.POINTER(MeshInfo)],
    "fsim_set_actuation_dev": [_P, C.c_int, C.c_void_p, C.c_void_p],
    "fsim_get_stream": [_P, C.POINTER(C.c_void_p)],
    "fsim_profile": [_P, C.c_uint32],
    "fsim_profile_read": [_P, C.c_int, _I64, _D],
    "fsim_profile_reset": [_P],
    "fsim_ccd_noalloc": [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p,
                         C.c_int64, C.c_double, C.c_double, C.c_int32, C.c_void_p, C.c_void_p],
    "fsim_server_create": [_P, C.POINTER(ServerConfig), C.POINTER(_P)],
    "fsim_server_submit": [_P, C.POINTER(Request), _I64],
    "fsim_server_poll": [_P, C.c_int64, _I32],
    "fsim_server_wait": [_P, C.c_int64, _D, C.POINTER(FrameStats), _D, _D],
    "fsim_server_info_get": [_P, C.POINTER(ServerInfo)],
    "fsim_server_destroy": [_P],
    "fsim_solve_frames": [_P, C.c_int32, C.POINTER(Request), C.c_int32, C.POINTER(_D),
                          C.POINTER(FrameStats)],
    "fsim_solve_batch": [_P, C.c_int32, C.POINTER(Request), C.c_int32, C.POINTER(_D),
                         C.POINTER(FrameStats)],
    "fsim_select_region": [_D, C.c_int64, _I32, C.c_int64, _U8, C.c_double, C.c_int32, _I32,
                           C.c_int64, _I64, _I32, C.c_int64, _I64],
}

PROF_CLASSES = ["local_step", "detect", "trsv_fwd", "trsv_bwd", "chol", "barrier", "ccd",
                "sigma_gemv", "reduced", "pcg", "schur"]
SOLVER_WOODBURY = 0
SOLVER_PCG = 1
SOLVER_SCHUR = 2

_libs = {}


def load(path: str = LIB_PATH):
    """Load libfsim.so, or another build of it such as the bounds-checked
    libfsim_check.so (raises if it has not been built)."""
    if path in _libs:
        return _libs[path]
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} (run paper_2312_02999_gb300.build)")
    lib = C.CDLL(path)
    for name, args in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_int
    _libs[path] = lib
    return lib


def exported_symbols():
    return sorted(_SIGS)


def _d(a):
    return a.ctypes.data_as(_D) if a is not None else None


def _i32(a):
    return a.ctypes.data_as(_I32) if a is not None else None


def _u8(a):
    return a.ctypes.data_as(_U8) if a is not None else None


def _chk(st, what):
    if st != FSIM_OK:
        raise FsimError(st, what)


def default_params(**kw) -> Params:
    p = Params()
    _chk(load().fsim_default_params(C.byref(p)), "fsim_default_params")
    for k, v in kw.items():
        setattr(p, k, v)
    return p


class Context:
    """One fsim context on a CUDA device."""

    def __init__(self, device: int = 0, lib_path: str = LIB_PATH):
        self.lib = load(lib_path)
        h = _P()
        _chk(self.lib.fsim_create(C.byref(h), int(device)), "fsim_create")
        self.h = h

    def check_status(self):
        """(enabled, word) of fsim_check_status: whether this library was built
        with index checks, and the first failed check (0: none)."""
        en, w = C.c_int32(), C.c_uint64()
        _chk(self.lib.fsim_check_status(self.h, C.byref(en), C.byref(w)), "fsim_check_status")
        return bool(en.value), int(w.value)

    def close(self):
        if self.h:
            self.lib.fsim_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def launch_count(self) -> int:
        v = C.c_int64()
        _chk(self.lib.fsim_launch_count(self.h, C.byref(v)), "fsim_launch_count")
        return int(v.value)

    def stream_ptr(self) -> int:
        v = C.c_void_p()
        _chk(self.lib.fsim_get_stream(self.h, C.byref(v)), "fsim_get_stream")
        return int(v.value or 0)

    def profile(self, mask: int):
        _chk(self.lib.fsim_profile(self.h, int(mask)), "fsim_profile")

    def profile_reset(self):
        _chk(self.lib.fsim_profile_reset(self.h), "fsim_profile_reset")

    def profile_read(self, cls: int):
        n = C.c_int64()
        ms = C.c_double()
        _chk(self.lib.fsim_profile_read(self.h, int(cls), C.byref(n), C.byref(ms)),
             "fsim_profile_read")
        return int(n.value), float(ms.value)

    def upload(self, mesh) -> "Mesh":
        rest = np.ascontiguousarray(mesh.rest, dtype=np.float64)
        tets = np.ascontiguousarray(mesh.tets, dtype=np.int32)
        pinned = np.ascontiguousarray(mesh.pinned, dtype=np.uint8)
        tris = np.ascontiguousarray(mesh.proxy_tris, dtype=np.int32)
        rp = np.ascontiguousarray(mesh.W_rowptr, dtype=np.int64)
        col = np.ascontiguousarray(mesh.W_col, dtype=np.int32)
        val = np.ascontiguousarray(mesh.W_val, dtype=np.float64)
        region = None if mesh.region is None else np.ascontiguousarray(mesh.region, dtype=np.uint8)
        mid = C.c_int()
        st = self.lib.fsim_mesh_upload(
            self.h, C.byref(mid), _d(rest), rest.shape[0], _i32(tets), tets.shape[0],
            pinned.ctypes.data_as(_U8), _i32(tris), tris.shape[0], rp.ctypes.data_as(_I64),
            _i32(col), _d(val), rp.shape[0] - 1,
            region.ctypes.data_as(_U8) if region is not None else None)
        _chk(st, "fsim_mesh_upload")
        return Mesh(self, mid.value, rest.shape[0], tets.shape[0], rp.shape[0] - 1)


class Mesh:
    """A mesh resident in a Context (thin wrapper over the mesh id)."""

    def __init__(self, ctx: Context, mid: int, n: int, T: int, Ns: int):
        self.ctx, self.id, self.n, self.T, self.Ns = ctx, mid, n, T, Ns
        self.lib = ctx.lib

    def prefactor(self, params: Params):
        _chk(self.lib.fsim_prefactor(self.ctx.h, self.id, C.byref(params)), "fsim_prefactor")

    def set_actuation(self, fiber, stretch):
        f = np.ascontiguousarray(fiber, dtype=np.float64)
        a = np.ascontiguousarray(stretch, dtype=np.float64)
        _chk(self.lib.fsim_set_actuation(self.ctx.h, self.id, _d(f), _d(a)), "fsim_set_actuation")

    def set_actuation_dev(self, fiber_ptr: int, stretch_ptr: int):
        _chk(self.lib.fsim_set_actuation_dev(self.ctx.h, self.id, C.c_void_p(fiber_ptr),
                                             C.c_void_p(stretch_ptr)), "fsim_set_actuation_dev")

    def info(self) -> dict:
        i = MeshInfo()
        _chk(self.lib.fsim_mesh_info_get(self.ctx.h, self.id, C.byref(i)), "fsim_mesh_info_get")
        return i.as_dict()

    def solve_frame(self, x_init=None, precision=FP64, check=True):
        """Returns (status, stats dict); positions stay resident."""
        st = FrameStats()
        x = None if x_init is None else np.ascontiguousarray(x_init, dtype=np.float64).reshape(-1)
        rc = self.lib.fsim_solve_frame(self.ctx.h, self.id, _d(x), int(precision), C.byref(st))
        if check and rc not in (FSIM_OK,):
            raise FsimError(rc, "fsim_solve_frame")
        return rc, st.as_dict()

    def solve_frame_dev(self, x_init_ptr=None, precision=FP64):
        st = FrameStats()
        rc = self.lib.fsim_solve_frame_dev(self.ctx.h, self.id,
                                           C.c_void_p(x_init_ptr) if x_init_ptr else None,
                                           int(precision), C.byref(st))
        return rc, st.as_dict()

    def positions(self) -> np.ndarray:
        out = np.empty((self.n, 3))
        _chk(self.lib.fsim_read_positions(self.ctx.h, self.id, _d(out)), "fsim_read_positions")
        return out

    def read_positions_dev(self, ptr: int):
        _chk(self.lib.fsim_read_positions_dev(self.ctx.h, self.id, C.c_void_p(ptr)),
             "fsim_read_positions_dev")

    def contacts(self, cap: int = 1 << 22):
        keys = np.empty((cap, 3), dtype=np.int32)
        cnt = C.c_int64()
        _chk(self.lib.fsim_read_contacts(self.ctx.h, self.id, _i32(keys), cap, C.byref(cnt)),
             "fsim_read_contacts")
        return keys[: cnt.value].copy()

    # ---- step-level entry points ------------------------------------------
    def _x(self, x):
        return np.ascontiguousarray(x, dtype=np.float64).reshape(-1)

    def eval_elastic(self, x, precision=FP64, want_proj=False):
        xx = self._x(x)
        E = C.c_double()
        g = np.empty((self.n, 3))
        P = np.empty((self.T, 9)) if want_proj else None
        _chk(self.lib.fsim_eval_elastic(self.ctx.h, self.id, _d(xx), int(precision), C.byref(E),
                                        _d(g), _d(P)), "fsim_eval_elastic")
        return (E.value, g, P) if want_proj else (E.value, g)

    def eval_proxy(self, x):
        xx = self._x(x)
        s = np.empty((self.Ns, 3))
        _chk(self.lib.fsim_eval_proxy(self.ctx.h, self.id, _d(xx), _d(s)), "fsim_eval_proxy")
        return s

    def eval_contacts(self, x, cap: int = 1 << 22):
        xx = self._x(x)
        keys = np.empty((cap, 3), dtype=np.int32)
        cnt = C.c_int64()
        B = C.c_double()
        _chk(self.lib.fsim_eval_contacts(self.ctx.h, self.id, _d(xx), _i32(keys), cap,
                                         C.byref(cnt), C.byref(B)), "fsim_eval_contacts")
        return keys[: cnt.value].copy(), B.value

    def eval_barrier(self, x, want_bcheck=True):
        xx = self._x(x)
        g = np.empty((self.n, 3))
        nc = C.c_int32()
        info = self.info()
        clist = np.empty(max(int(info["n2"]), 1), dtype=np.int32)
        cap = 9 * int(info["n2"]) ** 2 if want_bcheck else 0
        B = np.empty(max(cap, 1)) if want_bcheck else None
        _chk(self.lib.fsim_eval_barrier(self.ctx.h, self.id, _d(xx), _d(g), C.byref(nc),
                                        _i32(clist), _d(B), cap), "fsim_eval_barrier")
        k = nc.value
        Bc = B[: 9 * k * k].reshape(3 * k, 3 * k) if want_bcheck else None
        return g, clist[:k].copy(), Bc

    def eval_global_step(self, x, precision=FP64, want_path=False):
        xx = self._x(x)
        dx = np.empty((self.n, 3))
        path = C.c_int32(-2)
        _chk(self.lib.fsim_eval_global_step(self.ctx.h, self.id, _d(xx), int(precision), _d(dx),
                                            C.byref(path)), "fsim_eval_global_step")
        return (dx, path.value) if want_path else dx

    def eval_sigma_inv_mr(self, y, tensor_cores=True):
        """u = Sigma^-1 y for an (n2, ncols) array in x2 order, as the batches form it."""
        y = np.ascontiguousarray(y, dtype=np.float64)
        if y.ndim != 2:
            raise ValueError("y must be (n2, ncols)")
        u = np.empty_like(y)
        _chk(self.lib.fsim_eval_sigma_inv_mr(self.ctx.h, self.id, _d(y), int(y.shape[1]),
                                             1 if tensor_cores else 0, _d(u)),
             "fsim_eval_sigma_inv_mr")
        return u

    def eval_ccd(self, x, dx):
        xx, dd = self._x(x), self._x(dx)
        a = C.c_double()
        _chk(self.lib.fsim_eval_ccd(self.ctx.h, self.id, _d(xx), _d(dd), C.byref(a)),
             "fsim_eval_ccd")
        return a.value

    def eval_energy(self, x, precision=FP64):
        xx = self._x(x)
        E = C.c_double()
        gn = C.c_double()
        _chk(self.lib.fsim_eval_energy(self.ctx.h, self.id, _d(xx), int(precision), C.byref(E),
                                       C.byref(gn)), "fsim_eval_energy")
        return E.value, gn.value


def params_for(mesh, **kw) -> Params:
    """Default parameters with the workload's dhat / weight / tolerances."""
    p = default_params(dhat=mesh.dhat, weight_scale=mesh.weight_scale, tol_abs=mesh.tol_abs,
                       tol_rel=mesh.tol_rel)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


class Server:
    """Continuous-batching request server (fsim_server_*): `workers` frame
    solves run at once, each on its own CUDA stream and workspace slot."""

    def __init__(self, ctx: "Context", workers: int = 4, mem_budget_bytes: int = 0,
                 batch_frames: int = 0):
        self.ctx = ctx
        self.lib = ctx.lib
        cfg = ServerConfig(int(workers), int(batch_frames), int(mem_budget_bytes))
        h = _P()
        _chk(self.lib.fsim_server_create(ctx.h, C.byref(cfg), C.byref(h)), "fsim_server_create")
        self.h = h
        self._n = {}

    def submit(self, mesh: "Mesh", fiber, stretch, x_init=None, precision: int = 1) -> int:
        fiber = np.ascontiguousarray(fiber, dtype=np.float64)
        stretch = np.ascontiguousarray(stretch, dtype=np.float64)
        if fiber.size != 3 * mesh.T or stretch.size != mesh.T:
            raise ValueError("actuation arrays do not match the mesh")
        xi = None
        if x_init is not None:
            xi = np.ascontiguousarray(x_init, dtype=np.float64)
            if xi.size != 3 * mesh.n:
                raise ValueError("x_init does not match the mesh")
        req = Request(mesh.id, int(precision), _d(fiber), _d(stretch), _d(xi), 0, 0, None)
        t = C.c_int64()
        _chk(self.lib.fsim_server_submit(self.h, C.byref(req), C.byref(t)), "fsim_server_submit")
        self._n[int(t.value)] = mesh.n
        return int(t.value)

    def submit_dev(self, mesh: "Mesh", fiber_ptr: int, stretch_ptr: int, x_init_ptr: int = 0,
                   x_out_ptr: int = 0, precision: int = 1) -> int:
        """Request whose inputs (and output) are device arrays (FSIM_REQ_DEVICE);
        they must stay valid until the request completes."""
        dp = lambda p: C.cast(C.c_void_p(p), _D) if p else None
        req = Request(mesh.id, int(precision), dp(fiber_ptr), dp(stretch_ptr), dp(x_init_ptr),
                      FSIM_REQ_DEVICE, 0, dp(x_out_ptr))
        t = C.c_int64()
        _chk(self.lib.fsim_server_submit(self.h, C.byref(req), C.byref(t)), "fsim_server_submit")
        self._n[int(t.value)] = 0
        return int(t.value)

    def poll(self, ticket: int) -> bool:
        d = C.c_int32()
        _chk(self.lib.fsim_server_poll(self.h, int(ticket), C.byref(d)), "fsim_server_poll")
        return bool(d.value)

    def wait(self, ticket: int):
        """(status, positions (n, 3), stats dict, latency ms, queue ms)"""
        n = self._n.pop(int(ticket))
        x = np.empty((n, 3), dtype=np.float64) if n else None
        st = FrameStats()
        lat, q = C.c_double(), C.c_double()
        rc = self.lib.fsim_server_wait(self.h, int(ticket), _d(x), C.byref(st), C.byref(lat),
                                       C.byref(q))
        return int(rc), x, st.as_dict(), float(lat.value), float(q.value)

    def info(self) -> dict:
        i = ServerInfo()
        _chk(self.lib.fsim_server_info_get(self.h, C.byref(i)), "fsim_server_info_get")
        return i.as_dict()

    def close(self):
        if self.h:
            self.lib.fsim_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_frames(ctx: "Context", requests, workers: int = 4):
    """Batched form (fsim_solve_frames): requests are (mesh, fiber, stretch,
    x_init or None, precision) tuples; returns (status, [positions], [stats])."""
    n = len(requests)
    keep, reqs = [], (Request * max(n, 1))()
    outs = []
    for i, (mesh, fiber, stretch, x_init, prec) in enumerate(requests):
        f = np.ascontiguousarray(fiber, dtype=np.float64)
        a = np.ascontiguousarray(stretch, dtype=np.float64)
        xi = None if x_init is None else np.ascontiguousarray(x_init, dtype=np.float64)
        keep += [f, a, xi]
        reqs[i] = Request(mesh.id, int(prec), _d(f), _d(a), _d(xi), 0, 0, None)
        outs.append(np.empty((mesh.n, 3), dtype=np.float64))
    ptrs = (_D * max(n, 1))(*[_d(o) for o in outs])
    stats = (FrameStats * max(n, 1))()
    rc = ctx.lib.fsim_solve_frames(ctx.h, n, reqs, int(workers), ptrs, stats)
    return int(rc), outs, [stats[i].as_dict() for i in range(n)]


def solve_batch(ctx: "Context", requests, max_frames: int = 16, want_positions: bool = True):
    """Lock-step batched form (fsim_solve_batch): requests are (mesh, fiber,
    stretch, x_init or None) host tuples of ONE mesh, mixed precision;
    returns (status, [positions or None], [stats])."""
    n = len(requests)
    keep, reqs = [], (Request * max(n, 1))()
    outs = []
    for i, (mesh, fiber, stretch, x_init) in enumerate(requests):
        f = np.ascontiguousarray(fiber, dtype=np.float64)
        a = np.ascontiguousarray(stretch, dtype=np.float64)
        xi = None if x_init is None else np.ascontiguousarray(x_init, dtype=np.float64)
        keep += [f, a, xi]
        reqs[i] = Request(mesh.id, MIXED, _d(f), _d(a), _d(xi), 0, 0, None)
        outs.append(np.empty((mesh.n, 3), dtype=np.float64) if want_positions else None)
    ptrs = (_D * max(n, 1))(*[_d(o) for o in outs])
    stats = (FrameStats * max(n, 1))()
    rc = ctx.lib.fsim_solve_batch(ctx.h, n, reqs, int(max_frames), ptrs, stats)
    return int(rc), outs, [stats[i].as_dict() for i in range(n)]


def solve_batch_dev(ctx: "Context", mesh: "Mesh", fiber_ptrs, stretch_ptrs, x_init_ptrs,
                    x_out_ptrs, max_frames: int = 16):
    """Lock-step batched form with device inputs and outputs (FSIM_REQ_DEVICE):
    per request the device pointers of its fiber (3T), stretch (T), start
    positions (3n, or 0 for the rest pose) and output positions (3n, or 0).
    Returns (status, [stats])."""
    n = len(fiber_ptrs)
    dp = lambda p: C.cast(C.c_void_p(p), _D) if p else None
    reqs = (Request * max(n, 1))()
    for i in range(n):
        reqs[i] = Request(mesh.id, MIXED, dp(fiber_ptrs[i]), dp(stretch_ptrs[i]),
                          dp(x_init_ptrs[i]), FSIM_REQ_DEVICE, 0, dp(x_out_ptrs[i]))
    stats = (FrameStats * max(n, 1))()
    rc = ctx.lib.fsim_solve_batch(ctx.h, n, reqs, int(max_frames), None, stats)
    return int(rc), [stats[i].as_dict() for i in range(n)]


def select_region(rest, tets, pinned, radius: float, rings: int):
    """fsim_select_region: (proxy triangles in proxy-vertex numbering, proxy
    vertex ids) of the automatically selected collision region (host only)."""
    lib = load()
    X = np.ascontiguousarray(rest, dtype=np.float64).reshape(-1)
    tt = np.ascontiguousarray(tets, dtype=np.int32).reshape(-1)
    pn = None if pinned is None else np.ascontiguousarray(pinned, dtype=np.uint8)
    nt, nv = C.c_int64(), C.c_int64()
    n, T = X.size // 3, tt.size // 4
    _chk(lib.fsim_select_region(_d(X), n, _i32(tt), T, _u8(pn) if pn is not None else None,
                                float(radius), int(rings), None, 0, C.byref(nt), None, 0,
                                C.byref(nv)), "fsim_select_region")
    tris = np.empty((max(nt.value, 1), 3), dtype=np.int32)
    verts = np.empty(max(nv.value, 1), dtype=np.int32)
    _chk(lib.fsim_select_region(_d(X), n, _i32(tt), T, _u8(pn) if pn is not None else None,
                                float(radius), int(rings), _i32(tris), nt.value, C.byref(nt),
                                _i32(verts), nv.value, C.byref(nv)), "fsim_select_region")
    return tris[: nt.value].copy(), verts[: nv.value].copy()
