"""Python binding of the C ABI in include/lbkm.h (argument marshalling only).

Every step of the model runs in the CUDA library ``_lib/libpaper_lbkm.so``;
this module converts arguments (NumPy arrays for host data, torch CUDA tensors
for device data, torch streams) and raises on error codes. There is no CPU
fallback: if the library is missing or fails to load, importing the binding
raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libpaper_lbkm.so")

F64, F32 = 0, 1
RECOVER_F64, RECOVER_DF32 = 0, 1
BC_PERIODIC, BC_ZERO_GRADIENT, BC_WALL, BC_DIRICHLET, BC_SPECULAR, BC_SIDES = 0, 1, 2, 3, 4, 5

STATUS = {0: "LBKM_OK", 1: "LBKM_EINVAL", 2: "LBKM_ENOMEM", 3: "LBKM_ECUDA",
          4: "LBKM_ESINGULAR", 5: "LBKM_EUNSTABLE", 6: "LBKM_ETIMEOUT", 7: "LBKM_ESTATE"}

EXPORTED = ["lbkm_default_params", "lbkm_create", "lbkm_destroy", "lbkm_set_stream",
            "lbkm_init_fields", "lbkm_step", "lbkm_sync", "lbkm_steps_taken", "lbkm_macros",
            "lbkm_tne", "lbkm_tne_history", "lbkm_state_bytes", "lbkm_get_state",
            "lbkm_set_state", "lbkm_last_error", "lbkm_version", "lbkm_tne_noalloc",
            "lbkm_create_batched", "lbkm_instances", "lbkm_tne_instances", "lbkm_autotune",
            "lbkm_set_wait_limit", "lbkm_grad", "lbkm_objective_value"]
EXPORTED24 = ["lbkm24_default_params", "lbkm24_create", "lbkm24_destroy", "lbkm24_init_fields",
              "lbkm24_step", "lbkm24_sync", "lbkm24_steps_taken", "lbkm24_macros", "lbkm24_tne",
              "lbkm24_tne_history", "lbkm24_state_bytes", "lbkm24_get_state", "lbkm24_set_state",
              "lbkm24_last_error"]


class LbkmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS.get(code, code), msg))
        self.code = code


# caller-owned device memory (lbkm_params.alloc / free)
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("recovery", ctypes.c_int32),
        ("gamma", ctypes.c_double), ("Pr", ctypes.c_double),
        ("orbit_kind", ctypes.c_int32 * 4), ("orbit_speed", ctypes.c_double * 4),
        ("orbit_eta", ctypes.c_double * 4), ("S", ctypes.c_double * 16),
        ("Q", ctypes.c_double), ("omega1", ctypes.c_double), ("omega2", ctypes.c_double),
        ("T_ig", ctypes.c_double),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dt", ctypes.c_double),
        ("bc_x", ctypes.c_int32), ("bc_y", ctypes.c_int32),
        ("tne_every", ctypes.c_int32), ("tne_capacity", ctypes.c_int32),
        ("wall_ux", ctypes.c_double * 2), ("wall_uy", ctypes.c_double * 2),
        ("wall_T", ctypes.c_double * 2),
        ("side_bc", ctypes.c_int32 * 4), ("side_rho", ctypes.c_double * 4),
        ("side_ux", ctypes.c_double * 4), ("side_uy", ctypes.c_double * 4),
        ("side_T", ctypes.c_double * 4), ("side_lam", ctypes.c_double * 4),
        ("time_scheme", ctypes.c_int32),
        ("collision", ctypes.c_int32),
        ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", ctypes.c_void_p),
    ]


class TorchAllocator:
    """Device memory of a handle from torch's caching allocator, through lbkm_params.alloc
    and free: each block is a uint8 CUDA tensor held here until the library frees it
    (torch's blocks are aligned to 512 bytes). Pass as Solver(..., allocator=...)."""

    def __init__(self):
        self.blocks = {}
        self.allocated = 0   # blocks handed out so far
        self._alloc = ALLOC_FN(self._a)
        self._free = FREE_FN(self._f)

    def _a(self, nbytes, stream, ctx):
        try:
            import torch
            t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
        except Exception:  # out of memory: the library reports LBKM_ENOMEM
            return None
        self.blocks[t.data_ptr()] = t
        self.allocated += 1
        return t.data_ptr()

    def _f(self, ptr, stream, ctx):
        self.blocks.pop(ptr, None)

    def install(self, params):
        params.alloc, params.free = self._alloc, self._free


class Objective(ctypes.Structure):
    _fields_ = [("rho_target", ctypes.c_void_p), ("w_mismatch", ctypes.c_double),
                ("w_tne", ctypes.c_double), ("steps", ctypes.c_int64),
                ("checkpoint_every", ctypes.c_int32)]


class GradOut(ctypes.Structure):
    _fields_ = [("J", ctypes.c_double), ("J_mismatch", ctypes.c_double),
                ("J_tne", ctypes.c_double), ("dS", ctypes.c_double * 16),
                ("dQ", ctypes.c_double), ("domega1", ctypes.c_double),
                ("drho0", ctypes.c_void_p), ("df0", ctypes.c_void_p),
                ("domega2", ctypes.c_double)]


class Params24(ctypes.Structure):
    """lbkm24_params: the paper's D2V24 (include/lbkm24.h)."""
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("gamma", ctypes.c_double), ("v", ctypes.c_double * 3), ("eta", ctypes.c_double * 3),
        ("S", ctypes.c_double * 24),
        ("Q", ctypes.c_double), ("omega1", ctypes.c_double), ("omega2", ctypes.c_double),
        ("T_ig", ctypes.c_double),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dt", ctypes.c_double),
        ("bc_x", ctypes.c_int32), ("bc_y", ctypes.c_int32),
        ("tne_every", ctypes.c_int32), ("tne_capacity", ctypes.c_int32),
        ("collision", ctypes.c_int32),
        ("side_bc", ctypes.c_int32 * 4), ("side_rho", ctypes.c_double * 4),
        ("side_ux", ctypes.c_double * 4), ("side_uy", ctypes.c_double * 4),
        ("side_T", ctypes.c_double * 4), ("side_lam", ctypes.c_double * 4),
    ]


def _tne_fields(nv):
    return [("sum", ctypes.c_double * nv), ("abs_sum", ctypes.c_double * nv),
            ("min", ctypes.c_double * nv), ("max", ctypes.c_double * nv),
            ("d_sum", ctypes.c_double), ("d2_sum", ctypes.c_double), ("step", ctypes.c_int64)]


class TneGlobal(ctypes.Structure):
    _fields_ = _tne_fields(16)

    def as_dict(self):
        return {"sum": np.array(self.sum[:]), "abs_sum": np.array(self.abs_sum[:]),
                "min": np.array(self.min[:]), "max": np.array(self.max[:]),
                "d_sum": self.d_sum, "d2_sum": self.d2_sum, "step": int(self.step)}


class TneGlobal24(ctypes.Structure):
    _fields_ = _tne_fields(24)
    as_dict = TneGlobal.as_dict


_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p


def load():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("CUDA library %s is missing: run __graft_entry__.build() "
                          "(nvcc, sm_103a) first; there is no CPU fallback" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    H = ctypes.c_void_p
    lib.lbkm_default_params.argtypes = [ctypes.POINTER(Params)]
    lib.lbkm_default_params.restype = None
    lib.lbkm_create.argtypes = [ctypes.POINTER(Params), _vp, ctypes.POINTER(H)]
    lib.lbkm_destroy.argtypes = [H]
    lib.lbkm_destroy.restype = None
    lib.lbkm_set_stream.argtypes = [H, _vp]
    lib.lbkm_init_fields.argtypes = [H, _vp, _vp, _vp, _vp, _vp, ctypes.c_int]
    lib.lbkm_step.argtypes = [H, ctypes.c_int64]
    lib.lbkm_sync.argtypes = [H]
    lib.lbkm_steps_taken.argtypes = [H]
    lib.lbkm_steps_taken.restype = ctypes.c_int64
    lib.lbkm_macros.argtypes = [H] + [_vp] * 6 + [ctypes.c_int]
    lib.lbkm_tne.argtypes = [H, _vp, ctypes.POINTER(TneGlobal), ctypes.c_int]
    lib.lbkm_tne_history.argtypes = [H, ctypes.POINTER(TneGlobal), ctypes.c_int32,
                                     ctypes.POINTER(ctypes.c_int32)]
    lib.lbkm_state_bytes.argtypes = [H]
    lib.lbkm_state_bytes.restype = ctypes.c_size_t
    lib.lbkm_get_state.argtypes = [H, _vp, ctypes.c_int]
    lib.lbkm_set_state.argtypes = [H, _vp, ctypes.c_int]
    lib.lbkm_last_error.argtypes = [H]
    lib.lbkm_last_error.restype = ctypes.c_char_p
    lib.lbkm_version.restype = ctypes.c_int32
    lib.lbkm_tne_noalloc.argtypes = [ctypes.POINTER(Params), _vp, ctypes.c_int64, _vp, _vp, _vp]
    lib.lbkm_tne_noalloc.restype = ctypes.c_int
    lib.lbkm_create_batched.argtypes = [ctypes.POINTER(Params), ctypes.c_int32, _vp, _vp, _vp,
                                        _vp, _vp, ctypes.POINTER(H)]
    lib.lbkm_create_batched.restype = ctypes.c_int
    lib.lbkm_instances.argtypes = [H]
    lib.lbkm_instances.restype = ctypes.c_int32
    lib.lbkm_tne_instances.argtypes = [H, ctypes.POINTER(TneGlobal)]
    lib.lbkm_tne_instances.restype = ctypes.c_int
    lib.lbkm_autotune.argtypes = [H, ctypes.c_int32, _vp]
    lib.lbkm_autotune.restype = ctypes.c_int
    lib.lbkm_grad.argtypes = [H, ctypes.POINTER(Objective), ctypes.POINTER(GradOut)]
    lib.lbkm_grad.restype = ctypes.c_int
    D = ctypes.POINTER(ctypes.c_double)
    lib.lbkm_objective_value.argtypes = [H, ctypes.POINTER(Objective), D, D, D]
    lib.lbkm_objective_value.restype = ctypes.c_int
    lib.lbkm_set_wait_limit.argtypes = [H, ctypes.c_int64, ctypes.c_int32]
    lib.lbkm_set_wait_limit.restype = ctypes.c_int
    for name in ("lbkm_create", "lbkm_set_stream", "lbkm_init_fields", "lbkm_step", "lbkm_sync",
                 "lbkm_macros", "lbkm_tne", "lbkm_tne_history", "lbkm_get_state",
                 "lbkm_set_state"):
        getattr(lib, name).restype = ctypes.c_int
    P24 = ctypes.POINTER(Params24)
    lib.lbkm24_default_params.argtypes = [P24]
    lib.lbkm24_default_params.restype = None
    lib.lbkm24_create.argtypes = [P24, _vp, ctypes.POINTER(H)]
    lib.lbkm24_destroy.argtypes = [H]
    lib.lbkm24_destroy.restype = None
    lib.lbkm24_init_fields.argtypes = [H, _vp, _vp, _vp, _vp, _vp, ctypes.c_int]
    lib.lbkm24_step.argtypes = [H, ctypes.c_int64]
    lib.lbkm24_sync.argtypes = [H]
    lib.lbkm24_steps_taken.argtypes = [H]
    lib.lbkm24_steps_taken.restype = ctypes.c_int64
    lib.lbkm24_macros.argtypes = [H] + [_vp] * 6 + [ctypes.c_int]
    lib.lbkm24_tne.argtypes = [H, _vp, ctypes.POINTER(TneGlobal24), ctypes.c_int]
    lib.lbkm24_tne_history.argtypes = [H, ctypes.POINTER(TneGlobal24), ctypes.c_int32,
                                       ctypes.POINTER(ctypes.c_int32)]
    lib.lbkm24_state_bytes.argtypes = [H]
    lib.lbkm24_state_bytes.restype = ctypes.c_size_t
    lib.lbkm24_get_state.argtypes = [H, _vp, ctypes.c_int]
    lib.lbkm24_set_state.argtypes = [H, _vp, ctypes.c_int]
    lib.lbkm24_last_error.argtypes = [H]
    lib.lbkm24_last_error.restype = ctypes.c_char_p
    for name in ("create", "init_fields", "step", "sync", "macros", "tne", "tne_history",
                 "get_state", "set_state"):
        getattr(lib, "lbkm24_" + name).restype = ctypes.c_int
    _lib = lib
    return lib


def default_params(**kw) -> Params:
    p = Params()
    load().lbkm_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if k in ("orbit_kind", "orbit_speed", "orbit_eta", "S"):
            arr = getattr(p, k)
            vals = np.broadcast_to(np.asarray(v), (len(arr),))
            for i in range(len(arr)):
                arr[i] = vals[i].item()
        elif k == "bc":
            p.bc_x, p.bc_y = v
        elif k == "walls":  # ((ux, uy, T) below row 0, (ux, uy, T) above row ny-1)
            for side in (0, 1):
                p.wall_ux[side], p.wall_uy[side], p.wall_T[side] = map(float, v[side])
        elif k == "sides":  # 4 x (code, rho, ux, uy, T, lambda): x = 0, x = nx, y = 0, y = ny
            for j, (code, r, u, w, T, lam) in enumerate(v):
                p.side_bc[j] = int(code)
                p.side_rho[j], p.side_ux[j], p.side_uy[j], p.side_T[j], p.side_lam[j] = (
                    float(r), float(u), float(w), float(T), float(lam))
        else:
            setattr(p, k, v)
    return p


def default_params24(**kw) -> Params24:
    """lbkm24_params from the defaults (the steady-detonation set of Sec. IV.A) and
    keyword overrides (v, eta: 3 values; S: 24 values or one; bc: (bc_x, bc_y))."""
    p = Params24()
    load().lbkm24_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if k in ("v", "eta", "S"):
            arr = getattr(p, k)
            vals = np.broadcast_to(np.asarray(v, float), (len(arr),))
            for i in range(len(arr)):
                arr[i] = float(vals[i])
        elif k == "bc":
            p.bc_x, p.bc_y = v
        elif k == "sides":  # 4 x (code, rho, ux, uy, T, lambda): x = 0, x = nx, y = 0, y = ny
            for j, (code, r, u, w, T, lam) in enumerate(v):
                p.side_bc[j] = int(code)
                p.side_rho[j], p.side_ux[j], p.side_uy[j], p.side_T[j], p.side_lam[j] = (
                    float(r), float(u), float(w), float(T), float(lam))
        else:
            setattr(p, k, v)
    return p


class _Api:
    """The C functions of one handle type, by name without their prefix."""

    def __init__(self, lib, prefix):
        self._lib, self._prefix = lib, prefix

    def __getattr__(self, name):
        return getattr(self._lib, self._prefix + name)


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _is_torch(a):
    return type(a).__module__.startswith("torch")


class Solver:
    """One MRT-LBKM grid on the GPU (a handle of the C ABI), 16-velocity model."""

    NV = 16
    _PREFIX = "lbkm_"
    _Tne = TneGlobal

    def __init__(self, params: Params = None, stream=None, allocator=None, **kw):
        lib = load()
        self._lib = lib
        self._api = _Api(lib, self._PREFIX)
        self.params = params if params is not None else self._default(**kw)
        self.allocator = allocator  # kept alive as long as the handle
        if allocator is not None:
            allocator.install(self.params)
        self.nx, self.ny = int(self.params.nx), int(self.params.ny)
        h = ctypes.c_void_p()
        rc = self._api.create(ctypes.byref(self.params), ctypes.c_void_p(_stream_ptr(stream)),
                              ctypes.byref(h))
        if rc != 0:
            raise LbkmError(rc, self._api.last_error(None).decode())
        self._h = h

    @staticmethod
    def _default(**kw):
        return default_params(**kw)

    @classmethod
    def batched(cls, inst_nx, inst_S=None, inst_Q=None, inst_omega1=None, params=None,
                stream=None, **kw):
        """Many 1-D instances in one handle (lbkm_create_batched); fields are the
        instances concatenated in order."""
        self = cls.__new__(cls)
        lib = load()
        self._lib = lib
        self._api = _Api(lib, cls._PREFIX)
        kw.setdefault("precision", F32)
        self.params = params if params is not None else default_params(**kw)
        nxs = np.ascontiguousarray(inst_nx, dtype=np.int32)
        keep = [nxs]

        def arr(a, shape):
            if a is None:
                return None
            b = np.ascontiguousarray(np.broadcast_to(np.asarray(a, np.float64), shape))
            keep.append(b)
            return b.ctypes.data
        h = ctypes.c_void_p()
        rc = lib.lbkm_create_batched(ctypes.byref(self.params), len(nxs),
                                     ctypes.c_void_p(nxs.ctypes.data),
                                     ctypes.c_void_p(arr(inst_S, (len(nxs), 16))),
                                     ctypes.c_void_p(arr(inst_Q, (len(nxs),))),
                                     ctypes.c_void_p(arr(inst_omega1, (len(nxs),))),
                                     ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(h))
        if rc != 0:
            raise LbkmError(rc, lib.lbkm_last_error(None).decode())
        self._h = h
        self.nx, self.ny = int(nxs.sum()), 1
        self.inst_nx = nxs.copy()
        return self

    @property
    def instances(self):
        return int(self._lib.lbkm_instances(self._h))

    def tne_instances(self):
        n = self.instances
        buf = (TneGlobal * n)()
        self._check(self._lib.lbkm_tne_instances(self._h, buf))
        return [buf[i].as_dict() for i in range(n)]

    def autotune(self, trial_steps=3):
        out = (ctypes.c_int32 * 3)()
        self._check(self._lib.lbkm_autotune(self._h, int(trial_steps), out))
        return tuple(out)

    def grad(self, rho_target, steps, w_mismatch=1.0, w_tne=1.0, checkpoint_every=64,
             want_f0=False):
        """lbkm_grad: J and dJ/d(S, Q, omega1, omega2, rho0 [, f0]) over `steps` steps from the
        current state (which is left unchanged)."""
        rt = np.ascontiguousarray(np.broadcast_to(np.asarray(rho_target, np.float64),
                                                  (self.nx,)))
        ob = Objective(rt.ctypes.data, float(w_mismatch), float(w_tne), int(steps),
                       int(checkpoint_every))
        drho0 = np.zeros(self.nx)
        df0 = np.zeros((16, self.nx)) if want_f0 else None
        out = GradOut()
        out.drho0 = drho0.ctypes.data
        out.df0 = df0.ctypes.data if want_f0 else None
        self._check(self._lib.lbkm_grad(self._h, ctypes.byref(ob), ctypes.byref(out)))
        return {"J": out.J, "J_mismatch": out.J_mismatch, "J_tne": out.J_tne,
                "dS": np.array(out.dS[:]), "dQ": out.dQ, "domega1": out.domega1,
                "domega2": out.domega2,
                "drho0": drho0, "df0": df0}

    def objective(self, rho_target, steps, w_mismatch=1.0, w_tne=1.0, checkpoint_every=64):
        """lbkm_objective_value: the J of `grad` (and its two terms) without the derivative."""
        rt = np.ascontiguousarray(np.broadcast_to(np.asarray(rho_target, np.float64),
                                                  (self.nx,)))
        ob = Objective(rt.ctypes.data, float(w_mismatch), float(w_tne), int(steps),
                       int(checkpoint_every))
        J, Jm, Jt = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.lbkm_objective_value(self._h, ctypes.byref(ob), ctypes.byref(J),
                                                   ctypes.byref(Jm), ctypes.byref(Jt)))
        return {"J": J.value, "J_mismatch": Jm.value, "J_tne": Jt.value}

    def set_wait_limit(self, timeout_ns, phantom_blocks=0):
        self._check(self._lib.lbkm_set_wait_limit(self._h, int(timeout_ns), int(phantom_blocks)))

    # ------------------------------------------------------------------
    def _check(self, rc):
        if rc != 0:
            raise LbkmError(rc, self._api.last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._api.destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------------
    def _field(self, a, keep):
        shape = (self.ny, self.nx)
        if a is None:
            return None, 0
        if _is_torch(a):
            import torch
            t = a.to(dtype=torch.float64).expand(shape).contiguous()
            keep.append(t)
            return t.data_ptr(), 1 if t.is_cuda else 0
        arr = np.ascontiguousarray(np.broadcast_to(np.asarray(a, np.float64), shape))
        keep.append(arr)
        return arr.ctypes.data, 0

    def init_fields(self, rho, ux, uy, T, lam=None):
        keep = []
        ptrs, dev = [], set()
        for a in (rho, ux, uy, T, lam):
            p, d = self._field(a, keep)
            ptrs.append(p)
            if a is not None:
                dev.add(d)
        if len(dev) != 1:
            raise ValueError("fields must be all host arrays or all CUDA tensors")
        self._check(self._api.init_fields(self._h, *[ctypes.c_void_p(p) for p in ptrs],
                                               dev.pop()))

    def step(self, n=1):
        self._check(self._api.step(self._h, int(n)))

    def sync(self):
        self._check(self._api.sync(self._h))

    @property
    def steps_taken(self):
        return int(self._api.steps_taken(self._h))

    def _out_ptr(self, a, name, device):
        # a caller's output buffer: ny * nx contiguous float64 values where `device` says
        n = self.ny * self.nx
        if _is_torch(a):
            import torch
            ok = (a.dtype == torch.float64 and a.is_contiguous() and a.numel() == n
                  and a.is_cuda == bool(device))
            if not ok:
                raise ValueError("out[%r] must be a contiguous float64 %s tensor of %d values"
                                 % (name, "CUDA" if device else "CPU", n))
            return a.data_ptr()
        if device:
            raise ValueError("out[%r] must be a CUDA tensor when device=True" % name)
        if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous
                and a.size == n and a.flags.writeable):
            raise ValueError("out[%r] must be a writable C-contiguous float64 array of %d values"
                             % (name, n))
        return a.ctypes.data

    def macros(self, device=False, out=None):
        """rho, ux, uy, T, p, lambda of the current state; with out (a dict of
        preallocated host or CUDA tensors/arrays) the results land there."""
        names = ("rho", "ux", "uy", "T", "p", "lam")
        if out is not None:
            ptrs = [self._out_ptr(out[k], k, device) if k in out else None for k in names]
            self._check(self._api.macros(self._h, *[ctypes.c_void_p(p) for p in ptrs],
                                              1 if device else 0))
            return out
        if device:
            import torch
            out = {k: torch.empty((self.ny, self.nx), dtype=torch.float64, device="cuda")
                   for k in names}
            ptrs = [out[k].data_ptr() for k in names]
        else:
            out = {k: np.empty((self.ny, self.nx)) for k in names}
            ptrs = [out[k].ctypes.data for k in names]
        self._check(self._api.macros(self._h, *[ctypes.c_void_p(p) for p in ptrs],
                                          1 if device else 0))
        return out

    def tne(self, fields=True, device=False):
        g = self._Tne()
        delta = None
        ptr = None
        if fields:
            if device:
                import torch
                delta = torch.empty((self.NV, self.ny, self.nx), dtype=torch.float64,
                                    device="cuda")
                ptr = delta.data_ptr()
            else:
                delta = np.empty((self.NV, self.ny, self.nx))
                ptr = delta.ctypes.data
        self._check(self._api.tne(self._h, ctypes.c_void_p(ptr), ctypes.byref(g),
                                       1 if device else 0))
        return delta, g.as_dict()

    def tne_history(self, max_records=None):
        cap = int(self.params.tne_capacity) if max_records is None else int(max_records)
        buf = (self._Tne * max(cap, 1))()
        n = ctypes.c_int32()
        self._check(self._api.tne_history(self._h, buf, cap, ctypes.byref(n)))
        return [buf[i].as_dict() for i in range(n.value)]

    def state_bytes(self):
        return int(self._api.state_bytes(self._h))

    def get_state(self, device=False):
        """State snapshot as bytes: a NumPy uint8 array, or a CUDA uint8 tensor."""
        if device:
            import torch
            buf = torch.empty(self.state_bytes(), dtype=torch.uint8, device="cuda")
            self._check(self._api.get_state(self._h, ctypes.c_void_p(buf.data_ptr()), 1))
            return buf
        buf = np.empty(self.state_bytes(), np.uint8)
        self._check(self._api.get_state(self._h, ctypes.c_void_p(buf.ctypes.data), 0))
        return buf

    def set_state(self, buf):
        if _is_torch(buf) and buf.is_cuda:
            import torch
            if not (buf.dtype == torch.uint8 and buf.is_contiguous()
                    and buf.numel() == self.state_bytes()):
                raise ValueError("a CUDA state buffer must be a contiguous uint8 tensor of %d "
                                 "bytes" % self.state_bytes())
            self._check(self._api.set_state(self._h, ctypes.c_void_p(buf.data_ptr()), 1))
            return
        if _is_torch(buf):
            buf = buf.numpy()
        buf = np.ascontiguousarray(buf, np.uint8)
        if buf.size != self.state_bytes():
            raise ValueError("state buffer has %d bytes, expected %d" % (buf.size,
                                                                        self.state_bytes()))
        self._check(self._api.set_state(self._h, ctypes.c_void_p(buf.ctypes.data), 0))

    def planes_device(self):
        """Current f_1..f_NV and lambda as a CUDA tensor [NV+1, ny, nx] in the state's dtype."""
        import torch
        raw = self.get_state(device=True)
        dt = torch.float64 if self.params.precision == F64 else torch.float32
        npl = self.NV + 1
        n = npl * self.ny * self.nx * (8 if dt == torch.float64 else 4)
        return raw[:n].view(dt).view(npl, self.ny, self.nx)

    def f_planes(self):
        """Current f_1..f_NV and lambda as FP64 NumPy arrays [NV+1, ny, nx] (state copy)."""
        raw = self.get_state()
        dt = np.float64 if self.params.precision == F64 else np.float32
        npl = self.NV + 1
        n = npl * self.ny * self.nx
        return np.frombuffer(raw[: n * np.dtype(dt).itemsize].tobytes(), dt).reshape(
            npl, self.ny, self.nx).astype(np.float64)


class Solver24(Solver):
    """One grid of the paper's D2V24 model on the GPU (a handle of include/lbkm24.h):
    the same calls as Solver (init_fields, step, sync, macros, tne, tne_history,
    get_state, set_state), with 24 velocities; no batched instances or gradients."""

    NV = 24
    _PREFIX = "lbkm24_"
    _Tne = TneGlobal24

    @staticmethod
    def _default(**kw):
        return default_params24(**kw)

    def _not_here(self, *a, **k):
        raise NotImplementedError("the D2V24 handle has no batched instances or gradients")

    batched = autotune = grad = set_wait_limit = tne_instances = instances = _not_here


def tne_noalloc(params: Params, state_ptr: int, pitch: int, delta_ptr, out_ptr: int, stream=None):
    """lbkm_tne_noalloc: TNE record of a caller-owned device state, allocating nothing.
    All pointers are device addresses; out receives one lbkm_tne_global (536 bytes)."""
    lib = load()
    rc = lib.lbkm_tne_noalloc(ctypes.byref(params), ctypes.c_void_p(state_ptr), int(pitch),
                              ctypes.c_void_p(delta_ptr), ctypes.c_void_p(out_ptr),
                              ctypes.c_void_p(_stream_ptr(stream)))
    if rc != 0:
        raise LbkmError(rc, lib.lbkm_last_error(None).decode())


def version():
    return int(load().lbkm_version())
