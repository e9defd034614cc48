"""Shared helpers of the GPU parity tests: one seeded configuration drives both the
CUDA library (through the C ABI) and the FP64 oracle."""
import numpy as np

from oracle import oracle
from paper_1411_6697_gb300 import lbkm

KEYS = ("gamma", "orbit_kind", "orbit_speed", "orbit_eta", "S", "Q", "omega1", "omega2",
        "T_ig", "dx", "dt", "walls", "sides", "time_scheme", "collision")


def solver(params, precision, recovery=0, tne_every=0, tne_capacity=1, allocator=None, **over):
    p = dict(params)
    p.update(over)
    kw = {k: p[k] for k in KEYS if k in p}
    return lbkm.Solver(nx=p["nx"], ny=p["ny"], precision=precision, recovery=recovery,
                       dy=p.get("dy", p["dx"]), bc=(p["bc_x"], p["bc_y"]),
                       tne_every=tne_every, tne_capacity=tne_capacity, allocator=allocator, **kw)


def make_oracle(params, **over):
    p = dict(params)
    p.update(over)
    nx, ny = p.pop("nx"), p.pop("ny")
    return oracle.Oracle(nx, ny, **p)


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def state_bytes(planes, precision, step=0):
    dt = np.float64 if precision == lbkm.F64 else np.float32
    return np.concatenate([np.ascontiguousarray(planes, dtype=dt).ravel().view(np.uint8),
                           np.array([step], np.int64).view(np.uint8)])


TOL = {lbkm.F64: 1e-12, lbkm.F32: 2e-5}
