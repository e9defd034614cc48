"""lbkm_tne_noalloc, the entry point for callers that cannot allocate device memory
(for example because their own memory pool already owns the device, or because a
latency-bound loop cannot afford cudaMalloc's implicit synchronisation). It must give
the same TNE record as the handle-based lbkm_tne, call after call, while its scratch
lives in a fixed array inside the library. Collected last on purpose."""
import ctypes

import numpy as np
import pytest

import lbkm_inputs as li
from paper_1411_6697_gb300 import lbkm

pytestmark = pytest.mark.gpu

REC_DOUBLES = ctypes.sizeof(lbkm.TneGlobal) // 8


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _record(t):
    raw = t.cpu().numpy()
    g = lbkm.TneGlobal.from_buffer_copy(raw.tobytes())
    return g.as_dict()


def _compare(g, g_ref, tol):
    scale = g_ref["abs_sum"].max()
    for k in ("sum", "abs_sum"):
        assert np.abs(g[k] - g_ref[k]).max() <= tol * scale, k
    for k in ("min", "max"):
        assert np.abs(g[k] - g_ref[k]).max() <= tol * np.abs(g_ref[k]).max(), k
    assert abs(g["d_sum"] - g_ref["d_sum"]) <= tol * g_ref["d_sum"]
    assert abs(g["d2_sum"] - g_ref["d2_sum"]) <= tol * g_ref["d2_sum"]
    assert g["step"] == -1


def _solver(nx, ny, prec, steps):
    x = np.arange(nx)[None, :] / nx
    y = np.arange(ny)[:, None] / ny
    s = lbkm.Solver(nx=nx, ny=ny, precision=prec, bc=(0, 0), Q=1.0, omega1=2e3, T_ig=1.05,
                    S=np.linspace(5e3, 1e5, 16), **li.DEFAULT_ORBITS)
    s.init_fields(1 + 0.1 * np.sin(2 * np.pi * x) + 0 * y, 0.2 * np.cos(2 * np.pi * y) + 0 * x,
                  -0.1 * np.sin(2 * np.pi * x) + 0 * y, 1.1 + 0.1 * np.cos(2 * np.pi * (x + y)),
                  0.3 + 0 * x * y)
    s.step(steps)
    return s


def _padded_state(s, prec, pad):
    """The solver's 17 planes copied into a caller-owned buffer whose rows are nx + pad
    elements apart; the padding holds NaN, so a read of it would show in the record."""
    import torch
    nx, ny = s.nx, s.ny
    dt = torch.float64 if prec == lbkm.F64 else torch.float32
    raw = s.get_state(device=True)
    planes = raw[: 17 * ny * nx * raw.new_empty(0, dtype=dt).element_size()].view(dt)
    buf = torch.full((17, ny, nx + pad), float("nan"), dtype=dt, device="cuda")
    buf[:, :, :nx] = planes.view(17, ny, nx)
    return buf


@pytest.mark.parametrize("prec", [lbkm.F64, lbkm.F32], ids=["f64", "f32"])
def test_noalloc_tne_matches_handle_tne(prec):
    import torch
    nx, ny = 150, 61
    s = _solver(nx, ny, prec, 12)
    state = s.get_state(device=True)  # [17][ny][nx] + step counter
    out = torch.zeros(REC_DOUBLES, dtype=torch.float64, device="cuda")
    delta = torch.empty((16, ny, nx), dtype=torch.float64, device="cuda")
    d_ref, g_ref = s.tne(fields=True)
    for _ in range(2):  # two calls in a row reuse the same scratch
        out.zero_()
        delta.fill_(np.nan)
        lbkm.tne_noalloc(s.params, state.data_ptr(), nx, delta.data_ptr(), out.data_ptr())
        torch.cuda.synchronize()
        _compare(_record(out), g_ref, 1e-12)
        assert np.abs(delta.cpu().numpy() - d_ref).max() <= 1e-12 * np.abs(d_ref).max()
    s.close()


@pytest.mark.parametrize("prec", [lbkm.F64, lbkm.F32], ids=["f64", "f32"])
def test_noalloc_tne_many_blocks_padded_pitch(prec):
    """350,000 cells (43 blocks, so the last block combines many partials) in a buffer
    with pitch nx + 32, two calls in a row."""
    import torch
    nx, ny, pad = 700, 500, 32
    s = _solver(nx, ny, prec, 3)
    buf = _padded_state(s, prec, pad)
    out = torch.zeros(REC_DOUBLES, dtype=torch.float64, device="cuda")
    delta = torch.empty((16, ny, nx), dtype=torch.float64, device="cuda")
    d_ref, g_ref = s.tne(fields=True)
    for _ in range(2):
        out.zero_()
        delta.fill_(np.nan)
        lbkm.tne_noalloc(s.params, buf.data_ptr(), nx + pad, delta.data_ptr(), out.data_ptr())
        torch.cuda.synchronize()
        _compare(_record(out), g_ref, 1e-12)
        assert np.abs(delta.cpu().numpy() - d_ref).max() <= 1e-12 * np.abs(d_ref).max()
    s.close()


def test_noalloc_tne_at_the_cell_limit_f32():
    """Exactly 4096 x 4096 cells (the largest grid the scratch serves), FP32 state."""
    import torch
    n = 4096
    s = _solver(n, n, lbkm.F32, 1)
    state = s.get_state(device=True)
    out = torch.zeros(REC_DOUBLES, dtype=torch.float64, device="cuda")
    _, g_ref = s.tne(fields=False)
    for _ in range(2):
        out.zero_()
        lbkm.tne_noalloc(s.params, state.data_ptr(), n, None, out.data_ptr())
        torch.cuda.synchronize()
        _compare(_record(out), g_ref, 1e-12)
    s.close()


def test_noalloc_rejects_grids_beyond_its_scratch():
    import torch
    p = lbkm.default_params(nx=5000, ny=5000)
    buf = torch.zeros(REC_DOUBLES, dtype=torch.float64, device="cuda")
    with pytest.raises(lbkm.LbkmError) as e:
        lbkm.tne_noalloc(p, buf.data_ptr(), 5000, None, buf.data_ptr())
    assert e.value.code == 1 and "16777216" in str(e.value)
