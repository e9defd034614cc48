"""Host-side validation of lbkm_create: every rejection happens before any CUDA call,
so these run without a GPU (stream 0 is passed explicitly)."""
import pytest

from paper_1411_6697_gb300 import lbkm


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1411_6697_gb300 import build
    build.build()


def create(**kw):
    base = dict(nx=16, ny=1)
    base.update(kw)
    return lbkm.Solver(stream=0, **base)


@pytest.mark.parametrize("kw,code", [
    (dict(nx=0), 1),
    (dict(ny=0), 1),
    (dict(precision=7), 1),
    (dict(recovery=3), 1),
    (dict(gamma=1.0), 1),
    (dict(gamma=2.5), 1),
    (dict(dt=3e-5), 1),                       # dt * S = 3 >= 2: Euler relaxation unstable
    (dict(dx=1e-5), 1),                        # CFL 2.7 > 1
    (dict(orbit_kind=(0, 0, 1, 1)), 1),        # order must be axis, diag, axis, diag
    (dict(orbit_speed=(2.7, -1.0, 1.2, 1.0)), 1),
    (dict(bc=(2, 0)), 1),                      # walls only in y
    (dict(bc=(0, 3)), 1),
    (dict(bc=(0, 2), walls=((0, 0, 1), (0.1, 0, 1))), 1),            # walls need ny >= 2
    (dict(ny=8, bc=(0, 2), walls=((0, 0, 1), (0.1, 0, 0.0))), 1),    # wall T must be > 0
    (dict(ny=8, bc=(0, 2), walls=((float("nan"), 0, 1), (0, 0, 1))), 1),
    # per-side conditions: specular and walls only on y sides, periodic only for both
    # sides of a direction, Dirichlet states physical
    (dict(ny=8, bc=(5, 0), sides=[(4, 1, 0, 0, 1, 0), (1, 1, 0, 0, 1, 0)] + [(1, 1, 0, 0, 1, 0)] * 2), 1),
    (dict(ny=8, bc=(0, 5), sides=[(1, 1, 0, 0, 1, 0)] * 2 + [(0, 1, 0, 0, 1, 0), (1, 1, 0, 0, 1, 0)]), 1),
    (dict(ny=8, bc=(5, 0), sides=[(3, 0.0, 0, 0, 1, 0), (1, 1, 0, 0, 1, 0)] + [(1, 1, 0, 0, 1, 0)] * 2), 1),
    (dict(ny=8, bc=(5, 0), sides=[(3, 1.0, 0, 0, 1, 1.5), (1, 1, 0, 0, 1, 0)] + [(1, 1, 0, 0, 1, 0)] * 2), 1),
    (dict(ny=1, bc=(0, 5), sides=[(1, 1, 0, 0, 1, 0)] * 2 + [(4, 1, 0, 0, 1, 0)] * 2), 1),
    (dict(tne_every=-1), 1),
    (dict(time_scheme=3), 1),
    (dict(tne_capacity=0), 1),
    (dict(omega1=-1.0), 1),
    (dict(collision=2), 1),                     # 0 (fast path where it applies) or 1
    (dict(alloc_ctx=None, alloc=lbkm.ALLOC_FN(lambda n, s, c: None)), 1),  # alloc without free
    # the paper's first two rings (shared speed and eta): singular M
    (dict(orbit_speed=(2.7, 2.7, 2.2, 2.2), orbit_eta=(5.0, 5.0, 3.0, 3.0)), 4),
])
def test_invalid_parameters_are_rejected(kw, code):
    with pytest.raises(lbkm.LbkmError) as e:
        create(**kw)
    assert e.value.code == code
    assert str(e.value)


def test_pr_sets_heat_conduction_rates():
    p = lbkm.default_params(nx=4, ny=1, Pr=0.5, S=[1e4] * 16)
    # the override happens inside lbkm_create; the stored copy keeps the caller's values
    assert p.Pr == 0.5 and p.S[7] == 1e4


@pytest.mark.parametrize("kw", [
    dict(nx=0), dict(precision=3), dict(gamma=1.0), dict(gamma=2.5),
    dict(v=(2.7, 0.0, 1.2)), dict(eta=(5.0, -1.0, 1.1)), dict(dt=5e-4),
    dict(dx=1e-6), dict(bc=(2, 0)), dict(bc=(0, 5)), dict(T_ig=float("nan")),
    dict(omega1=-1.0), dict(tne_every=-1),
    dict(v=(1.0, 1.0, 1.0), eta=(1.0, 1.0, 1.0)),  # three equal groups: singular M
])
def test_d2v24_invalid_parameters_are_rejected(kw):
    """lbkm24_create validates on the host before any CUDA call."""
    base = dict(nx=16, ny=1)
    base.update(kw)
    with pytest.raises(lbkm.LbkmError) as e:
        lbkm.Solver24(stream=0, **base)
    assert e.value.code in (1, 4)


def test_d2v24_collision_flag_is_checked():
    with pytest.raises(lbkm.LbkmError) as e:
        lbkm.Solver24(stream=0, nx=16, ny=1, collision=2)
    assert e.value.code == 1


@pytest.mark.parametrize("kw", [
    dict(ny=8, bc=(5, 0), sides=[(4, 1, 0, 0, 1, 0), (1, 1, 0, 0, 1, 0)] + [(1, 1, 0, 0, 1, 0)] * 2),
    dict(ny=8, bc=(5, 0), sides=[(2, 1, 0, 0, 1, 0)] + [(1, 1, 0, 0, 1, 0)] * 3),
    dict(ny=8, bc=(5, 0), sides=[(3, 0.0, 0, 0, 1, 0), (1, 1, 0, 0, 1, 0)] + [(1, 1, 0, 0, 1, 0)] * 2),
    dict(ny=1, bc=(0, 5), sides=[(1, 1, 0, 0, 1, 0)] * 2 + [(4, 1, 0, 0, 1, 0)] * 2),
    dict(ny=1, bc=(0, 5), sides=[(1, 1, 0, 0, 1, 0)] * 2 + [(2, 1, 0, 0, 1, 0)] * 2),
    dict(ny=8, bc=(0, 5), sides=[(1, 1, 0, 0, 1, 0)] * 2 + [(2, 1, 0, 0, 0.0, 0)] * 2),
])
def test_d2v24_side_conditions_are_checked(kw):
    """D2V24 per-side conditions: specular and walls only on y sides (and ny >= 2), a
    positive wall temperature, physical Dirichlet states."""
    base = dict(nx=16, ny=1, dx=1e-3, dy=1e-3, dt=1e-5)
    base.update(kw)
    with pytest.raises(lbkm.LbkmError) as e:
        lbkm.Solver24(stream=0, **base)
    assert e.value.code == 1


def _shell(nx, ny):
    # a Solver's Python side without a handle: only the buffer checks run
    s = lbkm.Solver.__new__(lbkm.Solver)
    s.nx, s.ny = nx, ny
    return s


def test_macros_output_buffers_are_checked_before_any_call():
    """Solver.macros(out=...) hands the library raw pointers that it fills with ny * nx
    doubles, so a buffer of another dtype, size, layout or device is refused first."""
    import numpy as np
    import torch
    s = _shell(8, 3)
    assert s._out_ptr(np.zeros((3, 8)), "rho", False) != 0
    assert s._out_ptr(torch.zeros((3, 8), dtype=torch.float64), "rho", False) != 0
    bad = [np.zeros((3, 8), np.float32), np.zeros((3, 7)), np.zeros((8, 3)).T,
           torch.zeros((3, 8)), torch.zeros((3, 9), dtype=torch.float64),
           torch.zeros((8, 3), dtype=torch.float64).t()]
    ro = np.zeros((3, 8))
    ro.flags.writeable = False
    bad.append(ro)
    for b in bad:
        with pytest.raises(ValueError):
            s._out_ptr(b, "rho", False)
    with pytest.raises(ValueError):  # host buffers where the call writes device memory
        s._out_ptr(np.zeros((3, 8)), "rho", True)
    with pytest.raises(ValueError):
        s._out_ptr(torch.zeros((3, 8), dtype=torch.float64), "rho", True)
