"""Boundary error behaviour that needs no GPU: the C ABI validates a scene description
and a solver configuration before it touches the device, and returns EINVAL (never
aborts) on what it cannot represent; calls on a null context return EINVAL."""
import copy
import ctypes

import pytest

from paper_2609_08800_gb300 import build as B
from paper_2609_08800_gb300 import ostrich as M
from paper_2609_08800_gb300 import scenes as S

OSTRICH_EINVAL = 1


@pytest.fixture(scope="module")
def lib():
    B.build()
    return M.lib()


def _create(lib, scene, cfg=None, n_worlds=4, ld=0, dtype=0, tape_slots=1):
    d, c = M.scene_desc(scene), M.solver_cfg(cfg or S.SolverConfig())
    h = ctypes.c_void_p()
    rc = lib.ostrich_create(ctypes.byref(d), ctypes.byref(c), n_worlds, ld, dtype, tape_slots, ctypes.byref(h))
    return rc, h


def _robot():
    return S.robot_plane_scene()


@pytest.mark.parametrize("case", ["zero_mass", "bad_inertia", "joint_self", "joint_out_of_range"])
def test_create_rejects_invalid_scenes(lib, case):
    sc = copy.deepcopy(_robot())
    if case == "zero_mass":
        sc.bodies[1].mass = 0.0
    elif case == "bad_inertia":
        sc.bodies[0].inertia = (1.0, -1.0, 1.0)
    elif case == "joint_self":
        sc.joints[0].child = sc.joints[0].parent
    else:
        sc.joints[2].child = 7
    rc, h = _create(lib, sc)
    assert rc == OSTRICH_EINVAL and not h.value


@pytest.mark.parametrize("kw", [dict(n_worlds=0), dict(ld=2, n_worlds=4), dict(dtype=7), dict(tape_slots=-1)])
def test_create_rejects_invalid_sizes(lib, kw):
    rc, h = _create(lib, _robot(), **kw)
    assert rc == OSTRICH_EINVAL and not h.value


def test_create_rejects_negative_budget(lib):
    rc, h = _create(lib, _robot(), cfg=S.SolverConfig(budget=-1))
    assert rc == OSTRICH_EINVAL and not h.value


def test_calls_on_a_null_context_return_einval(lib):
    assert lib.ostrich_adjoint(None, 0, None, 0.1, None, None, None) == OSTRICH_EINVAL
    assert lib.ostrich_adjoint_params(None, 0, None, 0.1, None, None, None, None, None, None, None) == OSTRICH_EINVAL
    assert lib.ostrich_set_adjoint_mode(None, 1, None) == OSTRICH_EINVAL
    assert lib.ostrich_set_linear_solver(None, 1, 0, 16, 256, 0.0) == OSTRICH_EINVAL
    assert lib.ostrich_step(None, None, None, 0.1, None, None, None, None, None, -1, None) == OSTRICH_EINVAL
    assert lib.ostrich_tape_clear(None) == OSTRICH_EINVAL


def _noalloc(lib, scene, n_worlds):
    """Call the allocation-free entry with placeholder (never dereferenced) pointers: the
    checks that refuse the call come before any device work."""
    d, c = M.scene_desc(scene), M.solver_cfg(S.SolverConfig())
    p = ctypes.c_void_p(4096)
    return lib.ostrich_step_adjoint_noalloc(ctypes.byref(d), ctypes.byref(c), n_worlds, 0, p, p, 0.1,
                                            ctypes.c_void_p(8192), p, ctypes.c_void_p(12288), None, None)


def test_noalloc_refuses_heightmap_scenes(lib):
    assert _noalloc(lib, S.terrain_scene(n=16), 4) == OSTRICH_EINVAL


def test_noalloc_refuses_worlds_beyond_its_array(lib):
    # 10432 B of tape per robot-over-box world: 1608 fit the 16 MiB array, 1609 do not
    assert _noalloc(lib, S.robot_box_scene(), 1609) == OSTRICH_EINVAL


@pytest.mark.parametrize("args", [(2, 0, 16, 256, 0.0), (1, 2, 16, 256, 0.0), (1, 0, 0, 256, 0.0),
                                  (1, 0, 16, 0, 0.0), (1, 1, 16, 256, -1.0)])
def test_linear_solver_rejects_invalid_settings(lib, args):
    """ostrich_set_linear_solver: unknown solver or preconditioner, counts below 1 and a
    negative tolerance are EINVAL; valid settings are accepted (host only, no device
    work: the context has no tape)."""
    rc, h = _create(lib, _robot(), tape_slots=0)
    if rc != 0:
        pytest.skip("context creation needs a device here")
    try:
        assert lib.ostrich_set_linear_solver(h, *args) == OSTRICH_EINVAL
        assert lib.ostrich_set_linear_solver(h, 1, 1, 16, 256, 0.0) == 0
        assert lib.ostrich_set_linear_solver(h, 0, 0, 1, 1, 1e-8) == 0
    finally:
        lib.ostrich_destroy(h)


def test_noalloc_capacity_of_the_robot_and_refusals(lib):
    """The capacity helper: 10432 B per robot-over-box world, 1608 worlds in the 16 MiB
    array; heightmap scenes refused (host only)."""
    mw, rb = M.noalloc_capacity(S.robot_box_scene())
    assert (mw, rb) == (1608, 10432)
    assert mw * rb <= 16 << 20 < (mw + 1) * rb
    with pytest.raises(ValueError):
        M.noalloc_capacity(S.terrain_scene(n=16))
    assert lib.ostrich_noalloc_capacity(None, None, None, None) == OSTRICH_EINVAL


def test_binding_checks_element_type_and_size_before_the_pointer():
    """The binding hands the library raw pointers, so it checks first what the library
    will assume: the element type and enough elements for [rows, ld] (a smaller array
    would be overrun on the device); a host tensor is refused as well."""
    torch = pytest.importorskip("torch")
    with pytest.raises(ValueError, match="element type"):
        M._checked(torch.zeros(8, dtype=torch.float64), torch.float32, 8, "state_in")
    with pytest.raises(ValueError, match="at least 9 elements"):
        M._checked(torch.zeros(8, dtype=torch.float32), torch.float32, 9, "state_in")
    with pytest.raises(ValueError, match="host tensor"):
        M._checked(torch.zeros(9, dtype=torch.float32), torch.float32, 9, "state_in")
    assert M._checked(None, torch.float32, 9, "state_in") is None
