"""sldm_mesh_create and sldm_stack_create reject invalid input on the host,
before any device call, so these checks need no GPU: each case returns
SLDM_EINVAL (SLDM_ENOTSUP for more layers than the multilayer kernel takes)
with its reason.

The formulation (Sec. II) takes every object as a closed surface with the
outward normal n; RWG functions need each interior edge shared by exactly two
triangles traversed in opposite directions; multiple objects (Sec. II-E) are
disjoint.
"""
import numpy as np
import pytest

from workloads.meshes import icosphere, merge


def _sl():
    from paper_2106_06184_gb300 import sldm
    return sldm


def _rejected(xyz, tri, obj=None):
    sl = _sl()
    with pytest.raises(sl.SldmError) as e:
        sl.Mesh(xyz, tri, obj)
    assert e.value.code == sl.EINVAL, str(e.value)
    return str(e.value)


@pytest.fixture(scope="module")
def sphere():
    return icosphere(1, 0.1)


def test_open_surface(sphere):
    v, f = sphere
    assert "not closed" in _rejected(v, f[:-1])


def test_directed_edge_used_twice(sphere):
    v, f = sphere
    g = f.copy()
    g[0] = g[0, [0, 2, 1]]                  # one triangle flipped: its edges run along its neighbours'
    assert "2-manifold" in _rejected(v, g)


def test_degenerate_triangle(sphere):
    v, f = sphere
    g = f.copy()
    g[0] = [g[0, 0], g[0, 0], g[0, 1]]
    assert "degenerate" in _rejected(v, g)


def test_collinear_triangle(sphere):
    v, f = sphere
    a, b = f[0, 0], f[0, 1]
    w = np.vstack([v, 0.5 * (v[a] + v[b])])  # a new vertex on the segment a-b
    g = f.copy()
    g[0] = [a, b, len(v)]
    assert "degenerate" in _rejected(w, g)


def test_inward_object(sphere):
    v, f = sphere
    assert "inward" in _rejected(v, f[:, ::-1].copy())


def test_second_object_inward(sphere):
    v, f = sphere
    v2, f2 = icosphere(1, 0.1, center=(0.5, 0.0, 0.0))
    xyz, tri, obj = merge((v, f), (v2, f2[:, ::-1].copy()))
    assert "object 1 is oriented inward" in _rejected(xyz, tri, obj)


def test_vertex_shared_by_two_objects(sphere):
    v, f = sphere
    xyz, tri, obj = merge((v, f), icosphere(1, 0.1, center=(0.5, 0.0, 0.0)))
    tri = tri.copy()
    tri[tri == len(v)] = 0                  # the second sphere takes a vertex of the first
    assert "two objects" in _rejected(xyz, tri, obj)


def test_vertex_index_out_of_range(sphere):
    v, f = sphere
    g = f.copy()
    g[3, 1] = len(v)
    assert "out of range" in _rejected(v, g)


def test_object_ids_not_sorted(sphere):
    v, f = sphere
    obj = np.zeros(len(f), np.int32)
    obj[: len(f) // 2] = 1
    assert "non-decreasing" in _rejected(v, f, obj)


def test_object_with_too_few_triangles(sphere):
    v, f = sphere
    # two triangles back to back: closed, but no surface encloses anything with fewer than four
    pv = np.array([[1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0]]) + 2.0
    pf = np.array([[0, 1, 2], [0, 2, 1]])
    xyz, tri, obj = merge((v, f), (pv, pf))
    assert "too few triangles" in _rejected(xyz, tri, obj)


def test_empty_mesh():
    assert "empty" in _rejected(np.zeros((0, 3)), np.zeros((0, 3), np.int32))


def _stack_rejected(layers, code=None, **kw):
    sl = _sl()
    with pytest.raises(sl.SldmError) as e:
        sl.Stack(layers, **kw)
    assert e.value.code == (sl.EINVAL if code is None else code), str(e.value)
    return str(e.value)


def test_valid_stacks_need_no_device():
    sl = _sl()
    sl.Stack([(1.0, 1.0, 0.0, 0.0)])
    sl.Stack([(1.0, 1.0, 0.0, 0.0), (3.9, 1.0, 0.0, 10e-6), (11.9, 1.0, 10.0, 200e-6)], z_top=0.0,
             bottom=sl.BOTTOM_PEC)
    sl.Stack([(1.0, 1.0, 0.0, 0.0), (2.25, 1.0, 0.0, np.inf)], bottom=sl.BOTTOM_HALFSPACE)  # half-spaces: any thickness


def test_invalid_stacks():
    sl = _sl()
    air = (1.0, 1.0, 0.0, 0.0)
    assert "invalid arguments" in _stack_rejected([])
    for bad in ((0.0, 1.0, 0.0, 0.0), (-2.0, 1.0, 0.0, 0.0), (2.0, 0.0, 0.0, 0.0), (2.0, 1.0, -1.0, 0.0),
                (np.nan, 1.0, 0.0, 0.0), (np.inf, 1.0, 0.0, 0.0), (2.0, 1.0, np.inf, 0.0)):
        assert "material" in _stack_rejected([air, bad])
    # a finite layer (between two interfaces, or any layer above a PEC bottom) needs a thickness
    for t in (0.0, -1e-3, np.inf, np.nan):
        assert "thickness" in _stack_rejected([air, (2.0, 1.0, 0.0, t), (4.0, 1.0, 0.0, 0.0)])
        assert "thickness" in _stack_rejected([air, (2.0, 1.0, 0.0, t)], bottom=sl.BOTTOM_PEC)
    assert "z_top" in _stack_rejected([air, (2.0, 1.0, 0.0, 0.0)], z_top=np.nan)
    assert "bottom" in _stack_rejected([air], bottom=7)
    assert "too many" in _stack_rejected([air] + [(2.0, 1.0, 0.0, 1e-3)] * 8 + [air], code=sl.ENOTSUP)
