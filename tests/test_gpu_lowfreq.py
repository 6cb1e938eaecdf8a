"""Low-frequency behaviour of the formulation (Sec. II-D: charges as unknowns keep
the system stable as the frequency drops): the copper bar, in free space and in
the wire's SiO2 / Si / PEC stack, solves to 1e-8 from 1 MHz down to 1 Hz with
GMRES iteration counts that stay within a small factor of the 1 MHz count."""
import numpy as np
import pytest

from workloads.meshes import box

pytestmark = pytest.mark.gpu

LAYERS = [(1.0, 1.0, 0.0, 0.0), (3.9, 1.0, 0.0, 10e-6), (11.9, 1.0, 10.0, 200e-6)]
COPPER = (1.0, 1.0, 5.8e7)


@pytest.mark.parametrize("background", ["free", "stack"])
def test_iterations_bounded_down_to_1Hz(background):
    import torch  # noqa: F401
    from paper_2106_06184_gb300 import sldm
    xyz, tri = box(20e-6, 2e-6, 1e-6, 6, 2, 1, center=(0.0, 0.0, -5e-6), jitter=0.01, seed=7)
    m = sldm.Mesh(xyz, tri)
    if background == "free":
        st, mat = sldm.Stack([(1.0, 1.0, 0.0, 0.0)]), COPPER
    else:
        st, mat = sldm.Stack(LAYERS, z_top=0.0, bottom=sldm.BOTTOM_PEC), COPPER + (1,)
    iters = {}
    for f in (1e6, 1e3, 1.0):
        op = sldm.Operator(m, st, [mat], f, precision=0)
        b = np.zeros(op.N, complex)
        op.rhs_planewave([0, 0, -1.0], [1.0, 0, 0], b)
        assert np.all(np.isfinite(b)) and np.linalg.norm(b) > 0
        x = np.zeros(op.N, complex)
        info = op.solve(b, x, tol=1e-8, maxit=3000)
        assert info["relres"] < 1e-8 and np.all(np.isfinite(x))
        iters[f] = info["iters"]
    assert max(iters.values()) <= 2 * iters[1e6] + 10, iters
