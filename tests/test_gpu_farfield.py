"""The multi-right-hand-side far field (sldm_farfield_n: phase factors or the
stack's waves shared by the right-hand sides of a CTA) against one call per
right-hand side, in free space and above a stack, with a ragged group (11
right-hand sides: groups of 8 and 3)."""
import numpy as np
import pytest

from workloads.meshes import icosphere

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("layered", [False, True])
def test_farfield_n_matches_single(layered):
    import torch  # noqa: F401
    from paper_2106_06184_gb300 import sldm
    v, f = icosphere(1, 0.1, (0.0, 0.0, 0.15))
    m = sldm.Mesh(v, f)
    st = (sldm.Stack([(1.0, 1.0, 0.0, 0.0), (4.0, 1.0, 0.01, 0.0)], z_top=0.0) if layered
          else sldm.Stack([(1.0, 1.0, 0.0, 0.0)]))
    op = sldm.Operator(m, st, [(4.0, 1.0, 0.0, 0)], 300e6)
    nr = 11
    th_inc = np.radians(np.linspace(0, 60, nr))
    khat = np.stack([np.sin(th_inc), 0 * th_inc, -np.cos(th_inc)], axis=1)
    pol = np.tile([0.0, 1.0, 0.0], (nr, 1))
    b = np.zeros((nr, op.N), complex)
    op.rhs_planewave(khat, pol, b)
    x = np.zeros_like(b)
    op.solve(b, x, nrhs=nr, tol=1e-10)
    th = np.radians(np.linspace(0, 85 if layered else 180, 19))
    got = op.farfield_n(x, th, 0.3, nr)
    for r in range(nr):
        ref = op.farfield(np.ascontiguousarray(x[r]), th, 0.3)
        assert np.max(np.abs(got[r] - ref)) <= 1e-12 * np.max(ref), r
