"""The allocation-free Kbar entry point (sldm_kbar_noalloc) against the
assembly's own Kbar, through the C ABI.

It exists for callers that may not allocate device memory on their hot path;
it keeps its temporaries in a fixed file-scope device array, so two calls in a
row must both give the assembly's result (the second call proves the shared
scratch is cleared where it must start at zero).  Collected last on purpose.
"""
import numpy as np
import pytest

from workloads.meshes import icosphere, merge

pytestmark = pytest.mark.gpu

C0 = 299792458.0


def test_kbar_noalloc_matches_assembly_twice():
    import torch
    from paper_2106_06184_gb300 import sldm
    # two objects (sphere + smaller sphere), lossy second object: non-trivial offsets and complex k
    xyz, tri, obj = merge(icosphere(2, 0.1), icosphere(1, 0.05, (0.3, 0.0, 0.0)))
    mats = [(4.0, 1.0, 0.0), (3.0, 1.0, 0.02)]
    f = 300e6
    m = sldm.Mesh(xyz, tri, obj)
    st = sldm.Stack([(1.0, 1.0, 0.0, 0.0)])
    op = sldm.Operator(m, st, mats, f, precision=sldm.PREC_F64)
    Ix = op.block(sldm.BLOCK_IX)
    k0 = 2 * np.pi * f / C0
    eps0 = 1.0 / (4e-7 * np.pi * C0 ** 2)
    uv, tp, tm = m.edges()
    e_obj = obj[tp]
    for o, (er, mr, sg) in enumerate(mats):
        k = k0 * np.sqrt((er - 1j * sg / (2 * np.pi * f * eps0)) * mr)
        ref = op.block(sldm.BLOCK_K, o)                              # Kbar + I_x / 2 from the assembly
        idx = np.nonzero(e_obj == o)[0]
        ix_o = Ix[np.ix_(idx, idx)]
        for call in range(2):
            out = torch.full((len(idx), len(idx)), complex("nan+nanj"), dtype=torch.complex128, device="cuda")
            m.kbar_noalloc(o, k, out)
            torch.cuda.synchronize()
            got = out.cpu().numpy() + 0.5 * ix_o
            err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            errmax = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
            assert err < 1e-10 and errmax < 1e-10, (o, call, err, errmax)


def test_kbar_noalloc_rejects_objects_beyond_the_scratch():
    import torch
    from paper_2106_06184_gb300 import sldm
    m = sldm.Mesh(*icosphere(3, 0.1))                                 # 1280 triangles: 1920 x 11520 entries
    out = torch.zeros((m.ne, m.ne), dtype=torch.complex128, device="cuda")
    with pytest.raises(sldm.SldmError) as e:
        m.kbar_noalloc(0, 2.0, out)
    assert e.value.code == sldm.EINVAL and "too large" in str(e.value)
