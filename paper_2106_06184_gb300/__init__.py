"""GB300 (sm_103a) implementation of the single-layer dual-mesh BEM hot path
(Sharma & Triverio, arXiv 2106.06184): a C-ABI CUDA library (``include/sldm.h``)
and this thin Python binding.  The binding only marshals arguments; every step
runs in the library's kernels and it raises if the library is missing."""
from .sldm import (Library, Mesh, Stack, Operator, Ports, Server, SldmError, load, port_ring, sparams,  # noqa: F401
                   PREC_F32, PREC_F64, PREC_F32X2, BOTTOM_HALFSPACE, BOTTOM_PEC,
                   BLOCK_LAM, BLOCK_LPM, BLOCK_LA, BLOCK_LP, BLOCK_K, BLOCK_Y11, BLOCK_Y21, BLOCK_IX, BLOCK_KBAR_L)
