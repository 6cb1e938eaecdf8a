"""CPU oracle for the single-layer dual-mesh BEM (SLDM) of Sharma & Triverio,
"A Single-Layer Dual-Mesh Boundary Element Method for Multiscale Electromagnetic
Modeling of Penetrable Objects in Layered Media" (arXiv 2106.06184).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 restatement of the
discrete system of Sec. II (Eqs. AEFIEintdis, AEFIEeqvdis, Yeqdef, AEFIEextdis,
finalsystem, Kmatdef, Aobj) written with numpy, for checking the CUDA library.
Only the tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it.  It shares no code,
tables or constants with the CUDA library and never calls it.

Modules
-------
topology    RWG edges, pulses, D/B/F, barycentric refinement, BC functions (Sec. II-B)
quadrature  6-point degree-4 Dunavant rule on triangles
singular    closed-form potential integrals over a flat triangle (1/R, R, grad 1/R)
fill        L^(A), L^(phi), K-bar, Gram I_x and plane-wave excitation (Sec. II-B, II-C)
system      per-object M_l, Y11/Y21, the final SLDM system and its dense solution (Sec. II-D, II-E)
farfield    far field / radar cross section of J_Delta in free space (Sec. IV-A) and above
            a stack (by reciprocity with the stack's plane waves); complex far-field amplitude
layered     multilayer kernel of one layer: stack reflections, quasistatic images, Sommerfeld
            tables and their bilinear remainder, reflected fill, plane wave through the stack
            (Sec. II-C, IV)
ports       delta-gap edge ports, port currents, Y and S parameters (Sec. IV-B, IV-C)
mie         Mie series of a dielectric sphere (independent pin for Sec. IV-A)
"""
