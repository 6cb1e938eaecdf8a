"""Writes href_sphere.txt: the oracle's bistatic RCS of the dielectric sphere of
Sec. IV-A (radius 0.1 m, eps_r 4, 300 MHz, x-polarised plane wave along -z) on
icospheres of subdivision 0 to 3, for the h-refinement pin in
tests/test_oracle_href.py.  Calls only the oracle (and the mesh generator); one
process per subdivision level (sub 3 takes several minutes).

    python tests/golden/make_href_sphere.py
"""
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
SUBS = (0, 1, 2, 3)
THETA_DEG = (0.0, 20.0, 40.0, 60.0, 120.0, 140.0, 160.0, 180.0)


def rcs_at(sub):
    sys.path.insert(0, ROOT)
    from oracle import farfield, system as S
    from oracle.topology import Mesh
    from workloads.meshes import icosphere
    v, f = icosphere(sub, 0.1)
    m = Mesh(v, f)
    A = S.assemble(m, [S.Material(4.0)], S.Material(), 300e6)
    x = S.solve(A, S.rhs(A))
    return farfield.rcs(m, A.k0, S.j_delta(A, x), np.radians(THETA_DEG))


if __name__ == "__main__":
    with mp.get_context("spawn").Pool(len(SUBS)) as pool:
        res = pool.map(rcs_at, SUBS)
    with open(os.path.join(HERE, "href_sphere.txt"), "w") as fh:
        fh.write("# oracle bistatic RCS (m^2), E-plane, theta = scattering direction from +z (0 = backscatter)\n")
        fh.write("# sphere r 0.1 m, eps_r 4, 300 MHz, icosphere subdivision s; written by make_href_sphere.py\n")
        fh.write("# theta_deg " + " ".join(f"{t:g}" for t in THETA_DEG) + "\n")
        for s, r in zip(SUBS, res):
            fh.write(f"{s} " + " ".join(f"{x:.15e}" for x in r) + "\n")
