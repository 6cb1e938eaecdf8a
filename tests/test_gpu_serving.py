"""The serving loop on the GPU: requests for several configurations (models x
frequencies) queued together, batched per operator, overlapped on two workers,
with operators cached under a device-memory budget.

* alone vs in the mix: every request's currents equal those of a solve of that
  request alone (its own operator, its own right-hand sides) to the solve
  tolerance times the conditioning (lockstep GMRES stops each right-hand side on
  its own residual);
* one configuration against the oracle (the sphere of the parity tests);
* a budget that holds one operator at a time: evictions happen, results unchanged;
* the statistics (latency quantiles, hits, batches) are consistent.
"""
import numpy as np
import pytest

from oracle import system as S
from oracle.topology import Mesh as OMesh
from workloads.meshes import icosphere, ellipsoid

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _waves(rng, n):
    th = rng.uniform(0, 1.2, n)
    ph = rng.uniform(-np.pi, np.pi, n)
    khat = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), -np.cos(th)], axis=1)
    e_te = np.stack([-np.sin(ph), np.cos(ph), np.zeros(n)], axis=1)
    e_tm = np.cross(e_te, khat)
    return khat, e_te if rng.random() < 0.5 else e_tm


@pytest.fixture(scope="module")
def setup():
    import torch  # noqa: F401
    from paper_2106_06184_gb300 import sldm
    v1, f1 = icosphere(1, 0.1)
    v2, f2 = ellipsoid(1, (0.08, 0.05, 0.06), (0.0, 0.0, 0.12))
    free = sldm.Stack([(1.0, 1.0, 0.0, 0.0)])
    ground = sldm.Stack([(1.0, 1.0, 0.0, 0.0), (4.0, 1.0, 0.01, 0.0)], z_top=0.0)
    m1, m2 = sldm.Mesh(v1, f1), sldm.Mesh(v2, f2)
    models = [(m1, free, [(4.0, 1.0, 0.0, 0)]), (m2, free, [(6.0, 1.0, 0.02, 0)]),
              (m2, ground, [(6.0, 1.0, 0.02, 0)])]
    return sldm, models, (v1, f1)


def _alone(sldm, model, freq, khat, pol, prec, tol):
    mesh, stack, mats = model
    op = sldm.Operator(mesh, stack, mats, freq, precision=prec)
    b = np.zeros((len(khat), op.N), complex)
    op.rhs_planewave(khat, pol, b)
    x = np.zeros_like(b)
    op.solve(b, x, nrhs=len(khat), tol=tol)
    return x


@pytest.mark.parametrize("prec", [0, 2])
def test_mix_equals_alone(setup, prec):
    sldm, models, _ = setup
    rng = np.random.default_rng(2106_06184 + 4)
    srv = sldm.Server(workers=2, max_batch=8, precision=prec)
    ids = [srv.add_model(*m) for m in models]
    freqs = [200e6, 300e6]
    reqs = []
    for i in range(14):
        mi = int(rng.integers(0, len(models)))
        f = freqs[int(rng.integers(0, 2))]
        n = int(rng.integers(1, 6))
        khat, pol = _waves(rng, n)
        reqs.append((mi, f, khat, pol))
    out = []
    for mi, f, khat, pol in reqs:
        x = np.zeros((len(khat), models[mi][0].n_unknowns), complex)
        out.append((srv.submit(ids[mi], f, khat, pol, x, tol=1e-10), x))
    res = [srv.wait(t, timeout=300) for t, _ in out]
    st = srv.stats()
    srv.close()
    assert all(r["code"] == sldm.OK for r in res), [r.get("error") for r in res if r["code"] != sldm.OK][:3]
    assert st["requests"] == len(reqs) and st["rhs"] == sum(len(r[2]) for r in reqs)
    assert st["batches"] < len(reqs)            # same-key requests were solved together
    assert st["hits"] > 0 and st["misses"] <= 6  # at most one assembly per (model, frequency)
    assert 0 < st["lat_p50"] <= st["lat_p99"] <= st["lat_max"]
    for (mi, f, khat, pol), (_, x), r in zip(reqs, out, res):
        xa = _alone(sldm, models[mi], f, khat, pol, prec, 1e-10)
        assert rel(x, xa) < 1e-6, (mi, f, rel(x, xa), r["batch_rhs"])


def test_served_sphere_matches_oracle(setup):
    sldm, models, (v1, f1) = setup
    srv = sldm.Server(workers=1, max_batch=4, precision=sldm.PREC_F32X2)
    mid = srv.add_model(*models[0])
    x = np.zeros((1, models[0][0].n_unknowns), complex)
    t = srv.submit(mid, 300e6, [[0, 0, -1.0]], [[1.0, 0, 0]], x, tol=1e-10)
    r = srv.wait(t, timeout=300)
    srv.close()
    assert r["code"] == sldm.OK
    om = OMesh(v1, f1)
    A = S.assemble(om, [S.Material(4.0)], S.Material(), 300e6)
    assert rel(x[0], S.solve(A, S.rhs(A))) < 1e-6


def test_budget_evicts_and_results_hold(setup):
    sldm, models, _ = setup
    op = sldm.Operator(*models[1], 200e6, precision=0)
    one = op.device_bytes
    N = op.N
    del op
    srv = sldm.Server(workers=1, max_batch=8, precision=0, budget_bytes=int(1.5 * one))
    mid = srv.add_model(*models[1])
    rng = np.random.default_rng(7)
    khat, pol = _waves(rng, 2)
    xs = []
    for f in (200e6, 300e6, 200e6, 300e6):
        x = np.zeros((2, N), complex)
        xs.append((srv.submit(mid, f, khat, pol, x, tol=1e-10), x, f))
        srv.wait(xs[-1][0], timeout=300)
    st = srv.stats()
    srv.close()
    assert st["evictions"] >= 2 and st["hits"] == 0 and st["cached_ops"] <= 1
    assert rel(xs[0][1], xs[2][1]) < 1e-8 and rel(xs[1][1], xs[3][1]) < 1e-8
