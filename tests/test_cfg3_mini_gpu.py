"""GPU parity of the small clustered-LTS scenario against the oracle.

`inputs.cfg3_mini_scenario`: the layered graded mesh with 16 x 16 x 8 Kuhn
boxes (12,288 tets, 32x grading), free surface on top, absorbing elsewhere,
the layer and half-space materials, degree 3, rate-2 clusters capped at 6,
the explosive Ricker source at 1010 m depth, the 8 LOHp receivers, 20 steps
of the largest cluster (0.67 s).  The oracle's run (`oracle.corrector.
LTSSimulation`, whose predictor is pinned to the dense LU solve) takes ~40
min of one host core, so its result is stored in tests/golden/cfg3_mini_N3.npz
by tests/golden/make_cfg3_mini.py, which calls only `oracle/`.

Tolerances: seismograms <= 1e-9 relative L2 per (receiver, quantity);
sampled elements' DOFs <= 1e-10 relative per element; every element's DOF
norm <= 1e-10 relative."""
import os

import numpy as np
import pytest

from paper_2108_10565_gb300 import inputs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "cfg3_mini_N3.npz")


@pytest.fixture(scope="module")
def L():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_10565_gb300 import _lib

    return _lib


@pytest.fixture(scope="module")
def ref():
    return dict(np.load(GOLDEN))


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_cfg3_mini_lts_run(L, ref, precision):
    sc = inputs.cfg3_mini_scenario()
    mesh, mats = sc["mesh"], sc["materials"]
    ne = mesh["tets"].shape[0]
    ctx = L.poro_create(0, sc["N"], precision)
    try:
        L.poro_set_mesh(ctx, mesh["vertices"], mesh["tets"], mesh["neighbors"], mesh["face_tag"])
        L.poro_set_materials(ctx, mats)
        dt, cl = L.poro_set_clusters(ctx, 0.5, sc["max_clusters"], n_elem=ne)
        assert dt == pytest.approx(float(ref["dt_min"]), rel=1e-13)
        assert np.array_equal(cl, ref["cluster"])
        L.poro_set_dofs(ctx, sc["Q0"])
        s = sc["source"]
        L.poro_add_point_source(ctx, s["x"], s["w"], s["f0"], s["t0"], s["amplitude"])
        for x in sc["receivers"]:
            L.poro_add_receiver(ctx, x)
        cycle = 2 ** (sc["max_clusters"] - 1)
        L.poro_advance(ctx, sc["n_cycles"] * cycle * dt * 1.0000001)
        Q = L.poro_get_dofs(ctx)
        seis = [L.poro_get_seismogram(ctx, r) for r in range(len(sc["receivers"]))]
    finally:
        L.poro_destroy(ctx)
    # seismograms
    for r, (t, q) in enumerate(seis):
        tr, qr = ref[f"t{r}"], ref[f"q{r}"]
        np.testing.assert_allclose(t, tr, rtol=1e-12)
        assert q.shape == qr.shape
        scale = np.abs(qr).max()
        for p in range(13):
            nr = np.linalg.norm(qr[:, p])
            err = np.linalg.norm(q[:, p] - qr[:, p])
            if nr > 1e-6 * scale:
                assert err <= 1e-9 * nr, f"receiver {r} quantity {p}: {err / nr:.3e}"
            else:
                assert err <= 1e-9 * scale
    # sampled elements, element by element
    idx = ref["sample"]
    err = np.linalg.norm((Q[idx] - ref["Q_sample"]).reshape(len(idx), -1), axis=1)
    nrm = np.linalg.norm(ref["Q_sample"].reshape(len(idx), -1), axis=1)
    assert (err <= 1e-10 * nrm).all(), (err / nrm).max()
    # every element's norm
    qn = np.linalg.norm(Q.reshape(ne, -1), axis=1)
    np.testing.assert_allclose(qn, ref["Q_norm"], rtol=1e-10)
