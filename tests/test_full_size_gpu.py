"""Parity at the clustered-LTS configuration's size: the layered graded mesh of
2,044,416 tetrahedra at N = 5, one global step of the mixed form (bf16 sweeps,
one refinement sweep, double-word corrector) through the C ABI.

The oracle cannot step two million elements, so six sampled elements are
checked one by one: each sampled element and its face neighbours carry random
DOFs (zeros elsewhere), and the element's DOFs after the step are compared
with the oracle's step (oracle/corrector.py GTSSimulation, with the mesh's
global time step) on the patch of the element and its neighbours, which is all
that one step of the element depends on.  Samples: an element on the free
surface, one on an absorbing boundary, one at the layer / half-space
interface and three at random.  Tolerance 1e-10 relative L2 per element."""
import numpy as np
import pytest

from oracle.corrector import GTSSimulation
from paper_2108_10565_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_10565_gb300 import _lib

    return _lib


def _patch(mesh, mats, e):
    """The element e (index 0) and its face neighbours as a small mesh: e's
    boundary faces keep their tags, the neighbours' other faces are absorbing
    (they do not enter e's step)."""
    nb, tag, tets = mesh["neighbors"], mesh["face_tag"], mesh["tets"]
    members = [e] + [int(r) for r in nb[e] if r >= 0]
    index = {m: i for i, m in enumerate(members)}
    vids = np.unique(tets[members].reshape(-1))
    vmap = {v: i for i, v in enumerate(vids)}
    ptets = np.array([[vmap[v] for v in tets[m]] for m in members], dtype=np.int64)
    pnb = -np.ones((len(members), 4), dtype=np.int64)
    ptag = np.full((len(members), 4), 2, dtype=np.int32)
    for f in range(4):
        r = int(nb[e, f])
        if r >= 0:
            pnb[0, f] = index[r]
            ptag[0, f] = 0
        else:
            ptag[0, f] = tag[e, f]
    for i, m in enumerate(members[1:], start=1):
        for f in range(4):
            if nb[m, f] == e:
                pnb[i, f] = 0
                ptag[i, f] = 0
    pmesh = {"vertices": mesh["vertices"][vids], "tets": ptets, "neighbors": pnb, "face_tag": ptag}
    return members, pmesh, mats[members]


def test_full_size_layered_mesh_step_sampled(L):
    N, B = 5, 56
    mesh, mats = inputs.layered_graded_mesh(44)
    ne = mesh["tets"].shape[0]
    assert ne == 2_044_416
    nb, tag = mesh["neighbors"], mesh["face_tag"]
    rng = np.random.default_rng(2108)
    free = np.where((nb < 0).any(axis=1) & (tag == 1).any(axis=1))[0]
    absorbing = np.where((nb < 0).any(axis=1) & (tag == 2).any(axis=1))[0]
    safe_nb = np.where(nb >= 0, nb, np.arange(ne)[:, None])
    interface = np.where((mats[safe_nb][:, :, 0] != mats[:, None, 0]).any(axis=1))[0]
    pools = [free, absorbing, interface, None, None, None]
    samples, used = [], set()
    for pool in pools:
        while True:
            e = int(rng.choice(pool)) if pool is not None else int(rng.integers(ne))
            patch = {e} | {int(r) for r in nb[e] if r >= 0}
            if not patch & used:
                break
        samples.append(e)
        used |= patch
    Q0 = np.zeros((ne, 13, B))
    for e in samples:
        members = [e] + [int(r) for r in nb[e] if r >= 0]
        Q0[members] = rng.standard_normal((len(members), 13, B))
    ctx = L.poro_create(0, N, L.PORO_BF16X3_REFINE)
    try:
        L.poro_set_mesh(ctx, mesh["vertices"], mesh["tets"], nb, tag)
        L.poro_set_materials(ctx, mats)
        dt, _ = L.poro_set_clusters(ctx, 0.5, 1, n_elem=ne)
        L.poro_set_dofs(ctx, Q0)
        L.poro_advance(ctx, 1.5 * dt)
        Q1 = L.poro_get_dofs(ctx)
    finally:
        L.poro_destroy(ctx)
    for e in samples:
        members, pmesh, pmats = _patch(mesh, mats, e)
        sim = GTSSimulation(pmesh, pmats, N)
        sim.dt = dt
        ref = sim.step(Q0[members], 0.0)[0]
        err = np.linalg.norm(Q1[e] - ref) / np.linalg.norm(ref)
        assert err <= 1e-10, (e, err)
