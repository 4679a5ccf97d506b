"""Continuous-batching server: every result is the same alone and in the
mix (bitwise: the kernels are deterministic and a request's arithmetic does
not depend on its neighbours on the device), a corrupt request fails alone,
cancellation, and admission by device-memory budget."""
import numpy as np
import pytest

from paper_2108_10565_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_10565_gb300 import _lib

    return _lib


def _scenarios():
    out = []
    sc0 = inputs.config0_scenario()
    m0 = sc0["mesh"]
    out.append(dict(N=2, mesh=m0, mat=sc0["materials"], C=1, prec=0, src=[sc0["source"]], rec=sc0["receivers"],
                    cycles=12))
    coords = [np.array([0, 0.05, 0.1, 0.2, 0.4, 0.8, 1.6]), np.linspace(0, 2.4, 4), np.linspace(0, 2.4, 4)]
    m1 = inputs.kuhn_box_mesh((6, 3, 3), periodic=(False, True, True), coords=coords, tags={"x-": 1, "x+": 2})
    ne1 = m1["tets"].shape[0]
    out.append(dict(N=2, mesh=m1, mat=np.tile(inputs.REFERENCE_MATERIAL, (ne1, 1)), C=3, prec=0,
                    src=[dict(x=np.array([0.07, 1.1, 1.3]), w=np.eye(13)[9], f0=2000.0, t0=2e-4, amplitude=1e6)],
                    rec=[np.array([0.03, 0.5, 0.5]), np.array([1.2, 1.0, 2.0])], cycles=4))
    m2 = inputs.kuhn_box_mesh((3, 3, 2), lo=(0, 0, -1), hi=(1.5, 1.5, 0), periodic=(False, False, False),
                              tags={"z+": 1})
    ne2 = m2["tets"].shape[0]
    out.append(dict(N=3, mesh=m2, mat=np.tile(inputs.REFERENCE_MATERIAL, (ne2, 1)), C=1, prec=1,
                    src=[dict(x=np.array([0.7, 0.7, -0.5]), w=-np.r_[np.ones(3), np.zeros(6), -1, np.zeros(3)],
                              f0=3000.0, t0=3e-4, amplitude=1e6)],
                    rec=[np.array([0.4, 0.5, -0.1])], cycles=10))
    out.append(dict(out[0], prec=1, cycles=8))
    # partners that share a batched group with the runs above (same degree,
    # precision, refinement and clusters; other sources, receivers, lengths)
    out.append(dict(out[0], src=[dict(sc0["source"], x=np.array([0.3, 0.6, 0.45]))], rec=sc0["receivers"][:2],
                    cycles=9))
    out.append(dict(out[1], src=[dict(out[1]["src"][0], x=np.array([0.5, 0.7, 2.0]))], cycles=3))
    out.append(dict(out[2], prec=2, cycles=6))
    out.append(dict(out[2], prec=2, cycles=11, rec=[np.array([1.1, 0.4, -0.7])]))
    return out


def _t_end(L, sc):
    ctx = L.poro_create(0, sc["N"], sc["prec"])
    try:
        L.poro_set_mesh(ctx, sc["mesh"]["vertices"], sc["mesh"]["tets"], sc["mesh"]["neighbors"],
                        sc["mesh"]["face_tag"])
        L.poro_set_materials(ctx, sc["mat"])
        dt, _ = L.poro_set_clusters(ctx, 0.5, sc["C"])
    finally:
        L.poro_destroy(ctx)
    return sc["cycles"] * dt * 2 ** (sc["C"] - 1) * (1 + 1e-9)


def _alone(L, sc, t_end):
    ctx = L.poro_create(0, sc["N"], sc["prec"])
    try:
        L.poro_set_mesh(ctx, sc["mesh"]["vertices"], sc["mesh"]["tets"], sc["mesh"]["neighbors"],
                        sc["mesh"]["face_tag"])
        L.poro_set_materials(ctx, sc["mat"])
        L.poro_set_clusters(ctx, 0.5, sc["C"])
        for s in sc["src"]:
            L.poro_add_point_source(ctx, s["x"], s["w"], s["f0"], s["t0"], s["amplitude"])
        for x in sc["rec"]:
            L.poro_add_receiver(ctx, x)
        # the server advances in chunks; the alone run in one call
        L.poro_advance(ctx, t_end)
        return [L.poro_get_seismogram(ctx, r) for r in range(len(sc["rec"]))]
    finally:
        L.poro_destroy(ctx)


def _submit(L, srv, sc, t_end):
    s, keep = L.make_scenario(sc["N"], sc["mesh"], sc["mat"], t_end, precision=sc["prec"], max_clusters=sc["C"],
                              sources=sc["src"], receivers=sc["rec"])
    return L.poro_submit(srv, s)


@pytest.mark.parametrize("batched", [True, False])
def test_alone_equals_in_the_mix(L, batched):
    """Every request's seismograms are bitwise those of the same simulation
    advanced alone: in batched mode (groups of equal degree, precision and
    clusters share every predictor launch; here groups of 2 in FP64 GTS, FP64
    3-cluster LTS and bf16 GTS, and single runs) and in stream mode."""
    scs = _scenarios()
    ends = [_t_end(L, sc) for sc in scs]
    alone = [_alone(L, sc, te) for sc, te in zip(scs, ends)]
    srv = L.poro_server_create(0, 64 << 30, 8)
    try:
        L.poro_server_set_batching(srv, batched)
        tickets = [_submit(L, srv, sc, te) for sc, te in zip(scs, ends)]
        for t in tickets:
            assert L.poro_wait(srv, t, 300_000) == L.PORO_REQ_DONE, L.poro_request_error(srv, t)
        for sc, t, ref in zip(scs, tickets, alone):
            for r in range(len(sc["rec"])):
                tt, q = L.poro_fetch(srv, t, r)
                assert np.array_equal(tt, ref[r][0]) and np.array_equal(q, ref[r][1])
            qd, run, total = L.poro_request_times(srv, t)
            assert total >= run >= 0.0 and qd >= 0.0
    finally:
        L.poro_server_destroy(srv)


def test_failure_isolation_and_cancel(L):
    scs = _scenarios()
    good = scs[0]
    te = _t_end(L, good)
    bad_mat = good["mat"].copy()
    bad_mat[7, 5] = np.nan                 # porosity NaN in one element
    long_run = dict(good, cycles=100000)
    srv = L.poro_server_create(0, 64 << 30, 3)
    try:
        t_bad = _submit(L, srv, dict(good, mat=bad_mat), te)
        t_long = _submit(L, srv, long_run, _t_end(L, long_run))
        t_good = _submit(L, srv, good, te)
        assert L.poro_wait(srv, t_bad, 300_000) == L.PORO_REQ_FAILED
        assert "element 7" in L.poro_request_error(srv, t_bad)
        L.poro_cancel(srv, t_long)
        assert L.poro_wait(srv, t_long, 300_000) == L.PORO_REQ_CANCELLED
        assert L.poro_wait(srv, t_good, 300_000) == L.PORO_REQ_DONE
        ref = _alone(L, good, te)
        tt, q = L.poro_fetch(srv, t_good, 0)
        assert np.array_equal(q, ref[0][1])
    finally:
        L.poro_server_destroy(srv)


def test_admission_by_memory_budget(L):
    """Budget for one request at a time: the second waits for the first to
    finish; a request larger than the whole budget fails."""
    sc = _scenarios()[0]
    te = _t_end(L, sc)
    ne = sc["mesh"]["tets"].shape[0]
    fp = L.poro_footprint_bytes(sc["N"], ne, 1, len(sc["rec"]))
    srv = L.poro_server_create(0, int(fp * 1.5), 4)
    try:
        t1 = _submit(L, srv, sc, te)
        t2 = _submit(L, srv, sc, te)
        big = dict(sc, N=6)
        t3 = _submit(L, srv, big, te)
        assert L.poro_wait(srv, t3, 300_000) == L.PORO_REQ_FAILED
        assert "budget" in L.poro_request_error(srv, t3)
        assert L.poro_wait(srv, t1, 300_000) == L.PORO_REQ_DONE
        assert L.poro_wait(srv, t2, 300_000) == L.PORO_REQ_DONE
        q1, r1, tot1 = L.poro_request_times(srv, t1)
        q2, r2, tot2 = L.poro_request_times(srv, t2)
        assert q2 >= r1 * 0.9          # admitted only after the first finished
        assert np.array_equal(L.poro_fetch(srv, t1, 0)[1], L.poro_fetch(srv, t2, 0)[1])
    finally:
        L.poro_server_destroy(srv)
