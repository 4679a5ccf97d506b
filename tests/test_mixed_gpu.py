"""GPU parity of the mixed-precision predictor (binary32 Algorithm 3 +
refinement against a double-binary32 residual) against the FP64 oracle.

Accuracy goal: relative L2 per element <= 1e-10 after refinement (one sweep
and two sweeps); without refinement the binary32 solve alone is ~1e-6 (shown,
so the tolerance tests the refinement and not the binary32 solve).
"""
import numpy as np
import pytest

from _oracle_cases import oracle_predictor, population, rel_l2

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-10


@pytest.fixture(scope="module")
def L():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_10565_gb300 import _lib

    return _lib


def _run(L, d, sweeps):
    ctx = L.poro_create(0, d["N"], L.PORO_FP32_REFINE)
    try:
        L.poro_set_refinement(ctx, sweeps)
        L.poro_set_isolated(ctx, d["vertices"], d["materials"], d["dt"])
        L.poro_set_dofs(ctx, d["Q0"])
        L.poro_predict(ctx)
        n = d["Q0"].shape[0]
        return L.poro_get_predictor(ctx, 0, n), L.poro_get_integrated(ctx, 0, n)
    finally:
        L.poro_destroy(ctx)


@pytest.mark.parametrize("N,n,n_dense", [(1, 33, 33), (2, 33, 33), (3, 33, 8), (4, 17, 3), (5, 11, 1), (6, 9, 1)])
@pytest.mark.parametrize("sweeps", [1, 2])
def test_mixed_refined_matches_oracle(L, N, n, n_dense, sweeps):
    d = population(n, N, seed=300 + N)
    qt, iout = _run(L, d, sweeps)
    errs = []
    for i in range(n):
        ref = oracle_predictor(d, i, dense=i < n_dense)
        errs.append(rel_l2(qt[i], ref))
        np.testing.assert_allclose(iout[i], d["dt"][i] * qt[i][:, :, 0], rtol=0, atol=1e-300)
    assert max(errs) <= TOL_MIXED, f"max rel err {max(errs):.3e}"


def test_unrefined_is_binary32_level(L):
    """Refinement is what brings the error down: the binary32 sweep alone is
    far from 1e-10 (and not garbage)."""
    d = population(9, 5, seed=11)
    qt, _ = _run(L, d, 0)
    errs = [rel_l2(qt[i], oracle_predictor(d, i)) for i in range(9)]
    assert 1e-9 < max(errs) < 1e-3


@pytest.mark.parametrize("visc", [0.0, 100.0])
def test_mixed_inviscid_and_very_stiff(L, visc):
    d = population(7, 6, seed=17, viscosity_scale=visc)
    qt, _ = _run(L, d, 1)
    for i in range(7):
        assert rel_l2(qt[i], oracle_predictor(d, i)) <= TOL_MIXED


def test_mixed_full_size_against_fp64(L):
    """The benchmark workload (200,000 elements, N = 6) in the bench's launch
    configuration: every element against the FP64 kernel (itself pinned to
    the oracle at 1e-12), and sampled elements against the oracle."""
    import torch

    from paper_2108_10565_gb300 import inputs

    N, n = 6, 200_000
    d = inputs.isolated_elements(n, N)
    dt = L.poro_cfl_dt(N, d["vertices"], d["materials"])
    q0 = torch.from_numpy(d["Q0"]).cuda()
    B = q0.shape[2]
    out = {}
    for prec in (L.PORO_FP64, L.PORO_FP32_REFINE):
        ctx = L.poro_create(0, N, prec)
        try:
            L.poro_set_isolated(ctx, d["vertices"], d["materials"], dt)
            qt = torch.empty((n, 13, B, N + 1), dtype=torch.float64, device="cuda")
            L.poro_predict_dev(ctx, 0, n, q0.data_ptr(), qt.data_ptr(), None,
                               stream=torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            out[prec] = qt
        finally:
            L.poro_destroy(ctx)
    a, b = out[L.PORO_FP32_REFINE], out[L.PORO_FP64]
    err = (torch.linalg.vector_norm((a - b).reshape(n, -1), dim=1)
           / torch.linalg.vector_norm(b.reshape(n, -1), dim=1)).cpu().numpy()
    assert np.isfinite(err).all()
    assert err.max() <= TOL_MIXED, f"max {err.max():.3e} median {np.median(err):.3e}"
    rng = np.random.default_rng(1)
    for i in [0, n - 1] + list(rng.choice(n, 4, replace=False)):
        sub = {"N": N, "vertices": d["vertices"][i:i + 1], "materials": d["materials"][i:i + 1],
               "Q0": d["Q0"][i:i + 1], "dt": dt[i:i + 1]}
        assert rel_l2(a[i].cpu().numpy(), oracle_predictor(sub, 0)) <= TOL_MIXED


@pytest.mark.parametrize("N", [3, 4, 5, 6])
@pytest.mark.parametrize("sweeps", [0, 1, 2])
def test_cta_size_variants_agree(L, N, sweeps):
    """Both CTA sizes of the mixed kernel (the autotuner's choices: different
    warp counts for the tensor-core epilogue, the time solves and the
    residual's balanced row lists) give bitwise identical predictors."""
    d = population(19, N, seed=2108 + N)
    out = []
    for variant in (0, 1):
        ctx = L.poro_create(0, N, L.PORO_FP32_REFINE)
        try:
            L.poro_set_refinement(ctx, sweeps)
            L.poro_set_variant(ctx, variant)
            L.poro_set_isolated(ctx, d["vertices"], d["materials"], d["dt"])
            L.poro_set_dofs(ctx, d["Q0"])
            L.poro_predict(ctx)
            out.append(L.poro_get_predictor(ctx, 0, 19))
        finally:
            L.poro_destroy(ctx)
    np.testing.assert_array_equal(out[0], out[1])


@pytest.mark.parametrize("N,n", [(3, 17), (4, 9), (5, 7), (6, 5)])
def test_bf16x3_refined_matches_oracle(L, N, n):
    """The bf16 split-product form reaches the 1e-10 goal with one refinement
    sweep (its default) and with two."""
    d = population(n, N, seed=31 + N)
    res = {}
    for sweeps in (1, 2):
        ctx = L.poro_create(0, N, L.PORO_BF16X3_REFINE)
        try:
            L.poro_set_refinement(ctx, sweeps)
            L.poro_set_isolated(ctx, d["vertices"], d["materials"], d["dt"])
            L.poro_set_dofs(ctx, d["Q0"])
            L.poro_predict(ctx)
            res[sweeps] = L.poro_get_predictor(ctx, 0, n)
        finally:
            L.poro_destroy(ctx)
    errs = {k: max(rel_l2(v[i], oracle_predictor(d, i)) for i in range(n)) for k, v in res.items()}
    print(f"N={N} bf16x3 max rel error: 1 sweep {errs[1]:.2e}, 2 sweeps {errs[2]:.2e}")
    assert errs[1] <= TOL_MIXED and errs[2] <= TOL_MIXED


def test_bf16x3_unrefined_is_low_precision(L):
    """Without refinement the bf16 form is far from 1e-10 (so the tolerance
    above tests the refinement)."""
    N, n = 4, 9
    d = population(n, N, seed=77)
    ctx = L.poro_create(0, N, L.PORO_BF16X3_REFINE)
    try:
        L.poro_set_refinement(ctx, 0)
        L.poro_set_isolated(ctx, d["vertices"], d["materials"], d["dt"])
        L.poro_set_dofs(ctx, d["Q0"])
        L.poro_predict(ctx)
        qt = L.poro_get_predictor(ctx, 0, n)
    finally:
        L.poro_destroy(ctx)
    err = max(rel_l2(qt[i], oracle_predictor(d, i)) for i in range(n))
    assert 1e-9 < err < 1e-2


@pytest.mark.parametrize("precision,sweeps", [(0, None), (1, 0), (1, 1), (1, 2), (2, 1)])
def test_non_finite_input_stays_in_its_element(L, precision, sweeps):
    """A NaN in one element's Q0 gives that element a non-finite predictor
    (every entry NaN once refinement rounds it onto the fixed-point grid) and
    leaves every other element bitwise as in a clean run."""
    N, n, bad = 3, 40, 7
    d = population(n, N, seed=99)
    out = []
    for poison in (False, True):
        q0 = d["Q0"].copy()
        if poison:
            q0[bad, 9, 0] = np.nan
        ctx = L.poro_create(0, N, precision)
        try:
            if sweeps is not None:
                L.poro_set_refinement(ctx, sweeps)
            L.poro_set_isolated(ctx, d["vertices"], d["materials"], d["dt"])
            L.poro_set_dofs(ctx, q0)
            L.poro_predict(ctx)
            out.append(L.poro_get_predictor(ctx, 0, n))
        finally:
            L.poro_destroy(ctx)
    clean, dirty = out
    keep = np.arange(n) != bad
    np.testing.assert_array_equal(clean[keep], dirty[keep])
    assert np.isfinite(clean).all()
    assert not np.isfinite(dirty[bad]).all()
    if precision != 0 and sweeps:
        assert np.isnan(dirty[bad]).all()


@pytest.mark.parametrize("scale", [1e-20, 1e20])
@pytest.mark.parametrize("precision", [1, 2])
def test_mixed_is_scale_invariant(L, scale, precision):
    """The predictor is linear in Q0: Q0 scaled by 1e-20 or 1e20 gives the
    oracle's predictor scaled alike, within 1e-10, so the fixed-point grid of
    the refinement (a power of two per quantity from its largest entry)
    follows the data's magnitude."""
    N, n = 4, 7
    d = population(n, N, seed=404)
    ctx = L.poro_create(0, N, precision)
    try:
        L.poro_set_isolated(ctx, d["vertices"], d["materials"], d["dt"])
        L.poro_set_dofs(ctx, d["Q0"] * scale)
        L.poro_predict(ctx)
        qt = L.poro_get_predictor(ctx, 0, n)
    finally:
        L.poro_destroy(ctx)
    err = max(rel_l2(qt[i] / scale, oracle_predictor(d, i)) for i in range(n))
    assert err <= TOL_MIXED, err


def _pade_exp(k, m, z):
    """(k, m) Pade approximant of exp(z), closed form (the P3 pin of the oracle)."""
    from math import factorial

    num = sum(factorial(k + m - j) * factorial(k) / (factorial(k + m) * factorial(j) * factorial(k - j)) * z ** j
              for j in range(k + 1))
    den = sum(factorial(k + m - j) * factorial(m) / (factorial(k + m) * factorial(j) * factorial(m - j)) * (-z) ** j
              for j in range(m + 1))
    return num / den


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("N", [3, 6])
def test_stiff_limit_is_radau_pade(L, N, precision):
    """Stiff Darcy limit on the GPU (the oracle's P3 pin, here for every
    precision form): constant-in-space data (mode 0 only) makes every spatial
    term vanish, so the predictor is DG in time for q' = E* q.  Its end value
    is the (N, N+1) Pade approximant R(e) of exp: uf(1) = R(e) uf0 and
    u(1) = u0 + g/e (R(e) - 1) uf0, the other quantities stay constant.
    The fluid viscosity is scaled by 1 ... 1e6, which puts e = dt E*_ufuf from
    about -2e2 down to about -2e8 (L-stable: R(e) -> 0)."""
    from oracle import material, predictor
    from paper_2108_10565_gb300 import inputs

    for scale in (1.0, 1e2, 1e4, 1e6):
        d = population(6, N, seed=500 + N, viscosity_scale=scale)
        q0 = np.zeros_like(d["Q0"])
        q0[:, :, 0] = d["Q0"][:, :, 0]
        d["Q0"] = q0
        ctx = L.poro_create(0, N, precision)
        try:
            L.poro_set_isolated(ctx, d["vertices"], d["materials"], d["dt"])
            L.poro_set_dofs(ctx, q0)
            L.poro_predict(ctx)
            qt = L.poro_get_predictor(ctx, 0, 6)
        finally:
            L.poro_destroy(ctx)
        assert np.abs(qt[:, :, 1:, :]).max() == 0.0  # higher modes stay exactly zero
        tol = 1e-12 if precision == 0 else TOL_MIXED
        for i in range(6):
            As, Es = predictor.element_operators(d["vertices"][i], inputs.material_dict(d["materials"][i]), d["dt"][i])
            end = qt[i].sum(axis=2)  # chi_s(1) = 1
            for v_, f_ in ((material.U, material.UF), (material.V, material.VF), (material.W, material.WF)):
                e, g = Es[f_, f_], Es[v_, f_]
                R = _pade_exp(N, N + 1, e)
                sc = np.abs(q0[i, :, 0]).max()
                assert abs(end[f_, 0] - R * q0[i, f_, 0]) <= tol * sc, (scale, e)
                assert abs(end[v_, 0] - (q0[i, v_, 0] + g / e * (R - 1) * q0[i, f_, 0])) <= tol * sc, (scale, e)
            for q in (0, 1, 2, 3, 4, 5, 9):
                assert abs(end[q, 0] - q0[i, q, 0]) <= tol * np.abs(q0[i, :, 0]).max()
            ref = predictor.predict_alg3(N, As, Es, q0[i])
            assert rel_l2(qt[i], ref) <= tol, (scale, rel_l2(qt[i], ref))
        if scale == 1e6:
            assert Es[material.UF, material.UF] < -1e7


@pytest.mark.parametrize("precision", [1, 2])
def test_bounded_wait_gives_up_and_context_recovers(L, precision):
    """The bounded-wait path of the mixed kernel: with a wait limit of one SM
    clock every wait that finds its MMA or bulk copy unfinished gives up.  The
    CTA then waits (with the default limit) for what it has in flight, frees
    its tensor memory and raises the context's status; the next synchronising
    call returns PORO_ETIMEOUT once.  With the default limit restored, the
    same context computes the correct predictor."""
    N, n = 4, 48
    d = population(n, N, seed=77)
    ctx = L.poro_create(0, N, precision)
    try:
        L.poro_set_isolated(ctx, d["vertices"], d["materials"], d["dt"])
        L.poro_set_dofs(ctx, d["Q0"])
        L.poro_set_wait_limit(ctx, 1)
        L.poro_predict(ctx)
        with pytest.raises(L.PoroError) as ei:
            L.poro_sync(ctx)
        assert ei.value.status == L.PORO_ETIMEOUT
        L.poro_sync(ctx)  # reported once, then cleared
        L.poro_set_wait_limit(ctx, 0)
        L.poro_predict(ctx)
        L.poro_sync(ctx)
        qt = L.poro_get_predictor(ctx, 0, n)
    finally:
        L.poro_destroy(ctx)
    errs = [rel_l2(qt[i], oracle_predictor(d, i)) for i in range(n)]
    assert max(errs) <= TOL_MIXED


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("N", [3, 4, 5, 6])
def test_tile_choices_agree_and_autotune(L, N, precision):
    """Every tile choice of the autotuner (CTA size x operand-buffer layout
    of the tensor-core sweeps: fewer A buffers or Khat slots serialise the
    directions differently) gives bitwise the predictor of the default
    choice; the autotuner times the available ones and keeps one of them."""
    d = population(23, N, seed=4100 + N)
    ctx = L.poro_create(0, N, precision)
    try:
        L.poro_set_isolated(ctx, d["vertices"], d["materials"], d["dt"])
        L.poro_set_dofs(ctx, d["Q0"])
        L.poro_predict(ctx)
        ref = L.poro_get_predictor(ctx, 0, 23)
        avail = [c for c in range(L.PORO_TILE_CHOICES) if precision == 1 or c < 6]
        for c in avail:
            L.poro_set_tiles(ctx, c)
            L.poro_predict(ctx)
            np.testing.assert_array_equal(L.poro_get_predictor(ctx, 0, 23), ref, err_msg=f"choice {c}")
        with pytest.raises(L.PoroError):
            if precision == 2:
                L.poro_set_tiles(ctx, 6)
            else:
                L.poro_set_tiles(ctx, 12)
        best, ms = L.poro_autotune_tiles(ctx, 0)
        assert best in avail and ms[best] > 0
        assert all((ms[c] > 0) == (c in avail) for c in range(L.PORO_TILE_CHOICES))
        L.poro_predict(ctx)
        np.testing.assert_array_equal(L.poro_get_predictor(ctx, 0, 23), ref)
    finally:
        L.poro_destroy(ctx)
