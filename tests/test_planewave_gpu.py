"""Full-scheme convergence on the GPU (pin P7 at scale): plane waves of the
Biot system (fast P + two S waves, k = (pi, pi, pi)) on the periodic cube
[-1, 1]^3 cut into 6 n^3 Kuhn tetrahedra, run through the C ABI with global
time stepping to t ~ 1e-4 s.  The error against the projected exact solution
must fall at the optimal rate N + 1 (paper, Section "Convergence"): within 0.3
on the finest pair of meshes 4^3, 8^3, 16^3, for N = 1..6."""
import numpy as np
import pytest

from oracle import planewave
from paper_2108_10565_gb300 import inputs

pytestmark = pytest.mark.gpu

K = np.array([np.pi, np.pi, np.pi])
T_END = 1e-4


@pytest.fixture(scope="module")
def L():
    from paper_2108_10565_gb300 import _lib

    return _lib


def _run(L, N, n, precision, norms=False):
    md = inputs.material_dict(inputs.REFERENCE_MATERIAL)
    modes = planewave.plane_wave_modes(md, K, 3)
    mesh = inputs.kuhn_box_mesh(n, lo=(-1, -1, -1), hi=(1, 1, 1))
    ne = len(mesh["tets"])
    ctx = L.poro_create(0, N, precision)
    try:
        L.poro_set_mesh(ctx, mesh["vertices"], mesh["tets"], mesh["neighbors"], mesh["face_tag"])
        L.poro_set_materials(ctx, np.tile(inputs.REFERENCE_MATERIAL, (ne, 1)))
        L.poro_set_clusters(ctx, 0.5, 1)
        v = mesh["vertices"][mesh["tets"]]
        L.poro_set_dofs(ctx, planewave.project(v, N, lambda x: planewave.plane_wave(x, 0.0, K, modes)))
        L.poro_advance(ctx, T_END)
        Q = L.poro_get_dofs(ctx)
        t, _ = L.poro_get_time(ctx)
    finally:
        L.poro_destroy(ctx)
    Qref = planewave.project(v, N, lambda x: planewave.plane_wave(x, t, K, modes))
    e, r = planewave.dg_error(v, N, Q, Qref)
    if norms:
        nr = planewave.error_norms(v, N, Q, lambda x: planewave.plane_wave(x, t, K, modes))
        return e / r, [a / b for a, b in zip(nr["err"], nr["ref"])]
    return e / r


@pytest.mark.parametrize("N,prec", [(1, "fp64"), (2, "fp64"), (3, "fp64"), (3, "mixed"), (4, "fp64"), (5, "fp64"),
                                    (6, "fp64"), (6, "bf16")])
def test_plane_wave_convergence_rate(L, N, prec):
    precision = {"fp64": L.PORO_FP64, "mixed": L.PORO_FP32_REFINE, "bf16": L.PORO_BF16X3_REFINE}[prec]
    errs = [_run(L, N, n, precision) for n in (4, 8, 16)]
    rates = [float(np.log2(errs[i] / errs[i + 1])) for i in range(2)]
    print(f"N={N} {prec}: rel L2 errors {errs}, rates {rates}")
    assert errs[0] > errs[1] > errs[2]
    assert abs(rates[1] - (N + 1)) < 0.3, (errs, rates)


@pytest.mark.parametrize("N", [2, 4])
def test_plane_wave_l1_linf_rates(L, N):
    """The pointwise error of the DG field against the exact plane wave in
    the L1 and L-infinity norms (oracle.planewave.error_norms) falls at about
    N + 1 too (L-infinity within 0.5: the maximum is taken over a finite
    point set)."""
    res = [_run(L, N, n, L.PORO_FP64, norms=True)[1] for n in (4, 8, 16)]
    for k, name in ((0, "L1"), (2, "Linf")):
        rate = float(np.log2(res[1][k] / res[2][k]))
        print(f"N={N} {name}: {[r[k] for r in res]}, finest rate {rate:.2f}")
        assert abs(rate - (N + 1)) < (0.3 if k == 0 else 0.5), (name, rate)
