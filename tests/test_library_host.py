"""CPU-side checks of libporoader: the library builds and loads, exports every
symbol include/poroader.h declares, and its host set-up (its own quadrature
and derivation) agrees with the oracle.  No GPU compute here."""
import os
import re

import numpy as np
import pytest

from oracle import basis, geometry, material
from paper_2108_10565_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2108_10565_gb300 import _lib

    if not os.path.exists(_lib.LIB_PATH):
        from paper_2108_10565_gb300 import build

        build.build()
    return _lib


def _declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(poro_[a-z0-9_]+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol(L):
    lib = L.load()
    declared = _declared_symbols()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    bound = {n for n, _, _ in L.SIGNATURES}
    assert declared == bound, f"binding and header differ: {declared ^ bound}"


@pytest.mark.parametrize("N", range(1, 7))
def test_reference_matrices_match_oracle(L, N):
    m, k = L.poro_reference_matrices(N)
    mo = np.diag(basis.mass_matrix(N))
    ko = np.stack(basis.khat_matrices(N))
    np.testing.assert_allclose(m, mo, rtol=1e-14)
    assert np.abs(k - ko).max() <= 1e-14 * np.abs(ko).max()
    np.testing.assert_array_equal(k != 0, ko != 0)  # identical structural zeros


def test_jacobians_and_speed_match_oracle(L):
    rng = np.random.default_rng(3)
    for row in inputs.perturbed_materials(rng, 5):
        abc, e = L.poro_material_jacobians(row)
        md = inputs.material_dict(row)
        A = np.stack(material.jacobians(md))
        E = material.source_matrix(md)
        assert np.abs(abc - A).max() <= 1e-15 * np.abs(A).max()
        assert np.abs(e - E).max() <= 1e-14 * np.abs(E).max()
        assert L.poro_max_wave_speed(row) == pytest.approx(geometry.max_wave_speed(md), rel=1e-13)


def test_cfl_matches_oracle(L):
    d = inputs.isolated_elements(20, 4, seed=9)
    dt = L.poro_cfl_dt(4, d["vertices"], d["materials"])
    ref = [geometry.cfl_dt(d["vertices"][i], inputs.material_dict(d["materials"][i]), 4) for i in range(20)]
    np.testing.assert_allclose(dt, ref, rtol=1e-13)


def test_invalid_inputs_rejected(L):
    bad = inputs.REFERENCE_MATERIAL.copy()
    bad[5] = 1.5  # porosity
    with pytest.raises(L.PoroError) as ex:
        L.poro_material_jacobians(bad)
    assert ex.value.status == L.PORO_EINVAL
    flat = np.zeros((1, 4, 3))
    with pytest.raises(L.PoroError) as ex:
        L.poro_cfl_dt(3, flat, inputs.REFERENCE_MATERIAL[None, :])
    assert ex.value.status == L.PORO_EINVAL
    with pytest.raises(L.PoroError) as ex:
        L.poro_reference_matrices(7)
    assert ex.value.status == L.PORO_EUNSUPPORTED


def test_flux_matrices_match_oracle(L):
    """The library's flux solvers (matrix sign function) against the
    oracle's (characteristic decomposition), in the impedance-scaled frame."""
    from oracle import flux

    rng = np.random.default_rng(0)
    mats = inputs.perturbed_materials(rng, 3)
    mats[1, 9] = 0.0  # inviscid neighbour
    for n in ([1, 0, 0], [0, 0, -1], np.array([1, 2, -2]) / 3.0):
        n = np.array(n, float)
        An = flux.normal_jacobian(inputs.material_dict(mats[0]), n)
        s = np.ones(13)
        s[[0, 1, 2, 3, 4, 5, 9]] = np.sqrt(np.abs(An[[0, 1, 2, 3, 4, 5, 9]]).max() /
                                           np.abs(An[[6, 7, 8, 10, 11, 12]]).max())
        sc = s[None, :] / s[:, None]
        amax = np.abs(An * sc).max()
        for kind, name in ((0, "interior"), (1, "free_surface"), (2, "absorbing")):
            Fm, Fp = L.poro_flux_matrices(mats[0], mats[1] if kind == 0 else None, n, kind)
            om, op = flux.flux_matrices(inputs.material_dict(mats[0]),
                                        inputs.material_dict(mats[1]) if kind == 0 else None, n, name)
            assert np.abs((Fm - om) * sc).max() < 1e-13 * amax
            assert np.abs((Fp - op) * sc).max() < 1e-13 * amax


@pytest.mark.parametrize("N", [3, 6])
def test_library_khat_rows_match_oracle_fractions(L, N):
    """The library's own quadrature gives the same rational rows (numerators
    over a common denominator) that its mixed residual packs."""
    from tests.test_oracle_pins import khat_row_fractions

    _, k = L.poro_reference_matrices(N)
    ko = basis.khat_matrices(N)
    for a in range(3):
        assert khat_row_fractions(k[a]) == khat_row_fractions(ko[a])


def test_perturbed_layer_materials_stay_physical():
    """The served-ensemble recipe (layer and half-space, +-20 %, skeleton
    moduli tied): every draw is in the model's domain, while independent
    draws of the soft layer's moduli are not (drained modulus above K_S)."""
    rng = np.random.default_rng(11)
    for base in (inputs.LAYER_MATERIAL, inputs.HALFSPACE_MATERIAL, inputs.REFERENCE_MATERIAL):
        for row in inputs.perturbed_materials(rng, 2000, base=base, tie_skeleton=True):
            material.check_physical(inputs.material_dict(row))
    bad = 0
    for row in inputs.perturbed_materials(rng, 2000, base=inputs.LAYER_MATERIAL):
        try:
            material.check_physical(inputs.material_dict(row))
        except ValueError:
            bad += 1
    assert bad > 0


def test_cfl_other_systems_match_oracle(L):
    """poro_cfl_dt_system: the CFL step of the damped Maxwell and viscoelastic
    material rows against the oracle's statement of each system."""
    from oracle import maxwell, viscoelastic

    for system, gen, mod, to_dict in ((L.PORO_SYSTEM_MAXWELL, inputs.maxwell_isolated_elements, maxwell,
                                       inputs.maxwell_dict),
                                      (L.PORO_SYSTEM_VISCOELASTIC, inputs.viscoelastic_isolated_elements,
                                       viscoelastic, inputs.viscoelastic_dict)):
        d = gen(40, 4)
        dt = L.poro_cfl_dt_system(system, 4, d["vertices"], d["materials"])
        ref = [mod.cfl_dt(d["vertices"][i], to_dict(d["materials"][i]), 4) for i in range(40)]
        np.testing.assert_allclose(dt, ref, rtol=1e-13)
    bad = inputs.maxwell_isolated_elements(2, 2)
    bad["materials"][1, 0] = -1.0
    with pytest.raises(L.PoroError):
        L.poro_cfl_dt_system(L.PORO_SYSTEM_MAXWELL, 2, bad["vertices"], bad["materials"])
