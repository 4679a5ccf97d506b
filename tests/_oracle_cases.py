"""Helpers shared by the GPU parity tests: seeded populations and their
oracle predictors.  Everything expected here comes from `oracle/` only."""
import numpy as np

from oracle import geometry, predictor
from paper_2108_10565_gb300 import inputs


def population(n, N, seed, viscosity_scale=1.0):
    d = inputs.isolated_elements(n, N, seed=seed)
    if viscosity_scale != 1.0:
        d["materials"] = d["materials"].copy()
        d["materials"][:, 9] *= viscosity_scale
    d["dt"] = np.array([geometry.cfl_dt(d["vertices"][i], inputs.material_dict(d["materials"][i]), N)
                        for i in range(n)])
    return d


def oracle_predictor(d, i, dense=False):
    """Oracle predictor of element i: dense LU of Y (definition) or
    Algorithm 3 written as plain loops (pinned to the dense solve)."""
    N = d["N"]
    As, Es = predictor.element_operators(d["vertices"][i], inputs.material_dict(d["materials"][i]), d["dt"][i])
    fn = predictor.predict_dense if dense else predictor.predict_alg3
    return fn(N, As, Es, d["Q0"][i])


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)
