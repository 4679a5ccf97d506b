"""Seeded synthetic inputs shared by the CUDA path, its tests and the oracle.

This module draws random numbers and shapes them; it holds none of the
predictor's arithmetic (no Jacobians, no basis, no time step).  Each side
derives everything else from these arrays on its own.

Workloads (the paper's meshes and data are not available, so these stand in
for them with the same shapes and value ranges):
  * `isolated_elements`: a population of unconnected tetrahedra, as in the
    paper's performance proxy (random data, one predictor per element,
    Section "Roofline model"), with per-element Biot material around the
    sandstone-like reference material and Q0 ~ N(0, 1).
"""
import numpy as np

# sandstone-like reference material (SI units); order of
# Table poroelastic_parameters: K_S, rho_S, lambda_M, mu_M, kappa, phi, T, K_F, rho_F, nu
REFERENCE_MATERIAL = np.array([40e9, 2650.0, 12e9, 12e9, 6e-13, 0.2, 2.0, 2.5e9, 1040.0, 1e-3])
PARAM_NAMES = ("K_S", "rho_S", "lambda_M", "mu_M", "kappa", "phi", "T", "K_F", "rho_F", "nu")

SEED_ISOLATED = 2108105651

_REF_TET = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])


def _random_rotations(rng, n):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def _aspect_ratio(v):
    """(longest edge) / (2 sqrt(6) r_in); 1 for the regular tetrahedron."""
    e = [v[:, b] - v[:, a] for a in range(4) for b in range(a + 1, 4)]
    longest = np.max(np.stack([np.linalg.norm(x, axis=1) for x in e]), axis=0)
    vol = np.abs(np.einsum("ij,ij->i", v[:, 1] - v[:, 0],
                           np.cross(v[:, 2] - v[:, 0], v[:, 3] - v[:, 0]))) / 6.0
    area = 0.0
    for i in range(4):
        a, b, c = [v[:, k] for k in range(4) if k != i]
        area = area + 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)
    r_in = 3.0 * vol / area
    return longest / (2.0 * np.sqrt(6.0) * r_in)


def random_tetrahedra(rng, n, h_range=(50.0, 200.0), max_aspect=4.0):
    """n tetrahedra x = c + h R1 diag(1, a, b) R2 (xi - 1/4), h log-uniform in
    h_range, a, b ~ U[0.5, 1], random rotations; aspect ratio <= max_aspect.
    Returns vertices [n][4][3]."""
    out = np.empty((0, 4, 3))
    while out.shape[0] < n:
        m = 2 * (n - out.shape[0]) + 16
        h = np.exp(rng.uniform(np.log(h_range[0]), np.log(h_range[1]), m))
        ab = rng.uniform(0.5, 1.0, (m, 2))
        R1, R2 = _random_rotations(rng, m), _random_rotations(rng, m)
        c = rng.uniform(-1000.0, 1000.0, (m, 3))
        D = np.zeros((m, 3, 3))
        D[:, 0, 0], D[:, 1, 1], D[:, 2, 2] = 1.0, ab[:, 0], ab[:, 1]
        L = h[:, None, None] * R1 @ D @ R2
        v = c[:, None, :] + np.einsum("nij,kj->nki", L, _REF_TET - 0.25)
        keep = _aspect_ratio(v) <= max_aspect
        out = np.concatenate([out, v[keep]])
    return np.ascontiguousarray(out[:n])


def perturbed_materials(rng, n, spread=0.2, base=REFERENCE_MATERIAL):
    """Each of the 10 parameters scaled by an independent U[1-spread, 1+spread].
    For spread <= 0.2 around the reference material every draw is physical
    (porosity in (0,1), positive coupling modulus and Biot mass determinant)."""
    return np.ascontiguousarray(base[None, :] * rng.uniform(1.0 - spread, 1.0 + spread, (n, 10)))


def isolated_elements(n, N, seed=SEED_ISOLATED, q0_scale=1.0):
    """The isolated-element population: dict with vertices [n][4][3],
    materials [n][10] and Q0 [n][13][B(N)] ~ N(0, q0_scale^2).

    The three arrays are drawn from three independent child streams of
    `seed`, so the first k elements of a population of n > k are identical
    to a population of k (samples of the full workload are reproducible)."""
    B = (N + 1) * (N + 2) * (N + 3) // 6
    ss = np.random.SeedSequence(seed)
    g_geo, g_mat, g_dof = [np.random.Generator(np.random.PCG64(s)) for s in ss.spawn(3)]
    vert = _blockwise(lambda r, k: random_tetrahedra(r, k), g_geo, n, (4, 3))
    mat = _blockwise(lambda r, k: perturbed_materials(r, k), g_mat, n, (10,))
    q0 = _blockwise(lambda r, k: q0_scale * r.standard_normal((k, 13, B)), g_dof, n, (13, B))
    return dict(vertices=vert, materials=mat, Q0=q0, N=N)


_CHUNK = 1024


def _blockwise(fn, rng, n, shape):
    """Draw in chunks of _CHUNK items from per-chunk child streams so that a
    prefix of the population does not depend on n."""
    out = np.empty((n,) + shape)
    seeds = np.random.SeedSequence(int(rng.integers(0, 2 ** 63))).spawn((n + _CHUNK - 1) // _CHUNK)
    for c, s in enumerate(seeds):
        lo, hi = c * _CHUNK, min(n, (c + 1) * _CHUNK)
        # always draw a full chunk, then truncate: the draws do not depend on n
        out[lo:hi] = fn(np.random.Generator(np.random.PCG64(s)), _CHUNK)[: hi - lo]
    return out


def material_dict(row):
    return {k: float(v) for k, v in zip(PARAM_NAMES, row)}
