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


def perturbed_materials(rng, n, spread=0.2, base=REFERENCE_MATERIAL, tie_skeleton=False):
    """Each of the 10 parameters scaled by an independent U[1-spread, 1+spread].
    For spread <= 0.2 around the reference material every draw is physical
    (porosity in (0,1), positive coupling modulus and Biot mass determinant).

    tie_skeleton: K_S, lambda_M and mu_M share the first draw, so the ratio of
    drained to grain bulk modulus stays the base material's.  Needed for soft
    bases such as LAYER_MATERIAL, whose drained modulus is close to K_S: with
    independent draws the drained modulus can exceed K_S and the coupling
    modulus M turns negative.  The same random numbers are consumed either way."""
    f = rng.uniform(1.0 - spread, 1.0 + spread, (n, 10))
    if tie_skeleton:
        f[:, 2] = f[:, 0]
        f[:, 3] = f[:, 0]
    return np.ascontiguousarray(base[None, :] * f)


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


# ---------------------------------------------------------------- meshes
SEED_CFG0 = 2108105650


def kuhn_box_mesh(n, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), periodic=(True, True, True),
                  tags=None, coords=None):
    """Structured tetrahedral mesh: an n[0] x n[1] x n[2] grid of boxes, each
    cut into the 6 Kuhn tetrahedra around its main diagonal (a
    translation-invariant split, so the mesh is conforming, also across
    periodic boundaries).

    Returns dict(vertices [nv][3], tets [ne][4] (vertex ids), neighbors
    [ne][4] (element across face i, the face opposite local vertex i; -1 on
    a boundary), face_tag [ne][4] (0 interior/periodic, 1 free surface,
    2 absorbing)).  `tags` maps a boundary side ('x-', 'x+', ..., 'z+') to a
    tag for non-periodic directions (default absorbing).  `coords` (optional)
    gives the n[a] + 1 grid coordinates of each axis (graded meshes)."""
    n = (n, n, n) if np.isscalar(n) else tuple(n)
    for ax in range(3):
        if periodic[ax] and n[ax] < 3:
            raise ValueError("a periodic direction needs at least 3 boxes (wrapped faces would coincide)")
    lo, hi = np.asarray(lo, float), np.asarray(hi, float)
    h = (hi - lo) / np.asarray(n)
    nx, ny, nz = n
    gi = np.arange(nx + 1)[:, None, None]
    gj = np.arange(ny + 1)[None, :, None]
    gk = np.arange(nz + 1)[None, None, :]

    def vid(i, j, k):
        return (i * (ny + 1) + j) * (nz + 1) + k

    if coords is None:
        coords = [lo[a] + np.arange(n[a] + 1) * h[a] for a in range(3)]
    coords = [np.asarray(c, float) for c in coords]
    assert all(len(coords[a]) == n[a] + 1 for a in range(3))
    vert = np.stack(np.broadcast_arrays(coords[0][gi], coords[1][gj], coords[2][gk]), -1).reshape(-1, 3)
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    # tets in box order (i, j, k), then the 6 vertex paths of the Kuhn split
    bi, bj, bk = [a.reshape(-1) for a in np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")]
    steps = np.zeros((6, 4, 3), dtype=np.int64)
    for p_, pm in enumerate(perms):
        c = np.zeros(3, dtype=np.int64)
        for v, ax in enumerate(pm):
            c[ax] += 1
            steps[p_, v + 1] = c
    ci = bi[:, None, None] + steps[None, :, :, 0]
    cj = bj[:, None, None] + steps[None, :, :, 1]
    ck = bk[:, None, None] + steps[None, :, :, 2]
    tets = vid(ci, cj, ck).reshape(-1, 4).astype(np.int64)
    # face matching on wrapped vertex keys: the 3 sorted keys of every face,
    # sorted; an interior face's key occurs twice
    ijk = np.stack(np.unravel_index(np.arange(vert.shape[0]), (nx + 1, ny + 1, nz + 1)), -1)
    wrapped = ijk.copy()
    for ax, m in enumerate(n):
        if periodic[ax]:
            wrapped[:, ax] %= m
    wkey = (wrapped[:, 0] * (ny + 1) + wrapped[:, 1]) * (nz + 1) + wrapped[:, 2]
    ne = tets.shape[0]
    opp = np.array([[v for v in range(4) if v != f] for f in range(4)])
    fk = np.sort(wkey[tets[:, opp]], axis=2).reshape(-1, 3)  # [ne*4][3]
    order = np.lexsort((fk[:, 2], fk[:, 1], fk[:, 0]))
    sk = fk[order]
    same = np.all(sk[1:] == sk[:-1], axis=1)
    nb = -np.ones(ne * 4, dtype=np.int64)
    a, b = order[:-1][same], order[1:][same]
    nb[a], nb[b] = b // 4, a // 4
    nb = nb.reshape(ne, 4)
    tag = np.zeros((ne, 4), dtype=np.int32)
    tags = tags or {}
    be, bf = np.nonzero(nb < 0)
    if be.size:
        fv = ijk[tets[be[:, None], opp[bf]]]   # [nb][3][3]
        side = np.full(be.size, "", dtype=object)
        for ax, name in enumerate("xyz"):
            side[np.all(fv[:, :, ax] == 0, axis=1)] = name + "-"
            side[np.all(fv[:, :, ax] == n[ax], axis=1)] = name + "+"
        tag[be, bf] = [tags.get(sd, 2) if sd else 2 for sd in side]
    return dict(vertices=vert, tets=tets, neighbors=nb, face_tag=tag)


def config0_scenario():
    """Plain method, small: unit cube, 4^3 boxes x 6 = 384 tetrahedra, periodic,
    degree 2, 50 steps, homogeneous sandstone-like material, pressure point
    source at the centre with a Ricker wavelet f0 = 10 kHz, t0 = 1e-4 s
    (10 Hz scaled from km to m), 4 receivers at seeded positions in
    [0.1, 0.9]^3, Q0 = 0."""
    mesh = kuhn_box_mesh(4)
    rng = np.random.Generator(np.random.PCG64(SEED_CFG0))
    rec = rng.uniform(0.1, 0.9, (4, 3))
    w = np.zeros(13)
    w[9] = 1.0
    ne = mesh["tets"].shape[0]
    return dict(mesh=mesh, N=2, n_steps=50, materials=np.tile(REFERENCE_MATERIAL, (ne, 1)),
                source=dict(x=np.array([0.5, 0.5, 0.5]), w=w, f0=1.0e4, t0=1.0e-4, amplitude=1.0),
                receivers=rec, Q0=np.zeros((ne, 13, 10)))


# layer over half-space (Table material_heterogeneous columns, viscous fluid)
LAYER_MATERIAL = np.array([7.6e9, 2210.0, 3.96e9, 3.96e9, 1e-12, 0.16, 2.0, 2.5e9, 1040.0, 1e-3])
HALFSPACE_MATERIAL = np.array([40e9, 2500.0, 12e9, 12e9, 6e-12, 0.2, 2.0, 2.5e9, 1040.0, 1e-3])
SEED_CFG2 = 2108105652
SEED_LOH = 2108105653
SEED_SERVING = 2108105654


def layered_graded_mesh(nz, radius=2000.0, grading=32.0, layer_depth=500.0):
    """Layer-over-half-space geometry on a graded tetrahedral mesh (the shape
    of the LOHp setting, scaled): a Kuhn mesh of the parameter box
    [-1, 1]^2 x [-1, 0] with 2nz x 2nz x nz boxes is mapped radially about
    the surface origin by rho' = R (exp(k rho) - 1) / (exp(k) - 1),
    k = ln(grading) / sqrt(3): z = 0 stays planar (free surface), edge
    lengths grow ~grading-fold from the origin outwards; absorbing faces
    elsewhere.  Elements with centroid depth < layer_depth get the layer
    material, the others the half-space material."""
    n = (2 * nz, 2 * nz, nz)
    mesh = kuhn_box_mesh(n, lo=(-1.0, -1.0, -1.0), hi=(1.0, 1.0, 0.0), periodic=(False, False, False),
                         tags={"z+": 1})
    v = mesh["vertices"]
    rho = np.linalg.norm(v, axis=1)
    k = np.log(grading) / np.sqrt(3.0)
    scale = np.where(rho > 0, radius * (np.exp(k * rho) - 1.0) / (np.exp(k) - 1.0) / np.maximum(rho, 1e-300), 0.0)
    mesh["vertices"] = v * scale[:, None]
    depth = -mesh["vertices"][mesh["tets"]].mean(axis=1)[:, 2]
    mats = np.where((depth < layer_depth)[:, None], LAYER_MATERIAL[None, :], HALFSPACE_MATERIAL[None, :])
    return mesh, np.ascontiguousarray(mats)


def uniform_box_mesh_for(n_target, extent=(20e3, 20e3, 10e3)):
    """Kuhn box mesh with about n_target tetrahedra, n_x = n_y = 2 n_z,
    free surface on top, absorbing elsewhere (the served-ensemble meshes)."""
    nz = max(1, int(round((n_target / 24.0) ** (1.0 / 3.0))))
    n = (2 * nz, 2 * nz, nz)
    return kuhn_box_mesh(n, lo=(0.0, 0.0, -extent[2]), hi=(extent[0], extent[1], 0.0),
                         periodic=(False, False, False), tags={"z+": 1})


# receivers of the LOHp layout (Section "Layer over half-space"): at the free
# surface, in the middle of the 500 m layer, 10 m below the interface and
# 200 m below the 1010 m deep source, at horizontal offsets from the source
LOH_RECEIVERS = np.array([
    [0.0, 0.0, -0.5], [500.0, 0.0, -0.5], [1000.0, 0.0, -0.5], [1900.0, 0.0, -0.5],
    [250.0, 0.0, -250.0], [1000.0, 0.0, -250.0], [500.0, 0.0, -510.0], [0.0, 0.0, -1210.0]])
EXPLOSIVE_WEIGHTS = -np.r_[np.ones(3), np.zeros(6), -1.0, np.zeros(3)]


def cfg3_mini_scenario(nz=8):
    """The small clustered-LTS case: `layered_graded_mesh(nz)` (nz = 8: 16 x 16 x
    8 boxes, 12,288 tets) with 32x grading, degree 3, rate-2 clusters capped at
    6, the explosive source at 1010 m depth (Ricker f0 = 5 Hz, t0 = 0.25 s),
    the 8 LOHp receivers, 20 steps of the largest cluster.  Initial DOFs are
    seeded N(0, 1), so that every element carries data from the first tick
    (the source alone reaches a few elements in this time)."""
    mesh, mats = layered_graded_mesh(nz, grading=32.0)
    ne = mesh["tets"].shape[0]
    rng = np.random.Generator(np.random.PCG64(SEED_LOH))
    q0 = rng.standard_normal((ne, 13, 20))
    return dict(mesh=mesh, materials=mats, N=3, max_clusters=6, n_cycles=20, Q0=q0,
                source=dict(x=np.array([0.0, 0.0, -1010.0]), w=EXPLOSIVE_WEIGHTS.copy(), f0=5.0, t0=0.25,
                            amplitude=1e9),
                receivers=LOH_RECEIVERS.copy())


# damped Maxwell (Section "Other applications"): per-element (eps, mu, sigma)
SEED_MAXWELL = 2108105655


def maxwell_isolated_elements(n, N, seed=SEED_MAXWELL, sigma_scale=1.0):
    """Isolated tetrahedra (the geometry of `isolated_elements`) with
    material rows (eps, mu, sigma): eps ~ U[1, 4], mu ~ U[1, 2], sigma =
    sigma_scale * U[0.5, 1.5]; Q0 [n][6][B] ~ N(0, 1)."""
    B = (N + 1) * (N + 2) * (N + 3) // 6
    ss = np.random.SeedSequence(seed)
    g_geo, g_mat, g_dof = [np.random.Generator(np.random.PCG64(s)) for s in ss.spawn(3)]
    vert = _blockwise(lambda r, k: random_tetrahedra(r, k), g_geo, n, (4, 3))
    mat = _blockwise(lambda r, k: np.stack([r.uniform(1.0, 4.0, k), r.uniform(1.0, 2.0, k),
                                            sigma_scale * r.uniform(0.5, 1.5, k)], axis=1), g_mat, n, (3,))
    q0 = _blockwise(lambda r, k: r.standard_normal((k, 6, B)), g_dof, n, (6, B))
    return dict(vertices=vert, materials=mat, Q0=q0, N=N)


def maxwell_dict(row):
    return {"eps": float(row[0]), "mu": float(row[1]), "sigma": float(row[2])}


SEED_VISCO = 2108105656


def viscoelastic_isolated_elements(n, N, seed=SEED_VISCO, omega_scale=1.0):
    """Isolated tetrahedra (the geometry of `isolated_elements`) with
    viscoelastic material rows of 12 values (rho, lam_u, mu_u, omega_1..3,
    Ylam_1..3, Ymu_1..3): rho ~ U[2000, 3000] kg/m^3, S speed ~ U[1500, 3500]
    m/s, P speed = S speed x U[1.7, 2.0]; relaxation frequencies 2 pi f_c
    (0.1, 1, 10) with f_c = 1 Hz, times omega_scale; anelastic coefficients
    U[0.005, 0.03] of the unrelaxed modulus each (quality factors of about
    20 to 100 over the band).  Q0 [n][27][B] ~ N(0, 1)."""
    B = (N + 1) * (N + 2) * (N + 3) // 6
    ss = np.random.SeedSequence(seed)
    g_geo, g_mat, g_dof = [np.random.Generator(np.random.PCG64(s)) for s in ss.spawn(3)]
    vert = _blockwise(lambda r, k: random_tetrahedra(r, k), g_geo, n, (4, 3))

    def mats(r, k):
        rho = r.uniform(2000.0, 3000.0, k)
        cs = r.uniform(1500.0, 3500.0, k)
        cp = cs * r.uniform(1.7, 2.0, k)
        mu = rho * cs ** 2
        lam = rho * cp ** 2 - 2 * mu
        om = np.tile(omega_scale * 2 * np.pi * np.array([0.1, 1.0, 10.0]), (k, 1))
        ylam = lam[:, None] * r.uniform(0.005, 0.03, (k, 3))
        ymu = mu[:, None] * r.uniform(0.005, 0.03, (k, 3))
        return np.concatenate([rho[:, None], lam[:, None], mu[:, None], om, ylam, ymu], axis=1)

    mat = _blockwise(mats, g_mat, n, (12,))
    q0 = _blockwise(lambda r, k: r.standard_normal((k, 27, B)), g_dof, n, (27, B))
    return dict(vertices=vert, materials=mat, Q0=q0, N=N)


def viscoelastic_dict(row):
    return {"rho": float(row[0]), "lam": float(row[1]), "mu": float(row[2]), "omega": np.array(row[3:6], float),
            "Ylam": np.array(row[6:9], float), "Ymu": np.array(row[9:12], float)}


SEED_SUBCELL = 2108105657


def subcell_isolated_elements(n, N, seed=SEED_SUBCELL, spread=0.1):
    """Isolated tetrahedra (the geometry of `isolated_elements`) whose four
    vertices carry their own material: each element's centre material is
    scaled per parameter by U[0.8, 1.2] around REFERENCE_MATERIAL (skeleton
    moduli tied), and each vertex material by a further U[1 - spread,
    1 + spread] per parameter (skeleton moduli tied).  materials [n][4][10],
    Q0 [n][13][B] ~ N(0, 1)."""
    B = (N + 1) * (N + 2) * (N + 3) // 6
    ss = np.random.SeedSequence(seed)
    g_geo, g_mat, g_dof = [np.random.Generator(np.random.PCG64(s)) for s in ss.spawn(3)]
    vert = _blockwise(lambda r, k: random_tetrahedra(r, k), g_geo, n, (4, 3))

    def mats(r, k):
        centre = perturbed_materials(r, k, tie_skeleton=True)
        f = r.uniform(1.0 - spread, 1.0 + spread, (k, 4, 10))
        f[:, :, 2] = f[:, :, 0]
        f[:, :, 3] = f[:, :, 0]
        return centre[:, None, :] * f

    mat = _blockwise(mats, g_mat, n, (4, 10))
    q0 = _blockwise(lambda r, k: r.standard_normal((k, 13, B)), g_dof, n, (13, B))
    return dict(vertices=vert, materials=mat, Q0=q0, N=N)
