"""ctypes binding of libporoader (include/poroader.h).

Argument marshalling only: every function has the C name and forwards to the
shared library.  The library is built in-tree (paper_2108_10565_gb300/build.py);
if it is missing, importing the binding raises: there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libporoader.so")

PORO_OK, PORO_EINVAL, PORO_ENOMEM, PORO_ECUDA, PORO_ETIMEOUT, PORO_ESTATE, PORO_ENUMERIC, PORO_EUNSUPPORTED = (
    0, -1, -2, -3, -4, -5, -6, -7)
PORO_FP64, PORO_FP32_REFINE, PORO_BF16X3_REFINE = 0, 1, 2
PORO_SOLVE_BLOCK, PORO_SOLVE_LU = 0, 1
PORO_SYSTEM_BIOT, PORO_SYSTEM_MAXWELL, PORO_SYSTEM_VISCOELASTIC = 0, 1, 2

_c = ctypes
_i32, _i64, _dbl, _vp = _c.c_int32, _c.c_int64, _c.c_double, _c.c_void_p
_pd = _c.POINTER(_c.c_double)

class poro_scenario(ctypes.Structure):
    _fields_ = [("degree_N", ctypes.c_int32), ("precision", ctypes.c_int32), ("refine_sweeps", ctypes.c_int32),
                ("max_clusters", ctypes.c_int32), ("cfl_c", ctypes.c_double), ("t_end", ctypes.c_double),
                ("n_vert", ctypes.c_int64), ("xyz", ctypes.c_void_p), ("n_elem", ctypes.c_int64),
                ("tet", ctypes.c_void_p), ("nb", ctypes.c_void_p), ("face_tag", ctypes.c_void_p),
                ("mat", ctypes.c_void_p), ("Q0", ctypes.c_void_p), ("n_sources", ctypes.c_int32),
                ("n_receivers", ctypes.c_int32), ("src_xyz", ctypes.c_void_p), ("src_w", ctypes.c_void_p),
                ("src_f0", ctypes.c_void_p), ("src_t0", ctypes.c_void_p), ("src_amp", ctypes.c_void_p),
                ("rec_xyz", ctypes.c_void_p)]


PORO_REQ_QUEUED, PORO_REQ_RUNNING, PORO_REQ_DONE, PORO_REQ_FAILED, PORO_REQ_CANCELLED = 0, 1, 2, 3, 4

# (name, restype, argtypes) for every symbol declared in include/poroader.h
SIGNATURES = [
    ("poro_create", _i32, [_c.c_int, _c.c_int, _c.c_int, _c.POINTER(_vp)]),
    ("poro_create_system", _i32, [_c.c_int, _c.c_int, _c.c_int, _c.c_int, _c.POINTER(_vp)]),
    ("poro_get_system", _i32, [_vp, _c.POINTER(_i32), _c.POINTER(_i32)]),
    ("poro_set_isolated_maxwell", _i32, [_vp, _i64, _vp, _vp, _vp]),
    ("poro_set_isolated_viscoelastic", _i32, [_vp, _i64, _vp, _vp, _vp]),
    ("poro_set_isolated_subcell", _i32, [_vp, _i64, _vp, _vp, _vp]),
    ("poro_set_subcell_tolerance", _i32, [_vp, _dbl, _i32]),
    ("poro_get_subcell_iterations", _i32, [_vp, _i64, _i64, _vp]),
    ("poro_cfl_dt_system", _i32, [_i32, _i32, _i64, _vp, _vp, _dbl, _vp]),
    ("poro_destroy", _i32, [_vp]),
    ("poro_last_error", _c.c_char_p, [_vp]),
    ("poro_get_info", _i32, [_vp, _c.POINTER(_i32), _c.POINTER(_i32), _c.POINTER(_i64)]),
    ("poro_reference_matrices", _i32, [_c.c_int, _vp, _vp]),
    ("poro_material_jacobians", _i32, [_vp, _vp, _vp]),
    ("poro_max_wave_speed", _i32, [_vp, _pd]),
    ("poro_cfl_dt", _i32, [_c.c_int, _i64, _vp, _vp, _dbl, _vp]),
    ("poro_set_isolated", _i32, [_vp, _i64, _vp, _vp, _vp]),
    ("poro_set_dofs", _i32, [_vp, _vp]),
    ("poro_predict", _i32, [_vp, _i32, _c.c_int]),
    ("poro_get_predictor", _i32, [_vp, _i64, _i64, _vp]),
    ("poro_get_integrated", _i32, [_vp, _i64, _i64, _vp]),
    ("poro_sync", _i32, [_vp, _i32]),
    ("poro_predict_dev", _i32, [_vp, _i64, _i64, _vp, _vp, _vp, _c.c_int, _vp]),
    ("poro_predict_host", _i32, [_vp, _vp, _vp, _i64, _c.c_int]),
    ("poro_flop_count", _i32, [_vp, _i32, _pd]),
    ("poro_set_refinement", _i32, [_vp, _i32]),
    ("poro_set_wait_limit", _i32, [_vp, _i64]),
    ("poro_lu_bytes", _i32, [_c.c_int, _i64, _c.POINTER(_c.c_size_t)]),
    ("poro_lu_factor", _i32, [_vp, _i64, _i64]),
    ("poro_lu_release", _i32, [_vp]),
    ("poro_lu_predict_static", _i32, [_vp, _i64, _i64, _vp, _vp, _vp, _vp]),
    ("poro_set_mesh", _i32, [_vp, _i64, _vp, _i64, _vp, _vp, _vp]),
    ("poro_set_materials", _i32, [_vp, _vp]),
    ("poro_set_clusters", _i32, [_vp, _dbl, _i32, _pd, _vp]),
    ("poro_add_point_source", _i32, [_vp, _vp, _vp, _dbl, _dbl, _dbl]),
    ("poro_add_receiver", _i32, [_vp, _vp, _c.POINTER(_i32)]),
    ("poro_advance", _i32, [_vp, _dbl]),
    ("poro_cluster_times", _i32, [_vp, _dbl, _vp]),
    ("poro_correct", _i32, [_vp, _i32]),
    ("poro_get_dofs", _i32, [_vp, _vp]),
    ("poro_get_seismogram", _i32, [_vp, _i32, _i64, _vp, _vp, _c.POINTER(_i64)]),
    ("poro_get_time", _i32, [_vp, _pd, _pd]),
    ("poro_flux_matrices", _i32, [_vp, _vp, _vp, _i32, _vp, _vp]),
    ("poro_autotune", _i32, [_vp, _i64, _c.POINTER(_i32), _vp]),
    ("poro_set_variant", _i32, [_vp, _i32]),
    ("poro_autotune_tiles", _i32, [_vp, _i64, _c.POINTER(_i32), _vp]),
    ("poro_set_tiles", _i32, [_vp, _i32]),
    ("poro_set_graphs", _i32, [_vp, _i32]),
    ("poro_server_create", _i32, [_c.c_int, _c.c_size_t, _i32, _c.POINTER(_vp)]),
    ("poro_server_destroy", _i32, [_vp]),
    ("poro_server_set_batching", _i32, [_vp, _i32]),
    ("poro_server_last_error", _c.c_char_p, [_vp]),
    ("poro_submit", _i32, [_vp, _c.POINTER(poro_scenario), _c.POINTER(_c.c_uint64)]),
    ("poro_poll", _i32, [_vp, _c.c_uint64, _c.POINTER(_i32), _pd]),
    ("poro_wait", _i32, [_vp, _c.c_uint64, _i32, _c.POINTER(_i32)]),
    ("poro_fetch", _i32, [_vp, _c.c_uint64, _i32, _i64, _vp, _vp, _c.POINTER(_i64)]),
    ("poro_request_times", _i32, [_vp, _c.c_uint64, _pd, _pd, _pd]),
    ("poro_request_error", _i32, [_vp, _c.c_uint64, _c.c_char_p, _c.c_size_t]),
    ("poro_cancel", _i32, [_vp, _c.c_uint64]),
    ("poro_footprint_bytes", _i32, [_c.c_int, _i64, _i32, _i32, _c.POINTER(_c.c_size_t)]),
]


class PoroError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"poroader error {status}: {msg}")
        self.status = status


def load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libporoader.so not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        _LIB = load()
    return _LIB


def _check(status, ctx=None):
    if status != PORO_OK:
        raise PoroError(status, lib().poro_last_error(ctx).decode())
    return status


def _ptr(a):
    """Host pointer of a C-contiguous numpy array (or None)."""
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"], "arrays passed to libporoader must be C-contiguous"
    return a.ctypes.data


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ------------------------------------------------------------ same-name wrappers
def poro_create(device, degree_N, precision=PORO_FP64, system=PORO_SYSTEM_BIOT):
    h = _vp()
    if system == PORO_SYSTEM_BIOT:
        _check(lib().poro_create(device, degree_N, precision, ctypes.byref(h)))
    else:
        _check(lib().poro_create_system(device, degree_N, precision, system, ctypes.byref(h)))
    return h.value


def poro_get_system(ctx):
    s, q = _i32(), _i32()
    _check(lib().poro_get_system(ctx, ctypes.byref(s), ctypes.byref(q)), ctx)
    return s.value, q.value


def poro_destroy(ctx):
    return _check(lib().poro_destroy(ctx))


def poro_last_error(ctx=None):
    return lib().poro_last_error(ctx).decode()


def poro_get_info(ctx):
    n, p, e = _i32(), _i32(), _i64()
    _check(lib().poro_get_info(ctx, ctypes.byref(n), ctypes.byref(p), ctypes.byref(e)), ctx)
    return n.value, p.value, e.value


def poro_reference_matrices(N):
    B = (N + 1) * (N + 2) * (N + 3) // 6
    m = np.zeros(B)
    k = np.zeros((3, B, B))
    _check(lib().poro_reference_matrices(N, _ptr(m), _ptr(k)))
    return m, k


def poro_material_jacobians(mat10):
    m = _f64(mat10)
    abc = np.zeros((3, 13, 13))
    e = np.zeros((13, 13))
    _check(lib().poro_material_jacobians(_ptr(m), _ptr(abc), _ptr(e)))
    return abc, e


def poro_max_wave_speed(mat10):
    m = _f64(mat10)
    v = _dbl()
    _check(lib().poro_max_wave_speed(_ptr(m), ctypes.byref(v)))
    return v.value


def poro_cfl_dt(N, vert, mat, cfl_c=0.5):
    v, m = _f64(vert), _f64(mat)
    n = v.shape[0]
    dt = np.zeros(n)
    _check(lib().poro_cfl_dt(N, n, _ptr(v), _ptr(m), cfl_c, _ptr(dt)))
    return dt


def poro_cfl_dt_system(system, N, vert, mat, cfl_c=0.5):
    v, m = _f64(vert), _f64(mat)
    n = v.shape[0]
    dt = np.empty(n)
    _check(lib().poro_cfl_dt_system(system, N, n, _ptr(v), _ptr(m), cfl_c, _ptr(dt)))
    return dt


def poro_set_isolated(ctx, vert, mat, dt):
    v, m, d = _f64(vert), _f64(mat), _f64(dt)
    return _check(lib().poro_set_isolated(ctx, v.shape[0], _ptr(v), _ptr(m), _ptr(d)), ctx)


def poro_set_isolated_maxwell(ctx, vert, mat, dt):
    """mat[n][3] = (eps, mu, sigma) per element."""
    v, m, d = _f64(vert), _f64(mat), _f64(dt)
    return _check(lib().poro_set_isolated_maxwell(ctx, v.shape[0], _ptr(v), _ptr(m), _ptr(d)), ctx)


def poro_set_isolated_subcell(ctx, vert, mat, dt):
    """mat[n][4][10]: the material rows of each element's four vertices."""
    v, m, d = _f64(vert), _f64(mat), _f64(dt)
    if m.size != v.shape[0] * 4 * 10:
        raise ValueError("mat must hold 4 material rows of 10 values per element")
    return _check(lib().poro_set_isolated_subcell(ctx, v.shape[0], _ptr(v), _ptr(m), _ptr(d)), ctx)


def poro_set_subcell_tolerance(ctx, tol, max_iter):
    return _check(lib().poro_set_subcell_tolerance(ctx, tol, max_iter), ctx)


def poro_get_subcell_iterations(ctx, first, count):
    out = np.empty(count, dtype=np.int32)
    _check(lib().poro_get_subcell_iterations(ctx, first, count, out.ctypes.data_as(ctypes.c_void_p)), ctx)
    return out


def poro_set_isolated_viscoelastic(ctx, vert, mat, dt):
    """mat[n][12] = (rho, lam_u, mu_u, omega_1..3, Ylam_1..3, Ymu_1..3) per element."""
    v, m, d = _f64(vert), _f64(mat), _f64(dt)
    return _check(lib().poro_set_isolated_viscoelastic(ctx, v.shape[0], _ptr(v), _ptr(m), _ptr(d)), ctx)


def _out(out, shape):
    """A C-contiguous float64 buffer of `shape` for the library to fill:
    `out` if it is one, a new array if out is None."""
    if out is None:
        return np.empty(shape)
    if not (isinstance(out, np.ndarray) and out.dtype == np.float64 and out.flags.c_contiguous
            and out.size == int(np.prod(shape))):
        raise ValueError(f"out must be a C-contiguous float64 array of shape {shape}")
    return out


def poro_set_dofs(ctx, Q):
    N, _, n = poro_get_info(ctx)
    nq = poro_get_system(ctx)[1]
    q = _f64(Q)
    if n > 0 and q.size != n * nq * ((N + 1) * (N + 2) * (N + 3) // 6):
        raise ValueError(f"Q must hold {n} elements x {nq} quantities x B(N) modes")
    return _check(lib().poro_set_dofs(ctx, _ptr(q)), ctx)


def poro_predict(ctx, cluster=-1, solver=PORO_SOLVE_BLOCK):
    return _check(lib().poro_predict(ctx, cluster, solver), ctx)


def poro_get_predictor(ctx, first, count, out=None):
    N, _, _ = poro_get_info(ctx)
    nq = poro_get_system(ctx)[1]
    B, T = (N + 1) * (N + 2) * (N + 3) // 6, N + 1
    out = _out(out, (count, nq, B, T))
    _check(lib().poro_get_predictor(ctx, first, count, _ptr(out)), ctx)
    return out


def poro_get_integrated(ctx, first, count, out=None):
    N, _, _ = poro_get_info(ctx)
    nq = poro_get_system(ctx)[1]
    B = (N + 1) * (N + 2) * (N + 3) // 6
    out = _out(out, (count, nq, B))
    _check(lib().poro_get_integrated(ctx, first, count, _ptr(out)), ctx)
    return out


def poro_sync(ctx, timeout_ms=-1):
    return _check(lib().poro_sync(ctx, timeout_ms), ctx)


def poro_predict_host(ctx, Q0, out=None, chunk_elems=0, solver=PORO_SOLVE_BLOCK):
    """End to end from host arrays: Q0[n][Q][B] in, I[n][Q][B] out (Q the
    system's quantities), copies overlapped with the kernels (pass pinned
    arrays for the overlap)."""
    N, _, n = poro_get_info(ctx)
    nq = poro_get_system(ctx)[1]
    B = (N + 1) * (N + 2) * (N + 3) // 6
    q = _f64(Q0)
    if n > 0 and q.size != n * nq * B:
        raise ValueError(f"Q0 must hold {n} x {nq} x {B} values")
    out = _out(out, (n, nq, B))
    _check(lib().poro_predict_host(ctx, _ptr(q), _ptr(out), chunk_elems, solver), ctx)
    return out


def poro_predict_dev(ctx, first, count, q0_ptr, qt_ptr, i_ptr, solver=PORO_SOLVE_BLOCK, stream=None):
    """Device-pointer form; pointers are integers (e.g. torch.Tensor.data_ptr())."""
    return _check(lib().poro_predict_dev(ctx, first, count, q0_ptr, qt_ptr, i_ptr, solver, stream), ctx)


def poro_set_refinement(ctx, sweeps):
    return _check(lib().poro_set_refinement(ctx, sweeps), ctx)


def poro_set_wait_limit(ctx, cycles):
    return _check(lib().poro_set_wait_limit(ctx, cycles), ctx)


def poro_lu_bytes(N, count):
    b = ctypes.c_size_t()
    _check(lib().poro_lu_bytes(N, count, ctypes.byref(b)))
    return b.value


def poro_lu_factor(ctx, first, count):
    return _check(lib().poro_lu_factor(ctx, first, count), ctx)


def poro_lu_release(ctx):
    return _check(lib().poro_lu_release(ctx), ctx)


def poro_lu_predict_static(ctx, first, count, q0_ptr, qt_ptr, i_ptr, stream=None):
    """Allocation-free dense-LU predictor (device pointers as integers)."""
    return _check(lib().poro_lu_predict_static(ctx, first, count, q0_ptr, qt_ptr, i_ptr, stream), ctx)


def poro_set_mesh(ctx, vertices, tets, neighbors, face_tag):
    v = _f64(vertices)
    t = np.ascontiguousarray(tets, dtype=np.int64)
    nb = np.ascontiguousarray(neighbors, dtype=np.int64)
    tg = np.ascontiguousarray(face_tag, dtype=np.int32)
    return _check(lib().poro_set_mesh(ctx, v.shape[0], _ptr(v), t.shape[0], _ptr(t), _ptr(nb), _ptr(tg)), ctx)


def poro_set_materials(ctx, mat):
    m = _f64(mat)
    return _check(lib().poro_set_materials(ctx, _ptr(m)), ctx)


def poro_set_clusters(ctx, cfl_c=0.5, max_clusters=1, n_elem=None):
    dt = _dbl()
    cl = np.zeros(n_elem, dtype=np.int32) if n_elem else None
    _check(lib().poro_set_clusters(ctx, cfl_c, max_clusters, ctypes.byref(dt), _ptr(cl)), ctx)
    return dt.value, cl


def poro_add_point_source(ctx, xyz, w, f0, t0, amplitude=1.0):
    x, ww = _f64(xyz), _f64(w)
    return _check(lib().poro_add_point_source(ctx, _ptr(x), _ptr(ww), f0, t0, amplitude), ctx)


def poro_add_receiver(ctx, xyz):
    x = _f64(xyz)
    i = _i32()
    _check(lib().poro_add_receiver(ctx, _ptr(x), ctypes.byref(i)), ctx)
    return i.value


def poro_advance(ctx, t_end):
    return _check(lib().poro_advance(ctx, t_end), ctx)


def poro_cluster_times(ctx, t_end, n_clusters):
    """poro_advance without graphs; returns the GPU ms of each of the
    context's n_clusters clusters' launches."""
    ms = np.zeros(max(1, n_clusters))
    _check(lib().poro_cluster_times(ctx, t_end, _ptr(ms)), ctx)
    return ms


def poro_correct(ctx, cluster=-1):
    return _check(lib().poro_correct(ctx, cluster), ctx)


def poro_get_dofs(ctx, out=None):
    N, _, n = poro_get_info(ctx)
    nq = poro_get_system(ctx)[1]
    B = (N + 1) * (N + 2) * (N + 3) // 6
    out = _out(out, (n, nq, B))
    _check(lib().poro_get_dofs(ctx, _ptr(out)), ctx)
    return out


def poro_get_seismogram(ctx, rec):
    n = _i64()
    _check(lib().poro_get_seismogram(ctx, rec, 0, None, None, ctypes.byref(n)), ctx)
    t = np.empty(n.value)
    q = np.empty((n.value, 13))
    _check(lib().poro_get_seismogram(ctx, rec, n.value, _ptr(t), _ptr(q), ctypes.byref(n)), ctx)
    return t, q


def poro_get_time(ctx):
    t, dt = _dbl(), _dbl()
    _check(lib().poro_get_time(ctx, ctypes.byref(t), ctypes.byref(dt)), ctx)
    return t.value, dt.value


def poro_flux_matrices(matL, matR, n, kind):
    mL = _f64(matL)
    mR = _f64(matR) if matR is not None else None
    nn = _f64(n)
    Fm, Fp = np.zeros((13, 13)), np.zeros((13, 13))
    _check(lib().poro_flux_matrices(_ptr(mL), _ptr(mR), _ptr(nn), kind, _ptr(Fm), _ptr(Fp)))
    return Fm, Fp


PORO_FACE_INTERIOR, PORO_FACE_FREE_SURFACE, PORO_FACE_ABSORBING = 0, 1, 2


def poro_autotune(ctx, sample=0):
    v = _i32()
    ms = (ctypes.c_double * 2)()
    _check(lib().poro_autotune(ctx, sample, ctypes.byref(v), ms), ctx)
    return v.value, list(ms)


def poro_set_graphs(ctx, on):
    return _check(lib().poro_set_graphs(ctx, 1 if on else 0), ctx)


def poro_set_variant(ctx, variant):
    return _check(lib().poro_set_variant(ctx, variant), ctx)


PORO_TILE_CHOICES = 12


def poro_autotune_tiles(ctx, sample=0):
    """Returns (chosen tile choice, ms per choice; -1 where not available)."""
    c = _i32()
    ms = np.zeros(PORO_TILE_CHOICES)
    _check(lib().poro_autotune_tiles(ctx, sample, ctypes.byref(c), _ptr(ms)), ctx)
    return c.value, ms


def poro_set_tiles(ctx, choice):
    return _check(lib().poro_set_tiles(ctx, choice), ctx)


def poro_flop_count(ctx, refine_sweeps=0):
    f = (ctypes.c_double * 3)()
    _check(lib().poro_flop_count(ctx, refine_sweeps, f), ctx)
    return list(f)


# ------------------------------------------------------------ serving
def _srv_check(status, srv):
    if status != PORO_OK:
        raise PoroError(status, lib().poro_server_last_error(srv).decode())
    return status


def poro_server_create(device, hbm_budget, max_slots):
    h = _vp()
    _srv_check(lib().poro_server_create(device, hbm_budget, max_slots, ctypes.byref(h)), None)
    return h.value


def poro_server_destroy(srv):
    return lib().poro_server_destroy(srv)


def poro_server_set_batching(srv, on):
    return _srv_check(lib().poro_server_set_batching(srv, 1 if on else 0), srv)


def make_scenario(N, mesh, materials, t_end, precision=PORO_FP64, max_clusters=1, refine_sweeps=1, cfl_c=0.5,
                  sources=(), receivers=(), Q0=None):
    """Build a poro_scenario; returns (struct, keepalive) -- keep the second
    alive until poro_submit returned (it copies the arrays)."""
    keep = dict(xyz=_f64(mesh["vertices"]), tet=np.ascontiguousarray(mesh["tets"], dtype=np.int64),
                nb=np.ascontiguousarray(mesh["neighbors"], dtype=np.int64),
                tag=np.ascontiguousarray(mesh["face_tag"], dtype=np.int32), mat=_f64(materials))
    sc = poro_scenario()
    sc.degree_N, sc.precision, sc.refine_sweeps, sc.max_clusters = N, precision, refine_sweeps, max_clusters
    sc.cfl_c, sc.t_end = cfl_c, t_end
    sc.n_vert, sc.xyz = keep["xyz"].shape[0], _ptr(keep["xyz"])
    sc.n_elem, sc.tet, sc.nb = keep["tet"].shape[0], _ptr(keep["tet"]), _ptr(keep["nb"])
    sc.face_tag, sc.mat = _ptr(keep["tag"]), _ptr(keep["mat"])
    if Q0 is not None:
        keep["q0"] = _f64(Q0)
        sc.Q0 = _ptr(keep["q0"])
    if sources:
        keep["sx"] = _f64([s["x"] for s in sources])
        keep["sw"] = _f64([s["w"] for s in sources])
        keep["sf"] = _f64([s["f0"] for s in sources])
        keep["st"] = _f64([s["t0"] for s in sources])
        keep["sa"] = _f64([s.get("amplitude", 1.0) for s in sources])
        sc.n_sources = len(sources)
        sc.src_xyz, sc.src_w, sc.src_f0 = _ptr(keep["sx"]), _ptr(keep["sw"]), _ptr(keep["sf"])
        sc.src_t0, sc.src_amp = _ptr(keep["st"]), _ptr(keep["sa"])
    if len(receivers):
        keep["rx"] = _f64(receivers)
        sc.n_receivers = len(receivers)
        sc.rec_xyz = _ptr(keep["rx"])
    return sc, keep


def poro_submit(srv, scenario):
    t = ctypes.c_uint64()
    _srv_check(lib().poro_submit(srv, ctypes.byref(scenario), ctypes.byref(t)), srv)
    return t.value


def poro_poll(srv, ticket):
    st, t = _i32(), _dbl()
    _srv_check(lib().poro_poll(srv, ticket, ctypes.byref(st), ctypes.byref(t)), srv)
    return st.value, t.value


def poro_wait(srv, ticket, timeout_ms=-1):
    st = _i32()
    rc = lib().poro_wait(srv, ticket, timeout_ms, ctypes.byref(st))
    if rc not in (PORO_OK, PORO_ETIMEOUT):
        _srv_check(rc, srv)
    return st.value


def poro_fetch(srv, ticket, rec):
    n = _i64()
    _srv_check(lib().poro_fetch(srv, ticket, rec, 0, None, None, ctypes.byref(n)), srv)
    t = np.empty(n.value)
    q = np.empty((n.value, 13))
    _srv_check(lib().poro_fetch(srv, ticket, rec, n.value, _ptr(t), _ptr(q), ctypes.byref(n)), srv)
    return t, q


def poro_request_times(srv, ticket):
    a, b, c = _dbl(), _dbl(), _dbl()
    _srv_check(lib().poro_request_times(srv, ticket, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), srv)
    return a.value, b.value, c.value


def poro_request_error(srv, ticket):
    buf = ctypes.create_string_buffer(512)
    lib().poro_request_error(srv, ticket, buf, 512)
    return buf.value.decode()


def poro_cancel(srv, ticket):
    return _srv_check(lib().poro_cancel(srv, ticket), srv)


def poro_footprint_bytes(N, n_elem, max_clusters=1, n_receivers=0):
    b = ctypes.c_size_t()
    _check(lib().poro_footprint_bytes(N, n_elem, max_clusters, n_receivers, ctypes.byref(b)))
    return b.value
