"""Binding of the plain-loop C statement of Algorithm 3 (oracle/alg3_loop.c).

TEST INFRASTRUCTURE, like the rest of `oracle/`: the timed CPU baseline of
the benchmark and a second statement of Algorithm 3 that the tests check
against the dense LU solve.  `build()` compiles the C file with gcc
(-O2 -fopenmp -ffp-contract=off) into oracle/liboracle_alg3.so.
"""
import ctypes
import os
import subprocess

import numpy as np

from . import basis, timebasis

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "alg3_loop.c")
LIB = os.path.join(HERE, "liboracle_alg3.so")


def build():
    """Compile the C oracle (host code only: the same flags on x86 and Arm)."""
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11", SRC, "-o", LIB + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"oracle C build failed: {' '.join(cmd)}\n{r.stderr}")
    os.replace(LIB + ".tmp", LIB)
    return LIB


_LIBH = None


def _lib():
    global _LIBH
    if _LIBH is None:
        if not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
            build()
        h = ctypes.CDLL(LIB)
        vp = ctypes.c_void_p
        h.oracle_alg3_predict.restype = ctypes.c_int64
        h.oracle_alg3_predict.argtypes = [ctypes.c_int, ctypes.c_int64, vp, vp, vp, vp, vp, vp, vp, ctypes.c_int]
        h.oracle_alg3_default_threads.restype = ctypes.c_int
        _LIBH = h
    return _LIBH


def default_threads():
    return int(_lib().oracle_alg3_default_threads())


def reference_arrays(N):
    """Khat^j [3][B][B], Z [T][T] and S^{-1} w [T] from the Python oracle."""
    W, w, S, Kt = timebasis.time_matrices(N)
    Kh = np.ascontiguousarray(np.stack(basis.khat_matrices(N)), dtype=np.float64)
    Z = np.ascontiguousarray(np.linalg.solve(S, W - Kt))
    return Kh, Z, np.ascontiguousarray(np.linalg.solve(S, w))


def predict_alg3_c(N, Astar, Estar, Q0, threads=0, ref=None):
    """Qt[n][13][B][N+1] of n elements (Astar [n][3][13][13], Estar
    [n][13][13], Q0 [n][13][B]) by the C loops with `threads` threads
    (0: OpenMP's default)."""
    Astar = np.ascontiguousarray(Astar, dtype=np.float64)
    Estar = np.ascontiguousarray(Estar, dtype=np.float64)
    Q0 = np.ascontiguousarray(Q0, dtype=np.float64)
    n, B = Q0.shape[0], basis.n_modes(N)
    Kh, Z, sw = ref if ref is not None else reference_arrays(N)
    Qt = np.empty((n, 13, B, N + 1))
    done = _lib().oracle_alg3_predict(N, n, Astar.ctypes.data, Estar.ctypes.data, Q0.ctypes.data, Kh.ctypes.data,
                                      Z.ctypes.data, sw.ctypes.data, Qt.ctypes.data, int(threads))
    if done != n:
        raise ArithmeticError("oracle Algorithm 3 (C): a time-matrix pivot was zero")
    return Qt
