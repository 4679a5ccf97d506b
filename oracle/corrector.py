"""ADER-DG corrector and global time stepping, plain float64 statement.

Paper, Section "Spatial discretisation", Eq. semi_discrete, integrated over
one step [t_n, t_n + dt] (Section "Temporal discretisation with ADER"):

  |J| M_kk (Q^{n+1} - Q^n)_pk =  sum_j sum_l |J| K^j_lk (A^j I)_pl
                                - sum_faces int_face phi_k (A_n q*)_p dS
                                + |J| M_kk (E I)_pk  + source

with I = int Q~ dt the time-integrated predictor, A^j the reference
Jacobians without dt, K^j_lk = int phi_l d_j phi_k, and the Godunov flux
A_n q* = F^- q_L + F^+ q_R of `oracle.flux`.  The face integrals are done
here by quadrature on each physical face: the quadrature points are mapped
into both elements' reference coordinates (no orientation tables).

Point source (Section "Homogeneous full-space"): the Ricker wavelet
s(t) = (1 - 2a^2) exp(-a^2), a = pi f0 (t - t0), acting on the quantities with
weights w; its exact antiderivative (t - t0) exp(-a^2) gives int s dt, and
the projection onto the element containing x_s adds
w_p phi_k(xi_s) / (|J| M_kk) int s dt.  Receivers sample
q_p(x_r) = sum_l Q_pl phi_l(xi_r) at the end of every step.
Readings: the source or receiver on a shared vertex/edge/face belongs to
the lowest element id whose barycentric coordinates are all >= -1e-12;
receivers are sampled at the end of every step.
"""
from functools import lru_cache

import numpy as np
from scipy.special import roots_legendre

from . import basis, flux, geometry, material, timebasis

NQ = 13
REF_VERTS = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
FACE_TAGS = {0: "interior", 1: "free_surface", 2: "absorbing"}


# ---------------------------------------------------------------- basis in float
@lru_cache(maxsize=None)
def _monomial_table(N):
    """Exponents [n_mono][3] of every monomial of degree <= N and the
    coefficient matrix C[l][mono] of the exact integer expansions of phi_l."""
    exps = [(a, b, c) for a in range(N + 1) for b in range(N + 1 - a) for c in range(N + 1 - a - b)]
    col = {e: i for i, e in enumerate(exps)}
    C = np.zeros((basis.n_modes(N), len(exps)))
    for l, (i, j, k) in enumerate(basis.mode_triples(N)):
        for e, c in basis.dubiner_poly(i, j, k).items():
            C[l, col[e]] = float(c)
    return np.array(exps), C


def basis_values(N, pts):
    """phi_l at reference points pts[n][3] -> [n][B], from the exact integer
    monomial expansions: sum over monomials of coefficient x xi^a eta^b zeta^c."""
    pts = np.atleast_2d(np.asarray(pts, float))
    exps, C = _monomial_table(N)
    mono = np.prod(pts[:, None, :] ** exps[None, :, :], axis=2)   # [n][n_mono]
    return mono @ C.T


def triangle_quadrature(N):
    """Collapsed Gauss product rule on {a, b >= 0, a + b <= 1}, exact for
    polynomials of degree 2N + 1; weights sum to 1/2."""
    x, w = roots_legendre(N + 2)
    pts, wts = [], []
    for r, wr in zip(x, w):
        for s, ws in zip(x, w):
            pts.append(((1 + r) * (1 - s) / 4, (1 + s) / 2))
            wts.append(wr * ws * (1 - s) / 8)
    return np.array(pts), np.array(wts)


def ricker_antiderivative(t, f0, t0):
    a = np.pi * f0 * (t - t0)
    return (t - t0) * np.exp(-a * a)


# ---------------------------------------------------------------- batched predictor
def predict_alg3_batch(N, Astar, Estar, Q0):
    """Algorithm 3 for a batch of elements (same steps as
    predictor.predict_alg3, vectorised over the leading element axis)."""
    B, T = basis.n_modes(N), N + 1
    Kh = basis.khat_matrices(N)
    W, w, S, Kt = timebasis.time_matrices(N)
    Sinv_w = np.linalg.solve(S, w)
    Z = np.linalg.solve(S, W - Kt)
    ne = Q0.shape[0]
    b = Q0[:, :, :, None] * Sinv_w[None, None, None, :]
    Qt = np.zeros((ne, NQ, B, T))
    F = np.einsum("epp->ep", Estar)
    for g in range(N, -1, -1):
        blk = slice(basis.block_offset(g), basis.block_offset(g) + basis.block_size(g))
        for p in range(NQ - 1, -1, -1):
            Zinv = np.linalg.inv(Z[None] - F[:, p, None, None] * np.eye(T)[None])   # [e][T][T]
            Qt[:, p, blk, :] = np.einsum("emu,evu->emv", b[:, p, blk, :], Zinv)
            for o in range(p):
                G = Estar[:, o, p]
                if np.any(G != 0.0):
                    b[:, o, blk, :] += G[:, None, None] * Qt[:, p, blk, :]
        if g > 0:
            # green update: two n-mode products, the star matrix on the
            # quantity index, then Khat^j restricted to the block's columns
            for j in range(3):
                X = np.einsum("epq,eqmu->epmu", Astar[:, j], Qt[:, :, blk, :])
                b -= np.einsum("lm,epmu->eplu", Kh[j][:, blk], X)
    return Qt


# ---------------------------------------------------------------- mesh set-up
def locate(vert_e, x, tol=1e-12):
    """Reference coordinates of x in the tetrahedron and whether x lies in it."""
    x0, J, Jinv = geometry.affine(vert_e)
    xi = Jinv @ (np.asarray(x, float) - x0)
    bary = np.array([1 - xi.sum(), xi[0], xi[1], xi[2]])
    return xi, bool(np.all(bary >= -tol))


class GTSSimulation:
    """Global time stepping on a conforming tetrahedral mesh (plain loops over
    elements and faces, float64)."""

    def __init__(self, mesh, materials, N, cfl=0.5, source=None, receivers=()):
        self.N, self.B, self.T = N, basis.n_modes(N), N + 1
        self.vert = mesh["vertices"][mesh["tets"]]            # [ne][4][3]
        self.nb, self.tag = mesh["neighbors"], mesh["face_tag"]
        self.mats = [{k: float(v) for k, v in zip(material.PARAM_NAMES, row)} for row in materials]
        ne = self.ne = self.vert.shape[0]
        self.dt = min(geometry.cfl_dt(self.vert[e], self.mats[e], N, cfl) for e in range(ne))
        self.M = np.diag(basis.mass_matrix(N))
        self.K = basis.stiffness_matrices(N)
        self.detJ = np.array([abs(np.linalg.det(geometry.affine(self.vert[e])[1])) for e in range(ne)])
        self.Aj = np.stack([np.stack(geometry.reference_jacobians(self.vert[e], self.mats[e])) for e in range(ne)])
        self.E = np.stack([material.source_matrix(m) for m in self.mats])
        self._faces()
        self._source(source)
        self.rec = []
        for x in receivers:
            e, xi = self._owner(x)
            self.rec.append((e, basis_values(N, xi)[0]))

    def _owner(self, x):
        for e in range(self.ne):
            xi, inside = locate(self.vert[e], x)
            if inside:
                return e, xi
        raise ValueError("point outside the mesh")

    def _faces(self):
        N = self.N
        pts, wts = triangle_quadrature(N)
        self.qw = wts
        self.face = []   # per element, per face: (area, phiL[nq][B], phiR[nq][B] or None, Fm, Fp, nbr)
        for e in range(self.ne):
            x0, J, Jinv = geometry.affine(self.vert[e])
            faces = []
            for f in range(4):
                fv = [v for v in range(4) if v != f]
                a, b, c = REF_VERTS[fv[0]], REF_VERTS[fv[1]], REF_VERTS[fv[2]]
                xi = a[None] + pts[:, :1] * (b - a)[None] + pts[:, 1:2] * (c - a)[None]
                xphys = x0[None] + xi @ J.T
                pa, pb, pc = self.vert[e][fv]
                nrm = np.cross(pb - pa, pc - pa)
                area = 0.5 * np.linalg.norm(nrm)
                nrm /= np.linalg.norm(nrm)
                if np.dot(nrm, self.vert[e][f] - pa) > 0:
                    nrm = -nrm
                phiL = basis_values(N, xi)
                r = self.nb[e, f]
                kind = FACE_TAGS[int(self.tag[e, f])] if r < 0 else "interior"
                if r >= 0:
                    # the neighbour's face: the one whose vertices equal ours up to a translation
                    shift = None
                    for h in range(4):
                        hv = self.vert[r][[v for v in range(4) if v != h]]
                        d = hv.mean(axis=0) - np.array([pa, pb, pc]).mean(axis=0)
                        if all(np.min(np.linalg.norm(hv - (p + d)[None], axis=1)) < 1e-9 * (1 + np.abs(p).max())
                               for p in (pa, pb, pc)):
                            shift = d
                            break
                    assert shift is not None, "non-conforming face"
                    xr0, Jr, Jrinv = geometry.affine(self.vert[r])
                    xir = (xphys + shift[None] - xr0[None]) @ Jrinv.T
                    phiR = basis_values(N, xir)
                    Fm, Fp = flux.flux_matrices(self.mats[e], self.mats[r], nrm, "interior")
                else:
                    phiR = None
                    Fm, Fp = flux.flux_matrices(self.mats[e], None, nrm, kind)
                faces.append((area, phiL, phiR, Fm, Fp, r))
            self.face.append(faces)

    def _source(self, src):
        self.src = None
        if src is None:
            return
        e, xi = self._owner(src["x"])
        phi = basis_values(self.N, xi)[0]
        coef = np.outer(np.asarray(src["w"], float), phi) / (self.detJ[e] * self.M[None, :])
        self.src = (e, coef * src.get("amplitude", 1.0), src["f0"], src["t0"])

    def step(self, Q, t):
        """One global step from Q (ne, 13, B) at time t; returns Q(t + dt)."""
        dt, N = self.dt, self.N
        Qt = predict_alg3_batch(N, self.Aj * dt, self.E * dt, Q)
        I = dt * Qt[:, :, :, 0]
        Qn = Q.copy()
        for e in range(self.ne):
            # volume: M^{-1} sum_j K^{jT} (A^j I) and the source term E I
            dQ = sum((self.Aj[e, j] @ I[e]) @ self.K[j] for j in range(3)) / self.M[None, :]
            dQ += self.E[e] @ I[e]
            for (area, phiL, phiR, Fm, Fp, r) in self.face[e]:
                trace = (Fm @ (I[e] @ phiL.T))                    # [13][nq]
                if r >= 0:
                    trace += Fp @ (I[r] @ phiR.T)
                dQ -= (2.0 * area / self.detJ[e]) * (trace * self.qw[None, :]) @ phiL / self.M[None, :]
            Qn[e] += dQ
        if self.src is not None:
            e, coef, f0, t0 = self.src
            Qn[e] += coef * (ricker_antiderivative(t + dt, f0, t0) - ricker_antiderivative(t, f0, t0))
        return Qn

    def run(self, Q0, n_steps):
        """Returns final Q and seismograms [n_rec][n_steps][13] at t_1..t_n."""
        Q, t = np.array(Q0, float), 0.0
        seis = np.zeros((len(self.rec), n_steps, NQ))
        for n in range(n_steps):
            Q = self.step(Q, t)
            t += self.dt
            for i, (e, phi) in enumerate(self.rec):
                seis[i, n] = Q[e] @ phi
        return Q, seis


class LTSSimulation(GTSSimulation):
    """Clustered local time stepping (Section "Temporal discretisation with
    ADER": clustered LTS; the paper gives no algorithm, this is the reading).

    Element e has its CFL step dt_e; dt_min = min dt_e; its cluster is
    c_e = min(C - 1, floor(log2(dt_e / dt_min))) and it steps with
    dt_c = 2^c dt_min.  Ticks k of length dt_min run:
      (A) every cluster with k mod 2^c = 0 predicts from its current DOFs
          (own interval [t_k, t_k + dt_c]); an element whose neighbour lies in
          a larger cluster L adds its time-integrated predictor I to a buffer
          of level L (reset when k mod 2^L = 0);
      (B) every cluster with (k + 1) mod 2^c = 0 corrects over its interval
          [t_{k+1} - dt_c, t_{k+1}].  The neighbour's trace is integrated over
          exactly that interval: same cluster -> its I; smaller cluster -> its
          buffer (the chronological sum of its sub-step integrals); larger
          cluster -> dt_L sum_s Qt_s int_a^b chi_s over the sub-interval
          [a, b] of its reference time interval.
    Sources act over each element's own interval; receivers sample at the
    end of every step of their element.  With C = 1 this is global time
    stepping."""

    def __init__(self, mesh, materials, N, max_clusters, cfl=0.5, source=None, receivers=()):
        super().__init__(mesh, materials, N, cfl, source, receivers)
        self.C = max_clusters
        dte = np.array([geometry.cfl_dt(self.vert[e], self.mats[e], N, cfl) for e in range(self.ne)])
        self.dt_min = dte.min()
        self.cl = np.minimum(max_clusters - 1, np.floor(np.log2(dte / self.dt_min) + 1e-12)).astype(int)
        self.dtc = self.dt_min * 2.0 ** np.arange(max_clusters)
        # buffer levels each element needs (larger neighbour clusters)
        self.levels = [sorted({int(self.cl[r]) for r in self.nb[e] if r >= 0 and self.cl[r] > self.cl[e]})
                       for e in range(self.ne)]

    def run(self, Q0, n_cycles):
        """n_cycles steps of the largest cluster; returns final Q and, per
        receiver, (times, samples [n][13])."""
        N, C = self.N, self.C
        Q = np.array(Q0, float)
        Qt = np.zeros((self.ne, NQ, self.B, self.T))
        I = np.zeros((self.ne, NQ, self.B))
        buf = {}
        seis = [([], []) for _ in self.rec]
        rec_of = {}
        for i, (e, phi) in enumerate(self.rec):
            rec_of.setdefault(e, []).append(i)
        clusters = [np.nonzero(self.cl == c)[0] for c in range(C)]
        K = n_cycles * 2 ** (C - 1)
        for k in range(K):
            for c in range(C):
                els = clusters[c]
                if k % 2 ** c or len(els) == 0:
                    continue
                dt = self.dtc[c]
                Qt[els] = predict_alg3_batch(N, self.Aj[els] * dt, self.E[els] * dt, Q[els])
                I[els] = dt * Qt[els][:, :, :, 0]
                for e in els:
                    for L in self.levels[e]:
                        if k % 2 ** L == 0:
                            buf[(e, L)] = I[e].copy()
                        else:
                            buf[(e, L)] += I[e]
            for c in range(C):
                els = clusters[c]
                if (k + 1) % 2 ** c or len(els) == 0:
                    continue
                ks = k + 1 - 2 ** c
                for e in els:
                    dQ = sum((self.Aj[e, j] @ I[e]) @ self.K[j] for j in range(3)) / self.M[None, :]
                    dQ += self.E[e] @ I[e]
                    for (area, phiL, phiR, Fm, Fp, r) in self.face[e]:
                        trace = Fm @ (I[e] @ phiL.T)
                        if r >= 0:
                            cr = self.cl[r]
                            if cr == c:
                                Ir = I[r]
                            elif cr < c:
                                Ir = buf[(r, c)]
                            else:
                                m = (ks // 2 ** cr) * 2 ** cr
                                a, b = (ks - m) / 2 ** cr, (k + 1 - m) / 2 ** cr
                                Ir = self.dtc[cr] * np.einsum("qls,s->ql", Qt[r], timebasis.chi_integrals(N, a, b))
                            trace += Fp @ (Ir @ phiR.T)
                        dQ -= (2.0 * area / self.detJ[e]) * (trace * self.qw[None, :]) @ phiL / self.M[None, :]
                    Q[e] += dQ
                    if self.src is not None and self.src[0] == e:
                        _, coef, f0, t0 = self.src
                        Q[e] += coef * (ricker_antiderivative((k + 1) * self.dt_min, f0, t0)
                                        - ricker_antiderivative(ks * self.dt_min, f0, t0))
                    for i in rec_of.get(e, []):
                        seis[i][0].append((k + 1) * self.dt_min)
                        seis[i][1].append(Q[e] @ self.rec[i][1])
        return Q, [(np.array(t), np.array(q)) for t, q in seis]
