"""One-level Schwarz preconditioners, Section 3.1 (oracle; test infrastructure only).

* Partition (Fig. 1): the mesh is split into P_x x P_y x P_z non-overlapping
  boxes Omega_i, each extended by delta cells per side (corners included) to
  Omega_i^delta and cut off at the domain boundary.
  Reading: parts of an axis get floor(n/P) cells, the first n mod P parts one
  more.
* R_i^delta keeps the entries of Omega_i^delta; R_i^0 additionally zeroes the
  overlap ring Omega_i^delta minus Omega_i.
* A_i = R_i^delta A (R_i^delta)^T (Eq. equ:as-class), ordered lexicographically
  inside the box (x fastest).
* Preconditioners: classical AS (Eq. equ:as-class), left-RAS (Eq. equ:as-left),
  right-RAS (Eq. equ:as-right).
* Subdomain solver: exact LU (dense, small cases) or ILU(k) with the usual
  level-of-fill rule, natural order, no pivoting, no shift (reading: PETSc's
  defaults; the paper only names ILU(k)).
* Reduced-precision factors (the mixed-precision mode): the computed FP64
  factors are rounded to float32 or bfloat16 (round to nearest even) and the
  triangular solves run in float32.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

AS, LEFT_RAS, RIGHT_RAS = 0, 1, 2


def split_axis(n: int, parts: int):
    """Start offsets of `parts` contiguous pieces of n cells (remainder first)."""
    q, r = divmod(n, parts)
    starts = [p * q + min(p, r) for p in range(parts + 1)]
    return starts


class Box:
    """Owned box [o0, o1) and overlapped box [e0, e1) per axis (x, y, z)."""

    def __init__(self, o0, o1, e0, e1, grid_dims):
        self.o0, self.o1, self.e0, self.e1 = o0, o1, e0, e1
        nx, ny, _ = grid_dims
        ex = [np.arange(e0[a], e1[a]) for a in range(3)]
        kk, jj, ii = np.meshgrid(ex[2], ex[1], ex[0], indexing="ij")
        # global indices of Omega_i^delta in local lexicographic order (x fastest)
        self.idx = (ii + nx * (jj + ny * kk)).reshape(-1)
        own = ((ii >= o0[0]) & (ii < o1[0]) & (jj >= o0[1]) & (jj < o1[1])
               & (kk >= o0[2]) & (kk < o1[2]))
        self.own = own.reshape(-1)
        self.shape = tuple(e1[a] - e0[a] for a in range(3))


def partition(grid_dims, parts, overlap):
    """List of Boxes for P_x x P_y x P_z subdomains with overlap delta."""
    dims = grid_dims
    cuts = [split_axis(dims[a], parts[a]) for a in range(3)]
    boxes = []
    for pz in range(parts[2]):
        for py in range(parts[1]):
            for px in range(parts[0]):
                p = (px, py, pz)
                o0 = [cuts[a][p[a]] for a in range(3)]
                o1 = [cuts[a][p[a] + 1] for a in range(3)]
                e0 = [max(o0[a] - overlap, 0) if dims[a] > 1 else 0 for a in range(3)]
                e1 = [min(o1[a] + overlap, dims[a]) if dims[a] > 1 else 1 for a in range(3)]
                boxes.append(Box(o0, o1, e0, e1, dims))
    return boxes


# ----------------------------------------------------------------------------
# ILU(k): symbolic level-of-fill + numeric factorisation on CSR rows
# ----------------------------------------------------------------------------

def iluk_symbolic(A: sp.csr_matrix, k: int):
    """Pattern of ILU(k): lev(i,j) = min over m of lev(i,m) + lev(m,j) + 1 <= k.

    Returns, per row, the sorted column list of the factor pattern.
    """
    n = A.shape[0]
    pat = []
    levs = []
    for i in range(n):
        cols = list(A.indices[A.indptr[i]:A.indptr[i + 1]])
        lev = {c: 0 for c in cols}
        lev.setdefault(i, 0)
        done = set()
        while True:
            cand = sorted(c for c in lev if c < i and c not in done)
            if not cand:
                break
            m = cand[0]
            done.add(m)
            lim = lev[m]
            mcols, mlev = pat[m], levs[m]
            for c, lmc in zip(mcols, mlev):
                if c <= m:
                    continue
                nl = lim + lmc + 1
                if nl <= k and nl < lev.get(c, k + 1):
                    lev[c] = nl
        cols = sorted(lev)
        pat.append(cols)
        levs.append([lev[c] for c in cols])
    return pat


def ilu_numeric(A: sp.csr_matrix, pattern):
    """IKJ incomplete LU on the given pattern, no pivoting.

    Returns (L, U) as CSR, L unit lower (diagonal not stored), U upper with
    the pivots on its diagonal. Raises ZeroDivisionError on a zero pivot.
    """
    n = A.shape[0]
    rows = []
    for i in range(n):
        w = {c: 0.0 for c in pattern[i]}
        for t in range(A.indptr[i], A.indptr[i + 1]):
            w[A.indices[t]] = A.data[t]
        for m in sorted(c for c in w if c < i):
            um = rows[m]
            piv = um[m]
            if piv == 0.0:
                raise ZeroDivisionError(f"zero pivot in row {m}")
            lm = w[m] / piv
            w[m] = lm
            for c, v in um.items():
                if c > m and c in w:
                    w[c] -= lm * v
        if w[i] == 0.0:
            raise ZeroDivisionError(f"zero pivot in row {i}")
        rows.append(w)
    Lr, Lc, Lv, Ur, Uc, Uv = [], [], [], [], [], []
    for i, w in enumerate(rows):
        for c, v in w.items():
            if c < i:
                Lr.append(i); Lc.append(c); Lv.append(v)
            else:
                Ur.append(i); Uc.append(c); Uv.append(v)
    L = sp.csr_matrix((Lv, (Lr, Lc)), shape=(n, n))
    U = sp.csr_matrix((Uv, (Ur, Uc)), shape=(n, n))
    L.sort_indices(); U.sort_indices()
    return L, U


def ilu0_stencil_pivots(A: sp.csr_matrix):
    """ILU(0) pivots in closed form for a matrix whose pattern is a 5/7-point
    stencil in natural order: d_n = a_nn - sum_{m<n, m nbr} a_nm a_mn / d_m.

    (Only the diagonal changes because no two lower neighbours of a row share an
    upper neighbour other than the row itself.) Used as a pin of ilu_numeric.
    """
    n = A.shape[0]
    Ad = A.todok()
    d = np.zeros(n)
    for i in range(n):
        s = Ad.get((i, i), 0.0)
        for t in range(A.indptr[i], A.indptr[i + 1]):
            m = A.indices[t]
            if m < i:
                s -= A.data[t] * Ad.get((m, i), 0.0) / d[m]
        d[i] = s
    return d


def round_bf16(x):
    """Round float32 values to bfloat16 precision (round to nearest even)."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


class SubdomainSolver:
    """A_i^{-1} through ILU(k) factors, exact LU, or reduced-precision factors."""

    def __init__(self, Ai: sp.csr_matrix, kind="ilu", k=0, prec=64):
        self.n = Ai.shape[0]
        self.kind = kind
        self.prec = prec
        if kind == "lu":
            self.lu = sla.lu_factor(Ai.toarray())
            return
        L, U = ilu_numeric(Ai, iluk_symbolic(Ai, k))
        if prec == 64:
            self.L, self.U = L, U
            return
        # mixed precision: solve L y = r then U z = y in float32, with
        # L' = strictly-lower part, U' = strictly-upper part and dinv = 1/d
        Ld = L.tocsr()
        Ud = U.tocsr()
        diag = Ud.diagonal()
        Uoff = (Ud - sp.diags(diag)).tocsr()
        Uoff.eliminate_zeros()
        rnd = (lambda v: np.asarray(v, dtype=np.float32)) if prec == 32 else round_bf16
        self.Lf = sp.csr_matrix((rnd(Ld.data), Ld.indices, Ld.indptr), shape=Ld.shape)
        self.Uf = sp.csr_matrix((rnd(Uoff.data), Uoff.indices, Uoff.indptr), shape=Uoff.shape)
        self.dinv = rnd(1.0 / diag)

    def solve(self, r):
        if self.kind == "lu":
            return sla.lu_solve(self.lu, r)
        if self.prec == 64:
            y = _lower_unit_solve(self.L, r)
            return _upper_solve(self.U, y)
        r32 = np.asarray(r, dtype=np.float32)
        y = _lower_unit_solve_f32(self.Lf, r32)
        z = _upper_offdiag_solve_f32(self.Uf, self.dinv, y)
        return z.astype(np.float64)


def _lower_unit_solve(L, r):
    y = np.array(r, dtype=np.float64)
    ip, ix, dv = L.indptr, L.indices, L.data
    for i in range(y.size):
        s = y[i]
        for t in range(ip[i], ip[i + 1]):
            s -= dv[t] * y[ix[t]]
        y[i] = s
    return y


def _upper_solve(U, y):
    z = np.array(y, dtype=np.float64)
    ip, ix, dv = U.indptr, U.indices, U.data
    for i in range(z.size - 1, -1, -1):
        s = z[i]
        d = 0.0
        for t in range(ip[i], ip[i + 1]):
            c = ix[t]
            if c == i:
                d = dv[t]
            else:
                s -= dv[t] * z[c]
        z[i] = s / d
    return z


def _lower_unit_solve_f32(L, r):
    y = np.array(r, dtype=np.float32)
    ip, ix, dv = L.indptr, L.indices, L.data
    for i in range(y.size):
        s = np.float32(y[i])
        for t in range(ip[i], ip[i + 1]):
            s = np.float32(s - np.float32(dv[t] * y[ix[t]]))
        y[i] = s
    return y


def _upper_offdiag_solve_f32(U, dinv, y):
    z = np.array(y, dtype=np.float32)
    ip, ix, dv = U.indptr, U.indices, U.data
    for i in range(z.size - 1, -1, -1):
        s = np.float32(z[i])
        for t in range(ip[i], ip[i + 1]):
            s = np.float32(s - np.float32(dv[t] * z[ix[t]]))
        z[i] = np.float32(s * dinv[i])
    return z


class Schwarz:
    """One-level Schwarz preconditioner M^{-1} on a structured grid."""

    def __init__(self, A: sp.csr_matrix, grid_dims, parts, overlap, kind=LEFT_RAS,
                 sub="ilu", ilu_k=0, prec=64):
        self.A = A.tocsr()
        self.kind = kind
        self.boxes = partition(grid_dims, parts, overlap)
        self.solvers = []
        for b in self.boxes:
            Ai = self.A[b.idx][:, b.idx].tocsr()
            Ai.sort_indices()
            self.solvers.append(SubdomainSolver(Ai, sub, ilu_k, prec))

    def apply(self, r):
        r = np.asarray(r, dtype=np.float64)
        z = np.zeros_like(r)
        for b, s in zip(self.boxes, self.solvers):
            ri = r[b.idx].copy()
            if self.kind == RIGHT_RAS:
                ri[~b.own] = 0.0           # R_i^0 on the input
            zi = s.solve(ri)
            if self.kind == LEFT_RAS:
                z[b.idx[b.own]] = zi[b.own]  # (R_i^0)^T on the output
            else:
                np.add.at(z, b.idx, zi)      # (R_i^delta)^T
        return z

    def __call__(self, r):
        return self.apply(r)

    def dense(self):
        """M^{-1} as a dense matrix (tiny cases only)."""
        n = self.A.shape[0]
        return np.column_stack([self.apply(e) for e in np.eye(n)])
