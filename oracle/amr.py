"""Berger-Oliger evolution of a 2:1-refined, block-structured patch hierarchy,
with a Sommerfeld (radiative) outer boundary.

TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's
CPU-baseline leg use this module. It shares no code with the CUDA library.
The right-hand side, dissipation and transfer stencils come from the plain
FP64 oracle (bssn_oracle.cpp, through oracle/__init__.py); the composition
below is written out in numpy.

The paper runs its BSSN kernels on Cactus/Carpet block-structured grids and
plans adaptive refinement with ratio-2 levels (Sec. 1.1, Sec. 4); it does not
print the refinement algorithm. What this module follows is the textbook
Berger-Oliger scheme (Berger & Oliger 1984) in the cell-centred, time-
interpolating form that Carpet uses (Schnetter, Hawley & Hawke 2004):

Hierarchy
  * level l has spacing h_l = h_0 / 2^l; cell I of level l has its centre at
    xlo + (I + 1/2) h_l, so cells 2c and 2c+1 of level l+1 lie in cell c of
    level l. The level-l domain is cells [0, N 2^l) per axis.
  * a patch is the box of cells [o, o + n) of one level plus g ghost cells
    on every side (state layout of the oracle: (24, nz+2g, ny+2g, nx+2g)).
  * a box "fits" a run of cells [lo, lo + m) along an axis if, for the
    smallest k with lo + k P >= box_lo (P the period of a periodic domain,
    k = 0 otherwise), lo + k P + m <= box_hi.

Ghost points (global index G of a ghost cell of patch b at level l)
  1. level 0, non-periodic, G outside the domain: the outer boundary. Static:
     the patch's t = 0 value. Radiative: evolved with the stages by
     d_t u = -v (x^i / r) d_i u - v (u - u_inf) / r (second-order
     differences: centred where both neighbours are in the patch's padded
     box, one-sided at its faces; v = sqrt(2) for alpha and trK under 1+log
     slicing, 1 otherwise; u_inf = flat space).
  2. otherwise, the first patch of level l (input order, b itself included)
     whose interior fits the cell G: a copy of that patch's value at the
     same stage.
  3. otherwise (l >= 1), prolongation from level l-1: the tricubic Lagrange
     interpolant through the 4 nearest coarse centres per axis (fine G sits
     at coarse coordinate G/2 - 1/4), applied to the parent level's RK4
     stage states of its latest step (see "Ghost values in time"). The
     parent level is read as one field on cells: coarse cell C takes its
     value from the first level-(l-1) patch whose interior fits C, else from
     the first whose padded box does (where a padded box holds a ghost copy
     of another patch's interior cell, both give the same value).
  4. anything else is an error (the hierarchy is not properly nested).

Ghost values in time. The parent's step t -> t + dt keeps its stage states
y0, Y2 = y0 + dt/2 f1, Y3 = y0 + dt/2 f2, Y4 = y0 + dt f3 and the result
y1 = y0 + dt/6 (f1 + 2 f2 + 2 f3 + f4). With D2, D3, D4, D5 the differences
of Y2, Y3, Y4, y1 from y0, the slopes are dt f1 = 2 D2, dt f2 = 2 D3,
dt f3 = D4 and dt f4 = 6 D5 - 2 D2 - 4 D3 - 2 D4. The classic third-order
continuous extension of RK4 (Hairer, Norsett & Wanner, Sec. II.6),
    y(t + chi dt) = y0 + dt [ (chi - 3/2 chi^2 + 2/3 chi^3) f1
                    + (chi^2 - 2/3 chi^3)(f2 + f3) + (2/3 chi^3 - 1/2 chi^2) f4 ],
gives y and its first three time derivatives at the start t + chi dt of a
fine step (chi = 0 or 1/2). RK4's stage inputs are not the solution at the
stage times, so the fine ghosts take, at the stage inputs of a fine step of
size k = dt/2, the values RK4 itself makes there for a linear autonomous
system with those Taylor data:
    Y1 = y,  Y2 = y + k/2 y',  Y3 = y + k/2 y' + k^2/4 y'',
    Y4 = y + k y' + k^2/2 y'' + k^3/4 y'''
(the coarse-fine coupling of McCorquodale & Colella 2011 and Mongwane 2015
for subcycled Runge-Kutta steps); the fine result after the step takes the
dense output at chi + 1/2. Each such ghost value is P[y0] + sum_j d_j P[D_j],
P the spatial prolongation, d_j constants of (half, stage).

Time stepping (one call of step() advances level 0 by dt_0):
  advance(l, m):   m = which half of the parent's step (0 for level 0)
    set the ghosts of the state (fine stage 0 of half m);
    classic RK4 with dt_l = dt_0 / 2^l; before stage s = 1, 2, 3 the ghosts
    of the stage input are set (fine stage s of half m);
    the ghosts of the result are set (end of half m);
    if level l+1 exists: keep (y0, Y2, Y3, Y4, y1); advance(l+1, 0);
    advance(l+1, 1); restrict level l+1 into level l; set level l's ghosts
    again (end of half m).
  Restriction: every interior cell c of level l for which the first level-
  (l+1) patch whose interior fits the fine run 2c-1 .. 2c+2 on every axis
  takes the tricubic interpolant of that patch's values at its centre.
"""
import math
from fractions import Fraction

import numpy as np

from . import Params, rhs as _rhs

NVAR = 24
# flat space: W, gt11, gt22, gt33, alpha = 1
_UINF = np.zeros(NVAR)
_UINF[[0, 1, 4, 6, 17]] = 1.0


def radiative_speeds(p: Params):
    """Propagation speed per variable for the Sommerfeld condition: the
    gauge speed sqrt(f) (f = 2 for 1+log) for alpha and trK, light speed
    for everything else."""
    v = np.ones(NVAR)
    if p.lapse == 0:
        v[7] = v[17] = math.sqrt(2.0)
    return v


def _diff2(f, axis, h):
    """Second-order first derivative of f along axis: centred
    (f[i+1] - f[i-1]) / 2h inside, one-sided on the two faces,
    (4 (f1 - f0) - (f2 - f0)) / 2h and its mirror (differences of stored
    values first, so that a constant gives exactly zero)."""
    f = np.moveaxis(f, axis, 0)
    d = np.empty_like(f)
    d[1:-1] = (f[2:] - f[:-2]) / (2.0 * h)
    d[0] = (4.0 * (f[1] - f[0]) - (f[2] - f[0])) / (2.0 * h)
    d[-1] = -(4.0 * (f[-2] - f[-1]) - (f[-3] - f[-1])) / (2.0 * h)
    return np.moveaxis(d, 0, axis)


def sommerfeld_rhs(u, h, xyz0, speeds, uinf=_UINF):
    """d_t u = -v (x^i/r) d_i u - v (u - u_inf)/r at every point of the padded
    array u (24, Z, Y, X); xyz0 = coordinates of padded point (0, 0, 0).
    d_i: second-order centred differences inside the array, second-order
    one-sided differences on its faces (_diff2)."""
    hx, hy, hz = (h, h, h) if np.isscalar(h) else h
    nzp, nyp, nxp = u.shape[1:]
    x = xyz0[0] + np.arange(nxp) * hx
    y = xyz0[1] + np.arange(nyp) * hy
    z = xyz0[2] + np.arange(nzp) * hz
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    r = np.sqrt(X * X + Y * Y + Z * Z)
    out = np.empty_like(u)
    for v in range(NVAR):
        dx = _diff2(u[v], 2, hx)
        dy = _diff2(u[v], 1, hy)
        dz = _diff2(u[v], 0, hz)
        out[v] = -speeds[v] * (X * dx + Y * dy + Z * dz) / r - speeds[v] * (u[v] - uinf[v]) / r
    return out


def dense_taylor(chi):
    """Coefficients over (D2, D3, D4, D5) of dt^q y^(q)(t + chi dt) - [q = 0] y0,
    q = 0..3, from the RK4 continuous extension (exact Fractions)."""
    chi = Fraction(chi)
    # dt times the slopes f1..f4, over (D2, D3, D4, D5)
    f1 = [Fraction(2), Fraction(0), Fraction(0), Fraction(0)]
    f2 = [Fraction(0), Fraction(2), Fraction(0), Fraction(0)]
    f3 = [Fraction(0), Fraction(0), Fraction(1), Fraction(0)]
    f4 = [Fraction(-2), Fraction(-4), Fraction(-2), Fraction(6)]
    # y(t + chi dt) - y0 = chi c1 + chi^2 c2 + chi^3 c3
    c1 = f1
    c2 = [-Fraction(3, 2) * a + b + c - Fraction(1, 2) * d for a, b, c, d in zip(f1, f2, f3, f4)]
    c3 = [Fraction(2, 3) * (a - b - c + d) for a, b, c, d in zip(f1, f2, f3, f4)]
    y = [chi * a + chi ** 2 * b + chi ** 3 * c for a, b, c in zip(c1, c2, c3)]
    y1 = [a + 2 * chi * b + 3 * chi ** 2 * c for a, b, c in zip(c1, c2, c3)]
    y2 = [2 * b + 6 * chi * c for b, c in zip(c2, c3)]
    y3 = [6 * c for c in c3]
    return y, y1, y2, y3


def fine_ghost_coeffs(m, s):
    """d_j over (D2, D3, D4, D5) of the ghost value at the input of fine stage
    s (0..3) of half m (0 or 1) of the parent's step, or of the fine result
    (s = 4)."""
    chi = Fraction(m, 2)
    r = Fraction(1, 2)  # fine step / parent step
    if s == 4:
        return [float(x) for x in dense_taylor(chi + r)[0]]
    y, y1, y2, y3 = dense_taylor(chi)
    if s == 0:
        c = y
    elif s == 1:
        c = [a + r / 2 * b for a, b in zip(y, y1)]
    elif s == 2:
        c = [a + r / 2 * b + r * r / 4 * d for a, b, d in zip(y, y1, y2)]
    else:
        c = [a + r * b + r * r / 2 * d + r ** 3 / 4 * e for a, b, d, e in zip(y, y1, y2, y3)]
    return [float(x) for x in c]


def lagrange_weights(x, nodes):
    """1D Lagrange basis at x through the given nodes (arrays broadcast)."""
    w = []
    for j in range(len(nodes)):
        num = 1.0
        den = 1.0
        for m in range(len(nodes)):
            if m != j:
                num = num * (x - nodes[m])
                den = den * (nodes[j] - nodes[m])
        w.append(num / den)
    return w


def _fit(lo, m, box_lo, box_hi, period):
    """Shift k*period that places the run [lo, lo+m) inside [box_lo, box_hi)
    (elementwise over arrays lo); returns (ok, shifted lo)."""
    if period is None:
        k = np.zeros_like(lo)
    else:
        k = -((lo - box_lo) // period)  # smallest k with lo + k P >= box_lo
    s = lo + k * (period if period is not None else 0)
    return (s >= box_lo) & (s + m <= box_hi), s


class Patch:
    def __init__(self, level, origin, n, state, ghost_src=None):
        self.level = int(level)
        self.o = np.array(origin, dtype=np.int64)
        self.n = np.array(n, dtype=np.int64)
        self.state = np.ascontiguousarray(state, dtype=np.float64)
        self.ghost_src = ghost_src
        self.stages = None  # (y0, Y2, Y3, Y4, y1) of the latest step


class Hierarchy:
    """patches: list of Patch (any order; level-0 patches carry boundary
    values in ghost_src for the static boundary); ncells: level-0 domain
    cells per axis; xlo: domain lower corner; h0: level-0 spacing (scalar
    or 3); boundary 0 periodic, 1 static, 2 radiative; dt0: level-0 step."""

    def __init__(self, patches, g, ncells, xlo, h0, boundary, params: Params, dt0):
        self.P = list(patches)
        self.g = g
        self.N = np.array(ncells, dtype=np.int64)
        self.xlo = np.array(xlo, dtype=np.float64)
        self.h0 = np.array([h0] * 3 if np.isscalar(h0) else h0, dtype=np.float64)
        self.bc = boundary
        self.p = params
        self.dt0 = dt0
        self.nlev = 1 + max(q.level for q in self.P)
        self.at = [[b for b, q in enumerate(self.P) if q.level == l] for l in range(self.nlev)]
        if any(len(a) == 0 for a in self.at):
            raise ValueError("levels must be contiguous from 0")
        for q in self.P:
            top = self.N * 2 ** q.level
            if np.any(q.o < 0) or np.any(q.o + q.n > top) or np.any(q.n < 1):
                raise ValueError("every patch must lie inside its level's domain")
        self.speeds = radiative_speeds(params)
        self._pcache = {}
        self.plans = [self._ghost_plan(b) for b in range(len(self.P))]
        self.rplans = [self._restrict_plan(b) for b in range(len(self.P))]

    # -------------------------------------------------------------- geometry
    def h(self, l):
        return self.h0 / 2 ** l

    def period(self, l):
        return None if self.bc != 0 else self.N * 2 ** l

    def _ghost_plan(self, b):
        q, g = self.P[b], self.g
        l = q.level
        shape = tuple(int(s) for s in (q.n[2] + 2 * g, q.n[1] + 2 * g, q.n[0] + 2 * g))
        kk, jj, ii = np.meshgrid(*(np.arange(s) for s in shape), indexing="ij")
        inter = ((ii >= g) & (ii < g + q.n[0]) & (jj >= g) & (jj < g + q.n[1]) & (kk >= g) & (kk < g + q.n[2]))
        gz, gy, gx = np.nonzero(~inter)
        G = np.stack([gx + q.o[0] - g, gy + q.o[1] - g, gz + q.o[2] - g])  # (3, count), x first
        todo = np.ones(G.shape[1], dtype=bool)
        plan = dict(dst=(gz, gy, gx), boundary=None, copy=[], prolong=[])
        per = self.period(l)
        if l == 0 and self.bc != 0:
            out = np.any((G < 0) | (G >= self.N[:, None]), axis=0)
            plan["boundary"] = out
            todo &= ~out
        for s in self.at[l]:
            if not todo.any():
                break
            r = self.P[s]
            ok = todo.copy()
            src = []
            for a in range(3):
                fit, sh = _fit(G[a], 1, r.o[a], r.o[a] + r.n[a], None if per is None else per[a])
                ok &= fit
                src.append(sh - r.o[a] + g)
            if ok.any():
                plan["copy"].append((s, ok, (src[2][ok], src[1][ok], src[0][ok])))
                todo &= ~ok
        if l >= 1 and todo.any():
            base = np.where(G % 2 == 0, G // 2 - 2, G // 2 - 1)
            sel = todo.copy()
            Gs, bs = G[:, sel], base[:, sel]
            # 64 stencil cells per ghost point: source patch and padded index
            cells = []
            ok = np.ones(Gs.shape[1], dtype=bool)
            for a3 in range(4):
                for a2 in range(4):
                    for a1 in range(4):
                        C = np.stack([bs[0] + a1, bs[1] + a2, bs[2] + a3])
                        src, idx = self._coarse_cells(l - 1, C)
                        ok &= src >= 0
                        cells.append((src, idx))
            if not ok.all():
                raise ValueError(f"patch {b}: ghost points whose coarse stencil has no source (not properly nested)")
            x = [(0.5 * Gs[a] - 0.25) - bs[a] for a in range(3)]
            w = [lagrange_weights(x[a], [0.0, 1.0, 2.0, 3.0]) for a in range(3)]
            plan["prolong"].append((sel, cells, w))
            todo &= ~sel
        if todo.any():
            raise ValueError(f"patch {b}: {int(todo.sum())} ghost points have no source (not properly nested)")
        return plan

    def _coarse_cells(self, l, C):
        """Source of level-l cells C (3, count): the first patch whose
        interior fits the cell, else the first whose padded box does.
        Returns (patch index or -1, padded (z, y, x) indices)."""
        g = self.g
        per = self.period(l)
        src = np.full(C.shape[1], -1, dtype=np.int64)
        idx = np.zeros((3, C.shape[1]), dtype=np.int64)
        for pad in (0, g):
            for s in self.at[l]:
                r = self.P[s]
                ok = src < 0
                loc = []
                for a in range(3):
                    fit, sh = _fit(C[a], 1, r.o[a] - pad, r.o[a] + r.n[a] + pad, None if per is None else per[a])
                    ok &= fit
                    loc.append(sh - r.o[a] + g)
                src[ok] = s
                for a in range(3):
                    idx[2 - a][ok] = loc[a][ok]
        return src, idx

    def _restrict_plan(self, b):
        """Coarse interior cells of patch b and their fine sources (level l+1)."""
        q, g = self.P[b], self.g
        l = q.level
        if l + 1 >= self.nlev:
            return []
        kk, jj, ii = np.meshgrid(*(np.arange(int(q.n[a])) for a in (2, 1, 0)), indexing="ij")
        C = np.stack([ii.ravel() + q.o[0], jj.ravel() + q.o[1], kk.ravel() + q.o[2]])
        todo = np.ones(C.shape[1], dtype=bool)
        fper = self.period(l + 1)
        out = []
        w = lagrange_weights(1.5, [0.0, 1.0, 2.0, 3.0])  # coarse centre between fine 2c and 2c+1
        for s in self.at[l + 1]:
            if not todo.any():
                break
            r = self.P[s]
            ok = todo.copy()
            lo_idx = []
            for a in range(3):
                fit, sh = _fit(2 * C[a] - 1, 4, r.o[a], r.o[a] + r.n[a], None if fper is None else fper[a])
                ok &= fit
                lo_idx.append(sh - r.o[a] + g)
            if ok.any():
                dst = (C[2][ok] - q.o[2] + g, C[1][ok] - q.o[1] + g, C[0][ok] - q.o[0] + g)
                out.append((s, dst, [lo_idx[a][ok] for a in range(3)], w))
                todo &= ~ok
        return out

    # -------------------------------------------------------------- transfer
    @staticmethod
    def _interp(u, lo, w):
        """sum_{a,b,c} wz[a] wy[b] wx[c] u[:, lz+a, ly+b, lx+c] per point."""
        lx, ly, lz = lo
        wx, wy, wz = w
        s = 0.0
        for a in range(4):
            for bb in range(4):
                for c in range(4):
                    s = s + (np.asarray(wz[a]) * np.asarray(wy[bb]) * np.asarray(wx[c])) * u[:, lz + a, ly + bb, lx + c]
        return s

    def _prolong(self, cells, w, j):
        """Tricubic interpolant of stage state j of the parent level (j = 0:
        y0; j = 1..4: D_j = S_j - y0, formed cell by cell) at the fine
        points; cells[a3*16 + a2*4 + a1] = (source patch, (z, y, x))."""
        wx, wy, wz = w
        out = 0.0
        for a3 in range(4):
            for a2 in range(4):
                for a1 in range(4):
                    src, (iz, iy, ix) = cells[a3 * 16 + a2 * 4 + a1]
                    v = np.empty((24, src.size))
                    for s in np.unique(src):
                        m = src == s
                        st = self.P[s].stages
                        v[:, m] = st[0][:, iz[m], iy[m], ix[m]]
                        if j > 0:
                            v[:, m] = st[j][:, iz[m], iy[m], ix[m]] - v[:, m]
                    out = out + (wz[a3] * wy[a2] * wx[a1]) * v
        return out

    def _fill(self, l, arrays, m, s):
        """Set the ghosts of level l's arrays (list indexed like self.P) for
        the input of fine stage s (0..3) of half m of the parent's step, or
        for the result of that half (s = 4)."""
        for b in self.at[l]:
            pl = self.plans[b]
            gz, gy, gx = pl["dst"]
            u = arrays[b]
            if pl["boundary"] is not None and self.bc == 1:
                sel = pl["boundary"]
                u[:, gz[sel], gy[sel], gx[sel]] = self.P[b].ghost_src[:, gz[sel], gy[sel], gx[sel]]
            for sib, ok, src in pl["copy"]:
                u[:, gz[ok], gy[ok], gx[ok]] = arrays[sib][:, src[0], src[1], src[2]]
            if pl["prolong"]:
                d = fine_ghost_coeffs(m, s)
                for gi, (ok, cells, w) in enumerate(pl["prolong"]):
                    # P[y0], P[D2..D5] depend only on the parent level's latest step
                    key = (b, gi)
                    if key not in self._pcache:
                        self._pcache[key] = [self._prolong(cells, w, j) for j in range(5)]
                    Pj = self._pcache[key]
                    val = Pj[0]
                    for j in range(4):
                        if d[j] != 0.0:
                            val = val + d[j] * Pj[j + 1]
                    u[:, gz[ok], gy[ok], gx[ok]] = val

    def _restrict(self, l):
        for b in self.at[l]:
            for s, dst, lo, w in self.rplans[b]:
                self.P[b].state[:, dst[0], dst[1], dst[2]] = self._interp(self.P[s].state, lo, [w, w, w])

    # -------------------------------------------------------------- evolution
    def _k(self, l, b, ys):
        q = self.P[b]
        k = _rhs(ys, self.g, tuple(self.h(l)), self.p, ko=True)
        pl = self.plans[b]
        if l == 0 and self.bc == 2 and pl["boundary"] is not None:
            sel = pl["boundary"]
            gz, gy, gx = (d[sel] for d in pl["dst"])
            xyz0 = self.xlo + (q.o - self.g + 0.5) * self.h(l)
            sr = sommerfeld_rhs(ys, tuple(self.h(l)), xyz0, self.speeds)
            k[:, gz, gy, gx] = sr[:, gz, gy, gx]
        return k

    def _advance(self, l, m):
        dt = self.dt0 / 2 ** l
        bs = self.at[l]
        arrays = [None] * len(self.P)
        for b in bs:
            arrays[b] = self.P[b].state
        self._fill(l, arrays, m, 0)
        y0 = {b: self.P[b].state.copy() for b in bs}
        kept = {b: [y0[b]] for b in bs}
        cnode = (0.5, 0.5, 1.0)
        ks = []
        ys = dict(y0)
        for st in range(4):
            if st > 0:
                arrays = [None] * len(self.P)
                for b in bs:
                    arrays[b] = ys[b]
                self._fill(l, arrays, m, st)
                for b in bs:
                    kept[b].append(ys[b])
            k = {b: self._k(l, b, ys[b]) for b in bs}
            ks.append(k)
            if st < 3:
                ys = {b: y0[b] + (cnode[st] * dt) * k[b] for b in bs}
        for b in bs:
            self.P[b].state[...] = y0[b] + dt / 6.0 * (ks[0][b] + 2.0 * ks[1][b] + 2.0 * ks[2][b] + ks[3][b])
        arrays = [None] * len(self.P)
        for b in bs:
            arrays[b] = self.P[b].state
        self._fill(l, arrays, m, 4)
        if l + 1 < self.nlev:
            for b in bs:
                self.P[b].stages = tuple(kept[b]) + (self.P[b].state.copy(),)
            for b in self.at[l + 1]:
                for key in [k for k in self._pcache if k[0] == b]:
                    del self._pcache[key]
            self._advance(l + 1, 0)
            self._advance(l + 1, 1)
            self._restrict(l)
            self._fill(l, arrays, m, 4)

    def step(self):
        self._advance(0, 0)

    def updates_per_step(self):
        return sum(int(np.prod(q.n)) * 2 ** q.level for q in self.P)

    # -------------------------------------------------------------- regridding
    def regrid(self, geometry):
        """A new hierarchy at the current time on the patch boxes `geometry`
        (list of (level, origin, n)). Level 0 is not regridded: its boxes must
        be the current ones, in the same order, and keep their states. Every
        cell of a new patch's padded box on a level l >= 1 takes the value of
        the first current level-l patch (input order) whose interior holds it
        (periodic images included), else the tricubic prolongation of the new
        level l-1 read as one field on cells (the rule of the ghost cells),
        levels filled in increasing order. Returns the new Hierarchy."""
        g = self.g
        old0 = [(tuple(q.o), tuple(q.n)) for q in self.P if q.level == 0]
        new0 = [(tuple(o), tuple(n)) for lv, o, n in geometry if lv == 0]
        if old0 != new0:
            raise ValueError("level 0 is not regridded: its boxes must stay the same")
        pts = []
        it0 = iter([q for q in self.P if q.level == 0])
        for lv, o, n in geometry:
            if lv == 0:
                q = next(it0)
                pts.append(Patch(0, o, n, q.state.copy(), ghost_src=q.ghost_src))
            else:
                pts.append(Patch(lv, o, n, np.zeros((24, n[2] + 2 * g, n[1] + 2 * g, n[0] + 2 * g))))
        H = Hierarchy(pts, g, self.N, self.xlo, self.h0, self.bc, self.p, self.dt0)
        for l in range(1, H.nlev):
            old = [q for q in self.P if q.level == l]
            per = H.period(l)
            for b in H.at[l]:
                q = H.P[b]
                shape = q.state.shape[1:]
                kk, jj, ii = np.meshgrid(*(np.arange(s) for s in shape), indexing="ij")
                kk, jj, ii = kk.ravel(), jj.ravel(), ii.ravel()
                G = np.stack([ii + q.o[0] - g, jj + q.o[1] - g, kk + q.o[2] - g])
                todo = np.ones(G.shape[1], dtype=bool)
                for r in old:
                    ok = todo.copy()
                    src = []
                    for a in range(3):
                        fit, sh = _fit(G[a], 1, r.o[a], r.o[a] + r.n[a], None if per is None else per[a])
                        ok &= fit
                        src.append(sh - r.o[a] + g)
                    if ok.any():
                        q.state[:, kk[ok], jj[ok], ii[ok]] = r.state[:, src[2][ok], src[1][ok], src[0][ok]]
                        todo &= ~ok
                if todo.any():
                    Gs = G[:, todo]
                    base = np.where(Gs % 2 == 0, Gs // 2 - 2, Gs // 2 - 1)
                    x = [(0.5 * Gs[a] - 0.25) - base[a] for a in range(3)]
                    w = [lagrange_weights(x[a], [0.0, 1.0, 2.0, 3.0]) for a in range(3)]
                    val = 0.0
                    for a3 in range(4):
                        for a2 in range(4):
                            for a1 in range(4):
                                C = np.stack([base[0] + a1, base[1] + a2, base[2] + a3])
                                srcp, (iz, iy, ix) = H._coarse_cells(l - 1, C)
                                if np.any(srcp < 0):
                                    raise ValueError("regridded patch not properly nested")
                                v = np.empty((24, srcp.size))
                                for s in np.unique(srcp):
                                    m = srcp == s
                                    v[:, m] = H.P[s].state[:, iz[m], iy[m], ix[m]]
                                val = val + (w[2][a3] * w[1][a2] * w[0][a1]) * v
                    q.state[:, kk[todo], jj[todo], ii[todo]] = val
        return H
