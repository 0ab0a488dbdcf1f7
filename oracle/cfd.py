"""Incompressible Navier-Stokes on a staggered grid by the SOLA scheme: the
three-kernel CFD benchmark of the paper's Sec. 3.2 ("CFD with Chemora and
Physis": an explicit velocity update, an iterative mass-conservation kernel
that updates velocity and pressure, and a boundary kernel applied after each
iteration; single precision; 256^3 per GPU).

TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's
CPU-baseline leg use this module. It shares no code with the CUDA library.

The paper cites the discretisation (Hirt & Nichols 1981, Torrey et al.,
NASA-VOF2D) without printing it. This module follows the SOLA algorithm of
Hirt, Nichols & Romero (Los Alamos LA-5852, 1975), extended to 3D, without
the free-surface (VOF) part, in numpy; every array is of the given dtype
(float64 for the pins, float32 like the paper's benchmark).

Grid. nx x ny x nz cells of size dx, dy, dz plus one ghost layer; arrays have
shape (nz+2, ny+2, nx+2) and index [k+1, j+1, i+1] holds cell (i, j, k):
  p[k, j, i]  pressure at the cell centre (density 1);
  u[k, j, i]  x-velocity on the face between cells i and i+1 (i + 1/2);
  v[k, j, i]  y-velocity on the face j + 1/2;  w[k, j, i]  z-velocity on k + 1/2.
Boundaries, per axis: periodic, or walls on both sides. On a wall axis the
two wall faces (index -1 and n-1 of the normal component) hold zero normal
velocity and are never moved; tangential components get ghost values from
the no-slip condition, ghost = 2 U_wall - interior (U_wall = the lid speed
for the x-velocity on the top z wall, 0 elsewhere).

Kernel 1, velocity (for every face that is not a wall face):
  u~ = u + dt [ (p_i - p_{i+1})/dx + g_x - FUX - FUY - FUZ + VISX ]
with SOLA's advective fluxes, a blend of centred (alpha = 0) and donor-cell
(alpha = 1) differencing,
  FUX = [ (u_c+u_e)^2 + alpha|u_c+u_e|(u_c-u_e) - (u_w+u_c)^2 - alpha|u_w+u_c|(u_w-u_c) ] / (4 dx)
  FUY = [ (v_c+v_ce)(u_c+u_n) + alpha|v_c+v_ce|(u_c-u_n)
          - (v_s+v_se)(u_s+u_c) - alpha|v_s+v_se|(u_s-u_c) ] / (4 dy)
  (v_c, v_ce: v on faces j+1/2 of cells i and i+1; v_s, v_se: on faces j-1/2)
  FUZ  likewise with w,
  VISX = nu [ (u_e - 2u_c + u_w)/dx^2 + (u_n - 2u_c + u_s)/dy^2 + (u_t - 2u_c + u_b)/dz^2 ],
and the same with the roles of the axes permuted for v and w.

Kernel 2, mass conservation: one iteration is a red and then a black
half-sweep (colour (i + j + k) mod 2) over all cells; for a cell,
  D  = (u_i - u_{i-1})/dx + (v_j - v_{j-1})/dy + (w_k - w_{k-1})/dz,
  dp = -beta D,   beta = omega / (dt * sum over the cell's movable faces of 1/h_a^2),
  p += dp;  every movable face of the cell moves by dt dp / h_a, outward
  positive (u_i += dt dp/dx, u_{i-1} -= dt dp/dx, ...).
Cells of one colour share no face (a periodic axis needs an even number of
cells for that), so a half-sweep done for all of them at once equals SOLA's
sequential sweep over them; after a cell's update its own divergence is
(1 - omega) D. Wall faces are not movable (the sum then has
one term less per wall face), so no boundary reset undoes the correction.

Kernel 3, boundary: ghost layers of u, v, w and p (periodic wrap, or the
wall rules above; p on a wall axis: zero normal gradient), applied after the
velocity kernel and after every mass-conservation iteration.
"""
import numpy as np


class Flow:
    """nx, ny, nz cells; h = (dx, dy, dz); periodic = (bool per axis x, y, z);
    lid = x-velocity of the top z wall (walls only); nu, dt, omega, alpha,
    g = (gx, gy, gz)."""

    def __init__(self, n, h, periodic, nu, dt, omega=1.7, alpha=0.3, lid=0.0, g=(0.0, 0.0, 0.0),
                 dtype=np.float64):
        self.n = tuple(int(x) for x in n)
        self.h = tuple(float(x) for x in h)
        self.per = tuple(bool(x) for x in periodic)
        self.dt = dtype(dt)
        self.nu = dtype(nu)
        self.omega = dtype(omega)
        self.alpha = dtype(alpha)
        self.lid = dtype(lid)
        self.g = tuple(dtype(x) for x in g)
        self.dtype = dtype
        if any(p and (n % 2) for p, n in zip(self.per, self.n)):
            raise ValueError("a periodic axis needs an even number of cells (red-black colouring)")
        shape = (self.n[2] + 2, self.n[1] + 2, self.n[0] + 2)
        self.u, self.v, self.w, self.p = (np.zeros(shape, dtype=dtype) for _ in range(4))
        self._beta = self._beta_field()

    # ---------------------------------------------------------------- helpers
    def _movable(self, a):
        """Boolean masks over cells (nz, ny, nx): is the low / high face of
        the cell along axis a (0 x, 1 y, 2 z) movable?"""
        nx, ny, nz = self.n
        lo = np.ones((nz, ny, nx), dtype=bool)
        hi = np.ones((nz, ny, nx), dtype=bool)
        if not self.per[a]:
            sl_lo = [slice(None)] * 3
            sl_hi = [slice(None)] * 3
            sl_lo[2 - a] = 0
            sl_hi[2 - a] = self.n[a] - 1
            lo[tuple(sl_lo)] = False
            hi[tuple(sl_hi)] = False
        return lo, hi

    def _beta_field(self):
        dt = self.dtype
        s = np.zeros((self.n[2], self.n[1], self.n[0]), dtype=dt)
        for a in range(3):
            lo, hi = self._movable(a)
            ih2 = dt(1.0) / (dt(self.h[a]) * dt(self.h[a]))
            s = s + lo.astype(dt) * ih2 + hi.astype(dt) * ih2
        return self.omega / (self.dt * s)

    def interior(self, f):
        return f[1:-1, 1:-1, 1:-1]

    # ---------------------------------------------------------------- kernel 3: boundary
    def boundary(self):
        nx, ny, nz = self.n
        comps = (self.u, self.v, self.w)
        for a in range(3):            # axis of the boundary
            ax = 2 - a                # array axis
            for c, f in enumerate(comps + (self.p,)):
                lo = [slice(None)] * 3
                hi = [slice(None)] * 3
                lo_in = [slice(None)] * 3
                hi_in = [slice(None)] * 3
                if self.per[a]:
                    lo[ax], hi[ax], lo_in[ax], hi_in[ax] = 0, self.n[a] + 1, self.n[a], 1
                    f[tuple(lo)] = f[tuple(lo_in)]
                    f[tuple(hi)] = f[tuple(hi_in)]
                    continue
                if c == a:            # normal velocity: wall faces (index -1 and n-1) are zero
                    lo[ax], hi[ax] = 0, self.n[a]
                    f[tuple(lo)] = 0
                    f[tuple(hi)] = 0
                    hi2 = [slice(None)] * 3
                    hi2[ax] = self.n[a] + 1
                    f[tuple(hi2)] = 0
                    continue
                lo[ax], hi[ax], lo_in[ax], hi_in[ax] = 0, self.n[a] + 1, 1, self.n[a]
                if c == 3:            # pressure: zero normal gradient
                    f[tuple(lo)] = f[tuple(lo_in)]
                    f[tuple(hi)] = f[tuple(hi_in)]
                    continue
                wall_hi = self.lid if (a == 2 and c == 0) else self.dtype(0)
                f[tuple(lo)] = -f[tuple(lo_in)]
                f[tuple(hi)] = self.dtype(2) * wall_hi - f[tuple(hi_in)]

    # ---------------------------------------------------------------- kernel 1: velocity
    def _face_range(self, c, a):
        """Padded index range [start, stop) along axis a of the faces of
        component c that the velocity kernel advances (a wall axis leaves
        out its two wall faces, -1 and n-1)."""
        if a == c and not self.per[a]:
            return 1, self.n[a]
        return 1, self.n[a] + 1

    def velocity(self):
        D = self.dtype
        dt, al, nu = self.dt, self.alpha, self.nu
        h = [D(x) for x in self.h]
        comps = (self.u, self.v, self.w)
        new = []
        for c in range(3):
            rng = [self._face_range(c, a) for a in range(3)]  # x, y, z

            def S(arr, dx=0, dy=0, dz=0):
                d = (dx, dy, dz)
                return arr[rng[2][0] + d[2]:rng[2][1] + d[2], rng[1][0] + d[1]:rng[1][1] + d[1],
                           rng[0][0] + d[0]:rng[0][1] + d[0]]

            def off(a, t):
                o = [0, 0, 0]
                o[a] = t
                return o

            f = comps[c]
            fc = S(f)
            flux = D(0)
            vis = D(0)
            for b in range(3):
                fp = S(f, *off(b, 1))
                fm = S(f, *off(b, -1))
                if b == c:
                    sp = fc + fp
                    sm = fm + fc
                    F = (sp * sp + al * np.abs(sp) * (fc - fp) - sm * sm - al * np.abs(sm) * (fm - fc)) / (D(4) * h[b])
                else:
                    g = comps[b]
                    # velocity b on the faces b+1/2 (and b-1/2) of the two cells c and c+1
                    o_hi = off(c, 1)
                    o_lo = off(b, -1)
                    o_lo_hi = list(o_lo)
                    o_lo_hi[c] = 1
                    t_hi = S(g) + S(g, *o_hi)
                    t_lo = S(g, *o_lo) + S(g, *o_lo_hi)
                    F = (t_hi * (fc + fp) + al * np.abs(t_hi) * (fc - fp)
                         - t_lo * (fm + fc) - al * np.abs(t_lo) * (fm - fc)) / (D(4) * h[b])
                flux = flux + F
                vis = vis + (fp - D(2) * fc + fm) / (h[b] * h[b])
            grad = (S(self.p) - S(self.p, *off(c, 1))) / h[c]
            sl = tuple(slice(rng[a][0], rng[a][1]) for a in (2, 1, 0))
            new.append((sl, fc + dt * (grad + self.g[c] - flux + nu * vis)))
        for c, (sl, val) in enumerate(new):
            comps[c][sl] = val

    # ---------------------------------------------------------------- kernel 2: mass conservation
    def half_sweep(self, colour):
        """All cells with (i + j + k) % 2 == colour, at once."""
        nx, ny, nz = self.n
        kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        sel = (ii + jj + kk) % 2 == colour
        k, j, i = kk[sel] + 1, jj[sel] + 1, ii[sel] + 1
        # the low face of a cell (padded index - 1); on a periodic axis the
        # low face of cell 0 is face n-1 itself, not its ghost copy
        lo_idx = []
        for a, c in enumerate((i, j, k)):
            lo_idx.append(((c - 2) % self.n[a]) + 1 if self.per[a] else c - 1)
        il, jl, kl = lo_idx
        D = self.dtype
        dt = self.dt
        h = [D(x) for x in self.h]
        div = ((self.u[k, j, i] - self.u[k, j, il]) / h[0] + (self.v[k, j, i] - self.v[k, jl, i]) / h[1]
               + (self.w[k, j, i] - self.w[kl, j, i]) / h[2])
        dp = -self._beta[sel] * div
        self.p[k, j, i] += dp
        for a, (f, idx_hi, idx_lo) in enumerate((
                (self.u, (k, j, i), (k, j, il)),
                (self.v, (k, j, i), (k, jl, i)),
                (self.w, (k, j, i), (kl, j, i)))):
            lo, hi = self._movable(a)
            c = dt * dp / h[a]
            mh, ml = hi[sel], lo[sel]
            f[tuple(x[mh] for x in idx_hi)] += c[mh]
            f[tuple(x[ml] for x in idx_lo)] -= c[ml]

    def mass_iteration(self):
        self.half_sweep(0)
        self.half_sweep(1)

    def divergence(self):
        h = self.h
        u, v, w = self.u, self.v, self.w
        return ((u[1:-1, 1:-1, 1:-1] - u[1:-1, 1:-1, :-2]) / self.dtype(h[0])
                + (v[1:-1, 1:-1, 1:-1] - v[1:-1, :-2, 1:-1]) / self.dtype(h[1])
                + (w[1:-1, 1:-1, 1:-1] - w[:-2, 1:-1, 1:-1]) / self.dtype(h[2]))

    # ---------------------------------------------------------------- one time step
    def step(self, iterations=4):
        """Boundary, velocity, boundary, then `iterations` times (mass
        conservation iteration, boundary)."""
        self.boundary()
        self.velocity()
        self.boundary()
        for _ in range(iterations):
            self.mass_iteration()
            self.boundary()
