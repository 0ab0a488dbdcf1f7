"""Seeded synthetic inputs for the BSSN evolution: the gauge-wave exact
solution, Brill-Lindquist two-puncture data, seeded noise and smooth seeded
perturbations.

This module holds initial data only, none of the evolution's arithmetic
(no derivative, right-hand side, dissipation or time-integration step). It is
the one module that both the CUDA path's callers and the CPU oracle's tests
use to build their inputs.

Layout: numpy float64 array of shape (24, nz+2g, ny+2g, nx+2g), variable
order W, gt11, gt12, gt13, gt22, gt23, gt33, trK, At11, At12, At13, At22,
At23, At33, Gt1, Gt2, Gt3, alpha, beta1, beta2, beta3, B1, B2, B3. Points are
cell centred: x_i = lo + (i + 1/2) h for i = -g .. n+g-1.
"""
import numpy as np

VARS = ["W", "gt11", "gt12", "gt13", "gt22", "gt23", "gt33", "trK",
        "At11", "At12", "At13", "At22", "At23", "At33", "Gt1", "Gt2", "Gt3",
        "alpha", "beta1", "beta2", "beta3", "B1", "B2", "B3"]
NVAR = 24
IDX = {name: i for i, name in enumerate(VARS)}
SYM = ((0, 1, 2), (1, 3, 4), (2, 4, 5))

_MASK64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x):
    """SplitMix64 output function (Steele, Lea & Flood 2014) applied
    elementwise to uint64 array x (already offset by the caller)."""
    with np.errstate(over="ignore"):
        z = (x + np.uint64(0x9E3779B97F4A7C15)) & _MASK64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _MASK64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _MASK64
        return z ^ (z >> np.uint64(31))


def uniform_noise(seed, var, shape):
    """Uniform values in [-1, 1) from splitmix64(seed ^ (var << 40) ^ flat_index)."""
    n = int(np.prod(shape))
    idx = np.arange(n, dtype=np.uint64)
    key = np.uint64(seed) ^ (np.uint64(var) << np.uint64(40)) ^ idx
    z = splitmix64(key)
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return (2.0 * u - 1.0).reshape(shape)


def coords(n, g, lo, hi):
    h = (hi - lo) / n
    return lo + (np.arange(-g, n + g) + 0.5) * h, h


def empty_state(nx, ny, nz, g):
    return np.zeros((NVAR, nz + 2 * g, ny + 2 * g, nx + 2 * g))


def flat_space(nx, ny, nz, g, beta=(0.0, 0.0, 0.0)):
    u = empty_state(nx, ny, nz, g)
    u[IDX["W"]] = 1.0
    u[IDX["alpha"]] = 1.0
    for i in range(3):
        u[IDX["gt11"] + SYM[i][i]] = 1.0
        u[IDX["beta1"] + i] = beta[i]
    return u


def periodic_wrap(u, g):
    """Fill the ghost zones of every variable by periodic wrap (in place);
    works for any interior size, including n < g."""
    if g == 0:
        return u
    for axis in (1, 2, 3):
        n = u.shape[axis] - 2 * g
        idx = (np.arange(-g, n + g) % n) + g
        u[...] = np.take(u, idx, axis=axis)
    return u


def add_noise(u, g, amplitude, seed, periodic=True):
    """Add seeded uniform noise amplitude*[-1,1) to the interior of every
    variable, then (periodic=True) refill ghosts by periodic wrap."""
    nz, ny, nx = (s - 2 * g for s in u.shape[1:])
    for v in range(NVAR):
        u[v, g:g + nz, g:g + ny, g:g + nx] += amplitude * uniform_noise(seed, v, (nz, ny, nx))
    if periodic:
        periodic_wrap(u, g)
    return u


def gauge_wave(n, g, amplitude=0.01, wavelength=1.0, lo=-0.5, hi=0.5, t=0.0, noise=1e-10, seed=1307,
               ny=None, nz=None):
    """1D gauge wave along x: H = 1 - A sin(2 pi (x - t)/d); lapse sqrt(H),
    spatial metric diag(H, 1, 1), zero shift, in BSSN variables, on n points
    along x (ny, nz default to n; y and z use the same spacing).
    Returns (state, h). Ghosts are filled by periodic wrap."""
    x, h = coords(n, g, lo, hi)
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    A, d = amplitude, wavelength
    th = 2 * np.pi * (x - t) / d
    H = 1 - A * np.sin(th)
    dxH = -(2 * np.pi * A / d) * np.cos(th)
    Kxx = -(np.pi * A / d) * np.cos(th) / np.sqrt(H)
    u = empty_state(n, ny, nz, g)

    def put(name, f1d):
        u[IDX[name]] = np.broadcast_to(f1d[None, None, :], u.shape[1:])

    put("W", H ** (-1.0 / 6.0))
    put("gt11", H ** (2.0 / 3.0))
    put("gt22", H ** (-1.0 / 3.0))
    put("gt33", H ** (-1.0 / 3.0))
    put("trK", Kxx / H)
    put("At11", (2.0 / 3.0) * H ** (-1.0 / 3.0) * Kxx)
    put("At22", -(1.0 / 3.0) * H ** (-4.0 / 3.0) * Kxx)
    put("At33", -(1.0 / 3.0) * H ** (-4.0 / 3.0) * Kxx)
    put("Gt1", (2.0 / 3.0) * H ** (-5.0 / 3.0) * dxH)
    put("alpha", np.sqrt(H))
    if noise:
        add_noise(u, g, noise, seed, periodic=True)
    else:
        periodic_wrap(u, g)
    return u, h


def brill_lindquist(n, g, lo=-8.0, hi=8.0, masses=(0.5, 0.5), centers=((-1.5, 0, 0), (1.5, 0, 0)),
                    lapse_psi_power=-2.0):
    """Brill-Lindquist data: psi = 1 + sum m/(2 r); W = psi^-2,
    alpha = psi^lapse_psi_power (default psi^-2), gt = delta, everything else
    zero. Ghost points hold the same closed form. Returns (state, h)."""
    x, h = coords(n, g, lo, hi)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    psi = np.ones_like(X)
    for m, c in zip(masses, centers):
        r = np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2)
        psi += m / (2 * r)
    u = empty_state(n, n, n, g)
    u[IDX["W"]] = psi ** -2.0
    u[IDX["alpha"]] = psi ** lapse_psi_power
    for i in range(3):
        u[IDX["gt11"] + SYM[i][i]] = 1.0
    return u, h


def patch_tree(nblocks=192, seed=6488, sides=tuple(range(16, 97, 8)), h0=0.5, levels=4,
               centers=((-1.5, 0.0, 0.0), (1.5, 0.0, 0.0))):
    """Seeded set of refinement patches around two punctures: patch b has
    level L in [0, levels) (finer levels drawn more often), spacing
    h0 / 2^L (ratio-2 levels), per-axis sizes drawn from `sides`, and its
    centre near puncture b % 2 at an offset that shrinks with the level.
    Returns a list of dicts n=(nx, ny, nz), h, origin (lower corner of the
    interior cell faces), level."""
    out = []
    for b in range(nblocks):
        r = 0.5 * (uniform_noise(seed, b, (8,)) + 1.0)  # uniform [0, 1)
        level = min(levels - 1, int(levels * np.sqrt(r[0])))
        h = h0 / 2 ** level
        n = tuple(int(sides[min(len(sides) - 1, int(len(sides) * r[1 + a]))]) for a in range(3))
        reach = 3.0 / 2 ** level
        c = centers[b % len(centers)]
        centre = [c[a] + (2 * r[4 + a] - 1) * reach for a in range(3)]
        origin = tuple(centre[a] - n[a] * h / 2 for a in range(3))
        out.append(dict(n=n, h=h, origin=origin, level=level))
    return out


def bl_conformal_tricubic(n, g, h, origin, masses=(0.5, 0.5), centers=((-1.5, 0.0, 0.0), (1.5, 0.0, 0.0))):
    """psi^-2 of Brill-Lindquist data on one patch (interior and g ghosts,
    cell centres origin + (i + 1/2) h), by tricubic Lagrange interpolation of
    its values on the node lattice origin + j h: the 4-point midpoint weights
    (-1, 9, 9, -1)/16 applied along x, then y, then z. Shape (nz+2g, ny+2g,
    nx+2g). This is W = alpha of the patch."""
    nx, ny, nz = n
    ax = [origin[a] + np.arange(-g - 1, n[a] + g + 2) * h for a in range(3)]
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    psi = np.ones_like(X)
    for m, c in zip(masses, centers):
        psi += m / (2 * np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2))
    f = psi ** -2.0

    def mid(a, axis):
        m = a.shape[axis] - 3
        s = [slice(None)] * 3

        def take(k):
            s[axis] = slice(k, k + m)
            return a[tuple(s)]
        return (-take(0) + 9 * take(1) + 9 * take(2) - take(3)) / 16.0

    return mid(mid(mid(f, 2), 1), 0)


def smooth_perturbation(u, g, amplitude, seed, h, periodic=False):
    """Add a seeded smooth perturbation to every variable, ghosts included:
    a sum of three plane waves per variable with seeded wave vectors (1..3
    cycles over 16 h) and phases, times amplitude (and, for the diagonal of
    gt, W and alpha, kept so that they stay positive). With periodic=True,
    the interior is perturbed and ghosts are refilled by periodic wrap."""
    nzp, nyp, nxp = u.shape[1:]
    r = uniform_noise(seed, 63, (NVAR, 3, 5))
    zi, yi, xi = np.meshgrid(np.arange(nzp), np.arange(nyp), np.arange(nxp), indexing="ij")
    L = 16.0
    for v in range(NVAR):
        f = np.zeros(u.shape[1:])
        for w in range(3):
            kx, ky, kz, ph, a = r[v, w]
            f += (0.6 + 0.4 * a) * np.sin(2 * np.pi * ((1 + kx) * xi / L + (1 + ky) * yi / L + (1 + kz) * zi / L)
                                          + np.pi * ph)
        u[v] += amplitude * f
    if periodic:
        periodic_wrap(u, g)
    return u


# ------------------------------------------------------------------ patches of a refined hierarchy
def box_coords(origin, n, g, h, xlo):
    """Cell-centre coordinates (x, y, z) of the padded points of a patch whose
    interior is cells [origin, origin + n) of a level with spacing h
    (scalar or 3) over a domain whose lower corner is xlo."""
    hh = (h, h, h) if np.isscalar(h) else h
    return [xlo[a] + (origin[a] + np.arange(-g, n[a] + g) + 0.5) * hh[a] for a in range(3)]


def gauge_wave_box(origin, n, g, h, xlo, amplitude=0.01, wavelength=1.0, t=0.0):
    """The gauge-wave closed form of gauge_wave() at every padded point of a
    patch (ghosts included, no noise)."""
    x = box_coords(origin, n, g, h, xlo)[0]
    A, d = amplitude, wavelength
    th = 2 * np.pi * (x - t) / d
    H = 1 - A * np.sin(th)
    dxH = -(2 * np.pi * A / d) * np.cos(th)
    Kxx = -(np.pi * A / d) * np.cos(th) / np.sqrt(H)
    u = empty_state(n[0], n[1], n[2], g)

    def put(name, f1d):
        u[IDX[name]] = np.broadcast_to(f1d[None, None, :], u.shape[1:])

    put("W", H ** (-1.0 / 6.0))
    put("gt11", H ** (2.0 / 3.0))
    put("gt22", H ** (-1.0 / 3.0))
    put("gt33", H ** (-1.0 / 3.0))
    put("trK", Kxx / H)
    put("At11", (2.0 / 3.0) * H ** (-1.0 / 3.0) * Kxx)
    put("At22", -(1.0 / 3.0) * H ** (-4.0 / 3.0) * Kxx)
    put("At33", -(1.0 / 3.0) * H ** (-4.0 / 3.0) * Kxx)
    put("Gt1", (2.0 / 3.0) * H ** (-5.0 / 3.0) * dxH)
    put("alpha", np.sqrt(H))
    return u


def brill_lindquist_box(origin, n, g, h, xlo, masses=(0.5, 0.5), centers=((-1.5, 0, 0), (1.5, 0, 0))):
    """Brill-Lindquist data (W = alpha = psi^-2, gt = delta) at every padded
    point of a patch."""
    x, y, z = box_coords(origin, n, g, h, xlo)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    psi = np.ones_like(X)
    for m, c in zip(masses, centers):
        psi += m / (2 * np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2))
    u = empty_state(n[0], n[1], n[2], g)
    u[IDX["W"]] = psi ** -2.0
    u[IDX["alpha"]] = psi ** -2.0
    for i in range(3):
        u[IDX["gt11"] + SYM[i][i]] = 1.0
    return u


def bl_hierarchy(n0=96, nested=4, fine_half=24, split=2, extent=96.0,
                 centers=((-1.5, 0.0, 0.0), (1.5, 0.0, 0.0))):
    """Geometry of a properly nested refinement hierarchy for two punctures:
    level 0 is n0^3 cells over [-extent/2, extent/2]^3 (h0 = extent/n0);
    each level l = 1 .. nested-1 is n0^3 cells covering the middle half of
    level l-1; every level is cut into split^3 equal patches. Level `nested`
    has one box of (2 fine_half)^3 cells per puncture, centred on the
    puncture's cell (origins even). Returns (ncells, xlo, h0, list of
    (level, origin, n)); origins are in each level's cell index space."""
    h0 = extent / n0
    xlo = (-extent / 2,) * 3
    out = []
    s = n0 // split
    for lev in range(nested):
        off = (n0 // 2) * (2 ** lev - 1)  # the middle half of every coarser level
        for k in range(split):
            for j in range(split):
                for i in range(split):
                    out.append((lev, (off + i * s, off + j * s, off + k * s), (s, s, s)))
    hl = h0 / 2 ** nested
    for c in centers:
        org = []
        for a in range(3):
            cell = int(np.floor((c[a] - xlo[a]) / hl))
            org.append(2 * ((cell - fine_half) // 2))
        out.append((nested, tuple(org), (2 * fine_half,) * 3))
    return (n0, n0, n0), xlo, h0, out
