"""Seeded synthetic inputs for the S-fraction multiscale finite-volume method.

This module is shared by the FP64 oracle (``oracle/``) and the GPU library
(``paper_1406_6923_gb300``).  It holds no arithmetic of the method itself:
only velocity models, the subdomain cuts, ROM sizes, source and receiver
positions, the Ricker wavelet and the spatial weights that say where a point
source acts and where a receiver samples.  Everything the method computes
from these (operators, ROMs, S-fraction coefficients, projections, coupling,
time stepping) is implemented independently on each side.

Conventions
-----------
* A grid of ``nx*ny*nz`` cells of side ``h`` metres; cell-centred velocity
  ``c[nz, ny, nx]`` in m/s; nodes ``(i, j, k)`` sit at ``(i*h, j*h, k*h)``.
* Cuts are node indices along an axis, including 0 and n; subdomains are the
  boxes between consecutive cuts, numbered ``ix + ncx*(iy + ncy*iz)``.
* The paper's experiment (section "Numerical experiments") uses a velocity
  model that is only shown in a figure, so every model here is a seeded
  synthetic stand-in with the shapes of the workloads the method targets.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

SEED = 1406


@dataclass
class Problem:
    name: str
    nx: int
    ny: int
    nz: int
    h: float
    c: np.ndarray                      # [nz, ny, nx] cell velocities (m/s)
    xcuts: np.ndarray                  # node indices incl. 0 and nx
    ycuts: np.ndarray
    zcuts: np.ndarray
    m_sub: np.ndarray                  # [nsub] face modes requested per subdomain
    k_sub: np.ndarray                  # [nsub] number of S-fraction levels
    sigma: float                       # Krylov shift (s^-2)
    f_peak: float                      # Ricker peak frequency (Hz)
    src_xyz: np.ndarray                # [nshots, 3] metres
    rec_xyz: np.ndarray                # [nrec, 3] metres
    nsteps: int
    src_sigma: float = 0.0             # Gaussian width of the source (m); 0 -> h
    dt_safety: float = 0.9
    meta: dict = field(default_factory=dict)

    @property
    def ncuts(self):
        return (len(self.xcuts) - 1, len(self.ycuts) - 1, len(self.zcuts) - 1)

    @property
    def nsub(self):
        a, b, c = self.ncuts
        return a * b * c

    @property
    def nshots(self):
        return int(self.src_xyz.shape[0])

    @property
    def nrec(self):
        return int(self.rec_xyz.shape[0])

    def sub_index(self, ix, iy, iz):
        ncx, ncy, _ = self.ncuts
        return ix + ncx * (iy + ncy * iz)

    def sub_box(self, s):
        """Node-index box ``(x0, x1, y0, y1, z0, z1)`` (inclusive) of subdomain ``s``."""
        ncx, ncy, _ = self.ncuts
        ix = s % ncx
        iy = (s // ncx) % ncy
        iz = s // (ncx * ncy)
        return (int(self.xcuts[ix]), int(self.xcuts[ix + 1]),
                int(self.ycuts[iy]), int(self.ycuts[iy + 1]),
                int(self.zcuts[iz]), int(self.zcuts[iz + 1]))

    @property
    def src_width(self):
        return self.src_sigma if self.src_sigma > 0 else self.h


# ----------------------------------------------------------------------------
# wavelet
# ----------------------------------------------------------------------------

def ricker(t, f, delay=None):
    """Ricker wavelet ``(1 - 2 pi^2 f^2 tau^2) exp(-pi^2 f^2 tau^2)``, ``tau = t - 1.5/f``."""
    if delay is None:
        delay = 1.5 / f
    tau = np.asarray(t, dtype=np.float64) - delay
    a = (np.pi * f * tau) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def wavelet_samples(problem: Problem, dt: float, nsteps: int | None = None):
    """Source time function per shot sampled at ``t_n = n*dt``, n = 0..nsteps-1.

    Returns float64 ``[nshots, nsteps]`` (all shots share the Ricker of the
    problem's peak frequency)."""
    n = problem.nsteps if nsteps is None else nsteps
    s = ricker(np.arange(n) * dt, problem.f_peak)
    return np.tile(s, (problem.nshots, 1))


# ----------------------------------------------------------------------------
# point weights: where a source acts / where a receiver samples
# ----------------------------------------------------------------------------

def gaussian_node_weights(xyz, width, h, nx, ny, nz):
    """Normalised Gaussian ``exp(-r^2/2w^2)`` on the grid nodes within ``3w``
    of ``xyz`` (metres); returns ``(nodes[n,3] int, weights[n])`` with
    ``sum(weights) == 1``."""
    x = np.asarray(xyz, dtype=np.float64)
    rad = 3.0 * width
    lo = np.maximum(np.floor((x - rad) / h).astype(int), 0)
    hi = np.minimum(np.ceil((x + rad) / h).astype(int), [nx, ny, nz])
    ii, jj, kk = np.meshgrid(np.arange(lo[0], hi[0] + 1), np.arange(lo[1], hi[1] + 1),
                             np.arange(lo[2], hi[2] + 1), indexing="ij")
    nodes = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1)
    r2 = np.sum((nodes * h - x) ** 2, axis=1)
    keep = r2 <= rad * rad + 1e-9 * h * h
    nodes, r2 = nodes[keep], r2[keep]
    w = np.exp(-r2 / (2.0 * width * width))
    return nodes, w / w.sum()


def trilinear_node_weights(xyz, h, nx, ny, nz):
    """Trilinear interpolation weights of a point (metres) on the grid nodes.
    Returns ``(nodes[n,3] int, weights[n])``; zero weights are dropped."""
    x = np.asarray(xyz, dtype=np.float64) / h
    base = np.minimum(np.floor(x + 1e-12).astype(int), [nx - 1, ny - 1, nz - 1])
    base = np.maximum(base, 0)
    fr = np.clip(x - base, 0.0, 1.0)
    nodes, ws = [], []
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                w = ((fr[0] if dx else 1 - fr[0]) * (fr[1] if dy else 1 - fr[1])
                     * (fr[2] if dz else 1 - fr[2]))
                if w > 1e-14:
                    nodes.append(base + [dx, dy, dz])
                    ws.append(w)
    ws = np.array(ws)
    return np.array(nodes, dtype=int).reshape(-1, 3), ws / ws.sum()


# ----------------------------------------------------------------------------
# velocity models
# ----------------------------------------------------------------------------

def _cell_centres(nx, ny, nz, h):
    z, y, x = np.meshgrid((np.arange(nz) + 0.5) * h, (np.arange(ny) + 0.5) * h,
                          (np.arange(nx) + 0.5) * h, indexing="ij")
    return x, y, z


def two_layer(nx, ny, nz, zint, c_top=1500.0, c_bot=3000.0):
    """Two layers with a flat interface at cell index ``zint``."""
    c = np.full((nz, ny, nx), c_top)
    c[zint:] = c_bot
    return c


def layered_lens(nx, ny, nz, h, rng, avoid=24, nlay=None, lens_amp=1200.0,
                 lens_w=15.0, cmin=1500.0, cmax=4500.0):
    """Seeded horizontal layers (velocity rising with depth, +-10% jitter) at
    random depths that avoid multiples of ``avoid`` cells, plus a Gaussian
    high-velocity lens; clipped to ``[cmin, cmax]``."""
    if nlay is None:
        nlay = 6 + int(rng.integers(-2, 3))
    cand = np.array([z for z in range(1, nz) if z % avoid != 0])
    zs = np.sort(rng.choice(cand, size=nlay, replace=False))
    vel = np.linspace(cmin, cmax, nlay + 1) * (1.0 + 0.1 * rng.uniform(-1, 1, nlay + 1))
    c = np.empty((nz, ny, nx))
    edges = np.concatenate([[0], zs, [nz]])
    for i in range(nlay + 1):
        c[edges[i]:edges[i + 1]] = vel[i]
    x, y, z = _cell_centres(nx, ny, nz, h)
    ctr = rng.uniform(0.2, 0.8, 3) * np.array([nx, ny, nz]) * h
    r2 = (x - ctr[0]) ** 2 + (y - ctr[1]) ** 2 + (z - ctr[2]) ** 2
    c = c + lens_amp * np.exp(-r2 / (2.0 * (lens_w * h) ** 2))
    return np.clip(c, cmin, cmax)


def salt_bodies(nx, ny, nz, h, rng, nbody=None, c_salt=4500.0):
    """Layered background plus 2-3 star-shaped 'salt' bodies at ``c_salt``:
    the radius is a smooth random function of direction, the boundary sharp."""
    c = layered_lens(nx, ny, nz, h, rng, avoid=32, lens_amp=0.0)
    if nbody is None:
        nbody = 2 + int(rng.integers(0, 2))
    x, y, z = _cell_centres(nx, ny, nz, h)
    L = np.array([nx, ny, nz]) * h
    for _ in range(nbody):
        ctr = rng.uniform([0.2, 0.2, 0.35], [0.8, 0.8, 0.8]) * L
        r0 = rng.uniform(0.08, 0.16) * min(L[0], L[1])
        dx, dy, dz = x - ctr[0], y - ctr[1], z - ctr[2]
        r = np.sqrt(dx * dx + dy * dy + dz * dz) + 1e-9
        th = np.arccos(np.clip(dz / r, -1, 1))
        ph = np.arctan2(dy, dx)
        rad = r0 * np.ones_like(r)
        for l in range(1, 4):
            a, b = rng.normal(0, 0.12 / l, 2)
            rad = rad * (1.0 + a * np.cos(l * ph + rng.uniform(0, 2 * np.pi))
                         * np.sin(th) + b * np.cos(l * th))
        c[r < rad] = c_salt
    return c


def skew_fracture(nx, ny, nz, h, rng, c_max=1.0, c_frac=0.3, width=0.08):
    """A velocity c(x, y) that does not depend on z: 3-4 regions separated by
    skewed straight lines (values drawn in [0.55, 1] * c_max) crossed by a
    thin slow fracture, a polyline of three segments (two corners) of the
    given width at ``c_frac``, so that max(c) / min(c) = c_max / c_frac.
    Lengths are in the units of ``h``."""
    x, y, _ = _cell_centres(nx, ny, 1, h)
    x, y = x[0], y[0]
    Lx, Ly = nx * h, ny * h
    nreg = int(rng.integers(3, 5))
    vals = np.concatenate([[c_max], rng.uniform(0.55, 1.0, nreg - 1) * c_max])
    rng.shuffle(vals)
    region = np.zeros(x.shape, int)
    for y0 in np.sort(rng.uniform(0.15, 0.85, nreg - 1)) * Ly:
        slope = rng.uniform(-0.4, 0.4)
        region += (y > y0 + slope * (x - 0.5 * Lx)).astype(int)
    c2 = vals[region]
    # fracture: corners at x = Lx/3 and 2Lx/3, ends on the x-faces
    px = np.array([0.0, Lx / 3, 2 * Lx / 3, Lx])
    py = rng.uniform(0.25, 0.75, 4) * Ly
    dist = np.full(x.shape, np.inf)
    for i in range(3):
        a = np.array([px[i], py[i]])
        d = np.array([px[i + 1] - px[i], py[i + 1] - py[i]])
        t = np.clip(((x - a[0]) * d[0] + (y - a[1]) * d[1]) / (d @ d), 0.0, 1.0)
        dist = np.minimum(dist, np.hypot(x - a[0] - t * d[0], y - a[1] - t * d[1]))
    c2 = np.where(dist < 0.5 * width, c_frac, c2)
    return np.broadcast_to(c2, (nz, ny, nx)).copy()


def smooth_random_field(shape, rng, corr=4.0):
    """Zero-mean, unit-std Gaussian random field with Gaussian correlation
    length ``corr`` cells (FFT filtering of white noise)."""
    w = rng.standard_normal(shape)
    k = [np.fft.fftfreq(n) for n in shape]
    kk = np.meshgrid(*k, indexing="ij")
    filt = np.exp(-2.0 * (np.pi * corr) ** 2 * sum(q * q for q in kk))
    f = np.real(np.fft.ifftn(np.fft.fftn(w) * filt))
    return (f - f.mean()) / (f.std() + 1e-30)


def lognormal_block(n, h, rng, median=2500.0, sig=0.15, cmin=1500.0, cmax=4500.0):
    """One ``n^3`` velocity block: log-normal background plus 1-3 planar or
    spherical-cap interfaces of contrast 1.5-3x (the learned-surrogate data)."""
    c = median * np.exp(sig * smooth_random_field((n, n, n), rng))
    x, y, z = _cell_centres(n, n, n, h)
    L = n * h
    for _ in range(int(rng.integers(1, 4))):
        contrast = rng.uniform(1.5, 3.0)
        if rng.uniform() < 0.5:
            nrm = rng.normal(size=3)
            nrm /= np.linalg.norm(nrm)
            off = rng.uniform(0.3, 0.7) * L
            side = (x - L / 2) * nrm[0] + (y - L / 2) * nrm[1] + (z - L / 2) * nrm[2] + L / 2 > off
        else:
            ctr = rng.uniform(-0.5, 1.5, 3) * L
            rad = rng.uniform(0.5, 1.2) * L
            side = (x - ctr[0]) ** 2 + (y - ctr[1]) ** 2 + (z - ctr[2]) ** 2 < rad * rad
        if rng.uniform() < 0.5:
            c[side] *= contrast
        else:
            c[side] /= contrast
    return np.clip(c, cmin, cmax)


# ----------------------------------------------------------------------------
# cuts
# ----------------------------------------------------------------------------

def uniform_cuts(n, step):
    return np.arange(0, n + 1, step, dtype=int)


def uneven_cuts(n, rng, choices=(16, 20, 24, 32)):
    """Per-axis cut lengths drawn from ``choices`` until the axis is filled;
    the tail (at most two pieces) is chosen within the set so the lengths add
    up to ``n`` exactly (redrawn when impossible)."""
    ch = np.array(choices)
    pair = {int(a): (int(a),) for a in ch}
    for a in ch:
        for b in ch:
            pair.setdefault(int(a + b), (int(a), int(b)))
    for _ in range(1000):
        lens = []
        rem = n
        while rem > 2 * ch.max():
            v = int(rng.choice(ch))
            lens.append(v)
            rem -= v
        if rem in pair:
            lens.extend(pair[rem])
            return np.concatenate([[0], np.cumsum(lens)]).astype(int)
    raise RuntimeError("could not tile the axis")


# ----------------------------------------------------------------------------
# the workloads
# ----------------------------------------------------------------------------

def default_sigma(f_peak, factor=2.5):
    """Krylov shift ``(2 pi factor f_peak)^2``: the source band's upper edge by
    default (factor 2.5).  Deep ROMs (k >= 16) use a larger factor so that
    their S-fraction coefficients stay representable."""
    return (2.0 * np.pi * factor * f_peak) ** 2


def config1():
    """48^3 cells (h=10 m), 2x2x2 subdomains of 24^3, two layers 1500/3000 m/s
    with the interface at z=24 cells, m=4, k=8, one 15 Hz Ricker at the grid
    centre, 8 receivers, 500 steps (run in FP64, parity in FP32 too)."""
    n, h = 48, 10.0
    c = two_layer(n, n, n, 24)
    cuts = uniform_cuts(n, 24)
    rec = np.array([[(4 + 6 * i) * h, 24 * h, 12 * h] for i in range(8)])
    return Problem("cfg1_48c_2x2x2_m4_k8", n, n, n, h, c, cuts, cuts.copy(), cuts.copy(),
                   np.full(8, 4), np.full(8, 8), default_sigma(15.0), 15.0,
                   np.array([[24 * h, 24 * h, 24 * h]]), rec, 500)


def config2(seed=SEED):
    """192^3 cells, 8^3 = 512 subdomains of 24^3, layered model with a lens and
    jumps inside subdomains, m=8, k=16, one 20 Hz shot, 1024 surface receivers
    along x at y=96h, 4000 steps (FP32 stepping)."""
    n, h = 192, 10.0
    rng = np.random.default_rng(seed)
    c = layered_lens(n, n, n, h, rng)
    cuts = uniform_cuts(n, 24)
    xs = np.linspace(0.0, n * h, 1024)
    rec = np.stack([xs, np.full(1024, 96 * h), np.zeros(1024)], axis=1)
    return Problem("cfg2_192c_8x8x8_m8_k16", n, n, n, h, c, cuts, cuts.copy(), cuts.copy(),
                   np.full(512, 8), np.full(512, 16), default_sigma(20.0, 8.0), 20.0,
                   np.array([[96 * h, 96 * h, 8 * h]]), rec, 4000)


def config3(seed=SEED):
    """256x256x128 cells tiled by uneven subdomains (sides from {16,20,24,32}),
    m in {4,8} and k in 8..24 per subdomain (at most 20 where a side is 16
    cells), 64 shots on an 8x8 surface grid,
    256 receivers on a 16x16 surface grid, 3000 steps (batched, reduced
    precision)."""
    nx, ny, nz, h = 256, 256, 128, 10.0
    rng = np.random.default_rng(seed)
    c = layered_lens(nx, ny, nz, h, rng, avoid=4)
    xc, yc, zc = uneven_cuts(nx, rng), uneven_cuts(ny, rng), uneven_cuts(nz, rng)
    nsub = (len(xc) - 1) * (len(yc) - 1) * (len(zc) - 1)
    m = rng.choice([4, 8], size=nsub)
    k = rng.integers(8, 25, size=nsub)
    # depth cap on the smallest subdomains: a 16-cell side with k > 20
    # levels takes the S-fraction coefficients past FP64's dynamic range
    # (their coupled lambda_max exceeds the Galerkin ROM's)
    ncx, ncy = len(xc) - 1, len(yc) - 1
    for s in range(nsub):
        ix, iy, iz = s % ncx, (s // ncx) % ncy, s // (ncx * ncy)
        side = min(xc[ix + 1] - xc[ix], yc[iy + 1] - yc[iy], zc[iz + 1] - zc[iz])
        if side <= 16:
            k[s] = min(k[s], 20)
    g = (np.arange(8) * 32 + 16) * h
    sx, sy = np.meshgrid(g, g, indexing="ij")
    src = np.stack([sx.ravel(), sy.ravel(), np.full(64, 2 * h)], axis=1)
    r = (np.arange(16) * 16 + 8) * h
    rx, ry = np.meshgrid(r, r, indexing="ij")
    rec = np.stack([rx.ravel(), ry.ravel(), np.zeros(256)], axis=1)
    return Problem("cfg3_256x256x128_uneven_64shots", nx, ny, nz, h, c, xc, yc, zc, m, k,
                   default_sigma(20.0, 8.0), 20.0, src, rec, 3000)


def config5(seed=SEED):
    """512x512x256 cells in 32^3 subdomains (2048), m=8, k=24, 128 shots on a
    16x8 surface grid, 512 receivers, salt-like bodies, 6000 steps."""
    nx, ny, nz, h = 512, 512, 256, 10.0
    rng = np.random.default_rng(seed)
    c = salt_bodies(nx, ny, nz, h, rng)
    xc, yc, zc = uniform_cuts(nx, 32), uniform_cuts(ny, 32), uniform_cuts(nz, 32)
    gx = (np.arange(16) * 32 + 16) * h
    gy = (np.arange(8) * 64 + 32) * h
    sx, sy = np.meshgrid(gx, gy, indexing="ij")
    src = np.stack([sx.ravel(), sy.ravel(), np.full(128, 2 * h)], axis=1)
    rx = np.linspace(0, nx * h, 32)
    ry = np.linspace(0, ny * h, 16)
    qx, qy = np.meshgrid(rx, ry, indexing="ij")
    rec = np.stack([qx.ravel(), qy.ravel(), np.zeros(512)], axis=1)
    return Problem("cfg5_512x512x256_32c_128shots", nx, ny, nz, h, c, xc, yc, zc,
                   np.full(2048, 8), np.full(2048, 24), default_sigma(20.0, 8.0), 20.0,
                   src, rec, 6000)


def paper_layout(seed=SEED, cells_per_unit=20, m=25, k=3):
    """Stand-in for the paper's experiment (section "Numerical experiments"),
    in its dimensionless units: the box [0,7] x [0,7] x [0,3] split into
    7 x 7 x 3 unit cubes of ``cells_per_unit``^3 cells, m = 25 face modes
    (the 25 lowest p^2 + q^2 cosine modes), k = n = 3 levels, c(x, y) from ``skew_fracture`` (its model is
    shown only in a figure), one source at (3.5, 1.5, 1.5) whose Ricker band
    edge (2.5 f_peak) gives a shortest wavelength of 0.78 at c = 1, traces
    u(x, 0, 1.5) at every node x of the line, t in [0, 12.5].  The outer
    faces are homogeneous Neumann (the paper's absorbing conditions are not
    built).  The Krylov shift is small, sigma = (2 pi 0.1 f_peak)^2: the
    paper's subspace uses sigma = 0, which a subdomain with Neumann faces
    does not allow.  ``nsteps`` is left for the caller: it follows from the
    time step of the run."""
    h = 1.0 / cells_per_unit
    nx, ny, nz = 7 * cells_per_unit, 7 * cells_per_unit, 3 * cells_per_unit
    rng = np.random.default_rng(seed)
    c = skew_fracture(nx, ny, nz, h, rng)
    cuts = [uniform_cuts(n, cells_per_unit) for n in (nx, ny, nz)]
    nsub = 7 * 7 * 3
    f_peak = 1.0 / (2.5 * 0.78)
    rec = np.stack([np.arange(nx + 1) * h, np.zeros(nx + 1), np.full(nx + 1, 1.5)], axis=1)
    return Problem(f"paper_7x7x3_unit_cubes_m{m}_k{k}", nx, ny, nz, h, c, cuts[0], cuts[1],
                   cuts[2], np.full(nsub, m), np.full(nsub, k), default_sigma(f_peak, 0.1), f_peak,
                   np.array([[3.5, 1.5, 1.5]]), rec, 0, meta={"t_end": 12.5})


def gaussian_pulse(problem: Problem, xyz, width):
    """Initial displacement ``exp(-r^2 / 2 width^2)`` around ``xyz`` on the
    grid nodes, ``[nz+1, ny+1, nx+1]`` (the initial-value form of a source:
    Algorithm 1 starts from initial conditions).  For the paper layout a
    width of ``3 * 0.78 / (2 pi)`` puts the spectrum's 1% point at the
    shortest wavelength 0.78."""
    h = problem.h
    k, j, i = np.meshgrid(np.arange(problem.nz + 1), np.arange(problem.ny + 1),
                          np.arange(problem.nx + 1), indexing="ij")
    x = np.asarray(xyz, dtype=np.float64)
    r2 = (i * h - x[0]) ** 2 + (j * h - x[1]) ** 2 + (k * h - x[2]) ** 2
    return np.exp(-r2 / (2.0 * width * width))


def small_problem(ncell=(8, 8, 8), cuts=(4, 4, 4), m=4, k=3, h=10.0, seed=SEED,
                  model="layers", f_peak=None, nsteps=200, src=None, rec=None,
                  m_sub=None, k_sub=None, sigma=None):
    """A small problem for oracle pins and parity tests.  ``cuts`` is either a
    per-axis uniform subdomain size or explicit cut arrays."""
    nx, ny, nz = ncell
    rng = np.random.default_rng(seed)
    axes = []
    for n, cstep in zip(ncell, cuts):
        axes.append(uniform_cuts(n, cstep) if np.isscalar(cstep) else np.asarray(cstep, int))
    if model == "uniform":
        c = np.full((nz, ny, nx), 2000.0)
    elif model == "two_layer":
        c = two_layer(nx, ny, nz, nz // 2)
    elif model == "random":
        c = rng.uniform(1500.0, 4500.0, (nz, ny, nx))
    else:
        c = layered_lens(nx, ny, nz, h, rng, avoid=int(axes[2][1]), nlay=3, lens_w=2.0)
    nsub = (len(axes[0]) - 1) * (len(axes[1]) - 1) * (len(axes[2]) - 1)
    if f_peak is None:
        # keep the shortest wavelength around 8 cells
        f_peak = float(c.min()) / (8.0 * h)
    if src is None:
        src = np.array([[nx * h * 0.37, ny * h * 0.41, nz * h * 0.45]])
    if rec is None:
        rec = np.array([[nx * h * f, ny * h * 0.55, nz * h * 0.5] for f in (0.15, 0.5, 0.85)])
    return Problem(f"small_{nx}x{ny}x{nz}", nx, ny, nz, h, c, axes[0], axes[1], axes[2],
                   np.full(nsub, m) if m_sub is None else np.asarray(m_sub),
                   np.full(nsub, k) if k_sub is None else np.asarray(k_sub),
                   default_sigma(f_peak) if sigma is None else sigma, f_peak,
                   np.asarray(src, float), np.asarray(rec, float), nsteps)


def surrogate_blocks(count, n=24, h=10.0, seed=SEED):
    """``count`` velocity blocks of ``n^3`` cells for the learned surrogate."""
    rng = np.random.default_rng(seed)
    return np.stack([lognormal_block(n, h, rng) for _ in range(count)])
