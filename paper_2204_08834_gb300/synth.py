"""Seeded synthetic inputs for the projection step (shared by tests, smoke and bench).

This module holds no arithmetic of the projection method itself: it only draws the
fields that the method consumes (velocity predictor, density, two pressure levels)
and the z grid, with the shapes and structure of the paper's workloads:

  * sphere      - one sphere of density 10 in density 1, 32^3 periodic (a small case);
  * emulsion    - a dispersed-droplet field in a triply periodic box, the shape of the
                  emulsion-in-HIT run (Sec. 7.1: 512^3, dispersed droplets);
  * two_layer   - a heavy layer under a light one between walls with a perturbed flat
                  interface and tanh-stretched z, the shape of the two-layer
                  Rayleigh-Benard run (Sec. 7.2: 1024x1024x512, aspect ratio 2, walls in z).
  * solenoidal_velocity - a single-phase velocity u^n for the momentum predictor: the MAC
                  curl of a Gaussian-filtered random vector potential (discretely
                  divergence-free), rescaled to a given rms; taylor_green - the 2-D vortex.
  * droplet_density + velocity_series - windows of a time series for the learned p_hat:
                  a fixed droplet field (density ratio 20) and a velocity predictor that
                  evolves as an AR(1) sequence u^{m+1} = a u^m + sqrt(1 - a^2) xi with smooth
                  (Gaussian-filtered) noise xi; the pressures of the series are computed by
                  the library's exact variable-coefficient solve, not here.

Density follows the one-fluid rule rho = rho_1 phi + rho_2 (1 - phi) (Eq. material_prop)
with a tanh volume-fraction profile of width 1.5 cells:
phi = (1 - tanh(s / eps)) / 2, s the signed distance to the interface (positive outside
the dense phase), eps = 0.75 * cell width, evaluated at cell centres.

Every array is float64, C-contiguous, shape (nz, ny, nx); every random stream is a
numpy PCG64 generator keyed by a fixed seed per field.
"""

import numpy as np

__all__ = ["Case", "stretched_dzf", "sphere", "emulsion", "two_layer", "ensemble_member", "random_fields",
           "droplet_density", "smooth_noise", "velocity_series", "solenoidal_velocity", "taylor_green"]


class Case(dict):
    """A dict of inputs with attribute access: u, v, w, rho, pn, pnm1, dt, dx, dy, dzf, lz, bc."""

    __getattr__ = dict.__getitem__

    @property
    def shape(self):
        return self["rho"].shape

    @property
    def npts(self):
        return int(np.prod(self["rho"].shape))


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def stretched_dzf(nz, lz, beta):
    """Cell widths of the wall-clustered grid z_f(k) = lz (1 + tanh(beta (2k/nz - 1)) / tanh beta) / 2."""
    k = np.arange(nz + 1, dtype=np.float64)
    zf = lz * 0.5 * (1.0 + np.tanh(beta * (2.0 * k / nz - 1.0)) / np.tanh(beta))
    zf[0], zf[-1] = 0.0, lz
    return np.diff(zf)


def _phi(s, eps):
    return 0.5 * (1.0 - np.tanh(s / eps))


def _droplet_phi(n, h, centres, radii, cutoff_cells=6.0):
    """phi = max over droplets, each evaluated on a periodic box of radius r + cutoff cells."""
    phi = np.zeros((n, n, n))
    eps = 0.75 * h
    for (cx, cy, cz), r in zip(centres, radii):
        ext = min(int(np.ceil(r / h + cutoff_cells)), (n - 2) // 2)
        idx = []
        for c in (cz, cy, cx):
            i0 = int(np.floor(c / h - 0.5))
            idx.append(np.arange(i0 - ext, i0 + ext + 2))
        kz, jy, ix = idx
        zc = (kz + 0.5) * h - cz
        yc = (jy + 0.5) * h - cy
        xc = (ix + 0.5) * h - cx
        dist = np.sqrt(zc[:, None, None] ** 2 + yc[None, :, None] ** 2 + xc[None, None, :] ** 2)
        s = dist - r
        local = np.where(s <= cutoff_cells * h, _phi(s, eps), 0.0)
        sub = np.ix_(kz % n, jy % n, ix % n)
        phi[sub] = np.maximum(phi[sub], local)
    return phi


def _place_droplets(rng, count, rmin, rmax, gap, max_tries=1_000_000):
    """Random non-overlapping droplets in the unit periodic box (minimum-image gap test)."""
    centres, radii = [], []
    tries = 0
    while len(centres) < count:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("droplet placement did not converge")
        c = rng.random(3)
        r = rng.uniform(rmin, rmax)
        ok = True
        for c2, r2 in zip(centres, radii):
            d = np.abs(c - c2)
            d = np.minimum(d, 1.0 - d)
            if np.sqrt(np.sum(d * d)) < r + r2 + gap:
                ok = False
                break
        if ok:
            centres.append(c)
            radii.append(r)
    return np.array(centres), np.array(radii)


def sphere(n=32, rho_in=10.0, rho_out=1.0, radius=0.25, dt=1e-3):
    """One sphere in a triply periodic unit box; u** ~ U[-1, 1]; p^n, p^{n-1} ~ U[-1, 1]."""
    h = 1.0 / n
    centre = _rng(1).random(3)  # (x, y, z)
    x = (np.arange(n) + 0.5) * h
    d2 = 0.0
    for axis, c in zip((2, 1, 0), centre):
        dd = np.abs(x - c)
        dd = np.minimum(dd, 1.0 - dd)
        shape = [1, 1, 1]
        shape[axis] = n
        d2 = d2 + (dd ** 2).reshape(shape)
    phi = _phi(np.sqrt(d2) - radius, 0.75 * h)
    rho = rho_in * phi + rho_out * (1.0 - phi)
    r2 = _rng(2)
    u, v, w = (r2.uniform(-1.0, 1.0, (n, n, n)) for _ in range(3))
    pn = _rng(3).uniform(-1.0, 1.0, (n, n, n))
    pnm1 = _rng(4).uniform(-1.0, 1.0, (n, n, n))
    return Case(u=u, v=v, w=w, rho=np.ascontiguousarray(rho), pn=pn, pnm1=pnm1, dt=dt,
                dx=h, dy=h, dzf=np.full(n, h), lz=1.0, bc="periodic", name=f"sphere{n}")


def emulsion(n=512, ratio=10.0, ndrops=200, rmin_cells=4.0, rmax_cells=12.0, dt=1e-3,
             seed=10):
    """Dispersed droplets (density `ratio`) in a carrier of density 1, triply periodic unit box.

    Droplet radii U[rmin, rmax] cells, centres U[0,1)^3, rejected until every pair has a
    minimum-image surface gap of at least 2 cells.  u** ~ N(0, 1);
    p^n, p^{n-1} ~ N(0, 1) * 0.1 * rho0 h / dt.
    """
    h = 1.0 / n
    centres, radii = _place_droplets(_rng(seed), ndrops, rmin_cells * h, rmax_cells * h, 2.0 * h)
    phi = _droplet_phi(n, h, centres, radii)
    rho = ratio * phi + 1.0 * (1.0 - phi)
    del phi
    r = _rng(seed + 1)
    u = r.standard_normal((n, n, n))
    v = r.standard_normal((n, n, n))
    w = r.standard_normal((n, n, n))
    scale = 0.1 * min(1.0, ratio) * h / dt
    pn = _rng(seed + 2).standard_normal((n, n, n))
    pn *= scale
    pnm1 = _rng(seed + 3).standard_normal((n, n, n))
    pnm1 *= scale
    return Case(u=u, v=v, w=w, rho=rho, pn=pn, pnm1=pnm1, dt=dt, dx=h, dy=h,
                dzf=np.full(n, h), lz=1.0, bc="periodic", name=f"emulsion{n}_r{ratio:g}")


def two_layer(nx=512, ny=512, nz=256, lx=2.0, ly=2.0, lz=1.0, beta=1.5, rho_low=1.5,
              rho_high=1.0, amp=0.02, dt=1e-3, seed=20, stretched=True):
    """Heavy layer (rho_low) under a light one between z walls; interface at z = lz/2 + eta(x, y).

    eta is a sum of three seeded sinusoidal modes scaled so that max |eta| = amp.
    z is tanh-stretched with parameter beta (uniform if stretched=False).
    u** ~ N(0, 1) with w = 0 on the top wall face; p^n, p^{n-1} as in `emulsion`.
    """
    dx, dy = lx / nx, ly / ny
    dzf = stretched_dzf(nz, lz, beta) if stretched else np.full(nz, lz / nz)
    zc = np.concatenate(([0.0], np.cumsum(dzf)[:-1])) + 0.5 * dzf
    r = _rng(seed)
    a = r.integers(1, 5, 3)
    b = r.integers(1, 5, 3)
    ph = r.uniform(0.0, 2.0 * np.pi, 3)
    am = r.uniform(0.5, 1.0, 3)
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dy
    eta = np.zeros((ny, nx))
    for m in range(3):
        eta += am[m] * np.sin(2.0 * np.pi * (a[m] * x[None, :] / lx + b[m] * y[:, None] / ly) + ph[m])
    eta *= amp / np.max(np.abs(eta))
    rho = np.empty((nz, ny, nx))
    for k in range(nz):
        phi = _phi(zc[k] - (0.5 * lz + eta), 0.75 * dzf[k])
        rho[k] = rho_low * phi + rho_high * (1.0 - phi)
    rr = _rng(seed + 1)
    u = rr.standard_normal((nz, ny, nx))
    v = rr.standard_normal((nz, ny, nx))
    w = rr.standard_normal((nz, ny, nx))
    w[-1] = 0.0
    scale = 0.1 * min(rho_low, rho_high) * dx / dt
    pn = _rng(seed + 2).standard_normal((nz, ny, nx))
    pn *= scale
    pnm1 = _rng(seed + 3).standard_normal((nz, ny, nx))
    pnm1 *= scale
    return Case(u=u, v=v, w=w, rho=rho, pn=pn, pnm1=pnm1, dt=dt, dx=dx, dy=dy, dzf=dzf,
                lz=lz, bc="walls", name=f"two_layer{nx}x{ny}x{nz}")


def ensemble_member(m, sizes=(32, 48, 64, 96, 128)):
    """Member m of the mixed-size ensemble: size sizes[m % 5]; periodic z for even m, uniform
    z walls for odd m; 8 droplets of density ratio U[1, 20]; seed 50 + m."""
    n = sizes[m % len(sizes)]
    r = _rng(50 + m)
    ratio = float(r.uniform(1.0, 20.0))
    rmin, rmax = max(2.0, n / 32.0), max(3.0, 3.0 * n / 32.0)
    c = emulsion(n, ratio=ratio, ndrops=8, rmin_cells=rmin, rmax_cells=rmax, seed=1000 + 10 * m)
    if m % 2 == 1:
        c["bc"] = "walls"
        c["w"][-1] = 0.0
    c["name"] = f"member{m}_n{n}_{c['bc']}"
    return c


def random_fields(nx, ny, nz, bc="periodic", stretched=False, lx=1.0, ly=1.3, lz=0.7, ratio=10.0,
                  seed=90, dt=1e-3):
    """Anisotropic grids for edge cases: a blob density (ratio `ratio`, tanh profile of a
    random ellipsoid), u** ~ U[-1, 1], p^n, p^{n-1} ~ U[-1, 1]; walls optional, z stretched
    with beta = 1.5 if asked."""
    r = _rng(seed)
    dx, dy = lx / nx, ly / ny
    dzf = stretched_dzf(nz, lz, 1.5) if stretched else np.full(nz, lz / nz)
    zc = np.concatenate(([0.0], np.cumsum(dzf)[:-1])) + 0.5 * dzf
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dy
    c = r.random(3) * np.array([lx, ly, lz])
    ax = 0.2 + 0.1 * r.random(3)
    d = np.sqrt(((zc[:, None, None] - c[2]) / (ax[2] * lz)) ** 2 + ((y[None, :, None] - c[1]) / (ax[1] * ly)) ** 2
                + ((x[None, None, :] - c[0]) / (ax[0] * lx)) ** 2)
    h = min(dx, dy, float(dzf.min()))
    phi = _phi((d - 1.0) * min(ax[0] * lx, ax[1] * ly, ax[2] * lz), 0.75 * h)
    rho = ratio * phi + 1.0 * (1.0 - phi)
    u = r.uniform(-1.0, 1.0, (nz, ny, nx))
    v = r.uniform(-1.0, 1.0, (nz, ny, nx))
    w = r.uniform(-1.0, 1.0, (nz, ny, nx))
    if bc == "walls":
        w[-1] = 0.0
    pn = r.uniform(-1.0, 1.0, (nz, ny, nx))
    pnm1 = r.uniform(-1.0, 1.0, (nz, ny, nx))
    return Case(u=u, v=v, w=w, rho=np.ascontiguousarray(rho), pn=pn, pnm1=pnm1, dt=dt, dx=dx, dy=dy,
                dzf=dzf, lz=lz, bc=bc, name=f"random{nx}x{ny}x{nz}_{bc}{'_str' if stretched else ''}")


def droplet_density(n, ndrops, rmin_cells, rmax_cells, ratio, seed):
    """Density of `ndrops` droplets (density `ratio`) in a carrier of density 1, n^3 periodic."""
    h = 1.0 / n
    centres, radii = _place_droplets(_rng(seed), ndrops, rmin_cells * h, rmax_cells * h, 2.0 * h)
    phi = _droplet_phi(n, h, centres, radii)
    return np.ascontiguousarray(ratio * phi + (1.0 - phi))


_FILTERS = {}


def _gauss_filter(n, sigma_cells):
    key = (n, sigma_cells)
    if key not in _FILTERS:
        k = 2.0 * np.pi * np.fft.fftfreq(n)
        kr = 2.0 * np.pi * np.fft.rfftfreq(n)
        k2 = k[:, None, None] ** 2 + k[None, :, None] ** 2 + kr[None, None, :] ** 2
        _FILTERS[key] = np.exp(-0.5 * sigma_cells ** 2 * k2)
    return _FILTERS[key]


def smooth_noise(rng, n, sigma_cells):
    """Periodic N(0,1) white noise filtered by a Gaussian of standard deviation `sigma_cells`
    cells (applied as exp(-sigma^2 |k|^2 / 2) in Fourier space), rescaled to unit rms."""
    import scipy.fft as sfft
    x = rng.standard_normal((n, n, n))
    y = sfft.irfftn(sfft.rfftn(x, workers=-1) * _gauss_filter(n, sigma_cells), s=x.shape, axes=(0, 1, 2),
                    workers=-1)
    return np.ascontiguousarray(y / np.sqrt(np.mean(y * y)))


def velocity_series(n, steps, seed, a=0.95, sigma_cells=2.0):
    """Yields `steps` velocity predictors (u, v, w) of an AR(1) sequence started in its
    stationary state: u^0 = xi_0, u^{m+1} = a u^m + sqrt(1 - a^2) xi_{m+1}, per component."""
    rng = _rng(seed)
    b = np.sqrt(1.0 - a * a)
    cur = [smooth_noise(rng, n, sigma_cells) for _ in range(3)]
    for m in range(steps):
        if m:
            cur = [a * c + b * smooth_noise(rng, n, sigma_cells) for c in cur]
        yield tuple(cur)


def learned_window(kind, w, n=None):
    """Window w of the learned-p_hat workload: (rho, velocity-series seed, n, dt).

    kind "train": 64^3, 50 droplets of radius U[2, 6] cells (seeds (30, w) and (31, w));
    kind "infer": 128^3, 50 droplets of radius U[4, 12] cells (seeds (32, w) and (33, w)).
    Density ratio 20 in both."""
    if kind == "train":
        n = n or 64
        rho = droplet_density(n, 50, 2.0, 6.0, 20.0, [30, w])
        return rho, [31, w], n, 1e-3
    n = n or 128
    rho = droplet_density(n, 50, 4.0, 12.0, 20.0, [32, w])
    return rho, [33, w], n, 1e-3


def solenoidal_velocity(n, seed=50, sigma_cells=4.0, urms=1.0, nz=None, ny=None):
    """(u, v, w) on an n^3 (or nz x ny x n) periodic MAC grid: the discrete curl of a vector
    potential of Gaussian-filtered noise (smooth_noise), so the discrete divergence is zero up to
    rounding; scaled so that the rms over the three components is `urms`.  Cell width 1/n."""
    nz, ny = nz or n, ny or n
    rng = _rng(seed)
    if nz == ny == n:
        psi = [smooth_noise(rng, n, sigma_cells) for _ in range(3)]
    else:
        psi = [rng.standard_normal((nz, ny, n)) for _ in range(3)]

    def d(a, ax):
        return a - np.roll(a, 1, axis=ax)
    u = d(psi[2], 1) - d(psi[1], 0)
    v = d(psi[0], 0) - d(psi[2], 2)
    w = d(psi[1], 2) - d(psi[0], 1)
    del psi
    s = urms / np.sqrt((np.mean(u * u) + np.mean(v * v) + np.mean(w * w)) / 3.0)
    return tuple(np.ascontiguousarray(q * s) for q in (u, v, w))


def taylor_green(nx, ny, nz, amplitude=1.0):
    """2-D Taylor-Green vortex u = A sin x cos y, v = -A cos x sin y, w = 0 on the MAC grid of a
    2 pi-periodic box (uniform in z): each component at its own face positions."""
    L = 2.0 * np.pi
    dx, dy = L / nx, L / ny
    xc = (np.arange(nx) + 0.5) * dx
    yc = (np.arange(ny) + 0.5) * dy
    u = amplitude * np.sin(xc + 0.5 * dx)[None, None, :] * np.cos(yc)[None, :, None] * np.ones((nz, 1, 1))
    v = -amplitude * np.cos(xc)[None, None, :] * np.sin(yc + 0.5 * dy)[None, :, None] * np.ones((nz, 1, 1))
    return np.ascontiguousarray(u), np.ascontiguousarray(v), np.zeros((nz, ny, nx))
