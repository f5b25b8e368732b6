"""Seeded synthetic inputs for the photoionization source evaluation.

This module is shared by the FP64 oracle (``oracle/``), the tests and
``bench.py``.  It holds no part of the method's arithmetic: it only draws
random numbers and lays out the emission field ``q`` and the electric-field
magnitude ``|E|`` on a uniform cell-centred grid (paper Section 4, uniform
mesh over the box ``[0,x_d] x [0,y_d] x [0,z_d]``).

Conventions
-----------
* Cell ``n = i + nx*(j + ny*k)`` (x fastest) has centre
  ``origin + h*(i+1/2, j+1/2, k+1/2)`` in cm.
* Every field is produced in FP64 and rounded once to FP32, so the oracle and
  the GPU path read bit-identical inputs.
* Random numbers come from SplitMix64 (Steele, Lea and Flood 2014): the n-th
  draw of a stream seeded with ``seed`` is ``mix(seed + (n+1)*0x9E3779B97F4A7C15)``
  and the uniform deviate is ``(x >> 11) * 2**-53``; draws are taken in
  linear-index order.
* Emission peak ``I0 = 1e26 m^-3 s^-1 = 1e20 cm^-3 s^-1``.
* ``source_scale`` is the factor that turns ``q`` into the emission term of
  Eq. Ifun: ``xi * p_q/(p + p_q)`` with the config's combined ``xi = 0.06``
  (= the paper's ``xi * omega/alpha = 0.1*0.6``) and ``p_q = 30`` Torr.
* ``pO2 = p * 150/760`` (the paper's air ratio).
"""
from __future__ import annotations

import dataclasses
import numpy as np

I0 = 1.0e20          # cm^-3 s^-1
CHI_MIN = 0.035      # cm^-1 Torr^-1  (Eq. gfun)
CHI_MAX = 2.0        # cm^-1 Torr^-1  (Eq. gfun)
P_Q = 30.0           # Torr
XI_EFF = 0.06        # xi * omega/alpha

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Draws ``offset .. offset+n-1`` of the SplitMix64 stream ``seed`` (uint64)."""
    with np.errstate(over="ignore"):
        idx = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed) + idx * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """U[0,1) deviates in FP64 from the SplitMix64 stream."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


@dataclasses.dataclass
class Problem:
    """One synthetic snapshot on a uniform grid (all lengths in cm)."""
    name: str
    nx: int
    ny: int
    nz: int
    h: float
    origin: tuple
    p_torr: float
    pO2_torr: float
    q: np.ndarray                 # float32[nx*ny*nz], emission shape (x fastest)
    emag: np.ndarray | None       # float32[nx*ny*nz], |E| in kV/cm, or None
    source_scale: float           # I = source_scale * q
    i_frac: float = 0.0           # 0 selects every cell as a source
    e_frac: float = 0.0
    e_applied: float = 0.0
    targets_all: bool = True      # True: every cell is a target (emag unused)
    leaf_size: int = 64
    seed: int = 0
    chi_min: float = CHI_MIN
    chi_max: float = CHI_MAX

    @property
    def ncell(self) -> int:
        return self.nx * self.ny * self.nz

    def centres(self):
        """FP64 cell-centre coordinate arrays (X, Y, Z), each shaped (nz, ny, nx)."""
        return _grid(self.nx, self.ny, self.nz, self.h, self.origin)


def _grid(nx, ny, nz, h, origin=(0.0, 0.0, 0.0)):
    x = origin[0] + h * (np.arange(nx, dtype=np.float64) + 0.5)
    y = origin[1] + h * (np.arange(ny, dtype=np.float64) + 0.5)
    z = origin[2] + h * (np.arange(nz, dtype=np.float64) + 0.5)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")   # shaped (nz, ny, nx): x fastest
    return X, Y, Z


def pO2_of(p_torr: float) -> float:
    return p_torr * 150.0 / 760.0


def scale_of(p_torr: float) -> float:
    return XI_EFF * P_Q / (p_torr + P_Q)


def _xp_ops(xp):
    """(exp, sqrt, where, maximum-with-scalar) for numpy or torch arrays."""
    if xp is np:
        return np.exp, np.sqrt, np.where, np.maximum
    return xp.exp, xp.sqrt, xp.where, lambda a, b: xp.clamp(a, min=b)


def streamer_emission(X, Y, Z, head, sigma_head, chan_len, chan_radius,
                      chan_level=1e-2, cloud=None, xp=np):
    """Gaussian head plus a Gaussian-profile channel behind it (head points -z).

    ``head`` = (x, y, z) of the head centre; the channel occupies
    ``z in [z_head, z_head + chan_len]`` on the axis through the head with
    radial profile ``chan_level * exp(-rho^2/chan_radius^2)``.  ``cloud`` =
    (centre, radius, level) adds a spherical Gaussian.  Peak value 1 (times I0).
    ``xp``: numpy (default) or torch, for arrays of either.
    """
    exp, _, where, _ = _xp_ops(xp)
    hx, hy, hz = head
    r2 = (X - hx) ** 2 + (Y - hy) ** 2 + (Z - hz) ** 2
    q = exp(-r2 / sigma_head ** 2)
    rho2 = (X - hx) ** 2 + (Y - hy) ** 2
    inside = (Z >= hz) & (Z <= hz + chan_len)
    q = q + where(inside, chan_level * exp(-rho2 / chan_radius ** 2), 0.0 * rho2)
    if cloud is not None:
        (cx, cy, cz), crad, clev = cloud
        q = q + clev * exp(-((X - cx) ** 2 + (Y - cy) ** 2 + (Z - cz) ** 2) / crad ** 2)
    return q


def streamer_efield(X, Y, Z, head, sigma_head, chan_len, chan_radius,
                    e_background=30.0, e_head=150.0, e_chan=30.0, xp=np):
    """|E| (kV/cm) of a synthetic streamer: background + charged ball + charged segment.

    * background ``(0, 0, -e_background)``;
    * a uniformly charged ball of radius ``sigma_head`` at the head whose
      surface field is ``e_head`` (linear inside, inverse-square outside);
    * a uniformly charged segment on the channel axis from ``z_head`` to
      ``z_head + chan_len`` with Plummer softening ``chan_radius``, its line
      density set so that the radial field at ``rho = chan_radius`` at
      mid-channel is ``e_chan``.
    """
    _, sqrt, where, maximum = _xp_ops(xp)
    hx, hy, hz = head
    dx, dy, dz = X - hx, Y - hy, Z - hz
    r = sqrt(dx * dx + dy * dy + dz * dz)
    R = sigma_head
    rs = maximum(r, 1e-300)
    fball = where(r < R, e_head * r / R, e_head * (R / rs) ** 2) / rs
    ex = fball * dx
    ey = fball * dy
    ez = fball * dz - e_background
    a = chan_radius
    L = chan_len
    z1, z2 = hz, hz + L
    k_lam = e_chan * 2.0 * a * float(np.sqrt(2.0 * a * a + L * L / 4.0)) / L
    rho2 = dx * dx + dy * dy
    b2 = rho2 + a * a
    u1 = Z - z1
    u2 = Z - z2
    s1 = sqrt(b2 + u1 * u1)
    s2 = sqrt(b2 + u2 * u2)
    erho_over_rho = k_lam / b2 * (u1 / s1 - u2 / s2)
    ex = ex + erho_over_rho * dx
    ey = ey + erho_over_rho * dy
    ez = ez + k_lam * (1.0 / s2 - 1.0 / s1)
    return sqrt(ex * ex + ey * ey + ez * ez)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float64).astype(np.float32).ravel()


def plain_gaussian(n=24, seed=1000, noise=1e-3, p_torr=760.0, box=0.2, sigma=0.02):
    """Plain direct-quadrature case: n^3 cells in a ``box`` cm cube, Gaussian + noise.

    ``q = exp(-|r-r0|^2/sigma^2) + noise*U[0,1)`` in units of I0, r0 at the
    box centre (a cell corner for even n); every cell is a source and a target.
    """
    h = box / n
    X, Y, Z = _grid(n, n, n, h)
    c = box / 2
    q = np.exp(-((X - c) ** 2 + (Y - c) ** 2 + (Z - c) ** 2) / sigma ** 2)
    q = q + noise * uniform01(seed, n ** 3).reshape(q.shape)
    return Problem("plain_gaussian_%d" % n, n, n, n, h, (0.0, 0.0, 0.0), p_torr,
                   pO2_of(p_torr), _f32(q * I0), None, scale_of(p_torr), seed=seed)


def streamer(n=128, box=1.0, p_torr=760.0, chan_len=0.5, i_frac=0.0, e_frac=0.1,
             e_applied=0.0, targets_all=True, leaf_size=64, seed=1001,
             sigma_head=0.015, chan_radius=0.02, with_efield=True, head=None,
             cloud=None, name=None):
    """Streamer-shaped emission (Gaussian head + channel) in an n^3 grid over a ``box`` cube.

    Head at (box/2, box/2, box/2 - chan_len/2) unless ``head`` is given; the
    channel runs ``chan_len`` cm towards +z.  ``|E|`` from :func:`streamer_efield`.
    """
    h = box / n
    X, Y, Z = _grid(n, n, n, h)
    if head is None:
        head = (box / 2, box / 2, box / 2 - chan_len / 2)
    q = streamer_emission(X, Y, Z, head, sigma_head, chan_len, chan_radius, cloud=cloud)
    em = None
    if with_efield:
        em = _f32(streamer_efield(X, Y, Z, head, sigma_head, chan_len, chan_radius))
    return Problem(name or "streamer_%d" % n, n, n, n, h, (0.0, 0.0, 0.0), p_torr,
                   pO2_of(p_torr), _f32(q * I0), em, scale_of(p_torr), i_frac=i_frac,
                   e_frac=e_frac, e_applied=e_applied, targets_all=targets_all,
                   leaf_size=leaf_size, seed=seed)


def plain_24():
    """24^3 plain direct quadrature in a 2 mm cube at 760 Torr, all cells source and target."""
    return plain_gaussian(24, seed=1000)


def streamer_full(n=128):
    """FMM without adaptivity: 128^3 streamer in a 1 cm cube at 760 Torr, all cells."""
    return streamer(n=n, box=1.0, p_torr=760.0, chan_len=0.5, i_frac=0.0,
                    targets_all=True, seed=1001, with_efield=False,
                    name="streamer_%d_full" % n)


def streamer_adaptive(n=256, p_torr=760.0, e_frac=0.1, e_applied=0.0):
    """Adaptive FMM: 256^3 streamer in a 1 cm cube, sources I >= 1e-4 max I,
    targets |E| >= e_applied + e_frac*(max|E| - e_applied)."""
    return streamer(n=n, box=1.0, p_torr=p_torr, chan_len=0.5, i_frac=1e-4,
                    e_frac=e_frac, e_applied=e_applied, targets_all=False, seed=1002,
                    name="streamer_%d_adaptive_p%d" % (n, int(p_torr)))


def snapshot_batch(count=24, seed=1003, sizes=(64, 96, 128, 192, 256), pressures=(76.0, 380.0, 760.0)):
    """Independent streamer snapshots for batched evaluation, drawn from one SplitMix64 stream.

    Per snapshot: grid n^3 with n from ``sizes``, a 1 cm cube, channel length
    U[0.1, 0.8] cm, pressure from ``pressures``, source threshold i_frac
    log-uniform in [1e-5, 1e-3], target threshold e_frac U[0.05, 0.2], head
    position jittered by up to 0.5 mm in x and y.
    """
    u = uniform01(seed, 8 * count).reshape(count, 8)
    out = []
    for k in range(count):
        n = int(sizes[min(int(u[k, 0] * len(sizes)), len(sizes) - 1)])
        chan = 0.1 + 0.7 * float(u[k, 1])
        p = float(pressures[min(int(u[k, 2] * len(pressures)), len(pressures) - 1)])
        i_frac = float(10.0 ** (-5.0 + 2.0 * u[k, 3]))
        e_frac = 0.05 + 0.15 * float(u[k, 4])
        head = (0.5 + 0.1 * (u[k, 5] - 0.5), 0.5 + 0.1 * (u[k, 6] - 0.5), 0.5 - chan / 2.0)
        out.append(streamer(n=n, box=1.0, p_torr=p, chan_len=chan, i_frac=i_frac, e_frac=e_frac,
                            targets_all=False, seed=seed * 1000 + k, head=head,
                            name="snap%02d_n%d_p%d" % (k, n, int(p))))
    return out


def stress_batch(count=4, seed=1006, sizes=(128, 192, 256, 256), pressures=(76.0, 380.0, 760.0)):
    """Snapshots with wide channels (many sources): the channel radius steps log-uniformly from
    0.2 to 1.0 mm over the batch (snapshot k of n: 0.2 mm x 5^(k / (n - 1))), its length is
    U[0.6, 0.8] cm and the source threshold 1e-5, so that the last snapshot (256^3, 1 mm) selects
    about three million sources.  Grid edges from ``sizes`` in order, pressures and target
    thresholds drawn as in :func:`snapshot_batch`."""
    u = uniform01(seed, 8 * count).reshape(count, 8)
    out = []
    for k in range(count):
        n = int(sizes[min(k, len(sizes) - 1)])
        chan = 0.6 + 0.2 * float(u[k, 1])
        p = float(pressures[min(int(u[k, 2] * len(pressures)), len(pressures) - 1)])
        radius = float(0.02 * 5.0 ** (k / max(count - 1, 1)))
        e_frac = 0.05 + 0.15 * float(u[k, 4])
        head = (0.5 + 0.1 * (u[k, 5] - 0.5), 0.5 + 0.1 * (u[k, 6] - 0.5), 0.5 - chan / 2.0)
        out.append(streamer(n=n, box=1.0, p_torr=p, chan_len=chan, i_frac=1e-5, e_frac=e_frac,
                            targets_all=False, seed=seed * 1000 + k, head=head, chan_radius=radius,
                            name="stress%02d_n%d_p%d_r%.2fmm" % (k, n, int(p), 10 * radius)))
    return out


def streamer_cloud(n=256, box=1.5, p_torr=760.0, i_frac=1e-4, seed=1004):
    """Streamer head approaching a plasma cloud: n^3 grid in a 1.5 cm cube at 760 Torr.

    Head (sigma 0.15 mm) at (0.75, 0.75, 0.6) cm with its channel up to z = 1.1 cm; a
    spherical Gaussian cloud of radius 1 mm and level 1e-3 I0 centred 3 mm ahead of the
    head, at (0.75, 0.75, 0.3) cm.  Every cell is a target.
    """
    return streamer(n=n, box=box, p_torr=p_torr, chan_len=0.5, i_frac=i_frac, targets_all=True,
                    seed=seed, head=(0.75, 0.75, 0.6), cloud=((0.75, 0.75, 0.3), 0.1, 1e-3),
                    name="streamer_cloud_%d" % n)


def cloud_geometry(k, seed=1005):
    """Seeded random streamer-and-cloud geometry k (training set of the surrogate), 1.5 cm cube.

    Head at (0.75 +- 0.1, 0.75 +- 0.1, U[0.45, 0.75]) cm, sigma U[0.10, 0.25] mm, channel
    length U[2, 6] mm and radius U[0.15, 0.3] mm; cloud U[2, 4] mm ahead of the head (-z),
    radius U[0.5, 1.5] mm, level 10^U[-4, -2.5].
    """
    u = uniform01(seed * 7919 + k, 10)
    head = (0.75 + 0.2 * (u[0] - 0.5), 0.75 + 0.2 * (u[1] - 0.5), 0.45 + 0.3 * u[2])
    cz = head[2] - (0.2 + 0.2 * u[6])
    return dict(head=head, sigma_head=0.010 + 0.015 * u[3], chan_len=0.2 + 0.4 * u[4],
                chan_radius=0.015 + 0.015 * u[5],
                cloud=((head[0], head[1], cz), 0.05 + 0.1 * u[7], 10.0 ** (-4.0 + 1.5 * u[8])))


def fields_torch(n, box, geom, device="cuda", with_efield=True):
    """Emission shape q and |E| (float32 tensors on ``device``, x fastest) of a geometry dict
    from :func:`cloud_geometry`, computed in float64 by the same formulas as the numpy path."""
    import torch
    h = box / n
    ax = (torch.arange(n, dtype=torch.float64, device=device) + 0.5) * h
    Z, Y, X = torch.meshgrid(ax, ax, ax, indexing="ij")
    q = streamer_emission(X, Y, Z, geom["head"], geom["sigma_head"], geom["chan_len"], geom["chan_radius"],
                          cloud=geom.get("cloud"), xp=torch)
    em = None
    if with_efield:
        em = streamer_efield(X, Y, Z, geom["head"], geom["sigma_head"], geom["chan_len"], geom["chan_radius"],
                             xp=torch).float().reshape(-1).contiguous()
    return (q * I0).float().reshape(-1).contiguous(), em


def gaussian_box(nx, ny, nz, sigma_cells=8.0, h=1.25e-3, pO2_torr=150.0, center=None, name=None):
    """One spherical Gaussian emission exp(-|r - r0|^2 / sigma^2), sigma = sigma_cells * h, in an
    nx x ny x nz box of cell edge h (cm), r0 the box centre unless given; every cell a target.
    The pressure is given through the O2 partial pressure (Section 4.2 form)."""
    X, Y, Z = _grid(nx, ny, nz, h)
    sig = sigma_cells * h
    c = center if center is not None else (nx * h / 2, ny * h / 2, nz * h / 2)
    q = np.exp(-((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) / sig ** 2)
    p_torr = pO2_torr * 760.0 / 150.0
    return Problem(name or "gaussian_%dx%dx%d" % (nx, ny, nz), nx, ny, nz, h, (0.0, 0.0, 0.0), p_torr, pO2_torr,
                   _f32(q * I0), None, scale_of(p_torr), targets_all=True, leaf_size=64)


def random_mask(n_cells: int, frac: float, seed: int) -> np.ndarray:
    """uint8 mask with each cell set with probability ``frac`` (SplitMix64 stream)."""
    return (uniform01(seed, n_cells) < frac).astype(np.uint8)


def stratified_targets(p: Problem, T: np.ndarray, center, radius: float, n_uniform: int, seed: int = 5):
    """A seeded target sample for parity checks at full size: every target whose cell centre
    lies within ``radius`` (cm) of ``center`` (the ball of Eq. relativefun's local error around
    the streamer head), plus ``n_uniform`` distinct targets drawn uniformly from the rest.

    Returns (sample, in_ball, weight): the sample as ascending int32 cell indices, a bool array
    marking its ball members, and the weight of one uniform member when the sample stands for
    all of T (|T \\ ball| / n_uniform; ball members weigh 1).
    """
    T = np.asarray(T, np.int64)
    i = T % p.nx
    j = (T // p.nx) % p.ny
    k = T // (p.nx * p.ny)
    o = p.origin
    d2 = ((o[0] + p.h * (i + 0.5) - center[0]) ** 2 + (o[1] + p.h * (j + 0.5) - center[1]) ** 2
          + (o[2] + p.h * (k + 0.5) - center[2]) ** 2)
    ball = d2 <= radius * radius
    rest = T[~ball]
    m = min(int(n_uniform), rest.size)
    if 0 < m < rest.size:
        u = uniform01(seed, rest.size)
        pick = rest[np.sort(np.argpartition(u, m - 1)[:m])]
    else:
        pick = rest[:m]
    samp = np.concatenate([T[ball], pick])
    order = np.argsort(samp, kind="stable")
    in_ball = np.concatenate([np.ones(int(ball.sum()), bool), np.zeros(m, bool)])[order]
    w = rest.size / m if m > 0 else 0.0
    return samp[order].astype(np.int32), in_ball, w


def streamer_head(box=1.0, chan_len=0.5):
    """Head centre of :func:`streamer` with its default placement."""
    return (box / 2, box / 2, box / 2 - chan_len / 2)



def brick_structured(nx=64, ny=48, nz=48, seed=1007, h=1e-3, p_torr=760.0):
    """Fields built brick by brick (bricks of 16^3 cells, brick (i, j, k) = cells 16i .. 16i+15
    along x, and so on) so that a selection may decide whole bricks at once and every way of
    deciding one is exercised, with ties at the thresholds.  i_frac = e_frac = 0.5, no applied
    field: the source threshold is 0.5 (max q = 1) and the |E| threshold 0.5 (max |E| = 1).

      q: 0, except 1.0 at (3, 5, 20), 0.5 (a tie: a source) at (6, 21, 6), NaN at (20, 4, 4)
         and just below 0.5 (not a source) at (20, 20, 3);
      |E|: 0.8 + seeded noise in [0, 0.1) with 1.0 at (0, 0, 0), except
         brick (1, 0, 0): 0.2 everywhere (no target);
         brick (2, 0, 0): 0.2 except 0.5 (a tie: a target) at its first cell;
         brick (0, 1, 1): one cell just below 0.5 (the others targets);
         brick (1, 1, 1): one cell at exactly 0.5 (every cell a target);
         brick (0, 0, 2): one NaN (never a target);
         brick (2, 2, 0): NaN everywhere (no target).
    Bricks that reach past the grid are left as they fall."""
    n = nx * ny * nz
    q = np.zeros((nz, ny, nx), np.float32)
    e = (0.8 + 0.1 * uniform01(seed, n)).astype(np.float32).reshape(nz, ny, nx)
    below = np.nextafter(np.float32(0.5), np.float32(0.0))

    def put(a, x, y, z, v):
        if x < nx and y < ny and z < nz:
            a[z, y, x] = v

    def brick(a, i, j, k, v):
        a[16 * k:16 * k + 16, 16 * j:16 * j + 16, 16 * i:16 * i + 16] = v

    put(q, 3, 5, 20, 1.0)
    put(q, 6, 21, 6, 0.5)
    put(q, 20, 4, 4, np.nan)
    put(q, 20, 20, 3, below)
    put(e, 0, 0, 0, 1.0)
    brick(e, 1, 0, 0, 0.2)
    brick(e, 2, 0, 0, 0.2)
    put(e, 32, 0, 0, 0.5)
    put(e, 5, 17, 18, below)
    put(e, 19, 21, 30, 0.5)
    put(e, 7, 9, 35, np.nan)
    brick(e, 2, 2, 0, np.nan)
    return Problem("bricks_%dx%dx%d" % (nx, ny, nz), nx, ny, nz, h, (0.0, 0.0, 0.0), p_torr, pO2_of(p_torr),
                   q.reshape(-1), e.reshape(-1), scale_of(p_torr), i_frac=0.5, e_frac=0.5, e_applied=0.0,
                   targets_all=False, leaf_size=64, seed=seed)
