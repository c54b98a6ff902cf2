"""Seeded synthetic disk problems (input generation only).

This module builds the inputs of the line radiative-transfer march: node grids of the
axisymmetric (r, z/r) fields, the CO-layer surfaces, the viewing geometry, channel
velocities and the line constants, plus neural-field weights and serving request mixes.
It holds none of the march's arithmetic (no ray tracing, line profile, populations or
transfer): both the CUDA path and the FP64 oracle read the plain arrays produced here.

Disk family (arXiv 2509.03623, Methods, "Parametric Disk Modeling"; sizes and laws as
fixed by the workload definitions):
  * temperature  T(r,z) = T_mid(r) + (T_atm(r) - T_mid(r)) sin^2(pi z / 2 z_q) below z_q,
    T_atm above, with T_mid = T_mid0 (r/100 au)^-0.5, T_atm = T_atm0 (r/100 au)^-0.5 and
    z_q = z_q0 (r / r_scale)^1.3 (z_q0 = 70 au, r_scale = 150 au from Table 2); this is the
    paper's cos^{2 delta} blend with delta = 1;
  * density      Gaussian scale height: rho = Sigma / (sqrt(2 pi) H) exp(-z^2 / 2H^2),
    H = c_s / Omega, c_s^2 = k T_mid / m_mol, Omega^2 = G M / r^3,
    Sigma = Sigma0 (r/100 au)^-1 exp(-r/300 au), Sigma0 set by M_gas = 0.09 M_sun (Table 2)
    over 10-600 au; n_H2 = rho / m_mol;
  * CO layer     between surfaces z = c_lo r (r/100)^p and z = c_hi r (r/100)^p
    (c_lo = 0.1, c_hi = 0.35, p = 0.25), stored as z/r heights per radial node;
  * turbulence   v_turb = 0.05 km/s (absolute).
Random jitter, log-normal perturbations and rings/gaps follow the workload definitions.
"""

from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

# CGS constants used by the generator (CODATA 2018, IAU 2015 nominal).
K_BOLTZ = 1.380649e-16
H_PLANCK = 6.62607015e-27
C_LIGHT = 2.99792458e10
AMU_G = 1.66053906660e-24
GM_SUN = 1.3271244e26
M_SUN_G = 1.98840987e33  # GM_SUN / G with G = 6.67430e-8
AU_CM = 1.495978707e13
M_H_AMU = 1.007825
DEBYE = 1e-18

CO21_NU0 = 230.538e9
CO_MASS_AMU = 28.0101
MEAN_MOL_AMU = 2.37 * M_H_AMU


def dipole_A(nu0_hz: float, mu_debye: float, J_u: int) -> float:
    """Einstein A of a rigid-rotor J_u -> J_u-1 transition from its dipole moment
    (A = 64 pi^4 nu^3 mu^2 / (3 h c^3) * J_u / (2 J_u + 1)); stands in for the missing
    molecular table."""
    mu = mu_debye * DEBYE
    return (64.0 * math.pi ** 4 * nu0_hz ** 3 * mu ** 2 / (3.0 * H_PLANCK * C_LIGHT ** 3)
            * J_u / (2.0 * J_u + 1.0))


@dataclasses.dataclass
class Problem:
    """One render problem: plain arrays and scalars in the units of the C interface."""
    # grid
    nr: int
    nz: int
    r_in_au: float
    r_out_au: float
    zr_max: float
    r_log: int
    # node fields [nz][nr] float64 and surfaces [nr]
    T: np.ndarray
    n_h2: np.ndarray
    vturb: np.ndarray
    h_lo: np.ndarray
    h_hi: np.ndarray
    x_co: float = 1e-4
    edge_w: float = 0.01
    vturb_mach: int = 0
    # geometry
    incl_deg: float = 45.0
    pa_deg: float = 0.0
    dist_pc: float = 100.0
    mstar_msun: float = 2.0
    vsys_kms: float = 0.0
    # view
    nx: int = 64
    ny: int = 64
    half_fov_au: float = 0.0
    v_kms: np.ndarray = dataclasses.field(default_factory=lambda: np.linspace(-4, 4, 16))
    n_samples: int = 128
    I0: float = 0.0
    units: int = 0
    # line
    nu0_hz: float = CO21_NU0
    A_ul: float = dataclasses.field(default_factory=lambda: dipole_A(CO21_NU0, 0.112, 2))
    B_rot_hz: float = 0.0
    m_co_amu: float = CO_MASS_AMU
    m_mol_amu: float = MEAN_MOL_AMU
    J_u: int = 2
    # optional rotation field [nz][nr] km/s (pressure-corrected); None: Keplerian
    vphi: Optional[np.ndarray] = None
    # optional 3-D Cartesian grid (rt_render3d); when set the fields above are unused
    g3: Optional["Grid3"] = None
    # optional 3-D spherical grid (rt_render_sph); when set the fields above are unused
    gs: Optional["GridSph"] = None
    # provenance
    name: str = ""
    seed: int = 0
    # surface power-law parameters (c_lo, p_lo, c_hi, p_hi) and ring modulation per node
    surf: tuple = (0.1, 0.25, 0.35, 0.25)
    ring_mod: Optional[np.ndarray] = None

    @property
    def nch(self) -> int:
        return int(len(self.v_kms))

    @property
    def npix(self) -> int:
        return self.nx * self.ny

    @property
    def evals(self) -> int:
        """Nominal sample-channel evaluations of one render: N_pix N_ch N_s."""
        return self.nx * self.ny * self.nch * self.n_samples

    def r_nodes(self) -> np.ndarray:
        if self.r_log:
            return self.r_in_au * (self.r_out_au / self.r_in_au) ** (
                np.arange(self.nr) / (self.nr - 1))
        return np.linspace(self.r_in_au, self.r_out_au, self.nr)

    def zr_nodes(self) -> np.ndarray:
        return np.linspace(0.0, self.zr_max, self.nz)

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


@dataclasses.dataclass
class Chain:
    """Parameters of the physics-constrained field chain: surface density
    Sigma(r) = Sigma0 (r/r_c)^-gamma exp(-(r/r_c)^(2-gamma)), freeze-out temperature and the
    photodissociation column applied to 0.706 N_H2."""
    sigma0_gcm2: float
    r_c_au: float
    gamma: float
    T_freeze: float
    N_dissoc_cm2: float


def chain_params(p: "Problem", m_gas_msun: float = 0.09, r_c_au: float = 212.0,
                 gamma: float = 0.8, T_freeze: float = 19.0,
                 N_dissoc_cm2: float = 1.3e21) -> Chain:
    """Chain parameters for the grid of p: r_c = 10^2.326 au (the HD 163296 value in the
    paper's parameter table), gamma = 0.8, T_freeze = 19 K (the freeze-out threshold the paper
    quotes), N_dissoc = 1.3e21 cm^-2; Sigma0 holds M_gas between r_in and r_out, from the
    closed-form integral 2 pi Sigma0 r_c^2 / (2 - gamma) [exp(-x_in^(2-gamma)) -
    exp(-x_out^(2-gamma))], x = r / r_c."""
    k = 2.0 - gamma
    xi, xo = p.r_in_au / r_c_au, p.r_out_au / r_c_au
    mass_per_sigma0 = (2.0 * math.pi * (r_c_au * AU_CM) ** 2 / k
                       * (math.exp(-xi ** k) - math.exp(-xo ** k)))
    return Chain(m_gas_msun * M_SUN_G / mass_per_sigma0, r_c_au, gamma, T_freeze, N_dissoc_cm2)


def _sigma0_from_mass(m_gas_msun: float, r_in: float, r_out: float) -> float:
    """Sigma0 [g cm^-2] of Sigma = Sigma0 (r/100 au)^-1 exp(-r/300 au) holding M_gas
    between r_in and r_out (closed-form integral of 2 pi r Sigma dr)."""
    integral = (2.0 * math.pi * 100.0 * 300.0 * AU_CM ** 2
                * (math.exp(-r_in / 300.0) - math.exp(-r_out / 300.0)))
    return m_gas_msun * M_SUN_G / integral


def parametric_fields(r_au: np.ndarray, zr: np.ndarray, *, T_mid0: float, T_atm0: float,
                      sigma0: float, mstar: float, z_q0: float = 70.0,
                      r_scale: float = 150.0, vturb_kms: float = 0.05):
    """Node values [nz][nr] of T [K], n_H2 [cm^-3], v_turb [km/s]."""
    R, ZR = np.meshgrid(r_au, zr)  # [nz][nr]
    Z = ZR * R
    T_mid = T_mid0 * (R / 100.0) ** -0.5
    T_atm = T_atm0 * (R / 100.0) ** -0.5
    z_q = z_q0 * (R / r_scale) ** 1.3
    blend = np.where(Z < z_q, np.sin(math.pi * Z / (2.0 * z_q)) ** 2, 1.0)
    T = T_mid + (T_atm - T_mid) * blend
    m_mol = MEAN_MOL_AMU * AMU_G
    cs = np.sqrt(K_BOLTZ * T_mid / m_mol)
    omega = np.sqrt(GM_SUN * mstar / (R * AU_CM) ** 3)
    H = cs / omega  # cm
    sigma = sigma0 * (R / 100.0) ** -1 * np.exp(-R / 300.0)
    rho = sigma / (math.sqrt(2.0 * math.pi) * H) * np.exp(-(Z * AU_CM) ** 2 / (2.0 * H ** 2))
    n = rho / m_mol
    vt = np.full_like(T, vturb_kms)
    return T, n, vt


def surfaces(r_au: np.ndarray, c_lo: float, p_lo: float, c_hi: float, p_hi: float,
             ring_mod: Optional[np.ndarray] = None):
    """CO-layer heights in z/r: h_s(r) = c_s (r/100 au)^p_s (x ring modulation)."""
    h_lo = c_lo * (r_au / 100.0) ** p_lo
    h_hi = c_hi * (r_au / 100.0) ** p_hi
    if ring_mod is not None:
        h_lo = h_lo * ring_mod
        h_hi = h_hi * ring_mod
    return h_lo, h_hi


def disk(seed: int = 0, *, nr: int = 64, nz: int = 32, r_in: float = 10.0,
         r_out: float = 600.0, zr_max: float = 0.5, nx: int = 64, ny: int = 64,
         nch: int = 16, vmax: float = 4.0, n_samples: int = 128, incl: float = 45.0,
         pa: float = 0.0, dist: float = 100.0, mstar: float = 2.0, jitter: float = 0.1,
         lognormal: float = 0.0, rings: int = 0, edge_w: float = 0.01,
         name: str = "") -> Problem:
    """The parametric disk family with seeded jitter (PCG64). Each of T_mid0, T_atm0,
    Sigma0, M_star and the two surface coefficients is scaled by U(1-jitter, 1+jitter);
    `lognormal` multiplies T and n_H2 node values by exp(sigma N(0,1)); `rings` adds Gaussian
    rings/gaps a_k exp(-(r-r_k)^2/2w_k^2) (w_k ~ U(10,30) au, r_k ~ U(50,550) au,
    |a_k| ~ U(0.1,0.3) with alternating sign) to the CO-layer heights."""
    rng = np.random.Generator(np.random.PCG64(seed))
    j = rng.uniform(1.0 - jitter, 1.0 + jitter, size=6) if jitter > 0 else np.ones(6)
    T_mid0, T_atm0 = 20.0 * j[0], 60.0 * j[1]
    sigma0 = _sigma0_from_mass(0.09, r_in, r_out) * j[2]
    mstar_j = mstar * j[3]
    c_lo, c_hi = 0.1 * j[4], 0.35 * j[5]
    grid_r = r_in * (r_out / r_in) ** (np.arange(nr) / (nr - 1))
    grid_zr = np.linspace(0.0, zr_max, nz)
    T, n, vt = parametric_fields(grid_r, grid_zr, T_mid0=T_mid0, T_atm0=T_atm0,
                                 sigma0=sigma0, mstar=mstar_j)
    if lognormal > 0:
        T = T * np.exp(lognormal * rng.standard_normal(T.shape))
        n = n * np.exp(lognormal * rng.standard_normal(n.shape))
    ring_mod = None
    if rings > 0:
        ring_mod = np.ones(nr)
        for k in range(rings):
            w = rng.uniform(10.0, 30.0)
            rk = rng.uniform(50.0, 550.0)
            a = rng.uniform(0.1, 0.3) * (1.0 if k % 2 == 0 else -1.0)
            ring_mod = ring_mod + a * np.exp(-(grid_r - rk) ** 2 / (2.0 * w * w))
    h_lo, h_hi = surfaces(grid_r, c_lo, 0.25, c_hi, 0.25, ring_mod)
    return Problem(nr=nr, nz=nz, r_in_au=r_in, r_out_au=r_out, zr_max=zr_max, r_log=1,
                   T=T, n_h2=n, vturb=vt, h_lo=h_lo, h_hi=h_hi, edge_w=edge_w,
                   incl_deg=incl, pa_deg=pa, dist_pc=dist, mstar_msun=mstar_j,
                   nx=nx, ny=ny, v_kms=np.linspace(-vmax, vmax, nch), n_samples=n_samples,
                   name=name, seed=seed, surf=(c_lo, 0.25, c_hi, 0.25), ring_mod=ring_mod)


@dataclasses.dataclass
class Grid3:
    """3-D Cartesian node grid in the disk frame: nodes uniformly spaced over
    extent = (x0, x1, y0, y1, z0, z1) au; fields [nz][ny][nx] float64: T [K], n_h2 [cm^-3],
    vturb [km/s], x_co (CO abundance), vx, vy, vz [km/s]."""
    nx: int
    ny: int
    nz: int
    extent: tuple
    T: np.ndarray
    n_h2: np.ndarray
    vturb: np.ndarray
    x_co: np.ndarray
    vx: np.ndarray
    vy: np.ndarray
    vz: np.ndarray

    def nodes(self):
        x0, x1, y0, y1, z0, z1 = self.extent
        return (np.linspace(x0, x1, self.nx), np.linspace(y0, y1, self.ny),
                np.linspace(z0, z1, self.nz))


def box3d(seed: int = 0, *, n3=(64, 64, 32), half_xy: float = 600.0, half_z: float = 150.0,
          nx: int = 64, ny: int = 64, nch: int = 32, vmax: float = 6.0, n_samples: int = 256,
          incl: float = 45.0, pa: float = 0.0, mstar: float = 2.0, turb: float = 0.2,
          r_in: float = 10.0, name: str = "") -> Problem:
    """A 3-D box [-half_xy, half_xy]^2 x [-half_z, half_z] au standing in for a hydrodynamic
    simulation: the parametric disk's temperature and density (same family as `disk`, no
    axisymmetry imposed on the perturbations) evaluated at the nodes and multiplied by
    exp(turb f(x)) with f a seeded sum of 6 Fourier modes (wavelengths 100-400 au), a CO
    abundance layer 1e-4 exp(-((|z|/r - 0.2)/0.08)^2 / 2), Keplerian rotation
    sqrt(G M r^2 / (r^2+z^2)^{3/2}) (-y/r, x/r, 0) plus seeded velocity modes of 0.1 km/s
    amplitude in all three components, and v_turb = 0.05 km/s. No gas inside r_in."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gx, gy, gz = n3
    xs = np.linspace(-half_xy, half_xy, gx)
    ys = np.linspace(-half_xy, half_xy, gy)
    zs = np.linspace(-half_z, half_z, gz)
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")  # [nz][ny][nx]
    R = np.sqrt(X * X + Y * Y)
    Rs = np.maximum(R, r_in)
    sigma0 = _sigma0_from_mass(0.09, r_in, half_xy)
    T_mid0, T_atm0 = 20.0, 60.0
    T_mid = T_mid0 * (Rs / 100.0) ** -0.5
    T_atm = T_atm0 * (Rs / 100.0) ** -0.5
    z_q = 70.0 * (Rs / 150.0) ** 1.3
    blend = np.where(np.abs(Z) < z_q, np.sin(math.pi * np.abs(Z) / (2.0 * z_q)) ** 2, 1.0)
    T = T_mid + (T_atm - T_mid) * blend
    m_mol = MEAN_MOL_AMU * AMU_G
    cs = np.sqrt(K_BOLTZ * T_mid / m_mol)
    H = cs / np.sqrt(GM_SUN * mstar / (Rs * AU_CM) ** 3)
    sig = sigma0 * (Rs / 100.0) ** -1 * np.exp(-Rs / 300.0)
    n = sig / (math.sqrt(2.0 * math.pi) * H) * np.exp(-(Z * AU_CM) ** 2 / (2.0 * H ** 2)) / m_mol

    def modes(k):
        f = np.zeros_like(X)
        for _ in range(k):
            lam = rng.uniform(100.0, 400.0)
            d = rng.standard_normal(3)
            d /= np.linalg.norm(d)
            ph = rng.uniform(0.0, 2.0 * math.pi)
            f += np.cos(2.0 * math.pi * (d[0] * X + d[1] * Y + d[2] * Z) / lam + ph)
        return f / math.sqrt(k)

    T = T * np.exp(turb * modes(6))
    n = n * np.exp(turb * modes(6))
    n[R < r_in] = 0.0
    x_co = 1e-4 * np.exp(-0.5 * ((np.abs(Z) / Rs - 0.2) / 0.08) ** 2)
    vphi = np.sqrt(GM_SUN * mstar * (Rs * AU_CM) ** 2 / ((Rs * AU_CM) ** 2 + (Z * AU_CM) ** 2) ** 1.5) / 1e5
    vx = -vphi * Y / Rs + 0.1 * modes(3)
    vy = vphi * X / Rs + 0.1 * modes(3)
    vz = 0.1 * modes(3)
    g3 = Grid3(gx, gy, gz, (-half_xy, half_xy, -half_xy, half_xy, -half_z, half_z),
               T, n, np.full_like(T, 0.05), x_co, vx, vy, vz)
    z2 = np.zeros((2, 2))
    return Problem(nr=2, nz=2, r_in_au=1.0, r_out_au=2.0, zr_max=1.0, r_log=1,
                   T=z2 + 1.0, n_h2=z2, vturb=z2, h_lo=np.zeros(2), h_hi=np.zeros(2),
                   incl_deg=incl, pa_deg=pa, mstar_msun=mstar, nx=nx, ny=ny,
                   half_fov_au=1.05 * half_xy, v_kms=np.linspace(-vmax, vmax, nch),
                   n_samples=n_samples, g3=g3,
                   name=name or f"box{gx}x{gy}x{gz}_px{nx}_ch{nch}_ns{n_samples}", seed=seed)


def config_box(seed: int = 0) -> Problem:
    """3-D workload: 128^3-node box (+-600 au in x, y; +-150 au in z), 256^2 px, 64 channels
    over +-6 km/s, 256 samples, i = 45 deg."""
    return box3d(seed, n3=(128, 128, 128), nx=256, ny=256, nch=64, n_samples=256)


@dataclasses.dataclass
class GridSph:
    """3-D spherical node grid centred on the star: nr radial nodes log-spaced (r_log=1) or
    linear (r_log=0) over [r_in, r_out] au, nth colatitudes (from +z) linear over [th0, th1]
    rad, nph azimuths at 2 pi k / nph; fields [nph][nth][nr] float64 (r fastest): T [K],
    n_h2 [cm^-3], vturb [km/s], x_co, and the velocity components vr, vth, vph [km/s]."""
    nr: int
    nth: int
    nph: int
    r_log: int
    r_in: float
    r_out: float
    th0: float
    th1: float
    T: np.ndarray
    n_h2: np.ndarray
    vturb: np.ndarray
    x_co: np.ndarray
    vr: np.ndarray
    vth: np.ndarray
    vph: np.ndarray

    def nodes(self):
        if self.r_log:
            r = self.r_in * (self.r_out / self.r_in) ** (np.arange(self.nr) / (self.nr - 1))
        else:
            r = np.linspace(self.r_in, self.r_out, self.nr)
        return (r, np.linspace(self.th0, self.th1, self.nth),
                2.0 * math.pi * np.arange(self.nph) / self.nph)


def sphere3d(seed: int = 0, *, nsph=(128, 48, 64), r_in: float = 20.0, r_out: float = 600.0,
             th_half: float = 0.55, nx: int = 64, ny: int = 64, nch: int = 32,
             vmax: float = 6.0, n_samples: int = 256, incl: float = 45.0, pa: float = 0.0,
             mstar: float = 2.0, turb: float = 0.2, spiral: float = 0.3, r_log: int = 1,
             th_range: Optional[tuple] = None, name: str = "") -> Problem:
    """A spherical grid (r log-spaced over [r_in, r_out] au, colatitudes within th_half rad of
    the midplane, full azimuth) standing in for a planet-disk hydrodynamic simulation: the
    parametric disk's temperature and density (the family of `disk` and `box3d`) at the nodes,
    multiplied by exp(turb f(x)) with f a seeded sum of 6 Fourier modes (as in `box3d`) and
    the density by 1 + spiral a, with a = cos(2 (phi - phi_p) + ln(R / 150 au) / tan 15 deg)
    a two-armed logarithmic spiral of seeded phase; the CO layer of `box3d`; Keplerian
    v_phi (1 + 0.02 a) plus seeded modes of 0.1 km/s in all three components and 0.1 a km/s
    in v_r; v_turb = 0.05 km/s. r_log = 0 spaces the radii linearly (r_in may then be 0);
    th_range = (th0, th1) replaces the midplane wedge."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gnr, gnth, gnph = nsph
    th0, th1 = th_range if th_range is not None else (0.5 * math.pi - th_half,
                                                      0.5 * math.pi + th_half)
    rr = (r_in * (r_out / r_in) ** (np.arange(gnr) / (gnr - 1)) if r_log
          else np.linspace(r_in, r_out, gnr))
    ths = np.linspace(th0, th1, gnth)
    phs = 2.0 * math.pi * np.arange(gnph) / gnph
    PH, TH, RR = np.meshgrid(phs, ths, rr, indexing="ij")  # [nph][nth][nr]
    Rc = RR * np.sin(TH)
    Z = RR * np.cos(TH)
    X = Rc * np.cos(PH)
    Y = Rc * np.sin(PH)
    Rs = np.maximum(Rc, 1.0)
    sigma0 = _sigma0_from_mass(0.09, r_in, r_out)
    T_mid = 20.0 * (Rs / 100.0) ** -0.5
    T_atm = 60.0 * (Rs / 100.0) ** -0.5
    z_q = 70.0 * (Rs / 150.0) ** 1.3
    blend = np.where(np.abs(Z) < z_q, np.sin(math.pi * np.abs(Z) / (2.0 * z_q)) ** 2, 1.0)
    T = T_mid + (T_atm - T_mid) * blend
    m_mol = MEAN_MOL_AMU * AMU_G
    cs = np.sqrt(K_BOLTZ * T_mid / m_mol)
    H = cs / np.sqrt(GM_SUN * mstar / (Rs * AU_CM) ** 3)
    sig = sigma0 * (Rs / 100.0) ** -1 * np.exp(-Rs / 300.0)
    n = sig / (math.sqrt(2.0 * math.pi) * H) * np.exp(-(Z * AU_CM) ** 2 / (2.0 * H ** 2)) / m_mol

    def modes(k):
        f = np.zeros_like(X)
        for _ in range(k):
            lam = rng.uniform(100.0, 400.0)
            d = rng.standard_normal(3)
            d /= np.linalg.norm(d)
            ph = rng.uniform(0.0, 2.0 * math.pi)
            f += np.cos(2.0 * math.pi * (d[0] * X + d[1] * Y + d[2] * Z) / lam + ph)
        return f / math.sqrt(k)

    phi_p = rng.uniform(0.0, 2.0 * math.pi)
    arm = np.cos(2.0 * (PH - phi_p) + np.log(Rs / 150.0) / math.tan(math.radians(15.0)))
    T = T * np.exp(turb * modes(6))
    n = n * np.exp(turb * modes(6)) * (1.0 + spiral * arm)
    x_co = 1e-4 * np.exp(-0.5 * ((np.abs(Z) / Rs - 0.2) / 0.08) ** 2)
    vk = np.sqrt(GM_SUN * mstar * (Rs * AU_CM) ** 2 / ((Rs * AU_CM) ** 2 + (Z * AU_CM) ** 2) ** 1.5) / 1e5
    vph = vk * (1.0 + 0.02 * arm) + 0.1 * modes(3)
    vr = 0.1 * arm + 0.1 * modes(3)
    vth = 0.1 * modes(3)
    gs = GridSph(gnr, gnth, gnph, 1 if r_log else 0, r_in, r_out, th0, th1, T, n,
                 np.full_like(T, 0.05), x_co, vr, vth, vph)
    z2 = np.zeros((2, 2))
    return Problem(nr=2, nz=2, r_in_au=1.0, r_out_au=2.0, zr_max=1.0, r_log=1,
                   T=z2 + 1.0, n_h2=z2, vturb=z2, h_lo=np.zeros(2), h_hi=np.zeros(2),
                   incl_deg=incl, pa_deg=pa, mstar_msun=mstar, nx=nx, ny=ny,
                   half_fov_au=1.05 * r_out, v_kms=np.linspace(-vmax, vmax, nch),
                   n_samples=n_samples, gs=gs,
                   name=name or f"sph{gnr}x{gnth}x{gnph}_px{nx}_ch{nch}_ns{n_samples}", seed=seed)


def config_sph(seed: int = 0) -> Problem:
    """Spherical-grid workload on the node count of the paper's runtime benchmark (512 x 96
    x 256 in r, theta, phi; r 20-600 au log-spaced, theta within 0.55 rad of the midplane),
    256^2 px, 64 channels over +-6 km/s, 512 samples, i = 47 deg, PA = 133 deg."""
    return sphere3d(seed, nsph=(512, 96, 256), nx=256, ny=256, nch=64, n_samples=512,
                    incl=47.0, pa=133.0)


# --------------------------------------------------------------------------------------
# The workloads (small parity case, observation scale, neural field, serving mix)
# --------------------------------------------------------------------------------------

def config_small(seed: int = 0) -> Problem:
    """64x32 grid, 64x64 px, 16 channels over +-4 km/s, 128 samples, i=45, PA=0, 100 pc."""
    return disk(seed, name="disk64x32_px64_ch16_ns128")


def config_observation(seed: int = 0) -> Problem:
    """512x256 grid, 256x256 px, 64 channels over +-6 km/s, 512 samples, i=47, PA=133,
    log-normal (sigma=0.1) T and n_H2, three rings/gaps in the CO-layer height."""
    return disk(seed, nr=512, nz=256, nx=256, ny=256, nch=64, vmax=6.0, n_samples=512,
                incl=47.0, pa=133.0, lognormal=0.1, rings=3,
                name="disk512x256_px256_ch64_ns512")


def config_neural(seed: int = 0) -> Problem:
    """Neural-field render shape: 512x512 px, 128 channels over +-6 km/s, 256 samples."""
    return disk(seed, nx=512, ny=512, nch=128, vmax=6.0, n_samples=256,
                name="mlp_px512_ch128_ns256")


def noisy_target(cube: np.ndarray, seed: int, frac: float = 0.05) -> np.ndarray:
    """Target cube = cube + N(0, (frac * peak)^2) noise (seeded)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return cube + frac * float(np.max(np.abs(cube))) * rng.standard_normal(cube.shape)


# --------------------------------------------------------------------------------------
# Neural field weights
# --------------------------------------------------------------------------------------

@dataclasses.dataclass
class MLPWeights:
    """Fourier-feature MLP: features [sin(2 pi B x), cos(2 pi B x)] of x = (rhat, zhat),
    Linear layers with SiLU on hidden layers. W[l] is [out][in] float32 (master copy)."""
    B: np.ndarray            # [n_freq][2]
    W: List[np.ndarray]
    b: List[np.ndarray]
    h_scale: float = 0.02

    @property
    def dims(self) -> List[int]:
        return [self.W[0].shape[1]] + [w.shape[0] for w in self.W]


def mlp_weights(seed: int = 0, n_freq: int = 32, width: int = 128, hidden: int = 4,
                n_out: int = 4, sigma_b: float = 4.0, out_gain: float = 1.0) -> MLPWeights:
    """Xavier-uniform weights (bound sqrt(6/(fan_in+fan_out))), zero biases, Gaussian
    Fourier directions B ~ N(0, sigma_b^2); all float32 from a PCG64 seed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    B = (sigma_b * rng.standard_normal((n_freq, 2))).astype(np.float32)
    dims = [2 * n_freq] + [width] * hidden + [n_out]
    W, b = [], []
    for l in range(len(dims) - 1):
        fi, fo = dims[l], dims[l + 1]
        bound = math.sqrt(6.0 / (fi + fo))
        w = rng.uniform(-bound, bound, size=(fo, fi))
        if l == len(dims) - 2:
            w = w * out_gain
        W.append(w.astype(np.float32))
        b.append(np.zeros(fo, dtype=np.float32))
    return MLPWeights(B=B, W=W, b=b)


# --------------------------------------------------------------------------------------
# Serving request mix
# --------------------------------------------------------------------------------------

@dataclasses.dataclass
class Request:
    t_arrival_s: float
    problem: Problem
    adjoint: bool


def request_mix(n: int = 256, seed: int = 0, rate_hz: float = 200.0,
                pixels=(128, 256, 512), channels=(32, 64, 128), samples=(128, 256, 1024),
                adjoint_frac: float = 0.3) -> List[Request]:
    """Poisson arrivals (exponential gaps, mean 1/rate) of seeded small-family disks with
    uniformly drawn image size, channel count and samples per ray; a fraction are
    gradient requests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate_hz)
        px = int(rng.choice(pixels))
        ch = int(rng.choice(channels))
        ns = int(rng.choice(samples))
        adj = bool(rng.uniform() < adjoint_frac)
        prob = disk(seed * 100003 + i, nx=px, ny=px, nch=ch, n_samples=ns,
                    name=f"req{i}_px{px}_ch{ch}_ns{ns}")
        out.append(Request(t, prob, adj))
    return out
