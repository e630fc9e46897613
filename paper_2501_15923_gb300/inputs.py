"""Seeded synthetic inputs shaped like the workloads of Icarus 3.0 (arXiv 2501.15923).

The paper drives its heliosphere from WSA boundary maps at 0.1 AU (Sect. 2.1 and 3), injects
cone CMEs (Sect. 3.2, Table 2) and samples the solution along spacecraft trajectories (Sect. 2).
None of those data sets exist here, so this module synthesises stand-ins from a seed:

* boundary maps of a tilted current sheet: slow wind near the sheet, fast wind away from it,
  radial field of opposite sign on the two sides, a Parker-spiral azimuthal field;
* a random walk of the sheet tilt from one map to the next (time-dependent driving, Sect. 3);
* cone CMEs with speed / half-width / direction / onset drawn from stated ranges;
* circular or Keplerian-like probe orbits between 0.7 and 1.5 AU, knots every hour.

This module is the ONE piece shared by the CUDA library's tests/bench and the CPU oracle. It holds
no arithmetic of the method itself (no flux, no update, no interpolation the solver performs): it
only produces plain SI arrays. Random numbers come from splitmix64 (Steele, Lea & Flood 2014),
implemented here from its published definition so that every draw is reproducible bit for bit.

Array conventions (all SI):
  maps  [n_maps][5][n_theta][n_phi]   fields (v_r m/s, n m^-3, p Pa, B_r T, B_phi T), phi fastest,
        sampled at the grid's angular cell centres
  t_maps [n_maps]                     seconds from the start of the run
  cmes  [n_cme][8]                    (t_on s, duration s, lat rad, lon_corot rad, half_width rad,
                                       speed m/s, n m^-3, T K)
  traj  [n_probes][n_knots][4]        (t s, r m, lat rad, lon_inertial rad, unwrapped)
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# --- physical constants (SI; CODATA 2018, IAU 2012/2015 nominal values) -----------------------
AU = 1.495978707e11          # m
M_P = 1.67262192369e-27      # kg
K_B = 1.380649e-23           # J/K
MU0 = 1.25663706212e-6       # N/A^2
GM_SUN = 1.32712440018e20    # m^3/s^2
DAY = 86400.0                # s
OMEGA_SUN = 2.0 * math.pi / (25.38 * DAY)   # sidereal rotation rate used by the workloads, rad/s

# boundary condition codes (same numbering as include/icarus.h)
BC_PERIODIC, BC_CONT, BC_REFLECT, BC_DRIVEN, BC_FIXED = 0, 1, 2, 3, 4
GEOM_SPHERICAL, GEOM_CARTESIAN = 0, 1
LIM_MINMOD, LIM_VANLEER, LIM_MC = 0, 1, 2
FLUX_TVDLF, FLUX_HLL, FLUX_HLLD = 0, 1, 2
DIVB_NONE, DIVB_LINDE, DIVB_GLM, DIVB_POWELL = 0, 1, 2, 3
IC_COROTATING, IC_INERTIAL_RADIAL = 0, 1     # initial v_phi: at rest co-rotating / radial inertial flow
CME_WINDOW, CME_SPHERE = 0, 1                # cone footprint over a fixed window / spherical cloud crossing


class SplitMix64:
    """splitmix64 counter-based generator (Steele, Lea, Flood 2014; constants from that paper)."""

    MASK = (1 << 64) - 1

    def __init__(self, seed: int):
        self.state = seed & self.MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & self.MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & self.MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & self.MASK
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        """Uniform double in [lo, hi) from the top 53 bits."""
        u = (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] (inclusive)."""
        return lo + int(self.uniform() * (hi - lo + 1))


@dataclass
class Grid:
    """Logical grid description, mirrored by the icarus_grid C struct."""
    n1: int
    n2: int
    n3: int
    geometry: int = GEOM_SPHERICAL
    stretch: int = 1                      # 1: geometric radial spacing (dr ~ r); 0: uniform
    x1min: float = 0.1                    # spherical: r in AU
    x1max: float = 2.0
    x2min: float = math.radians(30.0)     # spherical: colatitude in rad (latitude +-60 deg)
    x2max: float = math.radians(150.0)
    x3min: float = 0.0                    # spherical: longitude in the co-rotating frame, rad
    x3max: float = 2.0 * math.pi
    bc: tuple = (BC_DRIVEN, BC_CONT, BC_CONT, BC_CONT, BC_PERIODIC, BC_PERIODIC)
    band_refine: int = 1                  # > 1: radial cells this many times narrower in the band
    band_lo: float = 0.0                  # the refined radial band [band_lo, band_hi] (AU)
    band_hi: float = 0.0

    @property
    def ncell(self) -> int:
        return self.n1 * self.n2 * self.n3

    def theta_centres(self) -> np.ndarray:
        d = (self.x2max - self.x2min) / self.n2
        return self.x2min + (np.arange(self.n2) + 0.5) * d

    def phi_centres(self) -> np.ndarray:
        d = (self.x3max - self.x3min) / self.n3
        return self.x3min + (np.arange(self.n3) + 0.5) * d


@dataclass
class Options:
    """Numerical options, mirrored by the icarus_options C struct."""
    cfl: float = 0.8
    limiter: int = LIM_VANLEER
    flux: int = FLUX_TVDLF
    gravity: int = 1
    divb: int = DIVB_LINDE
    divb_coef: float = 0.8
    rho_floor: float = 1e-6               # code units (n in cm^-3)
    p_floor: float = 1e-9                 # code units (p / (m_p 1e6 m^-3 (100 km/s)^2))
    init_vphi: int = IC_COROTATING        # initial v_phi: IC_COROTATING (0) or IC_INERTIAL_RADIAL
    cme_model: int = CME_WINDOW           # CME_WINDOW (0) or CME_SPHERE (1)
    tracer: int = 0                       # 1: carry the CME tracer c (passive, rho c conserved)
    glm_alpha: float = 0.1                # GLM (divb = DIVB_GLM): psi damped by exp(-alpha c_h dt / dmin)
    strict_floors: int = 0                # 1: a floor activation makes the solver's status EFLOOR


@dataclass
class Workload:
    name: str
    grid: Grid
    opts: Options
    gamma: float
    omega: float                          # rad/s
    t_maps: np.ndarray
    maps: np.ndarray
    cmes: np.ndarray
    traj: np.ndarray
    t_end: float                          # s (simulated time of the full workload)
    n_steps: int = 0                      # fixed step count (0: run to t_end)
    meta: dict = field(default_factory=dict)


# --- boundary maps ---------------------------------------------------------------------------
def current_sheet_map(theta_c: np.ndarray, phi_c: np.ndarray, tilt: float, phase: float,
                      omega: float, r_in_au: float, n_scale: float = 1.0) -> np.ndarray:
    """One boundary map [5][n_theta][n_phi] of a tilted current sheet (SI).

    Sheet normal n = (sin a sin p0, -sin a cos p0, cos a) for tilt a and phase p0. The angular
    distance to the sheet is d = |asin(r_hat . n)|. v_r = 350 + 350 S((d - 5 deg)/15 deg) km/s with
    the clamped smoothstep S(x) = 3x^2 - 2x^3; n = 300 (350 km/s / v_r)^2 cm^-3; T = 1.5 MK and
    p = 2 n k_B T (protons + electrons); B_r = +-300 nT by the side of the sheet;
    B_phi = -B_r omega r_in sin(theta) / v_r (Parker spiral at the inner radius).
    With n_scale = 1 (the stated recipe) the Alfven Mach number of the inflow is 0.926 everywhere
    (n ~ v^-2 at fixed |B| keeps v / v_A constant); n_scale = 2 makes it 1.31.
    """
    th, ph = np.meshgrid(theta_c, phi_c, indexing="ij")
    rx, ry, rz = np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)
    nx, ny, nz = math.sin(tilt) * math.sin(phase), -math.sin(tilt) * math.cos(phase), math.cos(tilt)
    dot = rx * nx + ry * ny + rz * nz
    d = np.abs(np.arcsin(np.clip(dot, -1.0, 1.0)))
    x = np.clip((d - math.radians(5.0)) / math.radians(15.0), 0.0, 1.0)
    s = 3.0 * x * x - 2.0 * x * x * x
    vr = (350.0 + 350.0 * s) * 1e3
    n = n_scale * 300e6 * (350e3 / vr) ** 2
    p = 2.0 * n * K_B * 1.5e6
    br = np.where(dot >= 0.0, 300e-9, -300e-9)
    bphi = -br * omega * (r_in_au * AU) * np.sin(th) / vr
    return np.stack([vr, n, p, br, bphi]).astype(np.float64)


def tilt_walk(rng: SplitMix64, n_maps: int, tilt0: float, step_deg: float = 5.0) -> list:
    """Tilt sequence a_{k+1} = clamp(a_k + U(-step, step) deg, 0, 90 deg) (step 5 deg by default)."""
    tilts = [tilt0]
    for _ in range(n_maps - 1):
        a = tilts[-1] + math.radians(rng.uniform(-step_deg, step_deg))
        tilts.append(min(max(a, 0.0), math.radians(90.0)))
    return tilts


# --- trajectories ----------------------------------------------------------------------------
def circular_orbit(t_knots: np.ndarray, r_au: float, lat_deg: float, lon0_deg: float,
                   period_days: float) -> np.ndarray:
    """[n_knots][4] knots of a circular orbit at fixed latitude, inertial longitude advancing."""
    lon = math.radians(lon0_deg) + 2.0 * math.pi * t_knots / (period_days * DAY)
    out = np.empty((t_knots.size, 4))
    out[:, 0] = t_knots
    out[:, 1] = r_au * AU
    out[:, 2] = math.radians(lat_deg)
    out[:, 3] = lon
    return out


def kepler_orbit(t_knots: np.ndarray, a_au: float, ecc: float, inc: float, m0: float) -> np.ndarray:
    """[n_knots][4] knots of a Keplerian orbit (node at longitude 0, periapsis at the node)."""
    a = a_au * AU
    nmean = math.sqrt(GM_SUN / a ** 3)
    m = m0 + nmean * t_knots
    e_an = m.copy()
    for _ in range(30):                   # Newton on Kepler's equation E - e sin E = M
        e_an = e_an - (e_an - ecc * np.sin(e_an) - m) / (1.0 - ecc * np.cos(e_an))
    r = a * (1.0 - ecc * np.cos(e_an))
    nu = 2.0 * np.arctan2(math.sqrt(1.0 + ecc) * np.sin(e_an / 2), math.sqrt(1.0 - ecc) * np.cos(e_an / 2))
    lat = np.arcsin(math.sin(inc) * np.sin(nu))
    lon = np.unwrap(np.arctan2(math.cos(inc) * np.sin(nu), np.cos(nu)))
    out = np.empty((t_knots.size, 4))
    out[:, 0], out[:, 1], out[:, 2], out[:, 3] = t_knots, r, lat, lon
    return out


def lon_corot(traj_p: np.ndarray, t: float, omega: float) -> float:
    """Co-rotating longitude of one probe's trajectory at time t (linear in the knots)."""
    lon = np.interp(t, traj_p[:, 0], traj_p[:, 3])
    return float((lon - omega * t) % (2.0 * math.pi))


def cme_row(t_on, duration, lat, lon, half_width, speed, n, temp) -> list:
    return [t_on, duration, lat, lon, half_width, speed, n, temp]


# --- workloads -------------------------------------------------------------------------------
def static_sheet(seed: int = 0, n_steps: int = 200, grid: Grid | None = None) -> Workload:
    """60x16x32 stretched grid, static tilted-sheet map (tilt 15 deg, random phase), 200 steps,
    two circular 1 AU probes (latitudes 0 and 7.25 deg, inertial longitudes 0 and 60 deg)."""
    g = grid or Grid(60, 16, 32)
    rng = SplitMix64(seed)
    phase = 2.0 * math.pi * rng.uniform()
    m = current_sheet_map(g.theta_centres(), g.phi_centres(), math.radians(15.0), phase, OMEGA_SUN, g.x1min)
    t_knots = np.arange(0.0, 3.0 * DAY + 1.0, 3600.0)
    traj = np.stack([circular_orbit(t_knots, 1.0, 0.0, 0.0, 365.25),
                     circular_orbit(t_knots, 1.0, 7.25, 60.0, 365.25)])
    return Workload("static_sheet_60x16x32", g, Options(), 1.5, OMEGA_SUN, np.zeros(1), m[None].copy(),
                    np.zeros((0, 8)), traj, t_end=0.0, n_steps=n_steps, meta={"phase": phase})


def dynamic_cme(seed: int = 1, grid: Grid | None = None, days: float = 10.0, n_scale: float = 1.0) -> Workload:
    """512x64x128 stretched grid, 10 daily maps with a random-walk tilt, one cone CME
    (1200 km/s, half-width 30 deg, 1000 cm^-3, 0.8 MK, 8 h, onset U(1, 3) d, aimed at probe 1),
    four Keplerian-like probes between 0.7 and 1.5 AU, 10 simulated days."""
    g = grid or Grid(512, 64, 128)
    rng = SplitMix64(seed)
    phase = 2.0 * math.pi * rng.uniform()
    tilts = tilt_walk(rng, 10, math.radians(15.0))
    th, ph = g.theta_centres(), g.phi_centres()
    maps = np.stack([current_sheet_map(th, ph, a, phase, OMEGA_SUN, g.x1min, n_scale) for a in tilts])
    t_maps = np.arange(10) * DAY
    t_knots = np.arange(0.0, (days + 1.0) * DAY + 1.0, 3600.0)
    probes = []
    for _ in range(4):
        a = rng.uniform(0.7, 1.5)
        e = min(rng.uniform(0.0, 0.05), 1.5 / a - 1.0, 1.0 - 0.7 / a)
        inc = math.radians(rng.uniform(-7.0, 7.0))
        m0 = rng.uniform(0.0, 2.0 * math.pi)
        probes.append(kepler_orbit(t_knots, a, max(e, 0.0), inc, m0))
    traj = np.stack(probes)
    t_on = rng.uniform(1.0, 3.0) * DAY
    cmes = np.array([cme_row(t_on, 8 * 3600.0, 0.0, lon_corot(traj[0], t_on, OMEGA_SUN),
                             math.radians(30.0), 1.2e6, 1000e6, 8e5)])
    return Workload("dynamic_cme_512x64x128", g, Options(), 1.5, OMEGA_SUN, t_maps, maps, cmes,
                    traj, t_end=days * DAY, meta={"phase": phase, "tilts": tilts})


def paper2019(seed: int = 7, days: float = 42.0, n_maps: int = 454, cadence_h: float = 2.0,
              grid: Grid | None = None) -> Workload:
    """Stand-in for the paper's 2019 dynamic run (Sect. 4): a uniform 600 x 64 x 192 grid over
    0.1-2 AU, 454 synthetic maps at a 2 h cadence (the current-sheet recipe of the production
    workload, tilt random-walking by U(-1.5, 1.5) deg per map, about +-5 deg per day), no CME,
    two probes on circular orbits (1 AU at latitude 0, and 0.96 AU 40 deg behind in longitude),
    42 simulated days (the maps stop after 37.8 d and the last one is held)."""
    g = grid or Grid(600, 64, 192, stretch=0)
    rng = SplitMix64(seed)
    phase = 2.0 * math.pi * rng.uniform()
    tilts = tilt_walk(rng, n_maps, math.radians(15.0), step_deg=1.5)
    th, ph = g.theta_centres(), g.phi_centres()
    maps = np.stack([current_sheet_map(th, ph, a, phase, OMEGA_SUN, g.x1min) for a in tilts])
    t_maps = np.arange(n_maps) * cadence_h * 3600.0
    t_knots = np.arange(0.0, (days + 1.0) * DAY + 1.0, 3600.0)
    traj = np.stack([circular_orbit(t_knots, 1.0, 0.0, 0.0, 365.25),
                     circular_orbit(t_knots, 0.96, 0.0, -40.0, 346.0)])
    return Workload(f"paper2019_{g.n1}x{g.n2}x{g.n3}_dynamic", g, Options(), 1.5, OMEGA_SUN, t_maps, maps,
                    np.zeros((0, 8)), traj, t_end=days * DAY, meta={"phase": phase, "tilts": tilts})


# The five eruptions of the paper's June-July 2015 case (Sect. 4, Table 2): time at 0.1 AU,
# latitude and longitude (HEEQ, deg), half-width (deg), speed (km/s).
PAPER2015_START = "2015-06-10T01:14"
PAPER2015_CMES = (("2015-06-18T20:00", 11.0, -50.0, 45.0, 1000.0),
                  ("2015-06-19T14:59", -33.0, 9.0, 54.0, 603.0),
                  ("2015-06-21T05:01", 7.0, -8.0, 47.0, 1250.0),
                  ("2015-06-22T21:10", 14.0, 3.0, 45.0, 1155.0),
                  ("2015-06-25T10:51", 23.0, 46.0, 41.0, 1450.0))


def paper2015(seed: int = 11, days: float = 29.875, cadence_h: float = 2.0, grid: Grid | None = None) -> Workload:
    """Stand-in for the paper's June-July 2015 dynamic case with five CMEs (Sect. 4): a uniform
    600 x 64 x 192 grid over 0.1-2 AU from 2015-06-10 01:14 for 29.875 days (to 2015-07-09 22:14:
    8 d relaxation, 7 d of CME insertion, the rest propagation); synthetic maps every 2 h from the
    production recipe (the paper's cadence for this case is not stated; its 2019 case used 2 h);
    the five cone CMEs of Table 2 at their times, latitudes, longitudes relative to Earth's,
    half-widths and speeds, with the production workload's density (1000 cm^-3) and temperature
    (0.8 MK), which the table does not give, inserted as spherical clouds; the CME tracer on; one
    probe at Earth (1 AU, latitude 0)."""
    from datetime import datetime
    g = grid or Grid(600, 64, 192, stretch=0)
    rng = SplitMix64(seed)
    phase = 2.0 * math.pi * rng.uniform()
    n_maps = int(math.ceil(days * 24.0 / cadence_h)) + 1
    tilts = tilt_walk(rng, n_maps, math.radians(15.0), step_deg=1.5)
    th, ph = g.theta_centres(), g.phi_centres()
    maps = np.stack([current_sheet_map(th, ph, a, phase, OMEGA_SUN, g.x1min) for a in tilts])
    t_maps = np.arange(n_maps) * cadence_h * 3600.0
    t_knots = np.arange(0.0, (days + 1.0) * DAY + 1.0, 3600.0)
    earth = circular_orbit(t_knots, 1.0, 0.0, 0.0, 365.25)
    t0 = datetime.fromisoformat(PAPER2015_START)
    cmes = []
    for when, lat, lon, hw, v in PAPER2015_CMES:
        t_on = (datetime.fromisoformat(when) - t0).total_seconds()
        lon_c = (lon_corot(earth, t_on, OMEGA_SUN) + math.radians(lon)) % (2.0 * math.pi)
        cmes.append(cme_row(t_on, 8 * 3600.0, math.radians(lat), lon_c, math.radians(hw), v * 1e3, 1000e6, 8e5))
    o = Options(cme_model=CME_SPHERE, tracer=1)
    return Workload(f"paper2015_{g.n1}x{g.n2}x{g.n3}_dynamic_5cme", g, o, 1.5, OMEGA_SUN, t_maps, maps,
                    np.array(cmes), earth[None].copy(), t_end=days * DAY, meta={"phase": phase, "tilts": tilts})


def ensemble(seed: int = 3, n_members: int = 64, nr_set=(128, 256, 384, 512), nth_range=(32, 64),
             nph_range=(64, 128), days: float = 10.0) -> list:
    """Cone-CME ensemble: speed U(600, 2000) km/s, half-width U(15, 45) deg, direction within
    +-20 deg of probe 1 in latitude and longitude, onset U(0, 2) d, uneven grids."""
    rng = SplitMix64(seed)
    phase = 2.0 * math.pi * rng.uniform()
    tilts = tilt_walk(rng, 10, math.radians(15.0))
    t_maps = np.arange(10) * DAY
    t_knots = np.arange(0.0, (days + 1.0) * DAY + 1.0, 3600.0)
    earth = circular_orbit(t_knots, 1.0, 0.0, 0.0, 365.25)
    members = []
    for _ in range(n_members):
        nr = nr_set[rng.randint(0, len(nr_set) - 1)]
        nth = 2 * rng.randint(nth_range[0] // 2, nth_range[1] // 2)
        nph = 2 * rng.randint(nph_range[0] // 2, nph_range[1] // 2)
        g = Grid(nr, nth, nph)
        speed = rng.uniform(600.0, 2000.0) * 1e3
        hw = math.radians(rng.uniform(15.0, 45.0))
        dlat = math.radians(rng.uniform(-20.0, 20.0))
        dlon = math.radians(rng.uniform(-20.0, 20.0))
        t_on = rng.uniform(0.0, 2.0) * DAY
        lon = (lon_corot(earth, t_on, OMEGA_SUN) + dlon) % (2.0 * math.pi)
        maps = np.stack([current_sheet_map(g.theta_centres(), g.phi_centres(), a, phase, OMEGA_SUN, g.x1min)
                         for a in tilts])
        cmes = np.array([cme_row(t_on, 8 * 3600.0, dlat, lon, hw, speed, 1000e6, 8e5)])
        members.append(Workload(f"member_{nr}x{nth}x{nph}", g, Options(), 1.5, OMEGA_SUN, t_maps, maps,
                                cmes, earth[None].copy(), t_end=days * DAY))
    return members


def perturbed_state(shape8, seed: int, base: np.ndarray, rel: float = 1e-3) -> np.ndarray:
    """base * (1 + rel * U(-1, 1)) elementwise, from splitmix64 (vectorised through numpy's
    reproducible integer stream seeded by one splitmix64 draw)."""
    rng = SplitMix64(seed)
    g = np.random.Generator(np.random.PCG64(rng.next_u64()))
    return base * (1.0 + rel * g.uniform(-1.0, 1.0, size=shape8))
