"""Seeded synthetic inputs shaped like the paper's workloads (FP64, host).

Nothing here belongs to the time step: these functions draw the initial
fields, winds and vertical grids that both the CPU oracle and the CUDA path
start from.  Every random number is drawn here from ``numpy.random`` with an
explicit seed; the base seed is 240408849 and member m of an ensemble uses
``seed + m``.

Workloads (the paper's own test cases - DCMIP2016 / JW06 - are not restated;
these are generic stand-ins with the same shapes, see the module functions):

* tracer under solid-body rotation (cosine bell; 12-day revolution)
* balanced zonal jet on a sigma-mass grid + a non-divergent spherical-harmonic
  perturbation (hydrostatic and non-hydrostatic dycore)
* the same jet plus a warm bubble on a stretched 30 km-top grid (NH)
* uneven tracer ensembles on steady non-divergent deformational winds
"""
from __future__ import annotations

import math

import numpy as np

from .mesh import lonlat

SEED = 240408849

# physical constants (one set, passed across the C ABI by value)
GRAVITY = 9.80616
RD = 287.04
CP = 1004.64
P0 = 1.0e5
KAPPA = RD / CP
GAMMA = CP / (CP - RD)
DAY = 86400.0


# ----------------------------------------------------------------------------
# winds from stream functions
# ----------------------------------------------------------------------------

def normal_wind_from_psi(mesh, psi_vertex):
    """Edge-normal wind of the non-divergent flow with vertex stream function
    psi: u_e = -(psi(v2) - psi(v1)) / dv_e.  With v1 -> v2 along t = k x n this
    is the edge-mean normal component of k x grad(psi), and its discrete
    divergence vanishes identically."""
    v1, v2 = mesh["vertices_on_edge"][:, 0], mesh["vertices_on_edge"][:, 1]
    return -(psi_vertex[..., v2] - psi_vertex[..., v1]) / mesh["edge_dv"]


def solid_body_psi(mesh, u0):
    """psi = -u0 R sin(lat): eastward solid-body rotation u = u0 cos(lat)."""
    _, lat = lonlat(mesh["vertex_xyz"])
    return -u0 * mesh["radius"] * np.sin(lat)


def great_circle(lon1, lat1, lon2, lat2):
    return np.arccos(np.clip(np.sin(lat1) * np.sin(lat2)
                             + np.cos(lat1) * np.cos(lat2) * np.cos(lon1 - lon2), -1.0, 1.0))


def cosine_bell(mesh, lon0, lat0, r0, h0, xyz=None):
    """h = (h0/2)(1 + cos(pi r / r0)) for r < r0, else 0 (r great-circle)."""
    lon, lat = lonlat(mesh["cell_xyz"] if xyz is None else xyz)
    r = mesh["radius"] * great_circle(lon, lat, lon0, lat0)
    return np.where(r < r0, 0.5 * h0 * (1.0 + np.cos(np.pi * r / r0)), 0.0)


def slotted_cylinder(mesh, lon0, lat0, r0, h0, slot_w, slot_l):
    """Disc of radius r0 and height h0 with a rectangular slot of width slot_w
    (radians of longitude) cut from the centre towards the south to slot_l."""
    lon, lat = lonlat(mesh["cell_xyz"])
    r = mesh["radius"] * great_circle(lon, lat, lon0, lat0)
    dlon = np.angle(np.exp(1j * (lon - lon0)))
    inside = r < r0
    slot = (np.abs(dlon) < slot_w / 2) & (lat < lat0 + slot_l) & (lat > lat0 - r0 / mesh["radius"])
    return np.where(inside & ~slot, h0, 0.0)


def gaussian_hill(mesh, lon0, lat0, width, h0):
    lon, lat = lonlat(mesh["cell_xyz"])
    r = mesh["radius"] * great_circle(lon, lat, lon0, lat0)
    return h0 * np.exp(-(r / width) ** 2)


# ----------------------------------------------------------------------------
# real spherical harmonics (normalised associated Legendre by recursion)
# ----------------------------------------------------------------------------

def _legendre_all(lmax, x):
    """Fully normalised associated Legendre functions P_l^m(x), 0<=m<=l<=lmax,
    by the standard three-term recursion in l (returns dict (l,m) -> array)."""
    out = {}
    s = np.sqrt(np.maximum(0.0, 1.0 - x * x))
    pmm = np.full_like(x, 1.0 / math.sqrt(4.0 * math.pi))
    for m in range(0, lmax + 1):
        if m > 0:
            pmm = -math.sqrt((2.0 * m + 1.0) / (2.0 * m)) * s * pmm
        out[(m, m)] = pmm
        if m + 1 <= lmax:
            out[(m + 1, m)] = math.sqrt(2.0 * m + 3.0) * x * pmm
        for l in range(m + 2, lmax + 1):
            a = math.sqrt((4.0 * l * l - 1.0) / (l * l - m * m))
            b = math.sqrt(((l - 1.0) ** 2 - m * m) / (4.0 * (l - 1.0) ** 2 - 1.0))
            out[(l, m)] = a * (x * out[(l - 1, m)] - b * out[(l - 2, m)])
    return out


def random_harmonic_field(xyz, lmin, lmax, rng):
    """Sum of real spherical harmonics of degree lmin..lmax with N(0,1)
    coefficients, evaluated at unit vectors xyz."""
    lon, lat = lonlat(xyz)
    P = _legendre_all(lmax, np.sin(lat))
    f = np.zeros(xyz.shape[0])
    for l in range(lmin, lmax + 1):
        for m in range(0, l + 1):
            c = rng.standard_normal()
            f += c * P[(l, m)] * np.cos(m * lon)
            if m > 0:
                f += rng.standard_normal() * P[(l, m)] * np.sin(m * lon)
    return f


def harmonic_perturbation(mesh, amp, lmax, rng):
    """Non-divergent edge-normal wind from a random vertex stream function of
    degree 1..lmax harmonics, scaled so max |u'| = amp."""
    psi = random_harmonic_field(mesh["vertex_xyz"], 1, lmax, rng)
    u = normal_wind_from_psi(mesh, psi)
    return u * (amp / np.max(np.abs(u)))


# ----------------------------------------------------------------------------
# tracer workloads
# ----------------------------------------------------------------------------

def tracer_rotation_case(mesh, n_levels=30, dt=1800.0, pi_top=225.0, ps=1.0e5):
    """Cosine bell (radius R/3, height 1000, centre lon 270, lat 0) under
    solid-body rotation u0 = 2 pi R / 12 days, same on every level; uniform
    layer mass dpi = (ps - pi_top)/L.  Returns q [1][nC][L], dpi [nC][L],
    mass flux [nE][L] (= dpi_e u_e), u [nE]."""
    R = mesh["radius"]
    u0 = 2.0 * math.pi * R / (12.0 * DAY)
    u = normal_wind_from_psi(mesh, solid_body_psi(mesh, u0))
    dpi0 = (ps - pi_top) / n_levels
    h = cosine_bell(mesh, math.radians(270.0), 0.0, R / 3.0, 1000.0)
    q = np.repeat(h[:, None], n_levels, 1)[None].copy()
    dpi = np.full((mesh["n_cells"], n_levels), dpi0)
    flux = np.repeat((dpi0 * u)[:, None], n_levels, 1)
    return {"q": q, "dpi": dpi, "mass_flux": flux, "u": u, "u0": u0, "dt": dt}


def bell_exact(mesh, t, u0, lon0=math.radians(270.0), lat0=0.0):
    """Analytic bell of the rotation case at time t (centre moved east)."""
    R = mesh["radius"]
    lon_c = lon0 + u0 * t / R
    return cosine_bell(mesh, lon_c, lat0, R / 3.0, 1000.0)


def deformational_psi(mesh, rng, umax=40.0):
    """Seeded smooth stream function: degree 2..4 harmonics, scaled so the
    induced edge wind peaks at umax."""
    psi = random_harmonic_field(mesh["vertex_xyz"], 2, 4, rng)
    u = normal_wind_from_psi(mesh, psi)
    return psi * (umax / np.max(np.abs(u)))


def tracer_mixture(mesh, n_tracers, n_levels, rng):
    """Seeded mixture of cosine bells, slotted cylinders and Gaussian hills,
    one shape per tracer (cycled), random centres / sizes, weak level
    dependence of the amplitude."""
    R = mesh["radius"]
    q = np.zeros((n_tracers, mesh["n_cells"], n_levels))
    lev = 1.0 + 0.1 * np.linspace(-1.0, 1.0, n_levels)
    for t in range(n_tracers):
        lon0 = rng.uniform(0, 2 * math.pi)
        lat0 = rng.uniform(-1.0, 1.0)
        kind = t % 3
        if kind == 0:
            h = cosine_bell(mesh, lon0, lat0, R * rng.uniform(0.2, 0.5), 1.0)
        elif kind == 1:
            h = slotted_cylinder(mesh, lon0, lat0, R * rng.uniform(0.3, 0.5), 1.0,
                                 rng.uniform(0.08, 0.15), rng.uniform(0.2, 0.4))
        else:
            h = gaussian_hill(mesh, lon0, lat0, R * rng.uniform(0.1, 0.3), 1.0)
        q[t] = 0.1 + h[:, None] * lev[None, :]
    return q


def ensemble_members(mesh, n_members=16, seed=SEED, tracers=(1, 4, 10, 25), levels=(30, 60),
                     pi_top=225.0, ps=1.0e5, cfl=0.4):
    """Uneven batched tracer workload: per member a tracer count from
    ``tracers``, a level count from ``levels``, a steady non-divergent
    deformational wind (amplitude x U(0.8, 1.2)), a tracer mixture.
    Returns a list of dicts and the common dt chosen from the CFL number."""
    members = []
    umax_all = 0.0
    for m in range(n_members):
        rng = np.random.default_rng(seed + m)
        T = int(rng.choice(tracers))
        L = int(rng.choice(levels))
        amp = rng.uniform(0.8, 1.2)
        psi = deformational_psi(mesh, rng) * amp
        u = normal_wind_from_psi(mesh, psi)
        umax_all = max(umax_all, float(np.max(np.abs(u))))
        dpi0 = (ps - pi_top) / L
        dpi = np.full((mesh["n_cells"], L), dpi0)
        flux = np.repeat((dpi0 * u)[:, None], L, 1)
        q = tracer_mixture(mesh, T, L, rng)
        members.append({"q": q, "dpi": dpi, "mass_flux": flux, "n_levels": L, "n_tracers": T})
    dt = cfl * float(np.min(mesh["edge_dc"])) / umax_all
    return members, dt


# ----------------------------------------------------------------------------
# dycore workloads
# ----------------------------------------------------------------------------

def sigma_uniform(n_levels):
    """B at interfaces, top (0) to surface (1), uniform spacing."""
    return np.linspace(0.0, 1.0, n_levels + 1)


def stretched_heights(n_levels, top=30.0e3, c=2.0):
    """Interface heights z = H (s + c s^2)/(1 + c), s uniform in [0, 1],
    returned top to bottom."""
    s = np.linspace(0.0, 1.0, n_levels + 1)
    z = top * (s + c * s * s) / (1.0 + c)
    return z[::-1].copy()


def sigma_from_heights(z_int, t_ref=250.0, ps_ref=P0):
    """sigma-mass interfaces matching heights z of an isothermal reference
    column p(z) = ps exp(-g z / (Rd T)); returns (B, pi_top)."""
    p = ps_ref * np.exp(-GRAVITY * z_int / (RD * t_ref))
    pi_top = p[0]
    B = (p - pi_top) / (ps_ref - pi_top)
    B[0], B[-1] = 0.0, 1.0
    return B, float(pi_top)


class ZonalJet:
    """Balanced zonal jet u(lat, p) = U(lat) S(p) on pressure surfaces.

    U(lat) = umax sin^2(2 lat) (mid-latitude jets in both hemispheres);
    S(p) = exp(-((ln p - ln p_j) / w)^2), p_j = 0.25 p0.  Gradient-wind
    balance on pressure surfaces, (2 Omega sin(lat) + u tan(lat)/a) u =
    -(1/a) dPhi/dlat, integrated numerically in latitude on a fine grid,
    gives Phi(lat, p) = Rd T0 ln(p0/p) - S G1(lat) - S^2 G2(lat); hydrostatic
    T = -(1/Rd) dPhi/dln p; surface pressure from Phi(lat, ps) = 0 (flat)."""

    def __init__(self, radius, omega, umax=35.0, t0=260.0, pj=0.25 * P0, width=1.4):
        self.a, self.omega, self.umax, self.t0 = radius, omega, umax, t0
        self.lpj, self.w = math.log(pj), width
        lat = np.linspace(0.0, math.pi / 2, 20001)
        U = umax * np.sin(2 * lat) ** 2
        g1 = radius * 2 * omega * np.sin(lat) * U
        g2 = U * U * np.tan(np.minimum(lat, math.pi / 2 - 1e-12))
        g2[-1] = 0.0
        dl = lat[1] - lat[0]
        self._lat = lat
        self._G1 = np.concatenate([[0], np.cumsum(0.5 * (g1[1:] + g1[:-1]) * dl)])
        self._G2 = np.concatenate([[0], np.cumsum(0.5 * (g2[1:] + g2[:-1]) * dl)])

    def U(self, lat):
        return self.umax * np.sin(2 * lat) ** 2

    def S(self, p):
        return np.exp(-((np.log(p) - self.lpj) / self.w) ** 2)

    def dS(self, p):     # dS / d ln p
        x = (np.log(p) - self.lpj) / self.w
        return -2.0 * x / self.w * np.exp(-x * x)

    def G(self, lat):
        al = np.abs(lat)
        return np.interp(al, self._lat, self._G1), np.interp(al, self._lat, self._G2)

    def temperature(self, lat, p):
        G1, G2 = self.G(lat)
        S, dS = self.S(p), self.dS(p)
        return self.t0 + (dS * G1 + 2.0 * S * dS * G2) / RD

    def surface_pressure(self, lat):
        G1, G2 = self.G(lat)
        ps = np.full_like(lat, P0)
        for _ in range(50):
            S = self.S(ps)
            ps = P0 * np.exp(-(S * G1 + S * S * G2) / (RD * self.t0))
        return ps

    def u(self, lat, p):
        return self.U(lat) * self.S(p)


def dycore_jet_case(mesh, n_levels, nonhydrostatic=False, seed=SEED, bubble=False,
                    pert_amp=1.0, pert_lmax=16, t0=260.0):
    """Balanced jet + seeded perturbation (+ warm bubble) on a sigma-mass grid.

    Hydrostatic: uniform sigma, pi_top = 225 Pa.  Non-hydrostatic: sigma at
    stretched heights with a 30 km top, pi_top = p(30 km) of the reference
    column.  Returns dict with ps [nC], u [nE][L], dpi_theta [nC][L],
    b_int [L+1], pi_top, phi_s [nC], and for NH w, phi [nC][L+1] with phi in
    discrete hydrostatic balance (so that the equation of state returns the
    hydrostatic mid-layer pressure)."""
    rng = np.random.default_rng(seed)
    R = mesh["radius"]
    jet = ZonalJet(R, mesh["omega"], t0=t0)
    if nonhydrostatic:
        B, pi_top = sigma_from_heights(stretched_heights(n_levels), t_ref=t0)
    else:
        B, pi_top = sigma_uniform(n_levels), 225.0
    dB = np.diff(B)
    lonc, latc = lonlat(mesh["cell_xyz"])
    ps = jet.surface_pressure(latc)
    pint = pi_top + B[None, :] * (ps[:, None] - pi_top)
    dpi = pint[:, 1:] - pint[:, :-1]
    pmid = 0.5 * (pint[:, 1:] + pint[:, :-1])
    T = jet.temperature(latc[:, None], pmid)
    theta = T * (P0 / pmid) ** KAPPA
    if bubble:
        r = R * great_circle(lonc, latc, math.radians(90.0), math.radians(30.0))
        z_approx = RD * t0 / GRAVITY * np.log(P0 / pmid)
        shape = np.exp(-(r / 250.0e3) ** 2)[:, None] * (z_approx < 5.0e3)
        theta = theta + 2.0 * shape
    # edge wind: eastward jet projected on the edge normal at the edge's
    # mid-layer pressure + non-divergent perturbation
    c1, c2 = mesh["cells_on_edge"][:, 0], mesh["cells_on_edge"][:, 1]
    xe, ne = mesh["edge_xyz"], mesh["edge_normal_xyz"]
    _, late = lonlat(xe)
    east = np.stack([-xe[:, 1], xe[:, 0], np.zeros_like(xe[:, 0])], 1)
    east /= np.maximum(np.linalg.norm(east, axis=1, keepdims=True), 1e-300)
    ncomp = np.sum(east * ne, 1)
    pe = 0.5 * (pmid[c1] + pmid[c2])
    u = jet.u(late[:, None], pe) * ncomp[:, None]
    u = u + harmonic_perturbation(mesh, pert_amp, pert_lmax, rng)[:, None]
    out = {"ps": ps, "u": u, "dpi_theta": dpi * theta, "b_int": B, "pi_top": pi_top,
           "phi_s": np.zeros(mesh["n_cells"]), "theta": theta, "dpi": dpi, "pmid": pmid}
    if nonhydrostatic:
        alpha = RD * theta * (pmid / P0) ** KAPPA / pmid
        phi = np.zeros((mesh["n_cells"], n_levels + 1))
        for k in range(n_levels - 1, -1, -1):
            phi[:, k] = phi[:, k + 1] + alpha[:, k] * dpi[:, k]
        out["phi"] = phi
        out["w"] = np.zeros_like(phi)
    return out


def resting_case(mesh, n_levels, nonhydrostatic=False, t0=250.0):
    """Resting, horizontally uniform isothermal atmosphere, flat surface,
    ps = p0; phi (NH) in discrete hydrostatic balance."""
    if nonhydrostatic:
        B, pi_top = sigma_from_heights(stretched_heights(n_levels), t_ref=t0)
    else:
        B, pi_top = sigma_uniform(n_levels), 225.0
    nC = mesh["n_cells"]
    ps = np.full(nC, P0)
    pint = pi_top + B[None, :] * (ps[:, None] - pi_top)
    dpi = pint[:, 1:] - pint[:, :-1]
    pmid = 0.5 * (pint[:, 1:] + pint[:, :-1])
    theta = t0 * (P0 / pmid) ** KAPPA
    out = {"ps": ps, "u": np.zeros((mesh["n_edges"], n_levels)), "dpi_theta": dpi * theta,
           "b_int": B, "pi_top": pi_top, "phi_s": np.zeros(nC), "theta": theta, "dpi": dpi}
    if nonhydrostatic:
        alpha = RD * theta * (pmid / P0) ** KAPPA / pmid
        phi = np.zeros((nC, n_levels + 1))
        for k in range(n_levels - 1, -1, -1):
            phi[:, k] = phi[:, k + 1] + alpha[:, k] * dpi[:, k]
        out["phi"] = phi
        out["w"] = np.zeros_like(phi)
    return out
