"""Seeded synthetic inputs for the Bragg-spot sum.

This module only *draws* inputs: crystal orientation, mosaic domain
matrices, a photon spectrum, a structure-factor table and detector
geometry.  It contains none of the per-pixel arithmetic of the method
(no scattering vectors, Miller indices, lattice transforms, lookups,
polarization, solid angle or phi rotation).  Both the CUDA path and the
FP64 CPU oracle consume the ``Shot`` objects built here, so the two sides
always see bit-identical inputs.

The paper (Sec. III-B) names only "crystal orientation, mosaicity and
photon energy" and (Sec. II) "one structure factor per Bragg spot"; the
concrete recipe below (uniform random orientation, Gaussian mosaic
angles, Gaussian spectrum, Wilson-like |F|^2) is the synthetic stand-in
for the experimental shots the paper simulates.

Conventions (lab frame, right-handed):
  * the sample sits at the origin, the beam travels along +z;
  * crystal axes are real-space vectors in Angstrom, rows a, b, c;
  * detector positions are in metres; a panel is described by the outer
    corner of pixel (slow 0, fast 0), unit fast/slow axes, the unit normal
    pointing away from the sample, and a square pixel size.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

HC_KEV_ANGSTROM = 12.398419843320026  # h*c in keV*Angstrom (CODATA 2018)

SHAPE_SINC = 0
SHAPE_GAUSS = 1
INTERP_NEAREST = 0
INTERP_TRICUBIC = 1


@dataclasses.dataclass
class Panel:
    origin: np.ndarray  # (3,) m, outer corner of pixel (0, 0)
    fdir: np.ndarray  # (3,) unit fast axis
    sdir: np.ndarray  # (3,) unit slow axis
    ndir: np.ndarray  # (3,) unit normal, away from the sample
    pixel_m: float
    nfast: int
    nslow: int

    @property
    def npix(self) -> int:
        return self.nfast * self.nslow


@dataclasses.dataclass
class Shot:
    """Every input of one Bragg-spot simulation (one detector image)."""

    # crystal
    axes: np.ndarray  # (3, 3) rows a, b, c in Angstrom, lab frame
    umats: np.ndarray  # (M, 3, 3) mosaic domain rotations
    n_phi: int
    phi0_deg: float
    phistep_deg: float
    spindle: np.ndarray  # (3,) unit
    ncells: np.ndarray  # (3,) Na, Nb, Nc
    shape: int  # SHAPE_SINC / SHAPE_GAUSS
    scale: float
    # structure factors
    F: np.ndarray  # (nh, nk, nl) float32, l fastest
    hkl_min: np.ndarray  # (3,) int
    interp: int  # INTERP_NEAREST / INTERP_TRICUBIC
    default_F: float
    # beam
    dirs: np.ndarray  # (S, 3) unit propagation directions
    lambdas: np.ndarray  # (S,) Angstrom
    weights: np.ndarray  # (S,)
    fluence: float  # photons / m^2
    kahn: float  # polarization factor K
    evec: np.ndarray  # (3,) E-vector direction of the polarized part
    # detector
    panels: List[Panel]
    oversample: int
    n_layers: int
    thickness_m: float
    atten_m: float

    @property
    def n_mosaic(self) -> int:
        return int(self.umats.shape[0])

    @property
    def n_src(self) -> int:
        return int(self.lambdas.shape[0])

    @property
    def npix(self) -> int:
        return sum(p.npix for p in self.panels)

    @property
    def hkl_n(self) -> np.ndarray:
        return np.array(self.F.shape, dtype=np.int32)

    @property
    def steps_per_pixel(self) -> int:
        return (self.oversample ** 2 * self.n_layers * self.n_src
                * self.n_mosaic * self.n_phi)

    @property
    def pixel_steps(self) -> int:
        return self.npix * self.steps_per_pixel

    def copy(self) -> "Shot":
        return dataclasses.replace(
            self,
            panels=[dataclasses.replace(p) for p in self.panels])


@dataclasses.dataclass
class Background:
    """Amorphous scatter (air / water around the crystal): the scattering
    factor F of one molecule (electrons) at increasing knots of
    stol = sin(theta)/lambda (1/Angstrom), interpolated linearly and held
    at the end values, and the number of molecules in the beam."""

    stol: np.ndarray  # (n,) strictly increasing
    F: np.ndarray  # (n,)
    n_molecules: float


# --------------------------------------------------------------------------
# random draws


def random_orientation(rng: np.random.Generator) -> np.ndarray:
    """Uniformly distributed rotation matrix (Shoemake's unit quaternion)."""
    u1, u2, u3 = rng.random(3)
    q1 = math.sqrt(1.0 - u1) * math.sin(2.0 * math.pi * u2)
    q2 = math.sqrt(1.0 - u1) * math.cos(2.0 * math.pi * u2)
    q3 = math.sqrt(u1) * math.sin(2.0 * math.pi * u3)
    q0 = math.sqrt(u1) * math.cos(2.0 * math.pi * u3)
    return _quat_to_matrix(q0, q1, q2, q3)


def _quat_to_matrix(w, x, y, z) -> np.ndarray:
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ], dtype=np.float64)


def _axis_angle_matrix(axis: np.ndarray, angle: float) -> np.ndarray:
    k = np.asarray(axis, dtype=np.float64)
    k = k / np.linalg.norm(k)
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + math.sin(angle) * K + (1 - math.cos(angle)) * (K @ K)


def mosaic_umats(rng: np.random.Generator, n: int,
                 spread_deg: float) -> np.ndarray:
    """n domain rotations: axis uniform on the sphere, angle ~ N(0, spread)."""
    out = np.empty((n, 3, 3), dtype=np.float64)
    for m in range(n):
        axis = rng.standard_normal(3)
        ang = math.radians(spread_deg) * rng.standard_normal()
        out[m] = _axis_angle_matrix(axis, ang)
    return out


def identity_umats(n: int) -> np.ndarray:
    return np.repeat(np.eye(3)[None], n, axis=0)


def monochromatic(lambda_A: float, direction=(0.0, 0.0, 1.0)):
    d = np.asarray(direction, dtype=np.float64)[None, :]
    return d / np.linalg.norm(d), np.array([lambda_A]), np.array([1.0])


def gaussian_spectrum(n: int, e0_keV: float, fwhm_frac: float,
                      direction=(0.0, 0.0, 1.0)):
    """n energies equispaced over E0 +- 3 sigma (FWHM = fwhm_frac * E0),
    Gaussian weights normalised to sum 1, all along one direction."""
    sigma = fwhm_frac * e0_keV / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    if n == 1:
        energies = np.array([e0_keV])
    else:
        energies = np.linspace(e0_keV - 3 * sigma, e0_keV + 3 * sigma, n)
    w = np.exp(-0.5 * ((energies - e0_keV) / sigma) ** 2)
    w = w / w.sum()
    lambdas = HC_KEV_ANGSTROM / energies
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    return np.repeat(d[None, :], n, axis=0), lambdas, w


def structure_factors(rng: np.random.Generator, hmax: int,
                      mean_I: float = 1.0e4) -> np.ndarray:
    """Amplitudes on h,k,l in [-hmax, hmax]^3 with |F|^2 ~ Exp(mean_I),
    Friedel-symmetric (F(-h) = F(h)) and F(000) = 0; float32, l fastest."""
    n = 2 * hmax + 1
    I = rng.exponential(mean_I, size=(n, n, n))
    I = 0.5 * (I + I[::-1, ::-1, ::-1])
    I[hmax, hmax, hmax] = 0.0
    return np.sqrt(I).astype(np.float32)


def orthorhombic_axes(a: float, b: float, c: float,
                      U: np.ndarray) -> np.ndarray:
    """Rows a, b, c of an orthorhombic cell (along x, y, z) rotated by U."""
    base = np.diag([a, b, c]).astype(np.float64)
    return (U @ base.T).T.copy()


def flat_detector(nfast: int, nslow: int, pixel_m: float,
                  dist_m: float, beam_center=None) -> Panel:
    """Panel perpendicular to the beam at distance dist_m, fast = +x,
    slow = +y, normal = +z; beam centre (fast, slow) in pixels from the
    outer corner of pixel (0, 0), default the panel centre."""
    if beam_center is None:
        beam_center = (nfast / 2.0, nslow / 2.0)
    cf, cs = beam_center
    return Panel(origin=np.array([-cf * pixel_m, -cs * pixel_m, dist_m]),
                 fdir=np.array([1.0, 0.0, 0.0]),
                 sdir=np.array([0.0, 1.0, 0.0]),
                 ndir=np.array([0.0, 0.0, 1.0]),
                 pixel_m=pixel_m, nfast=nfast, nslow=nslow)


def tiled_detector(n_tf: int, n_ts: int, nfast: int, nslow: int,
                   pixel_m: float, dist_m: float, gap_m: float) -> List[Panel]:
    """n_tf x n_ts coplanar panels with gaps, centred on the beam."""
    wf = nfast * pixel_m
    ws = nslow * pixel_m
    tot_f = n_tf * wf + (n_tf - 1) * gap_m
    tot_s = n_ts * ws + (n_ts - 1) * gap_m
    panels = []
    for js in range(n_ts):
        for jf in range(n_tf):
            x0 = -tot_f / 2 + jf * (wf + gap_m)
            y0 = -tot_s / 2 + js * (ws + gap_m)
            panels.append(Panel(origin=np.array([x0, y0, dist_m]),
                                fdir=np.array([1.0, 0.0, 0.0]),
                                sdir=np.array([0.0, 1.0, 0.0]),
                                ndir=np.array([0.0, 0.0, 1.0]),
                                pixel_m=pixel_m, nfast=nfast, nslow=nslow))
    return panels


def amorphous_background(n_knots: int = 64, stol_max: float = 1.0,
                         n_molecules: float = 3.3e10,
                         uneven: bool = False) -> Background:
    """Synthetic water-like scattering curve: a smooth ring (maximum near
    stol = 0.16/A, the 3.1 A water ring) over a slowly falling floor, F in
    electrons (about 2.4 at the ring), sampled at n_knots knots on
    [0, stol_max] (uneven:
    denser towards stol = 0).  n_molecules 3.3e10 is the water in one cubic
    micrometre."""
    x = np.linspace(0.0, 1.0, n_knots)
    st = stol_max * (x ** 1.5 if uneven else x)
    F = 2.6 * (0.35 + 0.65 * np.exp(-((st - 0.16) / 0.05) ** 2)) \
        * np.exp(-0.5 * st)
    return Background(stol=st, F=F, n_molecules=float(n_molecules))


# --------------------------------------------------------------------------
# the workloads


def _base_shot(**kw) -> Shot:
    d = dict(n_phi=1, phi0_deg=0.0, phistep_deg=0.0,
             spindle=np.array([0.0, 1.0, 0.0]), scale=1.0,
             default_F=0.0, fluence=1.0e24, kahn=0.0,
             evec=np.array([1.0, 0.0, 0.0]), oversample=1, n_layers=1,
             thickness_m=0.0, atten_m=0.0)
    d.update(kw)
    return Shot(**d)


def single_shot_small(seed: int = 0, n: int = 256) -> Shot:
    """256x256, 0.1 mm pixels at 100 mm, one source at 1.3 A, 10 mosaic
    domains (0.05 deg), 79x79x38 cell, Na=Nb=Nc=10 sinc, nearest lookup
    on hkl in [-30,30]^3, unpolarized, 1e24 ph/m^2."""
    rng = np.random.default_rng(seed)
    U = random_orientation(rng)
    umats = mosaic_umats(rng, 10, 0.05)
    F = structure_factors(rng, 30)
    dirs, lam, w = monochromatic(1.3)
    return _base_shot(
        axes=orthorhombic_axes(79.0, 79.0, 38.0, U), umats=umats,
        ncells=np.array([10.0, 10.0, 10.0]), shape=SHAPE_SINC,
        F=F, hkl_min=np.array([-30, -30, -30], dtype=np.int32),
        interp=INTERP_NEAREST, dirs=dirs, lambdas=lam, weights=w,
        panels=[flat_detector(n, n, 1.0e-4, 0.1)])


def large_shot(seed: int = 1, n: int = 3072, n_src: int = 100,
               n_mosaic: int = 50) -> Shot:
    """3072x3072, oversample 2, two layers of a 0.5 mm sensor (attenuation
    length 0.3 mm), 100 sources on a Gaussian 0.5 % spectrum at 9.5 keV,
    50 mosaic domains, Na=Nb=Nc=25 Gaussian, tricubic lookup on hkl in
    [-60,60]^3, Kahn factor 0.99 (E along x)."""
    rng = np.random.default_rng(seed)
    U = random_orientation(rng)
    umats = mosaic_umats(rng, n_mosaic, 0.05)
    F = structure_factors(rng, 60)
    dirs, lam, w = gaussian_spectrum(n_src, 9.5, 0.005)
    return _base_shot(
        axes=orthorhombic_axes(79.0, 79.0, 38.0, U), umats=umats,
        ncells=np.array([25.0, 25.0, 25.0]), shape=SHAPE_GAUSS,
        F=F, hkl_min=np.array([-60, -60, -60], dtype=np.int32),
        interp=INTERP_TRICUBIC, dirs=dirs, lambdas=lam, weights=w,
        kahn=0.99, panels=[flat_detector(n, n, 1.0e-4, 0.1)],
        oversample=2, n_layers=2, thickness_m=5.0e-4, atten_m=3.0e-4)


def precision_shot(ncells: float, seed: int = 2, n: int = 1024,
                   n_src: int = 100, n_mosaic: int = 20) -> Shot:
    """1024x1024 (0.1 mm at 100 mm), the 100-source spectrum of
    large_shot, 20 mosaic domains, Na=Nb=Nc=ncells sinc, nearest lookup
    on hkl in [-60,60]^3, oversample 1, one layer, unpolarized."""
    rng = np.random.default_rng(seed)
    U = random_orientation(rng)
    umats = mosaic_umats(rng, n_mosaic, 0.05)
    F = structure_factors(rng, 60)
    dirs, lam, w = gaussian_spectrum(n_src, 9.5, 0.005)
    return _base_shot(
        axes=orthorhombic_axes(79.0, 79.0, 38.0, U), umats=umats,
        ncells=np.array([ncells] * 3, dtype=np.float64), shape=SHAPE_SINC,
        F=F, hkl_min=np.array([-60, -60, -60], dtype=np.int32),
        interp=INTERP_NEAREST, dirs=dirs, lambdas=lam, weights=w,
        panels=[flat_detector(n, n, 1.0e-4, 0.1)])


def multipanel_shot(n_src: int, seed: int = 3, n_mosaic: int = 10,
                    tiles=(8, 8), panel=(194, 185)) -> Shot:
    """64 panels of 185x194 pixels (0.11 mm) tiled 8x8 at 100 mm with
    1 mm gaps, n_src sources on the 0.5 % spectrum at 9.5 keV, 10 mosaic
    domains, Na=Nb=Nc=15 Gaussian, nearest lookup on hkl in [-40,40]^3."""
    rng = np.random.default_rng(seed)
    U = random_orientation(rng)
    umats = mosaic_umats(rng, n_mosaic, 0.05)
    F = structure_factors(rng, 40)
    dirs, lam, w = gaussian_spectrum(n_src, 9.5, 0.005)
    return _base_shot(
        axes=orthorhombic_axes(79.0, 79.0, 38.0, U), umats=umats,
        ncells=np.array([15.0, 15.0, 15.0]), shape=SHAPE_GAUSS,
        F=F, hkl_min=np.array([-40, -40, -40], dtype=np.int32),
        interp=INTERP_NEAREST, dirs=dirs, lambdas=lam, weights=w,
        panels=tiled_detector(tiles[0], tiles[1], panel[0], panel[1],
                              1.1e-4, 0.1, 1.0e-3))


def shrink(shot: Shot, nfast: int, nslow: int, f0: int = None,
           s0: int = None) -> Shot:
    """A copy whose single panel is the nfast x nslow window starting at
    pixel (s0, f0) of the first panel (default: the window touching the
    beam centre's lower-right quadrant, where spots are dense)."""
    p = shot.panels[0]
    if f0 is None:
        f0 = p.nfast // 2 + p.nfast // 8
    if s0 is None:
        s0 = p.nslow // 2 + p.nslow // 8
    origin = p.origin + f0 * p.pixel_m * p.fdir + s0 * p.pixel_m * p.sdir
    out = shot.copy()
    out.panels = [Panel(origin=origin, fdir=p.fdir.copy(), sdir=p.sdir.copy(),
                        ndir=p.ndir.copy(), pixel_m=p.pixel_m,
                        nfast=nfast, nslow=nslow)]
    return out


def sample_pixels(shot: Shot, n_blocks: int, block: int, seed: int,
                  ) -> np.ndarray:
    """Global indices (panel-major, then slow, then fast) of n_blocks
    random square blocks of block x block pixels, for spot checks of a
    full-size image."""
    rng = np.random.default_rng(seed)
    out = []
    base = 0
    offs = []
    for p in shot.panels:
        offs.append(base)
        base += p.npix
    for _ in range(n_blocks):
        q = int(rng.integers(len(shot.panels)))
        p = shot.panels[q]
        s0 = int(rng.integers(0, max(1, p.nslow - block + 1)))
        f0 = int(rng.integers(0, max(1, p.nfast - block + 1)))
        for s in range(s0, min(p.nslow, s0 + block)):
            for f in range(f0, min(p.nfast, f0 + block)):
                out.append(offs[q] + s * p.nfast + f)
    return np.unique(np.array(out, dtype=np.int64))


def strided_rows(shot: Shot, every: int) -> np.ndarray:
    """Global indices of every `every`-th row of every panel."""
    out = []
    base = 0
    for p in shot.panels:
        for s in range(0, p.nslow, every):
            out.append(base + s * p.nfast + np.arange(p.nfast))
        base += p.npix
    return np.concatenate(out).astype(np.int64)


# --------------------------------------------------------------- serving


@dataclasses.dataclass
class ShotRequest:
    """One served shot: its own orientation, mosaic domains, spectrum and
    detector region of interest (f0, s0, nfast, nslow)."""
    axes: np.ndarray
    umats: np.ndarray
    lambdas: np.ndarray
    weights: np.ndarray
    scale: float
    roi: tuple

    @property
    def npix(self) -> int:
        return self.roi[2] * self.roi[3]

    @property
    def pixel_steps(self) -> int:
        return self.npix * self.umats.shape[0] * self.lambdas.shape[0]


def serving_detector_shot(seed: int = 4) -> Shot:
    """Resident state of the shot server: the 3072x3072 detector (0.1 mm at
    100 mm, oversample 1, one layer), Na=Nb=Nc=25 Gaussian, tricubic F on
    [-60,60]^3, beam along z, Kahn 0.99; crystal and spectrum per request."""
    rng = np.random.default_rng(seed)
    F = structure_factors(rng, 60)
    dirs, lam, w = gaussian_spectrum(1, 9.5, 0.005)
    return _base_shot(
        axes=orthorhombic_axes(79.0, 79.0, 38.0, np.eye(3)),
        umats=identity_umats(1), ncells=np.array([25.0, 25.0, 25.0]),
        shape=SHAPE_GAUSS, F=F, hkl_min=np.array([-60, -60, -60],
                                                 dtype=np.int32),
        interp=INTERP_TRICUBIC, dirs=dirs, lambdas=lam, weights=w,
        kahn=0.99, panels=[flat_detector(3072, 3072, 1.0e-4, 0.1)])


def serving_requests(n: int, seed: int = 5, max_src: int = 100,
                     max_mosaic: int = 50, min_pix: float = 1e3,
                     max_pix: float = 4e6, det: int = 3072):
    """n requests: random orientation of the 79x79x38 cell, S ~ U{1..max_src}
    sources on the 0.5 % spectrum at 9.5 keV, M ~ U{1..max_mosaic} domains
    (0.05 deg), an ROI of log-uniform area in [min_pix, max_pix] pixels with
    aspect ratio in [1/2, 2], placed uniformly on the det x det detector."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        U = random_orientation(rng)
        S = int(rng.integers(1, max_src + 1))
        M = int(rng.integers(1, max_mosaic + 1))
        area = math.exp(rng.uniform(math.log(min_pix), math.log(max_pix)))
        aspect = math.exp(rng.uniform(math.log(0.5), math.log(2.0)))
        nf = int(max(1, min(det, round(math.sqrt(area * aspect)))))
        ns = int(max(1, min(det, round(area / nf))))
        f0 = int(rng.integers(0, det - nf + 1))
        s0 = int(rng.integers(0, det - ns + 1))
        _, lam, w = gaussian_spectrum(S, 9.5, 0.005)
        out.append(ShotRequest(axes=orthorhombic_axes(79.0, 79.0, 38.0, U),
                               umats=mosaic_umats(rng, M, 0.05),
                               lambdas=lam, weights=w, scale=1.0,
                               roi=(f0, s0, nf, ns)))
    return out


def poisson_arrivals(n: int, rate: float, seed: int = 6) -> np.ndarray:
    """Arrival times (s) of a Poisson process of the given rate (1/s)."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))


def request_shot(base: Shot, req: ShotRequest) -> Shot:
    """The stand-alone Shot of a served request (its ROI as the panel)."""
    s = base.copy()
    s.axes = req.axes
    s.umats = req.umats
    s.lambdas = req.lambdas
    s.weights = req.weights
    s.dirs = np.repeat(base.dirs[:1], len(req.lambdas), axis=0)
    s.scale = req.scale
    f0, s0, nf, ns = req.roi
    return shrink(s, nf, ns, f0, s0)
