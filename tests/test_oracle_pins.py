"""Pins of the FP64 CPU oracle against what physics and mathematics fix.

None of these re-types the oracle's formula: each compares it with a
closed form, an invariance, a special case that collapses a loop, an
independent numerical integral or high-precision arithmetic.  A plausible
slip anywhere in the oracle (a dropped factor, a wrong sign or index, a
transposed operand, a wrong normalisation) fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2205_07976_gb300 import workloads as W

R_E = 2.8179403262e-15


def tiny_shot(shape=W.SHAPE_SINC, interp=W.INTERP_NEAREST, N=10.0, n=8,
              seed=5, n_src=1, n_mosaic=1, os_=1, hmax=20):
    rng = np.random.default_rng(seed)
    U = W.random_orientation(rng)
    umats = (W.mosaic_umats(rng, n_mosaic, 0.05) if n_mosaic > 1
             else W.identity_umats(1))
    F = W.structure_factors(rng, hmax)
    if n_src == 1:
        dirs, lam, w = W.monochromatic(1.3)
    else:
        dirs, lam, w = W.gaussian_spectrum(n_src, 9.5, 0.005)
    return W._base_shot(
        axes=W.orthorhombic_axes(79.0, 79.0, 38.0, U), umats=umats,
        ncells=np.array([N, N, N]), shape=shape, F=F,
        hkl_min=np.array([-hmax] * 3, dtype=np.int32), interp=interp,
        dirs=dirs, lambdas=lam, weights=w,
        panels=[W.flat_detector(n, n, 1e-4, 0.1,
                                beam_center=(-40.0, -30.0))],
        oversample=os_)


# ------------------------------------------------------------- F_latt


@pytest.mark.parametrize("N", [1, 2, 10, 25, 50, 200])
def test_sinc_peak_is_N_at_integer_h(N):
    for h in [-61, -7, -1, 0, 1, 2, 3, 17, 60]:
        assert abs(oracle.sincg(h, N)) == N


@pytest.mark.parametrize("N", [10, 25, 50, 200])
def test_sinc_matches_high_precision(N):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    rng = np.random.default_rng(N)
    for h in np.concatenate([rng.uniform(-65, 65, 40),
                             rng.integers(-60, 60, 10) + rng.normal(0, 1e-3, 10)]):
        hm = mp.mpf(float(h))
        ref = mp.sin(mp.pi * N * hm) / mp.sin(mp.pi * hm)
        # the argument pi N f is rounded once in FP64: absolute error is
        # bounded by a few ulp of pi N |f| relative to the peak N
        assert abs(oracle.sincg(h, N) - float(ref)) <= 1e-12 * N


@pytest.mark.parametrize("N", [10, 50])
def test_sinc_zeros(N):
    for n in [-5, 0, 3, 40]:
        for j in range(1, N // 2):
            f = j / N
            for h in (n + f, n - f):
                assert abs(oracle.sincg(h, N)) <= 1e-12 * N


def test_sinc_literal_and_reduced_agree_off_peak():
    rng = np.random.default_rng(7)
    for N in (10, 25):
        for h in rng.uniform(-40, 40, 50):
            a = oracle.sincg(h, N, "literal")
            b = oracle.sincg(h, N, "reduced")
            assert abs(a - b) <= 1e-10 * N


def test_gauss_closed_form():
    s = tiny_shot(shape=W.SHAPE_GAUSS, N=15.0)
    s.ncells = np.array([15.0, 12.0, 9.0])
    NN = 15.0 * 12.0 * 9.0
    assert oracle.flatt(s, [3, -4, 7]) == NN
    for x in [0.01, 0.1, 0.3, -0.2, 0.49]:
        assert math.isclose(oracle.flatt(s, [3 + x, -4, 7]),
                            NN * math.exp(-(15.0 * x) ** 2 / 0.63),
                            rel_tol=1e-13)
        assert math.isclose(oracle.flatt(s, [3, -4 + x, 7 - x]),
                            NN * math.exp(-((12.0 * x) ** 2 + (9 * x) ** 2)
                                          / 0.63), rel_tol=1e-13)


def test_sinc_product_over_axes():
    s = tiny_shot(N=10.0)
    s.ncells = np.array([10.0, 6.0, 4.0])
    hkl = [2.13, -0.37, 5.61]
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    ref = 1
    for h, N in zip(hkl, s.ncells):
        ref *= mp.sin(mp.pi * N * h) / mp.sin(mp.pi * h)
    assert math.isclose(oracle.flatt(s, hkl), float(ref), rel_tol=1e-12)


# -------------------------------------------------------------- F_cell


def test_nearest_lookup_and_ties():
    s = tiny_shot()
    F = s.F.astype(np.float64)
    hm = -20

    def at(h, k, l):
        return F[h - hm, k - hm, l - hm]

    assert oracle.fcell(s, [3, -2, 5]) == at(3, -2, 5)
    assert oracle.fcell(s, [3.4, -2.4, 5.49]) == at(3, -2, 5)
    assert oracle.fcell(s, [3.6, -2.6, 4.51]) == at(4, -3, 5)
    # ties round down: 2.5 -> 2, -2.5 -> -3
    assert oracle.fcell(s, [2.5, -2.5, 0.0]) == at(2, -3, 0)
    # outside the table -> default_F
    assert oracle.fcell(s, [20.6, 0, 0]) == 0.0
    s.default_F = 7.5
    assert oracle.fcell(s, [0, -21, 0]) == 7.5
    assert oracle.fcell(s, [20.4, 0, 0]) == at(20, 0, 0)


def test_tricubic_reproduces_cubic_polynomials():
    s = tiny_shot(interp=W.INTERP_TRICUBIC, hmax=6)
    rng = np.random.default_rng(3)
    C = rng.normal(size=(4, 4, 4))
    g = np.arange(-6, 7, dtype=np.float64)

    def poly(h, k, l):
        return sum(C[i, j, m] * h ** i * k ** j * l ** m
                   for i in range(4) for j in range(4) for m in range(4))

    H, K, L = np.meshgrid(g, g, g, indexing="ij")
    s.F = poly(H, K, L)  # the oracle reads the table as float64
    for hkl in rng.uniform(-4.9, 3.9, size=(25, 3)):
        assert math.isclose(oracle.fcell(s, hkl), poly(*hkl),
                            rel_tol=1e-9, abs_tol=1e-9 * np.abs(s.F).max())
    for hkl in [(0, 0, 0), (-3, 2, 1), (3, -5, 4)]:
        assert math.isclose(oracle.fcell(s, hkl), poly(*hkl), rel_tol=1e-12,
                            abs_tol=1e-12)


def test_tricubic_falls_back_to_nearest_at_table_edge():
    s = tiny_shot(interp=W.INTERP_TRICUBIC, hmax=6)
    F = s.F.astype(np.float64)
    # floor(h) + 2 = 7 > 6: the stencil leaves the table
    assert oracle.fcell(s, [5.3, 0.2, 0.1]) == F[5 + 6, 0 + 6, 0 + 6]
    assert oracle.fcell(s, [-5.7, 0.2, 0.1]) == F[-6 + 6, 6, 6]
    # continuity at the switch point: an interior node equals its entry
    a = oracle.fcell(s, [4.999999999, 1.0, 1.0])
    b = oracle.fcell(s, [5.0, 1.0, 1.0])
    assert math.isclose(a, b, rel_tol=1e-7)


# ----------------------------------------------- per-pixel physics terms


def test_polarization_thomson_limits():
    inc = np.array([0.0, 0.0, 1.0])
    e = np.array([1.0, 0.0, 0.0])
    for tth in np.radians([5.0, 30.0, 60.0, 90.0, 120.0]):
        c = math.cos(tth)
        in_plane = np.array([math.sin(tth), 0.0, c])   # along E
        perp = np.array([0.0, math.sin(tth), c])        # normal to E
        # unpolarized: (1 + cos^2 2theta) / 2
        assert math.isclose(oracle.polarization(in_plane, inc, 0.0, e),
                            0.5 * (1 + c * c), rel_tol=1e-14)
        # fully polarized: cos^2 2theta in the E plane, 1 normal to it
        assert math.isclose(oracle.polarization(in_plane, inc, 1.0, e),
                            c * c, rel_tol=1e-12, abs_tol=1e-15)
        assert math.isclose(oracle.polarization(perp, inc, 1.0, e), 1.0,
                            rel_tol=1e-14)
        # partial polarization interpolates linearly in K
        K = 0.99
        mid = np.array([math.sin(tth) * math.cos(0.3),
                        math.sin(tth) * math.sin(0.3), c])
        p0 = oracle.polarization(mid, inc, 0.0, e)
        p1 = oracle.polarization(mid, inc, 1.0, e)
        pk = oracle.polarization(mid, inc, K, e)
        assert math.isclose(pk, p0 + K * (p1 - p0), rel_tol=1e-13)
    # an E vector with a component along the beam uses its transverse part
    d = np.array([0.3, 0.4, math.sqrt(1 - 0.25)])
    assert math.isclose(oracle.polarization(d, inc, 1.0, [1.0, 0.0, 5.0]),
                        oracle.polarization(d, inc, 1.0, e), rel_tol=1e-14)


def test_solid_angle_integrates_to_rectangle():
    # solid angle of a centred 2a x 2b rectangle at distance D
    a, b, D = 0.06, 0.04, 0.1
    exact = 4 * math.atan(a * b / (D * math.sqrt(a * a + b * b + D * D)))
    px = 5e-4
    xs = np.arange(-a + px / 2, a, px)
    ys = np.arange(-b + px / 2, b, px)
    n = np.array([0.0, 0.0, 1.0])
    tot = sum(oracle.solid_angle(px, n, [x, y, D]) for x in xs for y in ys)
    assert math.isclose(tot, exact, rel_tol=2e-5)


def test_capture_matches_beer_lambert_integral():
    quad = pytest.importorskip("scipy.integrate").quad
    thick, atten, T = 5e-4, 3e-4, 2
    dt = thick / T
    for rho in (1.0, 0.8, 0.45):
        L = atten * rho  # attenuation length along the slanted ray
        tot = 0.0
        for t in range(T):
            c = oracle.capture(t, dt, atten, rho, thick)
            ref = quad(lambda z: math.exp(-z / L) / L, t * dt, (t + 1) * dt)[0]
            assert math.isclose(c, ref, rel_tol=1e-10)
            tot += c
        assert math.isclose(tot, 1 - math.exp(-thick / L), rel_tol=1e-12)
    assert oracle.capture(0, 0.0, 0.0, 1.0, 0.0) == 1.0


# ------------------------------------------------------ the whole sum


def bragg_pixel_shot(shape, interp, hkl, seed=11):
    """A one-pixel detector whose pixel centre sees reflection hkl exactly:
    lambda solves the Ewald condition |lambda S + i| = 1 for S = A^-1 hkl."""
    rng = np.random.default_rng(seed)
    inc = np.array([0.0, 0.0, 1.0])
    for _ in range(200):
        U = W.random_orientation(rng)
        A = W.orthorhombic_axes(79.0, 79.0, 38.0, U)
        S = np.linalg.solve(A, np.asarray(hkl, dtype=np.float64))
        if S @ inc >= 0:
            continue
        lam = -2 * (S @ inc) / (S @ S)
        d = lam * S + inc
        if 0.5 < lam < 3.0 and d[2] > 0.5:
            break
    else:
        raise RuntimeError("no orientation found")
    assert abs(np.linalg.norm(d) - 1) < 1e-14
    D = 0.1 / d[2]
    P = D * d
    px = 1e-4
    panel = W.Panel(origin=P - 0.5 * px * np.array([1.0, 1.0, 0.0]),
                    fdir=np.array([1.0, 0, 0]), sdir=np.array([0, 1.0, 0]),
                    ndir=np.array([0, 0, 1.0]), pixel_m=px, nfast=1, nslow=1)
    hmax = 20
    F = W.structure_factors(rng, hmax)
    s = W._base_shot(
        axes=A, umats=W.identity_umats(1), ncells=np.array([10.0, 11.0, 7.0]),
        shape=shape, F=F, hkl_min=np.array([-hmax] * 3, dtype=np.int32),
        interp=interp, dirs=inc[None, :], lambdas=np.array([lam]),
        weights=np.array([1.0]), panels=[panel], fluence=3e23, scale=1.7)
    c2t = d @ inc
    expected = (R_E ** 2 * s.fluence * s.scale
                * float(F[hkl[0] + hmax, hkl[1] + hmax, hkl[2] + hmax]) ** 2
                * (10.0 * 11.0 * 7.0) ** 2
                * 0.5 * (1 + c2t ** 2)
                * px * px * 0.1 / D ** 3)
    return s, expected


@pytest.mark.parametrize("shape,interp", [
    (W.SHAPE_SINC, W.INTERP_NEAREST), (W.SHAPE_GAUSS, W.INTERP_NEAREST),
    (W.SHAPE_GAUSS, W.INTERP_TRICUBIC), (W.SHAPE_SINC, W.INTERP_TRICUBIC)])
@pytest.mark.parametrize("hkl", [(1, 2, 3), (-4, 3, 2), (7, -1, -5)])
def test_single_step_on_a_bragg_condition(shape, interp, hkl):
    s, expected = bragg_pixel_shot(shape, interp, hkl)
    got = oracle.image(s)[0]
    assert math.isclose(got, expected, rel_tol=1e-11)


def test_friedel_inversion():
    for shape, interp in [(W.SHAPE_SINC, W.INTERP_NEAREST),
                          (W.SHAPE_GAUSS, W.INTERP_TRICUBIC)]:
        s = tiny_shot(shape=shape, interp=interp, n=12, n_src=3, n_mosaic=3)
        a = oracle.image(s)
        s2 = s.copy()
        s2.axes = -s.axes
        b = oracle.image(s2)
        np.testing.assert_allclose(b, a, rtol=1e-12, atol=1e-13 * a.max())


def _rotate_setup(s, Q):
    r = s.copy()
    r.axes = (Q @ s.axes.T).T
    r.umats = np.einsum("ij,mjk,lk->mil", Q, s.umats, Q)
    r.spindle = Q @ s.spindle
    r.dirs = (Q @ s.dirs.T).T
    r.evec = Q @ s.evec
    r.panels = [W.Panel(origin=Q @ p.origin, fdir=Q @ p.fdir, sdir=Q @ p.sdir,
                        ndir=Q @ p.ndir, pixel_m=p.pixel_m, nfast=p.nfast,
                        nslow=p.nslow) for p in s.panels]
    return r


@pytest.mark.parametrize("shape,interp,N,n", [
    (W.SHAPE_SINC, W.INTERP_NEAREST, 10.0, 10),
    (W.SHAPE_GAUSS, W.INTERP_TRICUBIC, 6.0, 24)])
def test_global_rotation_invariance(shape, interp, N, n):
    rng = np.random.default_rng(21)
    s = tiny_shot(shape=shape, interp=interp, n=n, n_src=2, n_mosaic=3,
                  os_=2, N=N)
    s.kahn = 0.9
    s.n_phi, s.phistep_deg = 3, 0.02
    s.n_layers, s.thickness_m, s.atten_m = 2, 4e-4, 3e-4
    s.spindle = np.array([0.3, 0.9, 0.1])
    a = oracle.image(s)
    Q = W.random_orientation(rng)
    b = oracle.image(_rotate_setup(s, Q))
    big = a > 1e-6 * a.max()
    assert big.sum() > 5
    np.testing.assert_allclose(b[big], a[big], rtol=1e-9)
    np.testing.assert_allclose(b, a, rtol=0, atol=1e-9 * a.max())


def test_identical_sources_collapse():
    s = tiny_shot(n=8)
    a = oracle.image(s)
    s3 = s.copy()
    s3.dirs = np.repeat(s.dirs, 3, axis=0)
    s3.lambdas = np.repeat(s.lambdas, 3)
    s3.weights = np.full(3, 1.0 / 3.0)
    np.testing.assert_allclose(oracle.image(s3), a, rtol=1e-13, atol=0)


def test_identical_domains_and_phi_steps_collapse():
    s = tiny_shot(n=8, shape=W.SHAPE_GAUSS, N=15.0)
    a = oracle.image(s)
    sm = s.copy()
    sm.umats = W.identity_umats(4)
    sm.n_phi, sm.phistep_deg = 3, 0.0
    np.testing.assert_allclose(oracle.image(sm), a, rtol=1e-13, atol=0)


def test_oversampling_equals_finer_pixels():
    s = tiny_shot(n=6, os_=2, N=10.0)
    a = oracle.image(s).reshape(6, 6)
    p = s.panels[0]
    f = s.copy()
    f.oversample = 1
    f.panels = [W.Panel(origin=p.origin, fdir=p.fdir, sdir=p.sdir,
                        ndir=p.ndir, pixel_m=p.pixel_m / 2, nfast=12,
                        nslow=12)]
    b = oracle.image(f).reshape(12, 12)
    bsum = b.reshape(6, 2, 6, 2).sum(axis=(1, 3))
    np.testing.assert_allclose(a, bsum, rtol=1e-9, atol=1e-12 * a.max())


def test_intensity_linear_in_fluence_scale_and_F():
    s = tiny_shot(n=6)
    a = oracle.image(s)
    t = s.copy()
    t.fluence *= 3.0
    t.scale = 0.5
    t.F = (s.F.astype(np.float64) * 2.0)
    np.testing.assert_allclose(oracle.image(t), a * 3.0 * 0.5 * 4.0,
                               rtol=1e-13)


def test_brute_force_high_precision_tiny_detector():
    """mpmath at 30 digits on a 2x2 detector (2 sources, 2 domains,
    oversample 2, 2 layers, Kahn 0.9): FP64 rounding of the oracle stays
    within 1e-11 relative."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    s = tiny_shot(n=2, n_src=2, n_mosaic=2, os_=2, shape=W.SHAPE_SINC,
                  N=10.0)
    s.kahn = 0.9
    s.n_layers, s.thickness_m, s.atten_m = 2, 4e-4, 3e-4
    got = oracle.image(s)
    M = [mp.matrix(u.tolist()) for u in s.umats]
    A = mp.matrix(s.axes.tolist())
    p = s.panels[0]
    F = s.F.astype(np.float64)

    def v(x):
        return mp.matrix([mp.mpf(float(t)) for t in x])

    O, fd, sd, nd = v(p.origin), v(p.fdir), v(p.sdir), v(p.ndir)
    px = mp.mpf(p.pixel_m)
    inc = v(s.dirs[0])
    e = v(s.evec)
    ep = e - (e.T * inc)[0] * inc
    ep = ep / mp.norm(ep)
    bp = mp.matrix([inc[1] * ep[2] - inc[2] * ep[1],
                    inc[2] * ep[0] - inc[0] * ep[2],
                    inc[0] * ep[1] - inc[1] * ep[0]])
    dt = mp.mpf(s.thickness_m) / 2
    out = []
    for q in range(4):
        ss, ff = divmod(q, 2)
        acc = mp.mpf(0)
        for i in range(2):
            for j in range(2):
                for t in range(2):
                    P = (O + (ff + (i + mp.mpf(0.5)) / 2) * px * fd
                         + (ss + (j + mp.mpf(0.5)) / 2) * px * sd + t * dt * nd)
                    R = mp.norm(P)
                    d = P / R
                    om = px ** 2 * (nd.T * P)[0] / R ** 3
                    rho = (d.T * nd)[0]
                    L = mp.mpf(s.atten_m) * rho
                    cap = mp.exp(-t * dt / L) - mp.exp(-(t + 1) * dt / L)
                    c2 = (d.T * inc)[0]
                    psi = mp.atan2((d.T * bp)[0], (d.T * ep)[0])
                    pol = (1 + c2 ** 2 - mp.mpf(s.kahn) * mp.cos(2 * psi)
                           * (1 - c2 ** 2)) / 2
                    for k in range(2):
                        S = (d - v(s.dirs[k])) / mp.mpf(s.lambdas[k])
                        for m in range(2):
                            Am = (M[m] * A.T).T
                            fl = mp.mpf(1)
                            hk = []
                            for a in range(3):
                                h = sum(Am[a, c] * S[c] for c in range(3))
                                fl *= mp.sin(mp.pi * 10 * h) / mp.sin(mp.pi * h)
                                hk.append(int(mp.ceil(h - mp.mpf(0.5))))
                            Fc = F[hk[0] + 20, hk[1] + 20, hk[2] + 20]
                            acc += (mp.mpf(float(Fc)) ** 2 * fl ** 2
                                    * mp.mpf(s.weights[k]) * cap * pol * om)
        out.append(mp.mpf(R_E) ** 2 * mp.mpf(s.fluence) * acc / (4 * 2))
    np.testing.assert_allclose(got, [float(x) for x in out], rtol=1e-11)


# --------------------------------------------------------- gradients


def _grad_shot():
    """A 12x10 panel (2 sources, 3 domains, N=15 Gaussian, nearest)
    centred on the brightest pixel of a 120x120 survey of the same shot."""
    s = W.multipanel_shot(2, tiles=(1, 1), panel=(120, 120), n_mosaic=3)
    U, cell, rot = _params(s)
    t = s.copy()
    t.axes, _ = oracle.param_axes(U, cell, rot)
    img = oracle.image(t).reshape(120, 120)
    js, jf = np.unravel_index(np.argmax(img), img.shape)
    p = s.panels[0]
    origin = (p.origin + (jf - 6) * p.pixel_m * p.fdir
              + (js - 5) * p.pixel_m * p.sdir)
    s.panels = [W.Panel(origin=origin, fdir=p.fdir, sdir=p.sdir, ndir=p.ndir,
                        pixel_m=p.pixel_m, nfast=12, nslow=10)]
    return s


def _params(s):
    rng = np.random.default_rng(3)
    U = W.random_orientation(rng)
    return U, np.array([79.0, 79.0, 38.0]), np.array([1e-3, -2e-3, 5e-4])


def test_param_axes_derivatives_match_finite_differences():
    U, cell, rot = _params(None)
    ax, dax = oracle.param_axes(U, cell, rot)
    # axes of an orthorhombic cell: orthogonal rows with the cell lengths
    np.testing.assert_allclose(np.linalg.norm(ax, axis=1), cell, rtol=1e-14)
    np.testing.assert_allclose(ax @ ax.T, np.diag(cell ** 2), atol=1e-10)
    x0 = np.concatenate([rot, cell])
    for r in range(6):
        h = 1e-6 * max(1.0, abs(x0[r]))
        xp, xm = x0.copy(), x0.copy()
        xp[r] += h
        xm[r] -= h
        ap, _ = oracle.param_axes(U, xp[3:], xp[:3])
        am, _ = oracle.param_axes(U, xm[3:], xm[:3])
        np.testing.assert_allclose(dax[r], (ap - am) / (2 * h), atol=1e-7)


@pytest.mark.parametrize("interp", [W.INTERP_NEAREST, W.INTERP_TRICUBIC])
def test_loss_gradient_matches_finite_differences(interp):
    s = _grad_shot()
    s.interp = interp
    U, cell, rot = _params(s)
    rng = np.random.default_rng(9)
    y = rng.poisson(2.0, size=s.npix).astype(np.float64)
    bkg = 1.0
    L0, g, gF, model = oracle.loss_grad(s, U, cell, rot, y, bkg)
    assert model.max() > 0.1, "the test panel must see spots"

    def loss_at(cell_=cell, rot_=rot, nc=None, scale=None, F=None):
        t = s.copy()
        if nc is not None:
            t.ncells = nc
        if scale is not None:
            t.scale = scale
        if F is not None:
            t.F = F
        return oracle.loss_grad(t, U, cell_, rot_, y, bkg, want_F=False)[0]

    x = np.concatenate([rot, cell, s.ncells, [s.scale]])
    for r in range(10):
        h = 1e-6 * max(abs(x[r]), 1e-3)
        xp, xm = x.copy(), x.copy()
        xp[r] += h
        xm[r] -= h
        fp = loss_at(xp[3:6], xp[:3], xp[6:9], xp[9])
        fm = loss_at(xm[3:6], xm[:3], xm[6:9], xm[9])
        fd = (fp - fm) / (2 * h)
        assert math.isclose(g[r], fd, rel_tol=2e-5,
                            abs_tol=1e-6 * np.abs(g).max()), (r, g[r], fd)
    # structure-factor gradient: the 8 entries with the largest gradient,
    # up to 24 other touched entries drawn at random, and an untouched one
    F64 = s.F.astype(np.float64)
    nz = np.flatnonzero(gF.ravel())
    assert nz.size >= 1
    order = nz[np.argsort(np.abs(gF.ravel()[nz]))]
    idx = list(order[-8:])
    rest = order[:-8]
    if rest.size:
        idx += list(rng.choice(rest, size=min(24, rest.size), replace=False))
    idx.append(int(np.flatnonzero(gF.ravel() == 0)[0]))  # an untouched entry
    for e in idx:
        h = 1e-4
        Fp, Fm = F64.copy().ravel(), F64.copy().ravel()
        Fp[e] += h
        Fm[e] -= h
        fd = (loss_at(F=Fp.reshape(F64.shape)) -
              loss_at(F=Fm.reshape(F64.shape))) / (2 * h)
        assert math.isclose(gF.ravel()[e], fd, rel_tol=1e-5,
                            abs_tol=1e-7 * np.abs(gF).max()), (e, fd)


def test_loss_model_equals_image():
    s = _grad_shot()
    U, cell, rot = _params(s)
    y = np.ones(s.npix)
    _, _, _, model = oracle.loss_grad(s, U, cell, rot, y, 1.0, want_F=False)
    t = s.copy()
    t.axes, _ = oracle.param_axes(U, cell, rot)
    np.testing.assert_allclose(model, oracle.image(t), rtol=1e-14)


# ------------------------------------------------- amorphous background


def bg_shot(n=64, px=1e-3, dist=0.05, os_=1, lam=1.3, kahn=0.0,
            beam_center=None, n_src=1):
    s = tiny_shot(n=n, os_=os_)
    s.panels = [W.flat_detector(n, n, px, dist, beam_center=beam_center)]
    if n_src == 1:
        s.dirs, s.lambdas, s.weights = W.monochromatic(lam)
    s.kahn = kahn
    return s


def flat_table(value, n_molecules=1.0):
    return W.Background(stol=np.array([0.0, 10.0]),
                        F=np.array([value, value]), n_molecules=n_molecules)


def test_background_integrates_to_rectangle_closed_form():
    # Constant F and an unpolarized beam along the normal through the
    # centre of a 2a x 2a panel at distance z: the summed background is
    # r_e^2 fluence n_mol F^2 (Omega + J) / 2 with Omega the rectangle's
    # solid angle and J = integral of cos^2(2 theta) dOmega.  With
    # Q(z) = Omega(z)/z = integral of 1/R^3 dx dy and d(1/R^3)/dz = -3z/R^5,
    # J = integral of z^3/R^5 dx dy = -(z^2/3) Q'(z) = (Omega - z Omega')/3.
    n, px, z = 64, 1e-3, 0.05
    a = b = n * px / 2
    s2 = math.sqrt(a * a + b * b + z * z)
    g = a * b / (z * s2)
    om = 4 * math.atan(g)
    dg = -a * b * (s2 * s2 + z * z) / (z * z * s2 ** 3)
    J = (om - z * 4 * dg / (1 + g * g)) / 3
    F, nm = 2.5, 7.0
    exact = R_E ** 2 * 1e24 * nm * F * F * (om + J) / 2
    sums = []
    for os_ in (4, 8):
        s = bg_shot(n=n, px=px, dist=z, os_=os_)
        sums.append(oracle.background(s, flat_table(F, nm)).sum())
    # midpoint rule: error ~ h^2, so Richardson's extrapolation is ~h^4
    rich = (4 * sums[1] - sums[0]) / 3
    assert abs(sums[1] - exact) < 1e-4 * exact
    assert abs(rich - exact) < 1e-8 * exact


def test_background_stol_is_sin_theta_over_lambda():
    # F = 1 up to stol*, 0 beyond: only pixels whose scattering angle is
    # below 2 arcsin(lambda stol*) see background.
    lam, st = 1.3, 0.25
    two_theta = 2 * math.asin(lam * st)
    s = bg_shot(n=48, px=2e-3, dist=0.05, lam=lam)
    bg = W.Background(stol=np.array([0.0, st, st * (1 + 1e-9), 5.0]),
                      F=np.array([1.0, 1.0, 0.0, 0.0]), n_molecules=1.0)
    img = oracle.background(s, bg).reshape(48, 48)
    idx = np.arange(48) + 0.5 - 24
    X, Y = np.meshgrid(idx * 2e-3, idx * 2e-3)
    ang = np.arctan2(np.hypot(X, Y), 0.05)
    inside = ang < two_theta - 1e-3
    outside = ang > two_theta + 1e-3
    assert inside.sum() > 100 and outside.sum() > 100
    assert (img[inside] > 0).all()
    assert (img[outside] == 0).all()


def test_background_wavelength_scaling():
    # stol scales as 1/lambda: doubling lambda and halving the knots of
    # the table gives the same image
    s1 = bg_shot(n=16, px=3e-3, dist=0.05, lam=1.0,
                 beam_center=(-2.0, 3.0))
    s2 = bg_shot(n=16, px=3e-3, dist=0.05, lam=2.0,
                 beam_center=(-2.0, 3.0))
    bg = W.amorphous_background(40)
    bg2 = W.Background(stol=bg.stol / 2, F=bg.F, n_molecules=bg.n_molecules)
    np.testing.assert_allclose(oracle.background(s1, bg),
                               oracle.background(s2, bg2), rtol=1e-13)


def test_background_table_is_piecewise_linear_and_held():
    # a table of a straight line gives the same image for any knots; ends
    # are held flat outside the table
    s = bg_shot(n=12, px=4e-3, dist=0.04, lam=1.0, beam_center=(0.0, 0.0))
    line = lambda x: 1.5 + 2.0 * x
    two = W.Background(stol=np.array([0.0, 3.0]), F=line(np.array([0.0, 3.0])),
                       n_molecules=2.0)
    rng = np.random.default_rng(1)
    knots = np.sort(np.concatenate([[0.0, 3.0], rng.uniform(0, 3, 30)]))
    many = W.Background(stol=knots, F=line(knots), n_molecules=2.0)
    a = oracle.background(s, two)
    np.testing.assert_allclose(oracle.background(s, many), a, rtol=1e-13)
    # a short table [0.1, 0.2] vs the same line held flat outside it
    short = W.Background(stol=np.array([0.1, 0.2]),
                         F=line(np.array([0.1, 0.2])), n_molecules=2.0)
    held = W.Background(stol=np.array([-1.0, 0.1, 0.2, 9.0]),
                        F=line(np.array([0.1, 0.1, 0.2, 0.2])),
                        n_molecules=2.0)
    np.testing.assert_allclose(oracle.background(s, short),
                               oracle.background(s, held), rtol=1e-13)
    assert oracle.background_factor(short, 0.15) == pytest.approx(line(0.15))
    assert oracle.background_factor(short, -5.0) == line(0.1)
    assert oracle.background_factor(short, 5.0) == line(0.2)


def test_background_oversampling_equals_finer_pixels():
    s = bg_shot(n=6, px=2e-3, dist=0.03, os_=2, beam_center=(1.0, 2.0))
    s.n_layers, s.thickness_m, s.atten_m = 2, 5e-4, 3e-4
    bg = W.amorphous_background(33)
    a = oracle.background(s, bg).reshape(6, 6)
    p = s.panels[0]
    f = s.copy()
    f.oversample = 1
    f.panels = [W.Panel(origin=p.origin, fdir=p.fdir, sdir=p.sdir,
                        ndir=p.ndir, pixel_m=p.pixel_m / 2, nfast=12,
                        nslow=12)]
    b = oracle.background(f, bg).reshape(12, 12)
    np.testing.assert_allclose(a, b.reshape(6, 2, 6, 2).sum(axis=(1, 3)),
                               rtol=1e-12)


def test_background_sources_collapse_and_scale():
    s = bg_shot(n=8, px=3e-3, dist=0.05, kahn=0.99,
                beam_center=(-1.0, 2.5))
    bg = W.amorphous_background(50)
    a = oracle.background(s, bg)
    m = s.copy()
    m.dirs = np.repeat(s.dirs, 4, axis=0)
    m.lambdas = np.repeat(s.lambdas, 4)
    m.weights = np.full(4, 0.25)
    np.testing.assert_allclose(oracle.background(m, bg), a, rtol=1e-14)
    # linear in fluence and n_mol, quadratic in F; the crystal plays no part
    t = s.copy()
    t.fluence *= 3.0
    t.axes = -t.axes
    t.ncells = t.ncells * 2
    bg3 = W.Background(stol=bg.stol, F=2 * bg.F, n_molecules=5 * bg.n_molecules)
    np.testing.assert_allclose(oracle.background(t, bg3), 60 * a, rtol=1e-14)


# ------------------------------------------------ phi steps, divergence


def test_phi_steps_equal_pre_rotated_axes():
    # n_phi steps of phistep about the spindle, starting at phi0, average
    # the images of the same crystal with its lab axes rotated by each angle
    # beforehand (right-hand rotation about the spindle; the mosaic domains
    # act after it)
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    s = tiny_shot(n=6, n_mosaic=3, N=10.0)
    k = np.array([0.3, 0.9, -0.2])
    k /= np.linalg.norm(k)
    s.spindle = k
    s.n_phi, s.phi0_deg, s.phistep_deg = 3, 0.7, 0.35
    got = oracle.image(s)
    parts = []
    for j in range(3):
        ang = np.deg2rad(0.7 + 0.35 * j)
        t = s.copy()
        t.n_phi, t.phi0_deg, t.phistep_deg = 1, 0.0, 0.0
        t.axes = Rot.from_rotvec(ang * k).apply(s.axes)
        parts.append(oracle.image(t))
    np.testing.assert_allclose(got, np.mean(parts, axis=0), rtol=1e-12,
                               atol=1e-14 * got.max())
    assert got.max() > 0


def test_sources_of_different_directions_add_up():
    # three sources of different directions and wavelengths: the image is
    # the weighted sum of one-source images (each with its own direction
    # in the scattering vector and the polarization)
    s = tiny_shot(n=6, N=10.0)
    s.kahn = 0.8
    dirs = np.array([[0.0, 0.0, 1.0], [2e-3, -1e-3, 1.0], [-1.5e-3, 0.0, 1.0]])
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    lam = np.array([1.30, 1.28, 1.32])
    w = np.array([0.5, 0.3, 0.2])
    s.dirs, s.lambdas, s.weights = dirs, lam, w
    got = oracle.image(s)
    want = np.zeros_like(got)
    for k in range(3):
        t = s.copy()
        t.dirs, t.lambdas, t.weights = dirs[k:k + 1], lam[k:k + 1], np.ones(1)
        want += w[k] * oracle.image(t)
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-15 * got.max())
    assert got.max() > 0
