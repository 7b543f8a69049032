"""GPU images vs the FP64 CPU oracle, element by element, through the C ABI.

Tolerances (max relative error per pixel):
  NB_F64    1e-12 on every pixel above 1e-250 photons (no floor relative
            to the maximum), and 1e-12 of the maximum in absolute terms
            everywhere;
  NB_MIXED  1e-5 on pixels above 1e-3 of the image maximum;
  NB_F32    reported only (the precision sweep's naive arm).
Windows are chosen with odd sizes so that every launch has ragged 16x8
tiles at its right and bottom edges.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2205_07976_gb300 import nbgb
from paper_2205_07976_gb300 import workloads as W
from tests.helpers import abs_err_frac, masked_rel_err, rel_err_above
from tests.test_oracle_pins import bragg_pixel_shot

pytestmark = pytest.mark.gpu

F64_TOL = 1e-12
MIXED_TOL = 1e-5


# Relative error is taken on every pixel above 1e-250 photons: far below
# any intensity, but above the range where a sum of terms of exp(-700)
# and less depends on how each libm rounds into the subnormal doubles
F64_FLOOR = 1e-250


def check_f64(got, ref):
    rel, n = rel_err_above(got, ref, F64_FLOOR)
    assert rel <= F64_TOL, (rel, n)
    assert abs_err_frac(got, ref) <= F64_TOL


def check_mixed(got, ref, tol=MIXED_TOL):
    rel, n = masked_rel_err(got, ref, 1e-3)
    assert rel <= tol, (rel, n)
    assert abs_err_frac(got, ref) <= tol


def run(shot, precision, pixels=None, variant="auto"):
    return nbgb.simulate(shot, precision, pixels, variant=variant)


# ------------------------------------------------------ single shot (c0)


@pytest.fixture(scope="module")
def c0():
    s = W.single_shot_small()
    return s, oracle.image(s)


def test_single_shot_f64(c0):
    s, ref = c0
    check_f64(run(s, "f64"), ref)


def test_single_shot_mixed(c0):
    s, ref = c0
    check_mixed(run(s, "mixed"), ref)


@pytest.mark.parametrize("shape,interp", [
    (W.SHAPE_SINC, W.INTERP_NEAREST), (W.SHAPE_GAUSS, W.INTERP_NEAREST),
    (W.SHAPE_GAUSS, W.INTERP_TRICUBIC), (W.SHAPE_SINC, W.INTERP_TRICUBIC)])
@pytest.mark.parametrize("hkl", [(1, 2, 3), (-4, 3, 2), (7, -1, -5)])
def test_single_step_on_a_bragg_condition(shape, interp, hkl):
    """One pixel whose centre sees reflection hkl exactly, one source, one
    domain: the closed form r_e^2 fluence scale F_hkl^2 (Na Nb Nc)^2 pol
    omega (the same case pins the oracle), from every kernel: the FP64
    form to 1e-11 (h is exact to a few ulp, so the sinc sits at its limit
    N), the FP32-mixed thread and warp kernels to 1e-5."""
    s, expected = bragg_pixel_shot(shape, interp, hkl)
    assert math.isclose(run(s, "f64")[0], expected, rel_tol=1e-11)
    assert math.isclose(run(s, "mixed", variant="thread")[0], expected,
                        rel_tol=MIXED_TOL)
    if shape == W.SHAPE_GAUSS:
        assert math.isclose(run(s, "mixed", variant="warp")[0], expected,
                            rel_tol=MIXED_TOL)


def test_single_shot_f32_is_finite_and_close(c0):
    s, ref = c0
    got = run(s, "f32")
    assert np.isfinite(got).all()
    rel, _ = masked_rel_err(got, ref, 1e-3)
    assert rel < 0.5  # N = 10, |h| <= 11: plain FP32 is still roughly right


# ---------------------------------------------- large shot windows (c1)


@pytest.fixture(scope="module", params=[(2500, 700, 37, 29),
                                        (1600, 1500, 33, 19)])
def c1win(request):
    f0, s0, nf, ns = request.param
    s = W.shrink(W.large_shot(), nf, ns, f0, s0)
    return s, oracle.image(s)


def test_large_shot_window_f64(c1win):
    s, ref = c1win
    check_f64(run(s, "f64"), ref)


@pytest.mark.parametrize("variant", ["thread", "warp"])
def test_large_shot_window_mixed(c1win, variant):
    s, ref = c1win
    check_mixed(run(s, "mixed", variant=variant), ref)


# ---------------------------------------------- precision sweep (c2)


@pytest.mark.parametrize("N", [10, 50, 200])
def test_precision_window(N):
    s = W.shrink(W.precision_shot(N), 45, 35, 600, 640)
    ref = oracle.image(s)
    # FP64 within 1e-12 on every pixel at every N: the kernel forms the
    # fractional offset before the sinc, as the oracle's reduced form does
    check_f64(run(s, "f64"), ref)
    check_mixed(run(s, "mixed"), ref)
    assert np.isfinite(run(s, "f32")).all()


@pytest.mark.parametrize("hmax,interp", [(20, W.INTERP_NEAREST),
                                         (6, W.INTERP_NEAREST),
                                         (20, W.INTERP_TRICUBIC)])
def test_sinc_table_edges(hmax, interp):
    """The sinc shape with one beam direction (the kernels' fixed-grid
    path) on a table of hkl in [-hmax, hmax]^3 that the detector's h
    exceeds (|h| reaches ~37 at its corners), with default_F = 35: a
    lattice point outside the table looks up default_F.  With hmax = 20
    some items have every step in the table, some a few steps outside and
    some every step outside; hmax = 6 is below the size at which the
    nearest lookup forms its index in FP32.  The whole 1024^2 image,
    compared on a grid of 4096 sampled pixels."""
    s = W.precision_shot(10, n_mosaic=4)
    s.F = W.structure_factors(np.random.default_rng(21), hmax)
    s.hkl_min = np.array([-hmax] * 3, dtype=np.int32)
    s.default_F = 35.0
    s.interp = interp
    pix = (np.arange(0, 1024, 32)[:, None] * 1024 +
           np.arange(0, 1024, 8)[None, :]).ravel().astype(np.int64)
    ref = oracle.image(s, pixels=pix)
    check_mixed(run(s, "mixed")[pix], ref)
    # the sample holds pixels whose terms all come from the table and
    # pixels with terms from default_F
    s0 = s.copy()
    s0.default_F = 0.0
    differ = oracle.image(s0, pixels=pix) != ref
    assert differ.any() and not differ.all()


# ---------------------------------------------- multi-panel (c3 forward)


@pytest.mark.parametrize("n_src", [1, 8])
def test_multipanel_full_detector(n_src):
    s = W.multipanel_shot(n_src)
    ref = oracle.image(s)
    check_f64(run(s, "f64"), ref)
    for variant in ("thread", "warp"):
        check_mixed(run(s, "mixed", variant=variant), ref)


# ---------------------------------------------- paths and edge cases


def test_pixel_list_path_matches_oracle():
    s = W.large_shot()
    pix = np.concatenate([W.sample_pixels(s, 3, 7, 11),
                          np.arange(700 * 3072 + 2500, 700 * 3072 + 2537)])
    ref = oracle.image(s, pix)
    for prec, chk in (("f64", check_f64), ("mixed", check_mixed)):
        sim = nbgb.Sim(prec).set_shot(s)
        sim.add_spots(pix)
        img = sim.image()
        chk(img[pix], ref)
        # untouched pixels stay exactly zero
        mask = np.ones(sim.npix, dtype=bool)
        mask[pix] = False
        assert not img[mask].any()
        sim.close()


def test_accumulate_is_the_fused_addarray():
    s = W.shrink(W.single_shot_small(), 21, 13, 150, 140)
    for prec in ("f64", "mixed"):
        sim = nbgb.Sim(prec).set_shot(s)
        sim.add_spots()
        one = sim.image()
        sim.add_spots()
        two = sim.image()
        # lhs += (double) rhs twice: exactly twice the first image
        assert np.array_equal(two, 2.0 * one)
        sim.zero()
        assert not sim.image().any()
        f32 = sim.image(np.float32)
        assert f32.dtype == np.float32 and not f32.any()
        sim.close()


def _edge_shot(seed=4):
    """Small shot with divergent sources, three phi steps about a tilted
    spindle, two sensor layers, oversample 3, Kahn 0.7 and a small F table
    (|h| exceeds it) with a non-zero default_F."""
    rng = np.random.default_rng(seed)
    U = W.random_orientation(rng)
    dirs = np.array([[0.0, 0.0, 1.0], [1e-3, 0.0, 1.0], [0.0, -2e-3, 1.0]])
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    s = W._base_shot(
        axes=W.orthorhombic_axes(79.0, 79.0, 38.0, U),
        umats=W.mosaic_umats(rng, 4, 0.1), n_phi=3, phi0_deg=0.5,
        phistep_deg=0.05, spindle=np.array([0.2, 1.0, 0.1]),
        ncells=np.array([12.0, 9.0, 7.0]), shape=W.SHAPE_GAUSS,
        F=W.structure_factors(rng, 6), hkl_min=np.array([-6, -6, -6],
                                                         dtype=np.int32),
        interp=W.INTERP_TRICUBIC, default_F=35.0, dirs=dirs,
        lambdas=np.array([1.2, 1.21, 1.19]), weights=np.array([.5, .3, .2]),
        kahn=0.7, evec=np.array([1.0, 0.2, 0.0]),
        panels=[W.flat_detector(29, 23, 1.5e-4, 0.08,
                                beam_center=(-60.0, -40.0))],
        oversample=3, n_layers=2, thickness_m=3e-4, atten_m=2e-4)
    return s


@pytest.mark.parametrize("shape,interp", [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_edge_case_shot(shape, interp):
    s = _edge_shot()
    s.shape, s.interp = shape, interp
    if shape == 0:
        s.ncells = np.array([12.0, 9.0, 7.0])
    ref = oracle.image(s)
    check_f64(run(s, "f64"), ref)
    for variant in ("thread", "warp"):
        check_mixed(run(s, "mixed", variant=variant), ref)


@pytest.mark.parametrize("variant", ["thread", "warp"])
def test_pixel_alone_equals_pixel_in_full_launch(variant):
    """A pixel's value depends on its own inputs only: launched alone (or
    in any subset) it is bitwise the value it has in the whole image."""
    s = W.shrink(W.large_shot(), 40, 24, 2490, 695)
    full = run(s, "mixed", variant=variant)
    rng = np.random.default_rng(0)
    sub = rng.choice(s.npix, 37, replace=False)
    sim = nbgb.Sim("mixed").set_shot(s).set_variant(variant)
    sim.add_spots(sub)
    part = sim.image()[sub]
    sim.close()
    assert np.array_equal(part, full[sub])


def test_stats_count_evaluated_terms():
    s = W.shrink(W.large_shot(), 24, 16, 2500, 700)
    counts = []
    for variant in ("thread", "warp"):
        sim = nbgb.Sim("mixed").set_shot(s).set_variant(variant)
        sim.add_spots()
        ev, ps = sim.stats()
        assert ps == s.pixel_steps
        assert 0 < ev < ps
        counts.append(ev)
        sim.close()
    # both variants skip exactly the same underflowing terms, up to the
    # rounding of f at the cut
    assert abs(counts[0] - counts[1]) <= 1e-4 * counts[0]


def test_work_counts_of_each_kernel():
    """nb_get_work: the counts fixed by the shot, and the ordering of what
    each kernel performed (terms <= pairs <= pixel-steps)."""
    s = W.shrink(W.large_shot(), 24, 16, 2500, 700)
    units = s.npix * s.oversample ** 2 * s.n_layers
    for prec, variant in (("mixed", "thread"), ("mixed", "warp"),
                          ("f64", "auto")):
        sim = nbgb.Sim(prec).set_shot(s).set_variant(variant)
        sim.add_spots()
        if variant == "warp":
            # counted only by the counting instantiation
            w = sim.work()
            assert w["pairs"] == w["intervals"] == w["blocks"] == -1
            img = sim.image()
            sim.count_work(True).zero()
            sim.add_spots()
            # which counts the same sum
            assert np.array_equal(sim.image(), img)
        w = sim.work()
        ev, ps = sim.stats()
        sim.close()
        assert w["pixel_steps"] == ps == s.pixel_steps
        assert w["units"] == units
        assert w["items"] == units * s.n_mosaic * s.n_phi
        if prec == "f64":
            assert w["pairs"] == w["terms"] == ps
            continue
        assert w["terms"] == ev
        if variant == "thread":
            assert w["pairs"] == ps and w["intervals"] == w["blocks"] == 0
        else:
            # N = 25: the exact intervals apply (block tests only where an
            # item's sweep reaches more than 8 lattice points); they skip
            # most steps and keep every surviving term
            assert w["intervals"] > 0
            assert ev <= w["pairs"] < ps


@pytest.mark.parametrize("precision", ["mixed", "f64"])
def test_fcell_device_upload_equals_host_upload(precision):
    """nb_set_fcell_device replaces the table's values from device memory:
    the image equals the one with the same table given on the host, for the
    nearest and the tricubic lookups and for the tables derived from F (the
    cell polynomials of NB_MIXED, the FP64 copy of NB_F64), which a launch
    before the replacement has built; a wrong size is rejected."""
    torch = pytest.importorskip("torch")
    for interp in (W.INTERP_NEAREST, W.INTERP_TRICUBIC):
        s = W.shrink(W.large_shot(), 24, 16, 2500, 700)
        s.interp = interp
        F2 = (s.F * np.float32(1.25) + np.float32(3.0)).astype(np.float32)
        t = s.copy()
        t.F = F2
        variant = "warp" if precision == "mixed" else "auto"
        ref = nbgb.simulate(t, precision, variant=variant)
        sim = nbgb.Sim(precision).set_shot(s).set_variant(variant)
        sim.add_spots()  # builds the derived tables of the first table
        dF = torch.from_numpy(F2).cuda()
        torch.cuda.synchronize()
        sim.set_fcell_device(dF.data_ptr(), dF.numel())
        sim.zero()
        sim.add_spots()
        got = sim.image()
        with pytest.raises(nbgb.NbError) as e:
            sim.set_fcell_device(dF.data_ptr(), dF.numel() - 1)
        assert e.value.code == nbgb.NB_EINVAL
        # the host route (nb_set_crystal with a new table) as well
        sim.upload_F(s.F)
        sim.zero()
        sim.add_spots()
        back = sim.image()
        sim.close()
        np.testing.assert_array_equal(got, ref)
        np.testing.assert_array_equal(
            back, nbgb.simulate(s, precision, variant=variant))
        assert back.max() > 0 and not np.array_equal(back, got)


def test_refused_allocations_fail_cleanly_and_leave_the_handle_usable():
    """Failure detection with the allocation-failure hook (no GPU fault): a
    call whose buffer is refused returns NB_ENOMEM and the handle works
    once memory is there; a refused table derived from F (the FP64 copy)
    makes the launch read F itself, with the same image."""
    base = W.shrink(W.large_shot(), 24, 16, 2500, 700)
    ref = nbgb.simulate(base, "f64")
    sim = nbgb.Sim("f64")
    try:
        sim.fail_allocations(1)
        with pytest.raises(nbgb.NbError) as e:
            sim.set_shot(base)  # the F table's buffer is the first
        assert e.value.code == nbgb.NB_ENOMEM
        sim.fail_allocations(0)
        sim.set_shot(base)
        sim.add_spots()
        np.testing.assert_array_equal(sim.image(), ref)
        # a larger table: its FP64 copy is the launch's only new buffer
        big = base.copy()
        big.F = W.structure_factors(np.random.default_rng(1), 62)
        big.hkl_min = np.array([-62, -62, -62], dtype=np.int32)
        ref_big = nbgb.simulate(big, "f64")
        sim.set_crystal(big)
        sim.fail_allocations(1)
        sim.zero()
        sim.add_spots()
        got = sim.image()
        # the refusal was spent on the FP64 copy: a new handle's buffers
        # are all granted
        probe = nbgb.Sim("f64").set_shot(base)
        probe.close()
        np.testing.assert_array_equal(got, ref_big)
    finally:
        sim.fail_allocations(0)
        sim.close()


def test_single_pixel_and_empty_list():
    s = W.shrink(W.single_shot_small(), 1, 1, 200, 170)
    ref = oracle.image(s)
    check_f64(run(s, "f64"), ref) if ref.max() > 0 else None
    sim = nbgb.Sim("mixed").set_shot(s)
    sim.add_spots(np.zeros(0, dtype=np.int64))
    assert not sim.image().any()
    sim.close()


def test_bad_arguments_are_rejected():
    s = W.single_shot_small()
    sim = nbgb.Sim("mixed")
    with pytest.raises(nbgb.NbError) as e:
        sim.add_spots()
    assert e.value.code == nbgb.NB_ESTATE
    sim.set_shot(s)
    with pytest.raises(nbgb.NbError) as e:
        sim.add_spots([sim.npix])
    assert e.value.code == nbgb.NB_EINVAL
    bad = s.copy()
    bad.ncells = np.array([10.5, 10.0, 10.0])
    with pytest.raises(nbgb.NbError) as e:
        sim.set_crystal(bad)
    assert e.value.code == nbgb.NB_EINVAL
    bad = s.copy()
    bad.lambdas = np.array([-1.0])
    with pytest.raises(nbgb.NbError):
        sim.set_beam(bad)
    bad = s.copy()
    bad.n_layers = 2
    with pytest.raises(nbgb.NbError):
        sim.set_detector(bad)
    assert sim.lib.nb_get_image(sim.h, None, sim.npix, 1, 0) == nbgb.NB_EINVAL
    out = np.empty(3)
    assert sim.lib.nb_get_image(sim.h, out.ctypes.data_as(nbgb._vp), 3, 1,
                                0) == nbgb.NB_EINVAL
    sim.close()


@pytest.mark.parametrize("precision,n_pm", [("mixed", 2048), ("f64", 1592)])
def test_largest_tables_that_fit_and_one_more(precision, n_pm):
    """Maximum sizes: 1024 sources (the nb_set_beam limit) with n_pm mosaic
    orientations, the most whose tables fit the kernels' 200 KB of shared
    memory: (18 PM + 12 S) x 4 bytes for the FP32 forms (so the
    nb_set_crystal limit of 2048), (9 PM + 11 S) x 8 bytes for FP64.  That
    shot matches the oracle on one 16x8 tile; one orientation or one
    source more is rejected with NB_EINVAL."""
    s = W.shrink(W.single_shot_small(), 16, 8, 150, 140)
    s.dirs, s.lambdas, s.weights = W.gaussian_spectrum(1024, 9.5, 0.005)
    rng = np.random.default_rng(5)
    s.umats = W.mosaic_umats(rng, n_pm, 0.05)
    assert s.n_mosaic * s.n_phi == n_pm and s.n_src == 1024
    ref = oracle.image(s)
    got = run(s, precision)
    (check_f64 if precision == "f64" else check_mixed)(got, ref)
    t = s.copy()
    t.umats = W.mosaic_umats(rng, n_pm + 1, 0.05)
    sim = nbgb.Sim(precision)
    with pytest.raises(nbgb.NbError) as e:
        sim.set_shot(t)  # n_pm + 1 > 2048 fails here, in nb_set_crystal
        sim.add_spots()  # FP64 tables over 200 KB fail here
    assert e.value.code == nbgb.NB_EINVAL
    sim.close()
    t = s.copy()
    t.dirs, t.lambdas, t.weights = W.gaussian_spectrum(1025, 9.5, 0.005)
    sim = nbgb.Sim(precision)
    with pytest.raises(nbgb.NbError) as e:
        sim.set_shot(t)
    assert e.value.code == nbgb.NB_EINVAL
    sim.close()


# ------------------------------------- full-size large shot, sampled rows


def test_large_shot_full_size_sampled_rows():
    """The whole 3072x3072 image in the launch configuration the benchmark
    times; the oracle computes three full rows (9216 pixels) of it."""
    s = W.large_shot()
    rows = [700, 1500, 2417]
    pix = np.concatenate([np.arange(r * 3072, (r + 1) * 3072) for r in rows])
    ref = oracle.image(s, pix)
    for variant in ("auto", "thread"):
        got = run(s, "mixed", variant=variant)[pix]
        check_mixed(got, ref)


def test_fp64_peak_probe_is_plausible():
    """The FP64 roofline's denominator: GB300's nominal FP64 rate is
    1.25 TFLOP/s (152 SMs at 2.07 GHz); the probe must land near it, and a
    second call must agree (it times the best of three launches)."""
    p1 = nbgb.fp64_peak_tflops(0)
    p2 = nbgb.fp64_peak_tflops(0)
    assert 0.3 < p1 < 3.0, p1
    assert abs(p1 - p2) <= 0.2 * max(p1, p2), (p1, p2)
    with pytest.raises(nbgb.NbError):
        nbgb.fp64_peak_tflops(10_000)
