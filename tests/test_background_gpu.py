"""Amorphous background (nb_add_background) vs the FP64 oracle, element by
element, through the C ABI.  Tolerances as for the spots: NB_F64 1e-12
relative, NB_MIXED 1e-5 relative (the background is smooth, so every
pixel is above 1e-3 of the maximum)."""
import numpy as np
import pytest

import oracle
from paper_2205_07976_gb300 import nbgb
from paper_2205_07976_gb300 import workloads as W
from tests.helpers import abs_err_frac, masked_rel_err

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "mixed": 1e-5}


def bg_image(shot, bg, precision, spots=False):
    sim = nbgb.Sim(precision).set_shot(shot).set_background(bg)
    try:
        if spots:
            sim.add_spots()
        sim.add_background()
        return sim.image()
    finally:
        sim.close()


def check(got, ref, precision):
    rel, _ = masked_rel_err(got, ref, 1e-3)
    assert rel <= TOL[precision], rel
    assert abs_err_frac(got, ref) <= TOL[precision]


def window_shot(n_src=100, kahn=0.99, os_=2, layers=2):
    """A 75x53 window (ragged 16x8 tiles) of the 3072x3072 large-shot
    detector, off the beam, with its spectrum, sensor and polarization."""
    s = W.shrink(W.large_shot(n_src=n_src, n_mosaic=2), 75, 53, 1400, 900)
    s.kahn = kahn
    s.oversample = os_
    s.n_layers = layers
    return s


@pytest.mark.parametrize("precision", ["f64", "mixed"])
@pytest.mark.parametrize("uneven", [False, True])
def test_background_matches_oracle(precision, uneven):
    s = window_shot()
    bg = W.amorphous_background(64, uneven=uneven)
    check(bg_image(s, bg, precision), oracle.background(s, bg), precision)


@pytest.mark.parametrize("precision", ["f64", "mixed"])
def test_background_beam_centre_and_table_edges(precision):
    # a panel around the direct beam (stol -> 0 at the centre) with a table
    # that starts above 0 and ends inside the detector's range: both held
    # ends and every knot bracket are used
    s = W.single_shot_small(n=67)
    s.panels = [W.flat_detector(67, 45, 1e-3, 0.05)]
    s.dirs, s.lambdas, s.weights = W.gaussian_spectrum(7, 9.5, 0.005)
    bg = W.Background(stol=np.linspace(0.02, 0.3, 29),
                      F=2.0 + np.sin(np.arange(29.0)), n_molecules=1e10)
    check(bg_image(s, bg, precision), oracle.background(s, bg), precision)


@pytest.mark.parametrize("precision", ["f64", "mixed"])
def test_background_divergent_sources_and_panels(precision):
    # three source directions, each with several wavelengths in arbitrary
    # order, on the 64-panel tiled detector (two panels kept)
    s = W.multipanel_shot(1)
    s.panels = s.panels[:2]
    rng = np.random.default_rng(11)
    dirs, lams, ws = [], [], []
    for tilt in (0.0, 2e-3, -1.5e-3):
        d = np.array([tilt, 0.5 * tilt, 1.0])
        d /= np.linalg.norm(d)
        for lam in rng.uniform(1.0, 1.4, 4):
            dirs.append(d)
            lams.append(lam)
            ws.append(rng.uniform(0.5, 1.5))
    order = rng.permutation(len(lams))
    s.dirs = np.array(dirs)[order]
    s.lambdas = np.array(lams)[order]
    s.weights = np.array(ws)[order] / np.sum(ws)
    s.kahn = 0.7
    bg = W.amorphous_background(200, uneven=True)
    check(bg_image(s, bg, precision), oracle.background(s, bg), precision)


@pytest.mark.parametrize("n_knots", [2, 4096])
def test_background_table_sizes(n_knots):
    s = window_shot(n_src=5, os_=1, layers=1)
    bg = W.amorphous_background(n_knots, stol_max=0.6)
    for precision in ("f64", "mixed"):
        check(bg_image(s, bg, precision), oracle.background(s, bg),
              precision)


def test_background_adds_onto_the_spots_image():
    s = W.shrink(W.single_shot_small(), 61, 37, 100, 120)
    bg = W.amorphous_background(64)
    both = bg_image(s, bg, "f64", spots=True)
    spots = nbgb.simulate(s, "f64")
    alone = bg_image(s, bg, "f64")
    np.testing.assert_array_equal(both, spots + alone)


def test_background_full_detector_sampled_rows():
    # the 3072x3072 large-shot detector with its 100 sources, oversample 2
    # and two layers, every pixel on the GPU; every 97th row by the oracle
    s = W.large_shot(n_mosaic=1)
    bg = W.amorphous_background(64)
    img = bg_image(s, bg, "mixed")
    rows = W.strided_rows(s, 97)
    ref = oracle.background(s, bg, rows)
    check(img[rows], ref, "mixed")
    assert np.all(img > 0)


def test_background_argument_errors():
    s = W.shrink(W.single_shot_small(), 16, 8)
    sim = nbgb.Sim("mixed").set_shot(s)
    with pytest.raises(nbgb.NbError) as e:
        sim.add_background()
    assert e.value.code == nbgb.NB_ESTATE
    bad = [W.Background(stol=np.array([0.0]), F=np.array([1.0]),
                        n_molecules=1.0),
           W.Background(stol=np.array([0.0, 0.0]), F=np.array([1.0, 1.0]),
                        n_molecules=1.0),
           W.Background(stol=np.array([0.0, 1.0]),
                        F=np.array([1.0, np.nan]), n_molecules=1.0),
           W.Background(stol=np.array([0.0, 1.0]), F=np.array([1.0, 1.0]),
                        n_molecules=-1.0),
           W.Background(stol=np.linspace(0, 1, 4097), F=np.ones(4097),
                        n_molecules=1.0)]
    for b in bad:
        with pytest.raises(nbgb.NbError) as e:
            sim.set_background(b)
        assert e.value.code == nbgb.NB_EINVAL
    sim.close()
