"""Host-side input recipes that feed both the oracle and the kernels, and
the flop counts of the roofline figures (no GPU)."""
import numpy as np

from paper_2205_07976_gb300 import flops
from paper_2205_07976_gb300 import workloads as W


def test_amorphous_background_recipe():
    for uneven in (False, True):
        bg = W.amorphous_background(64, uneven=uneven)
        assert bg.stol.shape == bg.F.shape == (64,)
        assert bg.stol[0] == 0.0 and bg.stol[-1] == 1.0
        assert np.all(np.diff(bg.stol) > 0)
        assert np.all(bg.F > 0)
        # the water ring: the curve peaks near stol = 0.16 / A
        assert abs(bg.stol[np.argmax(bg.F)] - 0.16) < 0.03
    even = W.amorphous_background(64).stol
    dense = W.amorphous_background(64, uneven=True).stol
    assert dense[1] < even[1]  # uneven knots crowd towards stol = 0


def test_gaussian_spectrum_is_equispaced_and_normalised():
    dirs, lam, w = W.gaussian_spectrum(100, 9.5, 0.005)
    E = 12.398419843 / lam
    np.testing.assert_allclose(np.diff(E), np.diff(E)[0], rtol=1e-9)
    assert abs(w.sum() - 1.0) < 1e-12
    assert abs(E.mean() - 9.5) < 1e-9
    # E0 +- 3 sigma with FWHM = 0.5 % of E0
    sigma = 0.005 * 9.5 / (2.0 * np.sqrt(2.0 * np.log(2.0)))
    assert abs((E.max() - E.min()) - 6 * sigma) < 1e-9


def test_flop_counts_scale_with_the_loop_nest():
    s = W.large_shot(n=64)
    a = flops.algorithmic_flops(s, 0)
    b = flops.algorithmic_flops(s, 1000)
    assert b > a > 0
    t = s.copy()
    t.lambdas = np.concatenate([s.lambdas, s.lambdas])
    t.weights = np.concatenate([s.weights, s.weights]) / 2
    t.dirs = np.concatenate([s.dirs, s.dirs])
    # twice the sources: twice the per-step work, the same per-unit work
    steps = s.npix * s.oversample ** 2 * s.n_layers * s.n_mosaic * s.n_src
    assert flops.algorithmic_flops(t, 0) - a == \
        steps * (flops.STEP_HKL + flops.STEP_GAUSS)
    bg1, bg2 = flops.background_flops(s), flops.background_flops(t)
    units = s.npix * s.oversample ** 2 * s.n_layers
    assert bg2 - bg1 == units * flops.BG_STEP * s.n_src
    assert abs(flops.fp32_peak_tflops(152, 2070.0) - 80.54784) < 1e-9
    # the FP64 form evaluates every step as a term: per step hkl (9) +
    # Gaussian (8) + term (exp 3, tricubic 198, accumulate 4) = 222, plus
    # the per-item and per-unit work
    per_px = flops.f64_flops(s, 1)
    items = s.oversample ** 2 * s.n_layers * s.n_mosaic * s.n_phi
    units = s.oversample ** 2 * s.n_layers
    assert per_px == 222 * s.steps_per_pixel + flops.ITEM * items + \
        flops.UNIT * units
    assert flops.f64_flops(s, 10) == 10 * per_px
