"""Algorithmic work of the Bragg-spot sum, for the roofline figure.

The count is the method's own arithmetic in FP32 flops (an FMA is 2), with
the loop invariants hoisted as the definition allows, independent of how a
kernel implements it (the double-float emulation of the fractional offset
in NB_MIXED costs ~3x more instructions and is NOT counted):

  per pixel-step (every step)
    h_x = G_x u_k + r_x (one FMA per axis)                      6
    f_x = h_x - rint(h_x)                                        3
    Gaussian: sum_x (N_x f_x)^2                                  8
    sinc:     per axis N f, reduction, sin(pi y) and sin(pi f)
              as degree-11 odd polynomials (14 flops each);
              the product and one division                     96
  per evaluated term (Gaussian terms whose F_latt^2 underflows in FP32
  are not evaluated; sinc terms always are)
    Gaussian: exponent scale, exp, (Na Nb Nc)^2                  3
    tricubic: 3 x 4 Lagrange weights (10 each) + 84 FMAs      198
    term = F^2 F_latt^2 w and its accumulation                   4
  per (subpixel, layer, phi x mosaic) item
    G = A . (d - i0): 3 dot products, r = u0 G - n0            21
  per (subpixel, layer) unit
    position, |P|, d, solid angle, capture, polarization      60
"""
from __future__ import annotations

STEP_HKL = 6 + 3
STEP_GAUSS = 8
STEP_SINC = 96
TERM_GAUSS = 3
TERM_TRICUBIC = 198
TERM_ACCUM = 4
ITEM = 21
UNIT = 60


def algorithmic_flops(shot, evaluated_terms: int, pixels: int = None) -> float:
    """FP32 flops of one image of `shot` (or of `pixels` of its pixels),
    given the number of evaluated terms reported by nb_get_stats."""
    npix = shot.npix if pixels is None else pixels
    units = npix * shot.oversample ** 2 * shot.n_layers
    items = units * shot.n_mosaic * shot.n_phi
    steps = items * shot.n_src
    per_step = STEP_HKL + (STEP_GAUSS if shot.shape == 1 else STEP_SINC)
    per_term = TERM_ACCUM + (TERM_GAUSS if shot.shape == 1 else 0) + (
        TERM_TRICUBIC if shot.interp == 1 else 0)
    return float(per_step * steps + per_term * evaluated_terms
                 + ITEM * items + UNIT * units)


# Work the kernels perform (nb_get_work counts) rather than the method's
# count.  The warp-per-pixel kernel does not visit every step: per item it
# bounds the lattice points its source sweep can reach, solves one source
# interval per lattice point (or tests 8-source blocks), and forms the
# offset and the cut test only for the (interval, source) pairs inside:
#   per pair tested: h and f (9) and the Gaussian exponent (8)          17
#   per interval: A, B, C of the quadratic in delta (3 x 8), its
#     discriminant, root and reciprocal (5), bounds and margins (8),
#     the lattice point's offsets (3)                                    40
#   per block test: per axis 2 FMAs, 2 margins, floor and ceil (3 x 6)   18
#   per item: G, r (21) and the lattice range per axis (3 x 6)           39
PAIR = STEP_HKL + STEP_GAUSS
INTERVAL = 40
BLOCK = 18
ITEM_RANGE = 18


def performed_flops(shot, work: dict) -> float:
    """FP32 flops a launch performed, from the nb_get_work counts of that
    launch (keys of nbgb.WORK_NAMES).  For the thread-per-pixel kernels
    (every step tested, no intervals) this equals algorithmic_flops."""
    per_term = TERM_ACCUM + (TERM_GAUSS if shot.shape == 1 else 0) + (
        TERM_TRICUBIC if shot.interp == 1 else 0)
    if work["intervals"] == 0 and work["blocks"] == 0:
        per_pair = STEP_HKL + (STEP_GAUSS if shot.shape == 1 else STEP_SINC)
        item = ITEM
    else:
        per_pair = PAIR
        item = ITEM + ITEM_RANGE
    return float(per_pair * work["pairs"] + INTERVAL * work["intervals"]
                 + BLOCK * work["blocks"] + per_term * work["terms"]
                 + item * work["items"] + UNIT * work["units"])


def f64_flops(shot, pixels: int) -> float:
    """Flops of the plain FP64 form on `pixels` pixels of `shot`: the same
    count in FP64 arithmetic, with every step a term (NB_F64 skips none)."""
    steps = (pixels * shot.oversample ** 2 * shot.n_layers * shot.n_mosaic
             * shot.n_phi * shot.n_src)
    return algorithmic_flops(shot, steps, pixels)


# amorphous background, per (subpixel, layer, source) step: stol = sin(theta)
# u_k (1), linear interpolation (sub + FMA, 3), F^2 w (2), accumulate (1);
# per (subpixel, layer, direction): |d - i|, polarization (25); per
# (subpixel, layer): position, |P|, solid angle, capture (35)
BG_STEP = 7
BG_GROUP = 25
BG_UNIT = 35


def background_flops(shot, n_directions: int = 1) -> float:
    """FP32 flops of the amorphous background of every pixel of `shot`."""
    units = shot.npix * shot.oversample ** 2 * shot.n_layers
    return float(units * (BG_UNIT + BG_GROUP * n_directions
                          + BG_STEP * shot.n_src))


def fp32_peak_tflops(sm_count: int = 152, mhz: float = 2070.0) -> float:
    """FP32 FMA peak: SMs x 128 lanes x 2 flops x clock."""
    return sm_count * 128 * 2 * mhz * 1e6 / 1e12
