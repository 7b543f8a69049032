"""The bounds-checked debug build (-DNB_CHECK=1) on small cases of every
kernel, against the FP64 oracle.  Its kernels check each table and image
index before use and make the call fail with the site and index instead
of reading out of bounds; here every case must pass the checks and still
match the oracle.  The cases run in a child process that loads the check
build (NBGB_VARIANT=check), so the release library of this process is
not replaced."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import numpy as np
import oracle
from paper_2205_07976_gb300 import nbgb
from paper_2205_07976_gb300 import workloads as W
from tests.helpers import masked_rel_err, rel_err_above

assert nbgb.load().nb_version().decode().endswith("+check")

def close(got, ref, tol, floor):
    rel, n = masked_rel_err(got, ref, floor)
    assert rel <= tol, (rel, n)

def close64(got, ref):
    rel, n = rel_err_above(got, ref, 1e-250)
    assert rel <= 1e-12, (rel, n)

# single shot (sinc, nearest): FP64, FP32-mixed, FP32
s = W.shrink(W.single_shot_small(), 37, 21, 150, 140)
ref = oracle.image(s)
close64(nbgb.simulate(s, "f64"), ref)
close(nbgb.simulate(s, "mixed"), ref, 1e-5, 1e-3)
assert np.isfinite(nbgb.simulate(s, "f32")).all()
# a large-shot window with spots (Gaussian, tricubic): both FP32-mixed
# kernels, FP64 on a few rows
s = W.shrink(W.large_shot(), 21, 13, 2500, 700)
ref = oracle.image(s)
assert ref.max() > 1e-6
for v in ("warp", "thread"):
    close(nbgb.simulate(s, "mixed", variant=v), ref, 1e-5, 1e-3)
rows = np.arange(2 * 21)
close64(nbgb.simulate(s, "f64", pixels=rows), ref[rows])
# the edge-case shot (a table smaller than the reached hkl, default_F,
# divergent sources, phi steps, layers): every shape and lookup
from tests.test_parity_gpu import _edge_shot
for shape in (0, 1):
    for interp in (0, 1):
        t = _edge_shot()
        t.shape, t.interp = shape, interp
        tref = oracle.image(t)
        close64(nbgb.simulate(t, "f64"), tref)
        for v in ("thread", "warp"):
            close(nbgb.simulate(t, "mixed", variant=v), tref, 1e-5, 1e-3)
# background
bg = W.amorphous_background(16)
sim = nbgb.Sim("mixed").set_shot(s).set_background(bg)
sim.add_background()
close(sim.image(), oracle.background(s, bg), 1e-5, 1e-3)
sim.close()
# adjoint, tricubic (term ring) and nearest, against the oracle gradient
import torch
from tests.test_grad_gpu import BKG, THETA, THETA_TRUE, grad_shot, with_theta
for interp in (W.INTERP_TRICUBIC, W.INTERP_NEAREST):
    shot, U = grad_shot(1, interp)
    truth = oracle.image(with_theta(shot, U, THETA_TRUE))
    y = np.random.default_rng(7).poisson(truth + BKG).astype(np.float64)
    m = with_theta(shot, U, THETA)
    L0, g0, gF0, _ = oracle.loss_grad(m, U, THETA["cell"], THETA["rot"], y,
                                      BKG)
    sim = nbgb.Sim("mixed").set_shot(m)
    sim.set_params(U, THETA["cell"], THETA["rot"], THETA["N"],
                   THETA["scale"])
    sim.add_spots()
    yd = torch.from_numpy(y).cuda()
    dL = torch.empty_like(yd)
    torch.cuda.synchronize()
    L = sim.poisson_loss(yd.data_ptr(), BKG, dL.data_ptr())
    gF = torch.zeros(m.F.size, dtype=torch.float64, device="cuda")
    g = sim.adjoint(dL.data_ptr(), gF.data_ptr())
    sim.close()
    assert abs(L - L0) <= 1e-6 * abs(L0)
    gm = np.abs(g0).max()
    assert gm > 0
    assert np.all(np.abs(g - g0) <= 1e-4 * np.abs(g0) + 1e-6 * gm), (g, g0)
print("check build ok")
'''


def test_check_build_passes_its_checks_and_matches_the_oracle():
    env = dict(os.environ, NBGB_VARIANT="check")
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "check build ok" in r.stdout
