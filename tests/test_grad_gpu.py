"""Gradients of the Poisson image loss through the hand-written adjoint
(nb_adjoint, FP32-mixed), against the FP64 oracle's analytic gradient and
against central finite differences of the GPU FP64 forward."""
import numpy as np
import pytest

import oracle
from paper_2205_07976_gb300 import nbgb
from paper_2205_07976_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

BKG = 1.0
THETA_TRUE = dict(rot=np.zeros(3), cell=np.array([79.0, 79.0, 38.0]),
                  N=np.array([15.0, 15.0, 15.0]), scale=1.0)
THETA = dict(rot=np.array([3e-4, -2e-4, 1e-4]),
             cell=np.array([79.05, 78.97, 38.02]),
             N=np.array([14.5, 15.5, 15.2]), scale=1.1)


def grad_shot(n_src, interp=W.INTERP_NEAREST, n_phi=1):
    """2x2 panels of 41x37 pixels (0.11 mm) around the brightest pixel of
    a 120x120 survey of the multi-panel shot (10 domains, N=15 Gaussian,
    table on [-40,40]^3), with the given lookup and phi steps of 0.02 deg
    about the spindle."""
    s = W.multipanel_shot(n_src, tiles=(1, 1), panel=(120, 120))
    s.interp = interp
    s.n_phi = n_phi
    s.phistep_deg = 0.02
    U = W.random_orientation(np.random.default_rng(3))
    img = oracle.image(s).reshape(120, 120)
    js, jf = np.unravel_index(np.argmax(img), img.shape)
    p = s.panels[0]
    c = p.origin + (jf + 0.5) * p.pixel_m * p.fdir + (js + 0.5) * p.pixel_m * p.sdir
    panels = []
    for ts in range(2):
        for tf in range(2):
            o = c + (tf * 42 - 41) * p.pixel_m * p.fdir + (ts * 38 - 37) * p.pixel_m * p.sdir
            panels.append(W.Panel(origin=o, fdir=p.fdir, sdir=p.sdir,
                                  ndir=p.ndir, pixel_m=p.pixel_m, nfast=41,
                                  nslow=37))
    s.panels = panels
    return s, U


def with_theta(shot, U, th):
    t = shot.copy()
    t.axes, _ = oracle.param_axes(U, th["cell"], th["rot"])
    t.ncells = th["N"].copy()
    t.scale = th["scale"]
    return t


CASES = [(1, W.INTERP_NEAREST, 1), (2, W.INTERP_NEAREST, 1),
         (1, W.INTERP_TRICUBIC, 1), (2, W.INTERP_TRICUBIC, 3)]


@pytest.fixture(scope="module", params=CASES,
                ids=["nearest-S1", "nearest-S2", "tricubic-S1",
                     "tricubic-S2-phi3"])
def case(request):
    shot, U = grad_shot(*request.param)
    truth = oracle.image(with_theta(shot, U, THETA_TRUE))
    y = np.random.default_rng(7).poisson(truth + BKG).astype(np.float64)
    s = with_theta(shot, U, THETA)
    L, g, gF, model = oracle.loss_grad(s, U, THETA["cell"], THETA["rot"], y,
                                       BKG)
    return shot, U, y, (L, g, gF, model)


def gpu_grad(shot, U, y, th, precision="mixed"):
    dev = torch.device("cuda", 0)
    sim = nbgb.Sim(precision).set_shot(with_theta(shot, U, th))
    sim.set_params(U, th["cell"], th["rot"], th["N"], th["scale"])
    sim.add_spots()
    yd = torch.from_numpy(y).to(dev)
    dL = torch.empty_like(yd)
    torch.cuda.synchronize()
    L = sim.poisson_loss(yd.data_ptr(), BKG, dL.data_ptr())
    if precision != "mixed":
        return L, None, None, sim.image()
    gF = torch.zeros(shot.F.size, dtype=torch.float64, device=dev)
    g = sim.adjoint(dL.data_ptr(), gF.data_ptr())
    img = sim.image()
    sim.close()
    return L, g, gF.cpu().numpy().reshape(shot.F.shape), img


def test_adjoint_matches_oracle_gradient(case):
    shot, U, y, (L0, g0, gF0, model0) = case
    L, g, gF, img = gpu_grad(shot, U, y, THETA)
    assert abs(L - L0) <= 1e-6 * abs(L0)
    gmax = np.abs(g0).max()
    for r in range(10):
        assert abs(g[r] - g0[r]) <= 1e-4 * abs(g0[r]) + 1e-6 * gmax, (
            r, g[r], g0[r])
    assert np.abs(gF - gF0).max() <= 1e-4 * np.abs(gF0).max()
    big = np.abs(gF0) > 1e-2 * np.abs(gF0).max()
    assert big.sum() >= 3
    np.testing.assert_allclose(gF[big], gF0[big], rtol=1e-4)


@pytest.mark.parametrize("interp", [W.INTERP_NEAREST, W.INTERP_TRICUBIC],
                         ids=["nearest", "tricubic"])
def test_adjoint_full_size_matches_oracle(interp):
    """The differentiation workload at its full size, as the benchmark runs
    it: 64 panels of 185x194 pixels, 8 sources, 10 domains, N=15 Gaussian,
    table on [-40,40]^3 (2.3e6 pixels, 1.8e8 pixel-steps).  The target is a
    Poisson draw of the oracle's image at the true parameters; loss, the 10
    scalars and every structure-factor gradient against the oracle's."""
    shot = W.multipanel_shot(8)
    shot.interp = interp
    U = W.random_orientation(np.random.default_rng(3))
    truth = oracle.image(with_theta(shot, U, THETA_TRUE))
    y = np.random.default_rng(7).poisson(truth + BKG).astype(np.float64)
    L0, g0, gF0, _ = oracle.loss_grad(with_theta(shot, U, THETA), U,
                                      THETA["cell"], THETA["rot"], y, BKG)
    L, g, gF, _ = gpu_grad(shot, U, y, THETA)
    assert abs(L - L0) <= 1e-6 * abs(L0)
    gmax = np.abs(g0).max()
    for r in range(10):
        assert abs(g[r] - g0[r]) <= 1e-4 * abs(g0[r]) + 1e-6 * gmax, (
            r, g[r], g0[r])
    assert np.abs(gF - gF0).max() <= 1e-4 * np.abs(gF0).max()
    big = np.abs(gF0) > 1e-2 * np.abs(gF0).max()
    assert big.sum() >= 10
    np.testing.assert_allclose(gF[big], gF0[big], rtol=1e-4)


def test_adjoint_matches_fd_of_f64_forward(case):
    shot, U, y, (L0, g0, _, _) = case
    _, g, _, _ = gpu_grad(shot, U, y, THETA)
    x0 = np.concatenate([THETA["rot"], THETA["cell"], THETA["N"],
                         [THETA["scale"]]])

    def loss_f64(x):
        th = dict(rot=x[0:3], cell=x[3:6], N=x[6:9], scale=x[9])
        sim = nbgb.Sim("f64").set_shot(with_theta(shot, U, th))
        sim.set_params(U, th["cell"], th["rot"], th["N"], th["scale"])
        sim.add_spots()
        m = sim.image() + BKG
        sim.close()
        return float(np.sum(m - y * np.log(m)))

    for r in range(10):
        h = 1e-6 if r < 3 else 1e-6 * abs(x0[r])
        xp, xm = x0.copy(), x0.copy()
        xp[r] += h
        xm[r] -= h
        fd = (loss_f64(xp) - loss_f64(xm)) / (2 * h)
        # the oracle's analytic gradient is exact up to FD's own error
        assert abs(fd - g0[r]) <= 1e-5 * abs(g0[r]) + 1e-6 * np.abs(g0).max()
        # the FP32-mixed adjoint, at the mixed tolerance
        assert abs(fd - g[r]) <= 1e-4 * abs(fd) + 1e-6 * np.abs(g0).max(), (
            r, fd, g[r])


def test_autograd_function_matches_adjoint(case):
    from paper_2205_07976_gb300.autograd import bragg_image
    shot, U, y, _ = case
    dev = torch.device("cuda", 0)
    sim = nbgb.Sim("mixed").set_shot(with_theta(shot, U, THETA))
    params = torch.tensor(np.concatenate([THETA["rot"], THETA["cell"],
                                          THETA["N"], [THETA["scale"]]]),
                          dtype=torch.float64, requires_grad=True)
    # a float64 leaf gets a float64 gradient (autograd casts to the
    # input's dtype); the table itself is uploaded as float32 either way
    F = torch.from_numpy(shot.F.astype(np.float64)).requires_grad_(True)
    img = bragg_image(params, F, sim, U)
    yd = torch.from_numpy(y).to(dev)
    loss = (img + BKG - yd * torch.log(img + BKG)).sum()
    loss.backward()
    L, g, gF, _ = gpu_grad(shot, U, y, THETA)
    assert abs(loss.item() - L) <= 1e-9 * abs(L)
    np.testing.assert_allclose(params.grad.numpy(), g, rtol=1e-8,
                               atol=1e-12 * np.abs(g).max())
    np.testing.assert_allclose(F.grad.numpy(), gF, rtol=1e-8,
                               atol=1e-12 * np.abs(gF).max())
    sim.close()


def _params(th, device="cpu"):
    return torch.tensor(np.concatenate([th["rot"], th["cell"], th["N"],
                                        [th["scale"]]]),
                        dtype=torch.float64, device=device,
                        requires_grad=True)


def test_autograd_keeps_F_on_the_device(case):
    """A CUDA table is uploaded device to device, once: a second forward
    with the same unchanged tensor uploads nothing, an in-place change
    uploads again, and the gradients (on the devices of params and F) still
    equal the adjoint's."""
    from paper_2205_07976_gb300.autograd import bragg_image
    shot, U, y, _ = case
    dev = torch.device("cuda", 0)
    sim = nbgb.Sim("mixed").set_shot(with_theta(shot, U, THETA))
    params = _params(THETA, dev)
    F = torch.from_numpy(shot.F.astype(np.float32)).to(dev).requires_grad_(
        True)
    yd = torch.from_numpy(y).to(dev)
    bragg_image(params, F, sim, U)
    assert sim.F_uploads == 1
    img = bragg_image(params, F, sim, U)
    assert sim.F_uploads == 1
    loss = (img + BKG - yd * torch.log(img + BKG)).sum()
    loss.backward()
    assert sim.F_uploads == 1
    assert params.grad.device == dev and F.grad.device == dev
    L, g, gF, _ = gpu_grad(shot, U, y, THETA)
    assert abs(loss.item() - L) <= 1e-9 * abs(L)
    np.testing.assert_allclose(params.grad.cpu().numpy(), g, rtol=1e-8,
                               atol=1e-12 * np.abs(g).max())
    # F is float32, so autograd hands back its gradient in float32
    assert F.grad.dtype == torch.float32
    np.testing.assert_allclose(F.grad.cpu().numpy(), gF, rtol=1.2e-7,
                               atol=1e-12 * np.abs(gF).max())
    with torch.no_grad():
        F.mul_(1.0)  # same values, new version
    bragg_image(params, F, sim, U)
    assert sim.F_uploads == 2
    sim.close()


def test_autograd_two_forwards_then_backward(case):
    """Two forwards on one handle at different parameters and tables, then
    the first one's backward: its gradient is the one at its own point."""
    from paper_2205_07976_gb300.autograd import bragg_image
    shot, U, y, _ = case
    dev = torch.device("cuda", 0)
    sim = nbgb.Sim("mixed").set_shot(with_theta(shot, U, THETA))
    p1 = _params(THETA)
    F1 = torch.from_numpy(shot.F.astype(np.float32)).to(dev).requires_grad_(
        True)
    th2 = dict(rot=THETA["rot"] * -1.5, cell=THETA["cell"] + 0.02,
               N=THETA["N"] + 0.3, scale=0.9)
    p2 = _params(th2)
    F2 = (F1.detach() * 1.05).requires_grad_(True)
    yd = torch.from_numpy(y).to(dev)
    img1 = bragg_image(p1, F1, sim, U)
    img2 = bragg_image(p2, F2, sim, U)
    loss1 = (img1 + BKG - yd * torch.log(img1 + BKG)).sum()
    loss1.backward()
    L, g, gF, _ = gpu_grad(shot, U, y, THETA)
    np.testing.assert_allclose(p1.grad.numpy(), g, rtol=1e-8,
                               atol=1e-12 * np.abs(g).max())
    np.testing.assert_allclose(F1.grad.cpu().numpy(), gF, rtol=1.2e-7,
                               atol=1e-12 * np.abs(gF).max())
    # and the second forward's image was its own
    s2 = with_theta(shot, U, th2)
    s2.F = (shot.F.astype(np.float32) * np.float32(1.05))
    sim2 = nbgb.Sim("mixed").set_shot(s2)
    sim2.set_params(U, th2["cell"], th2["rot"], th2["N"], th2["scale"])
    sim2.add_spots()
    np.testing.assert_array_equal(img2.detach().cpu().numpy(), sim2.image())
    sim2.close()
    sim.close()


def test_adjoint_rejects_unsupported_setups():
    shot, U = grad_shot(1)
    sim = nbgb.Sim("mixed").set_shot(shot)
    dev = torch.device("cuda", 0)
    buf = torch.zeros(sim.npix, dtype=torch.float64, device=dev)
    with pytest.raises(nbgb.NbError) as e:
        sim.adjoint(buf.data_ptr())
    assert e.value.code == nbgb.NB_ESTATE  # no nb_set_crystal_params yet
    t = shot.copy()
    t.shape = W.SHAPE_SINC
    sim.set_crystal(t)
    # sinc F_latt takes whole cell counts only
    with pytest.raises(nbgb.NbError) as e:
        sim.set_params(U, THETA["cell"], THETA["rot"], THETA["N"], 1.0)
    assert e.value.code == nbgb.NB_EINVAL
    sim.set_params(U, THETA["cell"], THETA["rot"], THETA_TRUE["N"], 1.0)
    with pytest.raises(nbgb.NbError) as e:
        sim.adjoint(buf.data_ptr())
    assert e.value.code == nbgb.NB_EINVAL  # sinc F_latt has no adjoint
    sim.close()
    sim = nbgb.Sim("f64").set_shot(shot)
    sim.set_params(U, THETA["cell"], THETA["rot"], THETA["N"], 1.0)
    with pytest.raises(nbgb.NbError) as e:
        sim.adjoint(buf.data_ptr())
    assert e.value.code == nbgb.NB_EINVAL  # the adjoint is FP32-mixed only
    sim.close()
