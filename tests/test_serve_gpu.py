"""The continuous-batching shot server (nb_server_*): each request's image
is bitwise the same alone and in the mix, equals the thread-per-pixel
kernel on the same pixels, matches the FP64 oracle at the FP32-mixed
tolerance, and admission respects the image pool and the slots."""
import numpy as np
import pytest

import oracle
from paper_2205_07976_gb300 import nbgb
from paper_2205_07976_gb300 import workloads as W
from tests.helpers import abs_err_frac, masked_rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def base():
    return W.serving_detector_shot()


def small_requests(n, seed):
    return W.serving_requests(n, seed=seed, max_src=12, max_mosaic=30,
                              min_pix=40, max_pix=2500)


def submit(srv, r):
    return srv.submit(r.axes, r.umats, r.lambdas, r.weights, r.scale, r.roi)


def run_alone(base, reqs):
    srv = nbgb.Server(base, max_slots=1, pool_bytes=64 << 20)
    out = []
    for r in reqs:
        rid = submit(srv, r)
        srv.run_all()
        out.append(srv.result(rid))
    srv.close()
    return out


def test_alone_equals_in_the_mix(base):
    reqs = small_requests(10, 11)
    alone = run_alone(base, reqs)
    # a small step budget forces many interleaved steps; later requests
    # arrive while earlier ones run
    srv = nbgb.Server(base, max_slots=4, pool_bytes=8 << 20,
                      step_budget=200000)
    ids = [submit(srv, r) for r in reqs[:5]]
    srv.step()
    srv.step()
    ids += [submit(srv, r) for r in reqs[5:]]
    done = srv.run_all()
    assert sorted(done) == sorted(ids)
    for rid, a in zip(ids, alone):
        b = srv.result(rid)
        assert np.array_equal(a, b)
    srv.close()


def test_server_equals_standalone_kernel_on_the_same_pixels(base):
    """The server runs each request with the kernel nb_add_spots would pick
    (one warp per pixel for >= 8 mosaic domains, else one thread per
    pixel): its images equal the stand-alone ones bit for bit."""
    reqs = W.serving_requests(6, seed=12, max_src=20, max_mosaic=40,
                              min_pix=40, max_pix=1500)
    assert any(r.umats.shape[0] >= 8 for r in reqs)
    assert any(r.umats.shape[0] < 8 for r in reqs)
    got = run_alone(base, reqs)
    for r, g in zip(reqs, got):
        s = base.copy()
        s.axes, s.umats = r.axes, r.umats
        s.lambdas, s.weights = r.lambdas, r.weights
        s.dirs = np.repeat(base.dirs[:1], len(r.lambdas), axis=0)
        f0, s0, nf, ns = r.roi
        pix = ((s0 + np.arange(ns))[:, None] * 3072
               + (f0 + np.arange(nf))[None, :]).ravel()
        sim = nbgb.Sim("mixed").set_shot(s)
        sim.add_spots(pix)
        ref = sim.image()[pix]
        sim.close()
        assert np.array_equal(g, ref)


def test_server_matches_oracle(base):
    reqs = small_requests(30, 13)
    got = run_alone(base, reqs)
    checked = 0
    for r, g in zip(reqs, got):
        ref = oracle.image(W.request_shot(base, r))
        if ref.max() < 1e-12:
            # no spot in the ROI: only Gaussian tails, which the FP32 forms
            # drop below FLT_MIN of the peak; compare in photons
            assert np.abs(g - ref).max() <= 1e-12
            continue
        rel, _ = masked_rel_err(g, ref, 1e-3)
        assert rel <= 1e-5
        assert abs_err_frac(g, ref) <= 1e-5
        checked += 1
    assert checked >= 3


def test_full_size_request_in_a_mix_matches_oracle_on_sampled_rows(base):
    """A request at the workload's largest sizes (a 2591x1351 ROI, 99
    sources, 49 domains: 1.7e10 pixel-steps, one warp per pixel) served
    between small ones with the benchmark's step budget of 2e9
    pixel-steps; the oracle computes six of its rows."""
    reqs = W.serving_requests(48, seed=40, min_pix=3.5e6, max_pix=4e6)
    big = max(reqs, key=lambda r: r.pixel_steps)
    assert big.pixel_steps > 1.5e10
    assert len(big.lambdas) >= 95 and big.umats.shape[0] >= 45
    others = small_requests(6, 41)
    srv = nbgb.Server(base, step_budget=2_000_000_000)
    ids = [submit(srv, r) for r in others[:3]]
    bid = submit(srv, big)
    ids += [submit(srv, r) for r in others[3:]]
    done = srv.run_all()
    assert sorted(done) == sorted(ids + [bid])
    got = srv.result(bid)
    srv.close()
    f0, s0, nf, ns = big.roi
    rows = [0, ns // 7, ns // 3, ns // 2, 2 * ns // 3, ns - 1]
    pix = np.concatenate([np.arange(r * nf, (r + 1) * nf) for r in rows])
    ref = oracle.image(W.request_shot(base, big), pix)
    assert (ref > 1e-3 * ref.max()).sum() >= 40
    rel, n = masked_rel_err(got[pix], ref, 1e-3)
    assert rel <= 1e-5, (rel, n)
    assert abs_err_frac(got[pix], ref) <= 1e-5


def test_admission_under_memory_pressure(base):
    reqs = small_requests(8, 14)
    alone = run_alone(base, reqs)
    biggest = max(r.npix for r in reqs)
    pool = int(1.5 * biggest) * 8  # room for one big request at a time
    srv = nbgb.Server(base, max_slots=8, pool_bytes=pool, step_budget=100000)
    ids = [submit(srv, r) for r in reqs]
    most = 0
    done = []
    while True:
        active = srv.step()
        info = srv.info()
        most = max(most, info["running"] + info["done"])
        assert info["pool_free_bytes"] >= 0
        for rid in srv.completed():
            done.append(rid)
        # fetch results as they complete, freeing slots and memory
        for rid in list(done):
            if srv.state(rid) == nbgb.NB_REQ_DONE:
                got = srv.result(rid)
                assert np.array_equal(got, alone[ids.index(rid)])
        if active == 0:
            break
    assert sorted(done) == sorted(ids)
    assert most < len(reqs)  # memory, not the slots, limited admission
    # a request larger than the whole pool is refused at submission
    big = W.ShotRequest(reqs[0].axes, reqs[0].umats, reqs[0].lambdas,
                        reqs[0].weights, 1.0, (0, 0, 3072, 3072))
    with pytest.raises(nbgb.NbError) as e:
        submit(srv, big)
    assert e.value.code == nbgb.NB_EINVAL
    srv.close()


def test_step_timeout_then_recovery(base):
    r = W.serving_requests(1, seed=15, max_src=100, max_mosaic=50,
                           min_pix=1e6, max_pix=2e6)[0]
    srv = nbgb.Server(base, max_slots=2, pool_bytes=64 << 20,
                      step_budget=1 << 62)
    rid = submit(srv, r)
    # the first step queues the whole request; the second has nothing new
    # to queue and waits for it, with no time to do so
    srv.step(timeout_s=0.0)
    with pytest.raises(nbgb.NbError) as e:
        srv.step(timeout_s=0.0)
    assert e.value.code == nbgb.NB_ETIMEOUT
    assert srv.state(rid) == nbgb.NB_REQ_RUNNING
    srv.run_all(timeout_s=60.0)
    assert srv.state(rid) == nbgb.NB_REQ_DONE
    img = srv.result(rid)
    assert img.shape == (r.npix,) and np.isfinite(img).all()
    srv.close()


def test_unfetched_results_stall_admission_instead_of_spinning(base):
    reqs = small_requests(3, 16)
    need = sorted(r.npix for r in reqs)
    srv = nbgb.Server(base, max_slots=4, pool_bytes=need[-1] * 8)
    ids = [submit(srv, r) for r in sorted(reqs, key=lambda r: -r.npix)]
    with pytest.raises(nbgb.NbError) as e:
        srv.run_all()
    assert e.value.code == nbgb.NB_ESTATE
    # fetching what completed frees the pool and the rest then runs
    for rid in ids:
        if srv.state(rid) == nbgb.NB_REQ_DONE:
            srv.result(rid)
    images = srv.run_all(fetch=True)
    assert len(images) >= 1
    srv.close()


def test_new_request_is_not_stuck_behind_a_large_old_one(base):
    """Half of each step's budget is shared equally by the running
    requests: a request submitted after a large one finishes within a few
    steps instead of advancing one work item per step."""
    # 3.4e6 pixels, 30 domains, 64 sources (33 budgets of work); 24198
    # pixels, 14 domains, 6 sources (378 warp-kernel items)
    big = W.serving_requests(1, seed=30, max_src=100, max_mosaic=50,
                             min_pix=2e6, max_pix=4e6)[0]
    small = W.serving_requests(1, seed=22, max_src=20, max_mosaic=20,
                               min_pix=2e4, max_pix=3e4)[0]
    assert big.pixel_steps > 30 * 2 * 10 ** 8 and small.npix > 300 * 64
    budget = 2 * 10 ** 8
    srv = nbgb.Server(base, max_slots=4, pool_bytes=64 << 20,
                      step_budget=budget)
    rb = submit(srv, big)
    srv.step()
    rs = submit(srv, small)
    steps = 0
    while srv.state(rs) != nbgb.NB_REQ_DONE:
        srv.step()
        steps += 1
        assert steps < 1000
    # the small request's share is budget / 4 per step (two requests
    # running); one more step for the pipelined completion
    share_steps = -(-small.pixel_steps // (budget // 4))
    assert steps <= share_steps + 3, (steps, share_steps)
    assert srv.state(rb) in (nbgb.NB_REQ_RUNNING, nbgb.NB_REQ_DONE)
    srv.run_all()
    srv.close()
