"""Batched projections (one persistent launch for many uneven grids) against
the FP64 CPU oracle, graph replay, and the autotuner."""
import json
import os

import numpy as np
import pytest

import oracle
import paris_inputs as pi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

P, W = pi.PERIODIC, pi.WALL


@pytest.fixture(scope="module")
def paris():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2012_11744_gb300 as m
    m.build()
    return m


GRIDS = [pi.Grid(16, 16, 16, 1 / 16), pi.Grid(24, 16, 8, 1 / 24, (P, P, W)), pi.Grid(32, 32, 32, 1 / 32),
         pi.Grid(12, 20, 16, 0.05, (W, P, P)), pi.Grid(8, 8, 8, 1 / 8), pi.Grid(48, 32, 16, 1 / 48)]


def run_batch(paris, probs, opts=None):
    grids = [p.grid for p in probs]
    with paris.Batch(grids, opts=opts or paris.default_opts()) as b:
        C = b.pack([p.C for p in probs], "C")
        u = b.pack([p.u for p in probs], "u")
        v = b.pack([p.v for p in probs], "v")
        w = b.pack([p.w for p in probs], "w")
        pp = torch.zeros_like(C)
        st = b.projection_step(C, [p.rho1 for p in probs], [p.rho2 for p in probs],
                               [p.dt for p in probs], u, v, w, pp)
        out = [(x.cpu().numpy(), (a.cpu().numpy(), bb.cpu().numpy(), c.cpu().numpy()))
               for x, a, bb, c in zip(b.unpack(pp, "p"), b.unpack(u, "u"), b.unpack(v, "v"), b.unpack(w, "w"))]
        return out, st, b.launch_ctas


def check_instance(pr, p, uvw, tol=1e-10, ref=None):
    g = pr.grid
    beta = oracle.face_coeffs(g, pr.C, pr.rho1, pr.rho2)
    b = oracle.divergence(g, pr.u, pr.v, pr.w, pr.dt)
    b -= oracle.mean(b)
    op = oracle.Operator(g, *beta)
    r = b - op.apply_L(p)
    assert np.linalg.norm(r) <= 1.01 * tol * np.linalg.norm(b)
    assert np.abs(r).max() <= 1.01 * tol * np.abs(b).max()
    umax = max(np.abs(x).max() for x in (pr.u, pr.v, pr.w))
    assert np.abs(oracle.divergence(g, *uvw, dt=1.0)).max() <= 1e-9 * umax / g.h
    if ref is not None:
        assert np.abs(p - ref.p).max() <= 1e-8 * np.abs(ref.p).max()
        for a in range(3):
            np.testing.assert_allclose(uvw[a], ref.u[a], rtol=0, atol=1e-7 * umax)
    op.close()


def test_batch_matches_oracle(paris):
    probs = [pi.random_problem(g, seed=30 + i, rho1=[10.0, 1000.0, 100.0, 1000.0, 3.0, 500.0][i])
             for i, g in enumerate(GRIDS)]
    out, st, ctas = run_batch(paris, probs)
    assert ctas >= len(probs)
    for pr, (p, uvw), s in zip(probs, out, st):
        assert s["converged"] == 1, s
        ref = oracle.projection_step(pr.grid, pr.C, pr.rho1, pr.rho2, pr.dt, pr.u, pr.v, pr.w)
        check_instance(pr, p, uvw, ref=ref)


def test_batch_graph_replay_with_new_inputs(paris):
    """The step is captured in a CUDA graph on the first call and replayed:
    a second step on the same pools with new C, u*, densities and time steps
    is still exact."""
    grids = GRIDS[:4]
    with paris.Batch(grids) as b:
        pools = None
        for rep in range(2):
            probs = [pi.random_problem(g, seed=60 + 10 * rep + i, rho1=[50.0, 200.0][rep],
                                       dt=[1e-3, 5e-4][rep], drops=1 + 2 * rep)
                     for i, g in enumerate(grids)]
            packs = {k: b.pack([getattr(q, k) for q in probs], k) for k in ("C", "u", "v", "w")}
            if pools is None:
                pools = dict(packs, p=torch.zeros_like(packs["C"]))
            else:
                for k, x in packs.items():
                    pools[k].copy_(x)
            st = b.projection_step(pools["C"], [q.rho1 for q in probs], [q.rho2 for q in probs],
                                   [q.dt for q in probs], pools["u"], pools["v"], pools["w"], pools["p"])
            for i, pr in enumerate(probs):
                assert st[i]["converged"] == 1
                p = b.unpack(pools["p"], "p")[i].cpu().numpy()
                uvw = tuple(b.unpack(pools[k], k)[i].cpu().numpy() for k in ("u", "v", "w"))
                check_instance(pr, p, uvw)


def test_batch_uneven_drop_fields(paris):
    """24 instances of the uneven-size recipe (axes from {32,48,64,96,128},
    1-8 drops, density ratio up to 1000): every instance converges to 1e-10."""
    probs = pi.config4(count=24)
    out, st, _ = run_batch(paris, probs)
    for pr, (p, uvw), s in zip(probs, out, st):
        assert s["converged"] == 1, s
        check_instance(pr, p, uvw)


def test_batch_autotune_and_cache(paris, tmp_path):
    probs = [pi.random_problem(g, seed=80 + i, rho1=100.0) for i, g in enumerate(GRIDS[:3])]
    grids = [p.grid for p in probs]
    cache = str(tmp_path / "tune.jsonl")
    with paris.Batch(grids) as b:
        C = b.pack([p.C for p in probs], "C")
        u = b.pack([p.u for p in probs], "u")
        v = b.pack([p.v for p in probs], "v")
        w = b.pack([p.w for p in probs], "w")
        u0 = u.clone()
        best = b.autotune(C, [p.rho1 for p in probs], [p.rho2 for p in probs], [p.dt for p in probs],
                          u, v, w, cache_path=cache)
        assert best > 0 and torch.equal(u, u0)  # inputs untouched
        nu, om, bps = b.tuning()
        assert nu in (1, 2, 3) and om in (1.0, 1.15, 1.3) and bps >= 1
        lines = open(cache).read().strip().splitlines()
        assert len(lines) == 1 and json.loads(lines[0])["nu"] == nu
        pp = torch.zeros_like(C)
        st = b.projection_step(C, [p.rho1 for p in probs], [p.rho2 for p in probs], [p.dt for p in probs],
                               u, v, w, pp)
        for i, pr in enumerate(probs):
            assert st[i]["converged"] == 1
            check_instance(pr, b.unpack(pp, "p")[i].cpu().numpy(),
                           tuple(b.unpack(x, k)[i].cpu().numpy() for x, k in ((u, "u"), (v, "v"), (w, "w"))))
    with paris.Batch(grids) as b2:  # a second batch reads the cache instead of timing
        C = b2.pack([p.C for p in probs], "C")
        u = b2.pack([p.u for p in probs], "u")
        v = b2.pack([p.v for p in probs], "v")
        w = b2.pack([p.w for p in probs], "w")
        b2.autotune(C, [p.rho1 for p in probs], [p.rho2 for p in probs], [p.dt for p in probs],
                    u, v, w, cache_path=cache)
        assert b2.tuning() == (nu, om, bps)
        assert len(open(cache).read().strip().splitlines()) == 1
