"""Full-size checks in the launch configuration the benchmark times.

256^3 drop field (periodic x/y, walls z, ratio 1000) and the 512x256x256 jet
(periodic x, walls y/z, ratio 1000).  The oracle cannot solve these in a test's
time, so the checks are (a) the FP64 residual of the GPU pressure under the
oracle's assembled operator, (b) the discrete divergence of the GPU velocity
under the oracle's divergence, (c) p and u at 4096 sampled points against a
stored full oracle solve (tests/golden/drops256_walls_z.json, written by
make_drops256_golden.py, which calls only the oracle), and (d) the
gradient-field property p = phi, u = 0, which holds exactly at any size.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
import paris_inputs as pi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def paris():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2012_11744_gb300 as m
    m.build()
    return m


@pytest.fixture(scope="module")
def drops256():
    return pi.config2(n=256)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def run_gpu(paris, pr, precision, tol=1e-10):
    g = pr.grid
    with paris.Context(g, opts=paris.default_opts(precision=precision, tol=tol)) as ctx:
        u, v, w = dev(pr.u), dev(pr.v), dev(pr.w)
        p = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
        st = ctx.projection_step(dev(pr.C), pr.rho1, pr.rho2, pr.dt, u, v, w, p)
        return host(p), (host(u), host(v), host(w)), st


def check_properties(pr, p, u, tol=1e-10):
    g = pr.grid
    beta = oracle.face_coeffs(g, pr.C, pr.rho1, pr.rho2)
    b = oracle.divergence(g, pr.u, pr.v, pr.w, pr.dt)
    b -= oracle.mean(b)
    op = oracle.Operator(g, *beta)
    r = b - op.apply_L(p)
    rel2 = np.linalg.norm(r) / np.linalg.norm(b)
    relinf = np.abs(r).max() / np.abs(b).max()
    assert rel2 <= tol * 1.01 and relinf <= tol * 1.01, (rel2, relinf)
    umax = max(np.abs(x).max() for x in (pr.u, pr.v, pr.w))
    d = oracle.divergence(g, *u, dt=1.0)
    assert np.abs(d).max() <= 1e-9 * umax / g.h
    op.close()
    return beta


@pytest.mark.parametrize("precision", ["MIXED", "FP64"])
def test_drops256_against_stored_oracle(paris, drops256, precision):
    pr = drops256
    path = os.path.join(HERE, "golden", "drops256_walls_z.json")
    if not os.path.exists(path):
        pytest.skip("stored oracle solve missing (run tests/golden/make_drops256_golden.py)")
    with open(path) as fh:
        gold = json.load(fh)
    assert gold["C_sha256"] == hashlib.sha256(np.ascontiguousarray(pr.C).tobytes()).hexdigest()
    p, u, st = run_gpu(paris, pr, getattr(paris, precision))
    assert st["converged"] == 1 and st["fell_back"] == 0, st
    check_properties(pr, p, u)
    cells = np.asarray(gold["cells"])
    err = np.abs(p.ravel()[cells] - np.asarray(gold["p"])).max() / gold["p_max_abs"]
    assert err <= 1e-8, err
    umax = max(np.abs(x).max() for x in (pr.u, pr.v, pr.w))
    for a in range(3):
        f = np.asarray(gold["faces"][a])
        du = np.abs(u[a].ravel()[f] - np.asarray(gold["u"][a])).max()
        assert du <= 1e-8 * umax, (a, du)


def test_drops256_gradient_field(paris, drops256):
    """u* = dt B G phi: the exact discrete answer is p = phi - mean(phi), u = 0.
    phi is smooth plus 1 % noise; the solve runs to 1e-12 so that the error
    bound (condition number times residual) is far below the 1e-8 bar."""
    pr = drops256
    g = pr.grid
    beta = oracle.face_coeffs(g, pr.C, pr.rho1, pr.rho2)
    c = (np.arange(256) + 0.5) / 256
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    phi = np.sin(2 * np.pi * X) * np.cos(4 * np.pi * Y) * np.cos(np.pi * Z) \
        + 0.01 * pi.random_field(g.shape, seed=256)
    phi -= phi.mean()
    gx = (phi - np.roll(phi, 1, axis=2)) / g.h
    gy = (phi - np.roll(phi, 1, axis=1)) / g.h
    gz = np.zeros(g.face_shape(2))
    gz[1:-1] = np.diff(phi, axis=0) / g.h
    us = [pr.dt * beta[0] * gx, pr.dt * beta[1] * gy, pr.dt * beta[2] * gz]
    pr2 = pi.Problem("gradfield256", g, pr.C, us[0], us[1], us[2], pr.rho1, pr.rho2, pr.dt)
    p, u, st = run_gpu(paris, pr2, paris.MIXED, tol=1e-12)
    assert st["converged"] == 1, st
    e = np.abs(p - phi).max() / np.abs(phi).max()
    assert e <= 1e-8, e
    umax = max(np.abs(x).max() for x in us)
    for a in range(3):
        assert np.abs(u[a]).max() <= 1e-8 * umax


def test_jet_512x256x256(paris):
    """The jet (BASELINE's third configuration), mixed form: the residual of
    the GPU pressure under the oracle's operator, the divergence bar, and the
    pointwise error against the stored full FP64 oracle solve
    (tests/golden/jet512x256x256.json, written by make_jet512_golden.py) at
    its 4096 sampled cells and 4096 sampled faces."""
    pr = pi.config3()
    p, u, st = run_gpu(paris, pr, paris.MIXED)
    assert st["converged"] == 1, st
    check_properties(pr, p, u)
    path = os.path.join(HERE, "golden", "jet512x256x256.json")
    if not os.path.exists(path):
        pytest.skip("stored oracle solve missing (run tests/golden/make_jet512_golden.py)")
    with open(path) as fh:
        gold = json.load(fh)
    assert gold["C_sha256"] == hashlib.sha256(np.ascontiguousarray(pr.C).tobytes()).hexdigest()
    cells = np.asarray(gold["cells"])
    err = np.abs(p.ravel()[cells] - np.asarray(gold["p"])).max() / gold["p_max_abs"]
    umax = max(np.abs(x).max() for x in (pr.u, pr.v, pr.w))
    du = max(np.abs(u[a].ravel()[np.asarray(gold["faces"][a])] - np.asarray(gold["u"][a])).max() for a in range(3))
    print(f"jet vs oracle: p {err:.3e} (relative to max|p|), u {du / umax:.3e} (relative to max|u*|), "
          f"oracle residual {gold['oracle']['rel_res_l2']:.2e}, its p bound {gold['bound']['p_rel_err_bound']:.2e}")
    assert err <= 1e-8, err
    assert du <= 1e-8 * umax, du


def test_batch_256_uneven_instances(paris):
    """The full batch: 256 periodic instances, axes from {32,48,64,96,128}
    (1.07e8 cells), one persistent launch: every instance converges; 12
    sampled instances are checked under the oracle's operator and divergence."""
    probs = pi.config4(count=256)
    with paris.Batch([p.grid for p in probs]) as b:
        C = b.pack([p.C for p in probs], "C")
        u = b.pack([p.u for p in probs], "u")
        v = b.pack([p.v for p in probs], "v")
        w = b.pack([p.w for p in probs], "w")
        pp = torch.zeros_like(C)
        st = b.projection_step(C, [p.rho1 for p in probs], [p.rho2 for p in probs],
                               [p.dt for p in probs], u, v, w, pp)
        assert all(s["converged"] == 1 for s in st)
        rng = np.random.default_rng(256)
        for i in rng.choice(len(probs), size=12, replace=False):
            p = b.unpack(pp, "p")[i].cpu().numpy()
            uvw = tuple(b.unpack(x, k)[i].cpu().numpy() for x, k in ((u, "u"), (v, "v"), (w, "w")))
            check_properties(probs[i], p, uvw)


def test_drops256_refinement_residual_matches_fp64(paris, drops256):
    """At 256^3 (the benchmark's field) the residual norms the mixed form
    reports, updated in double-float during refinement, agree with a full
    FP64 residual of the returned pressure to 2e-12 relative."""
    pr = drops256
    g = pr.grid
    with paris.Context(g, opts=paris.default_opts(precision=paris.MIXED)) as ctx:
        u, v, w = dev(pr.u), dev(pr.v), dev(pr.w)
        p = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
        st = ctx.projection_step(dev(pr.C), pr.rho1, pr.rho2, pr.dt, u, v, w, p)
        assert st["converged"] == 1 and st["fell_back"] == 0, st
        bx, by, bz = ctx.face_coeffs(dev(pr.C), pr.rho1, pr.rho2)
        rhs = torch.empty(g.shape, dtype=torch.float64, device="cuda")
        ctx.divergence(dev(pr.u), dev(pr.v), dev(pr.w), pr.dt, rhs)
        l2, linf = ctx.residual_norms(bx, by, bz, rhs, p)
    print(f"reported {st['rel_res_l2']:.4e} {st['rel_res_linf']:.4e}  FP64 {l2:.4e} {linf:.4e}")
    assert abs(st["rel_res_l2"] - l2) <= 2e-12 and abs(st["rel_res_linf"] - linf) <= 2e-12
    assert l2 <= 1e-10 and linf <= 1e-10
