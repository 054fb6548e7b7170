"""GPU path vs FP64 oracle, element by element, on identical seeded inputs.

Every case builds the state with the oracle's initial data (exact Kerr-Schild BSSN
slice + primitive profiles of the workload generator), hands the same array to the
C-ABI library (grmhd_set_state) and compares.

Bar (FP64: 1e-11 relative on every component): per variable v,
    max|gpu_v - oracle_v| <= max(1e-11, KAPPA floor_v) max|oracle_v|,
where floor_v is the oracle's own FP64 rounding floor of that component, measured in the
test by evaluating the oracle again with one more rounding at the unit roundoff after
every stage of its computation (oracle/rounding.py).  For a component that is not a residue of
cancelling terms the floor is ~1e-15 and the bar is the plain 1e-11 of max|oracle_v|; for a
cancellation residue (the right-hand side of the metric of a stationary Kerr-Schild slice,
the phi derivative of a nearly axisymmetric flux) rounding alone moves the oracle by more
than 1e-11 of the residue, and the bar is KAPPA times that measured movement.  Every case
prints, per variable, the plain ratio max|gpu_v - oracle_v| / max|oracle_v|, the floor and
the ratio to the bar.
"""
import os

import numpy as np
import pytest

from oracle import solver as so
from workloads import config

from oracle import rounding as fpf

pytestmark = pytest.mark.gpu

TOL = 1e-11


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2508_18221_gb300 as pkg
    if not os.path.exists(pkg.LIB_PATH):
        from paper_2508_18221_gb300 import _build
        _build.build()
    pkg.load()
    torch.cuda.init()
    return pkg


def _ctx(pkg, cfg, **kw):
    import torch
    opt_keys = ("evolve_metric", "gauge", "integrator", "filter", "contraction", "coupling", "glm", "precision",
                "c2p_lambda", "c2p_maxit", "c2p_tol")
    grid, phys, opts = pkg.make_structs(cfg, **{k: v for k, v in kw.items() if k in opt_keys})
    return pkg.Context(grid, phys, opts, torch.cuda.current_stream().cuda_stream)


def _oracle(cfg, **kw):
    pk = {k: v for k, v in kw.items() if k in ("evolve_metric", "gauge", "integrator", "coupling")}
    if "filter" in kw:
        pk["filter_mask"] = kw["filter"]
    return so.workload_state(cfg, **pk)


# canonical variables grouped by the tensor they are components of (a component whose
# oracle value is identically zero is compared against its tensor's scale)
TENSORS = [range(0, 6), [6], range(7, 13), [13], range(14, 17), [17], range(18, 21),
           range(21, 24), [24], range(25, 28), [28], range(29, 32), [32]]
TENSOR_OF = {v: list(t) for t in TENSORS for v in t}


def min_spacing(g):
    """Smallest node spacing min(dr, r dtheta, r sin(theta) dphi) of the grid (the CFL
    spacing)."""
    p = g.p
    h = np.inf
    for e in range(p.n_elem):
        h = min(h, np.diff(g.r[e]).min())
    h = min(h, g.r.min() * np.diff(g.theta).min(),
            g.r.min() * np.sin(g.theta).min() * 2 * np.pi / p.n_phi)
    return h


def _report_line(what, rows):
    out = os.environ.get("GRMHD_REPORT_DIR")
    if out:
        import json
        os.makedirs(out, exist_ok=True)
        with open(os.path.join(out, "parity_ratios.jsonl"), "a") as fh:
            fh.write(json.dumps({"case": what, "vars": rows}) + "\n")


def assert_parity(got, ref, what, fn, U, tol=TOL, eps=fpf.EPS64, trials=3, kappa=fpf.KAPPA):
    """Per variable v: max|got_v - ref_v| <= max(tol, kappa floor_v) max|ref_v|, floor_v
    the oracle's rounding floor of v at unit roundoff eps (fpf.floor of fn at U; fn(U) is
    the oracle result `ref`).  The mixed-precision modes pass the unit of their FP32 stages
    and kappa = 1 (their floor rounds every stage at that unit, the FP64 ones included).
    A variable whose oracle value is identically zero must match to tol times its
    tensor's largest value (exactly, when that is zero too).
    Prints per variable the plain ratio, the floor and the ratio to the bar; returns
    (worst plain ratio, worst ratio to the bar)."""
    nv = ref.shape[0]
    _, fl = fpf.floor(fn, U, trials=trials, eps=eps, ref=ref)
    worst_plain, worst_bar, rows, bad = 0.0, 0.0, [], []
    for v in range(nv):
        m = float(np.abs(ref[v]).max())
        err = float(np.abs(got[v] - ref[v]).max())
        if not np.isfinite(err):
            bad.append(f"variable {v}: non-finite result")
            continue
        if m > 0:
            bar = max(tol, kappa * fl[v]) * m
            plain = err / m
        else:
            bar = tol * max(float(np.abs(ref[w]).max()) for w in TENSOR_OF.get(v, [v]) if w < nv)
            plain = 0.0 if err == 0 else float("inf")
        r = err / bar if bar > 0 else (0.0 if err == 0 else float("inf"))
        worst_plain = max(worst_plain, plain if m > 0 else 0.0)
        worst_bar = max(worst_bar, r)
        rows.append({"v": v, "plain": plain, "floor": float(fl[v]), "err_over_bar": r})
        if not r <= 1.0:
            bad.append(f"variable {v}: error {err:.3e}, max|ref| {m:.3e}, plain {plain:.3e}, "
                       f"floor {fl[v]:.2e}, bar {bar:.3e}")
    resid = [row["v"] for row in rows if row["floor"] * kappa > tol]
    print(f"\n[parity] {what}: worst plain ratio {worst_plain:.2e}, worst error/bar {worst_bar:.3f}; "
          f"variables with a floor above tol/{kappa:g} (cancellation residues): {resid}")
    for row in rows:
        print(f"[parity]   v{row['v']:2d} plain {row['plain']:.2e} floor {row['floor']:.1e} "
              f"err/bar {row['err_over_bar']:.3f}")
    _report_line(what, rows)
    assert not bad, f"{what}: " + "; ".join(bad)
    return worst_plain, worst_bar


def _gpu_rhs(pkg, ctx, U):
    import torch
    Ud = torch.from_numpy(U.reshape(-1).copy()).cuda()
    ctx.set_state(Ud, True)
    out = torch.empty_like(Ud)
    ctx.rhs(out, True)
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(U.shape)


CASES = [
    ("c1", {}),                                             # 2 elements, 12 x 12 x 16
    ("c1", {"contraction": 1}),                             # contractions on the FP64 units
    ("c1", {"evolve_metric": 0}),                           # fixed Kerr-Schild metric
    ("c1", {"gauge": 1}),                                   # frozen gauge
    ("c1:ragged", {}),                                      # odd sizes, 3 elements
    ("c1:single", {}),                                      # one element (no interface)
    ("c1:wide", {}),                                        # full-width theta range
]


def _cfg(name):
    if name == "c1":
        return config("c1")
    if name == "c1:ragged":
        return config("c1", n_elem=3, n_r=9, n_theta=11, n_phi=6)
    if name == "c1:single":
        return config("c1", n_elem=1, n_r=7, n_theta=5, n_phi=4)
    if name == "c1:wide":
        return config("c1", theta_min=0.05, theta_max=np.pi - 0.05, n_theta=10)
    raise KeyError(name)


@pytest.mark.parametrize("name,kw", CASES)
def test_rhs_parity(pkg, name, kw):
    cfg = _cfg(name)
    g, p, U = _oracle(cfg, **kw)
    ctx = _ctx(pkg, cfg, **kw)
    R = _gpu_rhs(pkg, ctx, U)
    Rref = so.rhs(U, g, p)
    assert_parity(R, Rref, f"rhs {name} {kw}", lambda X: so.rhs(X, g, p), U)
    ctx.close()


@pytest.mark.parametrize("contraction", [0, 1])
def test_derivative_operators(pkg, contraction):
    import torch
    cfg = config("c1", n_elem=3, n_r=10, n_theta=9, n_phi=8)
    g, p, U = _oracle(cfg)
    ctx = _ctx(pkg, cfg, contraction=contraction)
    src = torch.from_numpy(U.reshape(-1).copy()).cuda()
    dst = torch.empty_like(src)
    for d, op in enumerate((g.d_r, g.d_t, g.d_p)):
        ctx.debug_deriv(src, dst, 32, d)
        D = dst.cpu().numpy().reshape(U.shape)
        ref = op(U)
        for v in range(32):
            den = np.abs(ref[v]).max()
            if den > 0:
                assert np.abs(D[v] - ref[v]).max() <= 1e-12 * den + 1e-13 * np.abs(U[v]).max(), (d, v)
    ctx.close()


def test_con2prim_parity(pkg):
    import torch
    cfg = config("c1")
    g, p, U = _oracle(cfg)
    prim = so.primitives(U, p)
    ctx = _ctx(pkg, cfg)
    ctx.set_state(torch.from_numpy(U.reshape(-1).copy()).cuda(), True)
    out = torch.empty(7 * U[0].size, dtype=torch.float64, device="cuda")
    nf = ctx.con2prim(out, True)
    P = out.cpu().numpy().reshape((7,) + U.shape[1:])
    assert nf == int(np.sum(~prim["ok"]))
    ref = [prim["rho"], prim["v"][..., 0], prim["v"][..., 1], prim["v"][..., 2], prim["eps"],
           prim["p"], prim["W"]]
    vmax = max(np.abs(ref[i]).max() for i in (1, 2, 3))
    for i in range(7):
        sc = vmax if i in (1, 2, 3) else np.abs(ref[i]).max()
        assert np.abs(P[i] - ref[i]).max() <= 1e-12 * sc, i
    ctx.close()


def _damped_prims(U, g, p, maxit, tol):
    """The oracle's damped recovery (the paper's iteration) from the dust estimates."""
    from oracle import valencia as va
    f = so.unpack_bssn(U)
    gam, sqg = so.metric_from_bssn(f)
    D = U[so.I_D] / sqg
    S = so.vec_from(U, so.I_S) / sqg[..., None]
    tau = U[so.I_TAU] / sqg
    B = so.vec_from(U, so.I_B) / sqg[..., None]
    r0, v0, e0 = va.con2prim_damped_guess(D, S, tau, gam, eps_min=p.eps_atm)
    rho, v, eps, pr, W, ok, _ = va.con2prim_damped(D, S, tau, B, gam, p.gamma_eos, r0, v0, e0, lam0=0.5,
                                                   maxit=maxit, tol=tol, eps_min=p.eps_atm)
    return {"rho": rho, "v": v, "eps": eps, "p": pr, "W": W, "ok": ok, "B": B}


@pytest.mark.parametrize("maxit", [40, 400])
def test_con2prim_damped_parity(pkg, maxit):
    """opts.c2p_lambda = 0.5: the paper's damped iteration on the GPU against the oracle's
    con2prim_damped from the same start (the dust estimates: the state was just set), with
    the same iteration limit and tolerance, and the right-hand side built on it; the
    distance of both to the exact root is printed (the paper's 40 iterations: ~1e-9)."""
    import torch
    cfg = config("c1")
    g, p, U = _oracle(cfg)
    tol = 1e-13
    ctx = _ctx(pkg, cfg, c2p_lambda=0.5, c2p_maxit=maxit, c2p_tol=tol)
    ctx.set_state(torch.from_numpy(U.reshape(-1).copy()).cuda(), True)
    out = torch.empty(7 * U[0].size, dtype=torch.float64, device="cuda")
    nf = ctx.con2prim(out, True)
    P = out.cpu().numpy().reshape((7,) + U.shape[1:])
    ref = _damped_prims(U, g, p, maxit, tol)
    exact = so.primitives(U, p)
    assert nf == int(np.sum(~ref["ok"]))
    names = ("rho", "v^r", "v^theta", "v^phi", "eps", "p", "W")
    refs = [ref["rho"], ref["v"][..., 0], ref["v"][..., 1], ref["v"][..., 2], ref["eps"], ref["p"], ref["W"]]
    exs = [exact["rho"], exact["v"][..., 0], exact["v"][..., 1], exact["v"][..., 2], exact["eps"],
           exact["p"], exact["W"]]
    vmax = max(np.abs(refs[i]).max() for i in (1, 2, 3))
    for i in range(7):
        sc = vmax if i in (1, 2, 3) else np.abs(refs[i]).max()
        err = np.abs(P[i] - refs[i]).max() / sc
        dist = np.abs(P[i] - exs[i]).max() / sc
        print(f"[c2p damped {maxit}] {names[i]}: GPU vs oracle iteration {err:.2e}, "
              f"GPU vs exact root {dist:.2e}")
        assert err <= 1e-10, (names[i], err)
    # the right-hand side on the damped primitives
    R = _gpu_rhs(pkg, ctx, U)
    fn = lambda X: so.rhs_from_prims(X, _damped_prims(X, g, p, maxit, tol), g, p)  # noqa: E731
    assert_parity(R, fn(U), f"rhs on the damped recovery ({maxit} iterations)", fn, U, trials=2)
    ctx.close()


@pytest.mark.parametrize("integrator,contraction,coupling", [(0, 0, 0), (1, 0, 0), (0, 1, 0), (1, 0, 1), (0, 0, 1)])
def test_step_parity(pkg, integrator, contraction, coupling):
    """2 steps; coupling = 1 is the paper's split loop (fluid RK on the frozen metric,
    then a forward-Euler BSSN + gauge step)."""
    import torch
    cfg = config("c1", n_elem=3, n_r=9, n_theta=10, n_phi=8)
    g, p, U = _oracle(cfg, integrator=integrator, coupling=coupling)
    ctx = _ctx(pkg, cfg, integrator=integrator, contraction=contraction, coupling=coupling)
    ctx.set_state(torch.from_numpy(U.reshape(-1).copy()).cuda(), True)
    dt = 2e-3
    ctx.step(dt, 2)
    got = np.empty(U.size)
    ctx.get_state(got, False)
    two = lambda X: so.rk_step(so.rk_step(X, dt, g, p), dt, g, p)  # noqa: E731
    assert_parity(got.reshape(U.shape), two(U),
                  f"2 steps integrator {integrator} contraction {contraction} coupling {coupling}", two, U,
                  trials=2)
    ctx.close()


def test_init_prims_matches_oracle(pkg):
    cfg = config("c1", n_elem=2, n_r=8, n_theta=8, n_phi=8)
    g, p, U = _oracle(cfg)
    from workloads import primitive_profiles
    ctx = _ctx(pkg, cfg)
    r, t, ph = ctx.coords()
    np.testing.assert_allclose(r.reshape(g.shape), g.R, rtol=1e-15)
    np.testing.assert_allclose(t.reshape(g.shape), g.T, rtol=1e-15)
    pr = primitive_profiles(cfg, r.reshape(g.shape), t.reshape(g.shape), ph.reshape(g.shape))
    ctx.init_prims(pr["rho"], pr["p"], pr["vr"], pr["vth"], pr["vph"], pr["A_phi"])
    got = np.empty(U.size)
    ctx.get_state(got, False)
    got = got.reshape(U.shape)
    for v in range(32):
        sc = max(np.abs(U[w]).max() for w in TENSOR_OF[v])
        assert np.abs(got[v] - U[v]).max() <= 1e-12 * sc, v
    ctx.close()


def test_cfl_and_diagnostics(pkg):
    import torch
    cfg = config("c1")
    g, p, U = _oracle(cfg)
    ctx = _ctx(pkg, cfg)
    ctx.set_state(torch.from_numpy(U.reshape(-1).copy()).cuda(), True)
    np.testing.assert_allclose(ctx.cfl_dt(), so.cfl_dt(U, g, p), rtol=1e-13)
    dg = ctx.diag()
    ref = so.diagnostics(U, g, p)
    np.testing.assert_allclose(dg[0], ref[0], rtol=1e-13)
    np.testing.assert_allclose(dg[1], ref[1], rtol=1e-12)
    assert dg[2] <= 1e-12 * np.abs(U[so.I_B:so.I_B + 3]).max() * 100
    # Hamiltonian constraint: max |H| and its quadrature RMS (a residual of O(1) cancelling
    # curvature terms: the RHS bar relative to the largest term, here max |H| itself)
    assert ref[4] > 0
    np.testing.assert_allclose(dg[5], ref[4], rtol=1e-9)
    np.testing.assert_allclose(dg[6], ref[5], rtol=1e-9)
    # the diagnostic leaves the state untouched
    after = np.empty(U.size)
    ctx.get_state(after, False)
    np.testing.assert_array_equal(after, U.reshape(-1))
    dg2 = ctx.diag()
    # (sums by atomic adds: equal up to their order)
    np.testing.assert_allclose(np.asarray(dg2)[[0, 1, 2, 5, 6]], np.asarray(dg)[[0, 1, 2, 5, 6]], rtol=1e-13)
    ctx.close()


def test_invalid_and_nan(pkg):
    import torch
    cfg = config("c1", n_elem=1, n_r=6, n_theta=6, n_phi=4)
    g, p, U = _oracle(cfg)
    ctx = _ctx(pkg, cfg)
    bad = U.copy()
    bad[so.I_TAU, 0, 2, 2, 1] = np.nan
    ctx.set_state(torch.from_numpy(bad.reshape(-1).copy()).cuda(), True)
    with pytest.raises(pkg.GrmhdError, match="-4"):
        ctx.step(1e-3, 1)
    with pytest.raises(pkg.GrmhdError, match="-1"):
        ctx.step(1e-3, 0)
    ctx.close()


@pytest.mark.slow
def test_rhs_parity_full_size(pkg):
    """The benchmarked 8-element 24 x 32 x 64 instance (393,216 nodes) in the launch
    configuration the benchmark uses: every node of one RHS evaluation against the
    oracle."""
    cfg = config("c2")
    g, p, U = _oracle(cfg)
    ctx = _ctx(pkg, cfg)
    R = _gpu_rhs(pkg, ctx, U)
    Rref = so.rhs(U, g, p)
    assert_parity(R, Rref, "rhs c2 full size", lambda X: so.rhs(X, g, p), U, trials=2)
    ctx.close()
