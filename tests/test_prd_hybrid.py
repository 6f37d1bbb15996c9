"""Hybrid PRD (redistribution angle-averaged in the frame of the moving gas,
Sect. 2.1) on the GPU against the FP64 oracle on moving columns: Lyman alpha
in PRD on a 3-level atom (24 points, 32 depths).  Fixed schedules per
iterate (FP64 within 1e-9, FP32 within 1e-3) without Ng (damped update) and
with the Jacobi step, whose derivative is the gas-frame one; the converged
FP64 fixed point; and at rest the hybrid kernel path is the static-frame one
to the bit."""
import numpy as np
import pytest

import rh_synth

pytestmark = pytest.mark.gpu

SCHEDULES = [(0, 5), (2, 50)]


@pytest.fixture(scope="module")
def rh():
    import paper_1411_1079_gb300 as m
    m.build()
    return m


def prd_atom():
    return rh_synth.hydrogen_like_atom(nbound=3, lyman_nlambda=24, line_nlambda=12, cont_nlambda=10, nmu=3,
                                       prd_lines=((1, 2),))


@pytest.fixture(scope="module")
def cols():
    c = rh_synth.subset(rh_synth.chromosphere_cube(nx=16, ny=16, ndep=32, seed=3), [0, 5, 9])
    assert np.max(np.abs(c["vz"])) > 2e3      # moving columns
    return c


@pytest.fixture(scope="module")
def oracle_hybrid(orc, cols):
    o = orc.Oracle()
    o.setup_atom(prd_atom())
    o.load_columns(cols)
    out = {}
    for ng, delay in SCHEDULES:
        for k in (3, 6):
            o.iterate(maxiter=k, tol=0.0, ng_order=ng, ng_delay=delay, prd_eps0=0.05, prd_hybrid=1)
            out[ng, k] = o.populations()[0]
    o.iterate(maxiter=3000, tol=1e-11, prd_hybrid=1)
    out["tight"] = o.populations()
    return out


@pytest.mark.parametrize("precision,tol", [(0, 1e-9), (1, 1e-3)])
def test_hybrid_fixed_schedule_matches_oracle(rh, cols, oracle_hybrid, precision, tol):
    g = rh.Context(0)
    g.setup_atom(prd_atom())
    g.load_columns(cols)
    for ng, delay in SCHEDULES:
        for k in (3, 6):
            g.iterate(maxiter=k, tol=0.0, ng_order=ng, ng_delay=delay, precision=precision, prd_eps0=0.05,
                      prd_hybrid=1)
            n = g.populations()[0]
            assert np.max(np.abs(n / oracle_hybrid[ng, k] - 1)) < tol, (precision, ng, k)


def test_hybrid_fp64_fixed_point(rh, cols, oracle_hybrid):
    g = rh.Context(0)
    g.setup_atom(prd_atom())
    g.load_columns(cols)
    g.iterate(maxiter=3000, tol=1e-11, precision=0, prd_hybrid=1)
    n, it, st, _ = g.populations()
    no, ito, sto, _ = oracle_hybrid["tight"]
    assert np.all(st == 0) and np.all(sto == 0)
    assert np.max(np.abs(n / no - 1)) < 1e-9


@pytest.mark.parametrize("precision", [0, 1])
def test_hybrid_at_rest_is_the_static_scheme(rh, cols, precision):
    c = {k: v.copy() for k, v in cols.items()}
    c["vz"] = np.zeros_like(c["vz"])
    out = []
    for hyb in (0, 1):
        g = rh.Context(0)
        g.setup_atom(prd_atom())
        g.load_columns(c)
        g.iterate(maxiter=12, tol=0.0, ng_order=2, ng_delay=3, ng_period=3, precision=precision, prd_eps0=0.05,
                  prd_hybrid=hyb)
        out.append(g.populations()[0])
    assert np.array_equal(out[0], out[1])


def test_solve_rescues_columns_with_the_bezier_solver(rh):
    """Four columns of the 512x512 x 128-height cube (seed 5678) on which
    every rung of the re-run ladder diverges with the linear formal solver
    (hybrid PRD, Lyman alpha and beta at 200 points): the final pass of
    solve with the Bezier solver converges at least three of them."""
    atom = rh_synth.hydrogen_like_atom(prd_lines=((1, 2), (1, 3)), prd_nlambda=200)
    sub = rh_synth.subset(rh_synth.chromosphere_cube(512, 512, 128, seed=5678), [15527, 15528, 28816, 28817])
    g = rh.Context(0)
    g.setup_atom(atom)
    g.load_columns(sub)
    s = g.solve(maxiter=500, tol=1e-3, precision=1, prd_eps0=0.05, prd_hybrid=1)
    st = g.populations()[2]
    assert s["rescue"]["formal"] == 1 and s["rescue"]["converged_before"] == 0
    assert s["rescue"]["converged_after"] >= 3 and int((st == 0).sum()) == s["n_converged"] >= 3
