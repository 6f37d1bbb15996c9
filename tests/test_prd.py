"""Angle-averaged partial redistribution on the GPU against the FP64 oracle
(Lyman alpha in PRD; R_II-A kernels computed by the column kernel with its
own quadrature)."""
import numpy as np
import pytest

import rh_synth

pytestmark = pytest.mark.gpu


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
    return rh_synth.subset(rh_synth.chromosphere_cube(nx=16, ny=16, ndep=32, seed=3), [0, 5])


@pytest.fixture(scope="module")
def oracle_runs(orc, cols):
    """Oracle populations after 1, 3 and 6 iterations (no Ng), and converged."""
    out = {}
    o = orc.Oracle()
    o.setup_atom(prd_atom())
    o.load_columns(cols)
    for k in (3, 6):
        o.iterate(maxiter=k, tol=0.0, ng_order=0, prd_eps0=0.05)
        out[k] = o.populations()[0]
    o.iterate(maxiter=400, tol=1e-3)
    out["conv"] = o.populations()
    return out


@pytest.mark.parametrize("precision,tol", [(0, 1e-9), (1, 1e-3)])
def test_prd_fixed_schedule_matches_oracle(rh, cols, oracle_runs, precision, tol):
    g = rh.Context(0)
    g.setup_atom(prd_atom())
    g.load_columns(cols)
    for k in (3, 6):
        g.iterate(maxiter=k, tol=0.0, ng_order=0, precision=precision, prd_eps0=0.05)
        n = g.populations()[0]
        assert np.max(np.abs(n / oracle_runs[k] - 1)) < tol, (precision, k)


def test_prd_converges_like_the_oracle(rh, cols, oracle_runs):
    g = rh.Context(0)
    g.setup_atom(prd_atom())
    g.load_columns(cols)
    s = g.solve(precision=1, maxiter=400, tol=1e-3)
    n, it, st, _ = g.populations()
    no, ito, sto, _ = oracle_runs["conv"]
    assert np.all(st == 0) and np.all(sto == 0)
    # both stop at 1e-3; the stopping points are compared within 3e-2
    assert np.max(np.abs(n / no - 1)) < 3e-2
    assert np.allclose(n.sum(axis=1), cols["nH"], rtol=1e-12)
    # PRD changes the solution (against CRD)
    a = prd_atom()
    a["line_prd"] = a["line_prd"] * 0
    h = rh.Context(0)
    h.setup_atom(a)
    h.load_columns(cols)
    h.solve(precision=1, maxiter=400, tol=1e-3)
    assert np.max(np.abs(h.populations()[0] / n - 1)) > 1e-2
