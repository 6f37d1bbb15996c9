"""Learned initial guess: the CUDA training kernels against the FP64 numpy
reference (oracle/mlp.py), training on GPU-converged columns, and what the
trained network gains over the LTE start at equal accuracy."""
import numpy as np
import pytest

import rh_synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rh():
    import paper_1411_1079_gb300 as m
    m.build()
    return m


def _oracle_features_targets(orc, atom, cols):
    """Populations after a few oracle iterations, and the reference features
    and targets ln(n/n*) from the oracle's own LTE values."""
    from oracle import mlp
    o = orc.Oracle()
    o.setup_atom(atom)
    o.load_columns(cols)
    o.iterate(maxiter=25, tol=1e-3)
    n = o.populations()[0]
    ns, ne = o.lte()
    X = mlp.features(cols["T"], ne, cols["nH"], cols["vz"])
    Y = np.log(n / ns).reshape(n.shape[0], -1)
    return n, X, Y


def _seeded_state(rng, dims4, X):
    """Network parameters drawn here (He-scaled weights, zero biases) and the
    standardisation of X, in the library's layout."""
    from oracle import mlp
    parts = []
    for di, do in mlp.layer_dims(*dims4):
        parts.append(rng.standard_normal(do * di) * np.sqrt(2.0 / di))
        parts.append(np.zeros(do))
    parts.append(X.mean(axis=0))
    parts.append(1.0 / np.maximum(X.std(axis=0), 1e-12 * (np.abs(X.mean(axis=0)) + 1)))
    return np.concatenate(parts)


@pytest.mark.parametrize("hidden,nhidden,ncols", [(64, 2, 96), (512, 3, 256)])
def test_gpu_gradient_matches_fp64_reference(rh, orc, hidden, nhidden, ncols):
    # every input of the reference comes from this test or the oracle: the
    # populations (targets), LTE values (features) and the seeded network
    from oracle import mlp
    atom = rh_synth.hydrogen_like_atom()
    cols = rh_synth.subset(rh_synth.chromosphere_cube(nx=32, ny=32, seed=11), slice(0, ncols))
    n, X, Y = _oracle_features_targets(orc, atom, cols)
    ctx = rh.Context(0)
    ctx.setup_atom(atom)
    ctx.load_columns(cols)
    ctx.set_populations(n)
    ctx.surrogate_init(hidden=hidden, nhidden=nhidden, seed=7)
    dims = (X.shape[1], hidden, nhidden, Y.shape[1])
    state32 = _seeded_state(np.random.default_rng(7), dims, X).astype(np.float32)
    ctx.surrogate_set_state(state32)
    state32 = state32.astype(np.float64)
    nwb = state32.size - 2 * X.shape[1]
    loss_g, grad_g = ctx.surrogate_loss_grad(np.arange(ncols))
    loss_o, grad_o = mlp.loss_grad(state32, dims, X, Y)
    gg, go = grad_g[:nwb].astype(np.float64), grad_o[:nwb]
    cos = gg @ go / (np.linalg.norm(gg) * np.linalg.norm(go))
    relL2 = np.linalg.norm(gg - go) / np.linalg.norm(go)
    # BF16 weights and activations against FP64: loss to 1 %, gradient direction
    assert loss_g == pytest.approx(loss_o, rel=1e-2)
    assert cos > 0.999 and relL2 < 1e-2, (cos, relL2)


def test_training_reduces_iterations_at_equal_accuracy(rh):
    atom = rh_synth.hydrogen_like_atom()
    train = rh_synth.chromosphere_cube(nx=64, ny=64, seed=4321)          # disjoint seed
    ctx = rh.Context(0)
    ctx.setup_atom(atom)
    ctx.load_columns(train)
    s = ctx.solve(precision=1)
    assert s["n_converged"] > 0.99 * 4096
    ctx.surrogate_init(hidden=512, nhidden=3, seed=0)
    t = ctx.surrogate_train(epochs=40, batch=256, lr=2e-3, seed=1)
    assert t["loss_last_epoch"] < 0.1 * t["loss_first_epoch"], t

    evalc = rh_synth.subset(rh_synth.chromosphere_cube(nx=64, ny=64, seed=99), slice(0, 1024))
    ctx.load_columns(evalc)
    s0 = ctx.iterate(maxiter=500, tol=1e-3, precision=1, start=0)
    it0, st0 = ctx.populations()[1:3]
    ctx.load_columns(evalc)
    s1 = ctx.iterate(maxiter=500, tol=1e-3, precision=1, start=1)
    it1, st1 = ctx.populations()[1:3]
    assert s1["guess_fallback_depths"] == 0
    ok = (st0 == 0) & (st1 == 0)
    assert ok.mean() > 0.99
    assert it1[ok].mean() < 0.8 * it0[ok].mean(), (it0[ok].mean(), it1[ok].mean())

    # the same solution from either start.  The discrete problem (rate
    # equations with the discrete transfer solution) can have more than one
    # solution in a column -- the FP64 oracle alone finds two, 5.7e-3 apart,
    # for some columns of this cube, each with a residual of 1e-11 -- and Ng
    # acceleration may converge to either.  A column whose two results differ
    # must therefore show that both satisfy the equations: one plain
    # iteration (no Ng) from each moves it by less than 1e-4.
    ctx.load_columns(evalc)
    ctx.iterate(maxiter=1000, tol=1e-6, precision=1, start=0)
    n0, _, a0, _ = ctx.populations()
    ctx.load_columns(evalc)
    ctx.iterate(maxiter=1000, tol=1e-6, precision=1, start=1)
    n1, _, a1, _ = ctx.populations()
    both = (a0 == 0) & (a1 == 0)
    assert both.mean() > 0.98
    differ = both & (np.abs(n1 / n0 - 1).max(axis=(1, 2)) > 2e-3)
    assert differ.mean() < 0.01, differ.sum()
    if differ.any():
        for n in (n0, n1):
            ctx.set_populations(n)
            ctx.iterate(maxiter=1, tol=0.0, ng_order=0, start=2, precision=1)
            resid = ctx.populations()[3]
            assert np.all(resid[differ] < 1e-4), resid[differ]

    # checkpoint round trip: the same network in a fresh context predicts the same
    state = ctx.surrogate_state()
    pred = ctx.surrogate_predict()
    ctx2 = rh.Context(0)
    ctx2.setup_atom(atom)
    ctx2.load_columns(evalc)
    ctx2.surrogate_init(hidden=512, nhidden=3, seed=5)
    ctx2.surrogate_set_state(state)
    assert np.array_equal(ctx2.surrogate_predict(), pred)


def test_surrogate_errors(rh):
    ctx = rh.Context(0)
    ctx.setup_atom(rh_synth.small_atom())
    with pytest.raises(rh.RhError):
        ctx.surrogate_init()                    # no columns yet
    ctx.load_columns(rh_synth.subset(rh_synth.chromosphere_cube(nx=16, ny=16, ndep=12, seed=1), [0, 1, 2]))
    with pytest.raises(rh.RhError) as e:
        ctx.iterate(start=1)                    # no network
    assert e.value.code == rh.RH_ESTATE
    ctx.surrogate_init(hidden=16, nhidden=1, seed=0)
    with pytest.raises(rh.RhError) as e:
        ctx.surrogate_train(epochs=1)           # nothing converged yet
    assert e.value.code == rh.RH_ESTATE
    bad = ctx.surrogate_state()
    bad[3] = np.nan
    with pytest.raises(rh.RhError):
        ctx.surrogate_set_state(bad)
