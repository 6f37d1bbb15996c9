"""The learned-start path (the bench's headline path) against the oracles.

* prediction: rh_surrogate_predict against the FP64 reference network
  (oracle/mlp.py) on the same weights and columns, element by element;
* gradients: the BF16 training kernels against the FP64 reference, tensor by
  tensor (every weight matrix and bias vector);
* guess application: the populations of the learned start (n = e^{ln b} n*,
  renormalised to n_H) against the same formula applied here to the
  library's own prediction;
* solve: rh_solve from the learned guess on the bench's 256x256 cube, 32
  sampled columns against the oracle's tight fixed point.

BF16 tolerances: weights and activations carry 8 significant bits (unit
roundoff u = 2^-9 ~ 2e-3).  A layer's pre-activation z = sum_i w_i h_i with
both factors rounded has the error sum_i w_i h_i (e_wi + e_hi), e uniform in
[-u, u]: a relative spread sqrt(2/3) u ~ 1.6e-3 per layer, four layers in
quadrature with some gain through the later layers ~ 5e-3 of the output's
RMS (measured 4.9e-3, worst of 126k elements 3.4e-2, the larger outputs
carrying the larger errors).  The prediction is held to twice that: RMS
error 1e-2 and worst element 6e-2 of the output's RMS (a dropped bias, a
transposed or missing layer moves the output by tens of per cent); the
gradients to cosine > 0.999 and relative L2 < 2e-2 per tensor (measured
>= 0.99999 and <= 3.5e-3).
"""
import numpy as np
import pytest

import rh_synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rh():
    import paper_1411_1079_gb300 as m
    m.build()
    return m


def _seeded_state(rng, dims4, X):
    """Network parameters drawn here (He-scaled weights, small biases) and the
    standardisation of X, in the library's layout."""
    from oracle import mlp
    parts = []
    for di, do in mlp.layer_dims(*dims4):
        parts.append(rng.standard_normal(do * di) * np.sqrt(2.0 / di))
        parts.append(0.1 * rng.standard_normal(do))
    parts.append(X.mean(axis=0))
    parts.append(1.0 / np.maximum(X.std(axis=0), 1e-12 * (np.abs(X.mean(axis=0)) + 1)))
    return np.concatenate(parts)


@pytest.fixture(scope="module")
def net_case(rh, orc):
    """256 cube columns, the oracle's populations after a few iterations
    (targets) and LTE n_e (features), and a seeded 328-512-512-512-492
    network loaded into a GPU context."""
    from oracle import mlp
    atom = rh_synth.hydrogen_like_atom()
    cols = rh_synth.subset(rh_synth.chromosphere_cube(nx=32, ny=32, seed=11), slice(0, 256))
    o = orc.Oracle()
    o.setup_atom(atom)
    o.load_columns(cols)
    o.iterate(maxiter=25, tol=1e-3)
    n = o.populations()[0]
    ns, ne = o.lte()
    X = mlp.features(cols["T"], ne, cols["nH"], cols["vz"])
    Y = np.log(n / ns).reshape(n.shape[0], -1)
    dims = (X.shape[1], 512, 3, Y.shape[1])
    state = _seeded_state(np.random.default_rng(7), dims, X).astype(np.float32)
    ctx = rh.Context(0)
    ctx.setup_atom(atom)
    ctx.load_columns(cols)
    ctx.set_populations(n)
    ctx.surrogate_init(hidden=512, nhidden=3, seed=7)
    ctx.surrogate_set_state(state)
    return dict(atom=atom, cols=cols, n=n, ns=ns, X=X, Y=Y, dims=dims, state=state.astype(np.float64), ctx=ctx)


def test_predict_matches_reference_network(net_case):
    from oracle import mlp
    c = net_case
    got = c["ctx"].surrogate_predict().astype(np.float64).reshape(c["Y"].shape)
    ref = mlp.forward(c["state"], c["dims"], c["X"])
    scale = np.sqrt(np.mean(ref ** 2))
    err = np.abs(got - ref)
    print("predict: max |d|/rms %.2e, rms(d)/rms %.2e" % (err.max() / scale, np.sqrt(np.mean(err ** 2)) / scale))
    assert np.all(np.isfinite(got))
    assert err.max() < 6e-2 * scale
    assert np.sqrt(np.mean(err ** 2)) < 1e-2 * scale


def test_gradients_match_reference_per_tensor(net_case):
    from oracle import mlp
    c = net_case
    cols = np.arange(c["X"].shape[0])
    loss_g, grad_g = c["ctx"].surrogate_loss_grad(cols)
    loss_o, grad_o = mlp.loss_grad(c["state"], c["dims"], c["X"], c["Y"])
    assert loss_g == pytest.approx(loss_o, rel=1e-2)
    off = 0
    for li, (di, do) in enumerate(mlp.layer_dims(*c["dims"])):
        for name, size in (("W", di * do), ("b", do)):
            gg = grad_g[off:off + size].astype(np.float64)
            go = grad_o[off:off + size]
            off += size
            cos = gg @ go / (np.linalg.norm(gg) * np.linalg.norm(go))
            rl2 = np.linalg.norm(gg - go) / np.linalg.norm(go)
            print("layer %d %s: cos %.6f relL2 %.2e" % (li, name, cos, rl2))
            assert cos > 0.999 and rl2 < 2e-2, (li, name, cos, rl2)


def test_learned_guess_application(net_case):
    """start kind 1: n_i = e^{ln b_i} n*_i scaled per depth to sum n = n_H,
    from the library's own prediction (the prediction itself is checked
    above): FP64 arithmetic, within 1e-12."""
    c = net_case
    ctx = c["ctx"]
    lnb = ctx.surrogate_predict().astype(np.float64)
    ctx.start_populations(1)
    n, _, st, _ = ctx.populations()
    ref = c["ns"] * np.exp(np.clip(lnb, -80.0, 80.0))
    ref *= c["cols"]["nH"][:, None, :] / ref.sum(axis=1, keepdims=True)
    assert np.max(np.abs(n / ref - 1)) < 1e-12
    assert np.all(st == 4)                              # RH_COL_NOTRUN
    assert np.max(np.abs(n / c["ns"] - 1)) > 1e-2       # not the LTE start
    ctx.set_populations(c["n"])


def test_learned_start_solve_of_the_bench_cube_matches_oracle(rh, orc):
    """The bench's headline path: a network trained on a disjoint cube that
    the GPU MALI converged, then rh_solve from the learned guess on the 256 x
    256 cube (seed 1234, 65536 columns).  Run to 1e-6, 32 sampled columns are
    within 1e-3 of the oracle's 1e-9 fixed point; at the paper's 1e-3
    criterion the true error of the same columns is reported and bounded."""
    atom = rh_synth.hydrogen_like_atom()
    ctx = rh.Context(0)
    ctx.setup_atom(atom)
    ctx.load_columns(rh_synth.chromosphere_cube(128, 128, 82, seed=4321))
    ctx.solve(precision=1)
    ctx.surrogate_init(hidden=512, nhidden=3, seed=0)
    ctx.surrogate_train(epochs=10, batch=512, lr=2e-3, seed=1)
    cube = rh_synth.chromosphere_cube(256, 256, 82, seed=1234)
    ctx.load_columns(cube)
    s6 = ctx.solve(precision=1, start=1, tol=1e-6, maxiter=1000)
    n6, _, st6, _ = ctx.populations()
    ctx.load_columns(cube)
    s3 = ctx.solve(precision=1, start=1, tol=1e-3)
    n3, it3, st3, _ = ctx.populations()
    assert s3["n_converged"] == 65536 and s3["guess_fallback_depths"] == 0
    idx = np.sort(np.random.default_rng(2024).choice(65536, 32, replace=False))
    o = orc.Oracle()
    o.setup_atom(atom)
    o.load_columns(rh_synth.subset(cube, idx))
    o.iterate(maxiter=2000, tol=1e-9)
    no, _, sto, _ = o.populations()
    assert np.all(sto == 0) and np.all(st6[idx] == 0)
    d6 = np.abs(n6[idx] / no - 1).max(axis=(1, 2))
    d3 = np.abs(n3[idx] / no - 1).max(axis=(1, 2))
    print("learned start, 32 columns: max |dn/n| vs oracle at tol 1e-6: %.2e; at tol 1e-3 (true error): "
          "max %.2e, median %.2e" % (d6.max(), d3.max(), np.median(d3)))
    # the discrete problem can have two solutions in a column (both satisfy
    # the equations; which one a run reaches depends on its path): a sampled
    # column off by more than 1e-3 must be such a case -- one plain FP64
    # iteration from the GPU's state moves it by less than 1e-6
    far = d6 >= 1e-3
    assert far.sum() <= 1, d6
    if far.any():
        sub = rh_synth.subset(cube, idx[far])
        h = rh.Context(0)
        h.setup_atom(atom)
        h.load_columns(sub)
        h.set_populations(n6[idx[far]])
        h.iterate(maxiter=1, tol=0.0, ng_order=0, start=2, precision=0)
        assert np.all(h.populations()[3] < 1e-6)
    assert np.max(d3[~far]) < 3e-2
