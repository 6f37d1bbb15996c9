"""Overlapping lines (Sect. 2.1: transitions overlapping in wavelength are
treated together).  With wide line wings the Lyman beta, gamma and delta
lines overlap each other, and two Balmer lines share wavelengths with a
continuum, so 32-wavelength tiles of the grid hold two or three lines: the
cross terms between lines and the per-line profile rows of the column
kernel's cache are exercised.  FP64: identical schedule without Ng against
the oracle, within 1e-9 per column.  FP32: the cached profiles (rh_iterate)
against the profiles evaluated in the sweep (rh_iterate_noalloc on a context
that never allocated the cache).  The profile arithmetic is the same in both
to the bit; the two kernels may fuse the sweep's other multiply-adds
differently, so they agree to FP32 rounding: FP32_SWEEP_TOL = 32 u (u =
2^-24), against 2.4 u seen after three iterations."""
import numpy as np
import pytest

import rh_synth

FP64_TOL = 1e-9
FP32_SWEEP_TOL = 32 * 2.0 ** -24
QWING = 1000.0        # line half-width in reference Doppler widths


@pytest.fixture(scope="module")
def atom():
    return rh_synth.hydrogen_like_atom(qwing=QWING)


@pytest.fixture(scope="module")
def cols():
    cube = rh_synth.chromosphere_cube(nx=32, ny=32, seed=11)
    base = rh_synth.chromosphere_column()
    pick = rh_synth.subset(cube, [17, 511, 1000])
    return {k: np.concatenate([base[k], pick[k]]) for k in base}


def test_grid_has_overlapping_lines(orc, atom):
    o = orc.Oracle()
    o.setup_atom(atom)
    g = o.grid()
    nline = len(atom["line_l"])
    lines_at = [int(np.sum(g["act"][i, :g["nact"][i]] < nline)) for i in range(len(g["nu"]))]
    assert max(lines_at) >= 2
    assert max(g["nact"]) <= 3


@pytest.mark.gpu
def test_fp64_fixed_schedule_matches_oracle(orc, atom, cols):
    import paper_1411_1079_gb300 as rh
    rh.build()
    g = rh.Context(0)
    g.setup_atom(atom)
    g.load_columns(cols)
    o = orc.Oracle()
    o.setup_atom(atom)
    o.load_columns(cols)
    sg = g.iterate(maxiter=3, tol=0.0, precision=0, ng_order=0)
    so = o.iterate(maxiter=3, tol=0.0, ng_order=0)
    ng, itg, stg, _ = g.populations()
    no, ito, sto, _ = o.populations()
    assert np.array_equal(itg, ito) and np.array_equal(stg, sto)
    assert float(np.max(np.abs(ng / no - 1))) < FP64_TOL
    assert sg["pts"] == so["pts"]


@pytest.mark.gpu
def test_fp32_cached_profiles_equal_profiles_in_sweep(atom, cols):
    import torch

    import paper_1411_1079_gb300 as rh
    rh.build()
    kw = dict(maxiter=3, tol=0.0, ng_order=0, precision=1)
    cached = rh.Context(0)
    cached.setup_atom(atom)
    cached.load_columns(cols)
    cached.iterate(**kw)
    n_ref = cached.populations()[0]
    fresh = rh.Context(0)          # no rh_iterate yet: no profile cache
    fresh.setup_atom(atom)
    fresh.load_columns(cols)
    ncol, ndep = cols["T"].shape
    n_out = torch.zeros((ncol, atom["nlev"], ndep), dtype=torch.float64, device="cuda")
    it_out = torch.zeros(ncol, dtype=torch.int32, device="cuda")
    st_out = torch.zeros(ncol, dtype=torch.uint8, device="cuda")
    dm_out = torch.zeros(ncol, dtype=torch.float64, device="cuda")
    fresh.iterate_noalloc(n_out, it_out, st_out, dm_out, **kw)
    torch.cuda.synchronize()
    assert float(np.max(np.abs(n_out.cpu().numpy() / n_ref - 1))) < FP32_SWEEP_TOL
