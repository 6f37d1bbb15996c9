"""Depth-grid optimisation (Sect. 2.3) in the oracle, pinned without a GPU.

The oracle interpolates each column onto points equidistant in a monitor
built from the steps in log10 hydrogen column density (the optical-depth
proxy), ln T, v_z and the height itself, optionally without the layers
above z_top.  Pins: the ends and the order of the grid; exact
interpolation of profiles that are linear (T, v_z) or exponential (n_H,
n_e) in height; a uniform grid where the monitor is uniform; more points
inside a temperature jump than a uniform grid puts there; the top cut; and
the purpose -- the emergent intensity of the NLTE solution converges as the
optimised grid is refined."""
import numpy as np
import pytest

import rh_synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _oracle(orc, cols, atom=None, ne=None):
    o = orc.Oracle()
    o.setup_atom(atom or rh_synth.small_atom())
    o.load_columns(cols, ne=ne)
    return o


def test_regrid_ends_order_and_exact_profiles(orc):
    """T and v_z linear in z, n_H and n_e exponential: every new point carries
    the exact profile values at its height; the ends are kept; z decreases."""
    z = np.linspace(2.0e6, -1.0e5, 57)[None, :]
    T = 4000.0 + 2.0e-3 * (2.0e6 - z)           # 4000 K .. 8200 K, linear
    vz = 3.0e3 - 2.5e-3 * (2.0e6 - z)            # linear, crosses zero
    nH = 1e23 * np.exp(-z / 1.7e5)
    ne = 1e18 * np.exp(-z / 2.3e5)
    o = _oracle(orc, {"z": z, "T": T, "nH": nH, "vz": vz}, ne=ne)
    o.regrid(90)
    c = o.columns()
    zn = c["z"][0]
    assert zn[0] == z[0, 0] and zn[-1] == z[0, -1]
    assert np.all(np.diff(zn) < 0)
    assert np.allclose(c["T"][0], 4000.0 + 2.0e-3 * (2.0e6 - zn), rtol=1e-13, atol=0)
    assert np.allclose(c["vz"][0], 3.0e3 - 2.5e-3 * (2.0e6 - zn), rtol=0, atol=1e-9)
    assert np.allclose(c["nH"][0], 1e23 * np.exp(-zn / 1.7e5), rtol=1e-12, atol=0)
    _, ne_new = o.lte()
    assert np.allclose(ne_new[0], 1e18 * np.exp(-zn / 2.3e5), rtol=1e-12, atol=0)
    # the monitor is not uniform here (T and v_z change): the grid is not either
    dz = -np.diff(zn)
    assert dz.max() / dz.min() > 1.05


def test_regrid_uniform_monitor_gives_uniform_grid(orc):
    """Isothermal, static, exponential n_H: every monitor term grows linearly
    with height, so the points are equally spaced."""
    z = np.linspace(2.0e6, -1.0e5, 60)[None, :]
    cols = {"z": z, "T": np.full_like(z, 6000.0), "nH": 1e23 * np.exp(-z / 1.5e5), "vz": np.zeros_like(z)}
    o = _oracle(orc, cols)
    o.regrid(41)
    dz = -np.diff(o.columns()["z"][0])
    assert np.ptp(dz) / dz.mean() < 1e-12


def test_regrid_resolves_a_temperature_jump(orc):
    """A transition-region jump (8 kK to 40 kK over 40 km) gets many more
    points than the uniform grid of the same size, and the steps inside
    it stay below a few per cent in ln T per point."""
    z = np.linspace(3.0e6, -1.0e5, 311)[None, :]
    zk = z / 1e3
    T = np.where(zk > 2540, 40000.0, np.where(zk < 2500, 8000.0, 8000.0 + (zk - 2500) / 40 * 32000.0))
    T = np.where(zk < 500, 6000.0, T)
    cols = {"z": z, "T": T, "nH": 1e23 * np.exp(-z / 1.5e5), "vz": np.zeros_like(z)}
    o = _oracle(orc, cols)
    o.regrid(100, dlnT=0.05)
    c = o.columns()
    zn = c["z"][0] / 1e3
    inside = np.sum((zn > 2500) & (zn < 2540))
    uniform = 40.0 / (3100.0 / 99)
    assert inside >= 8 * uniform, (inside, uniform)
    Tn = c["T"][0]
    jump = (zn[:-1] <= 2541) & (zn[1:] >= 2499)
    assert np.max(np.abs(np.diff(np.log(Tn)))[jump]) < 0.2


def test_regrid_top_cut(orc):
    """z_top removes the layers above it: the new top is z_top itself, with
    the profile interpolated there, and the grid below is the optimised grid
    of the remaining column."""
    cols = rh_synth.chromosphere_column(ndep=82)
    o = _oracle(orc, cols)
    o.regrid(60, z_top=1.8e6)
    c = o.columns()
    assert c["z"][0, 0] == 1.8e6 and c["z"][0, -1] == cols["z"][0, -1]
    zk = cols["z"][0]
    T_at = np.interp(1.8e6, zk[::-1], cols["T"][0][::-1])
    assert c["T"][0, 0] == pytest.approx(T_at, rel=1e-13)
    lnH_at = np.interp(1.8e6, zk[::-1], np.log(cols["nH"][0][::-1]))
    assert np.log(c["nH"][0, 0]) == pytest.approx(lnH_at, rel=1e-13)
    with pytest.raises(RuntimeError):
        o2 = _oracle(orc, cols)
        o2.regrid(60, z_top=-2.0e5)      # below the column: nothing left


def test_regrid_refinement_converges_the_emergent_intensity(orc):
    """The purpose of the optimised grid: the emergent intensities of the
    converged NLTE solution converge as the grid is refined -- successive
    differences (41, 82, 164, 328, 656 points) fall monotonically, four
    times or more from the first to the last -- in the Lyman alpha wing, the
    n = 2-3 line core and the Lyman continuum.  (The Lyman alpha core is
    left out: its optical depth at the column's top point is >> 1, so the
    emergent core samples the top layer, which every refinement thins, and
    it converges far more slowly.)"""
    atom = rh_synth.hydrogen_like_atom(nbound=3, lyman_nlambda=24, line_nlambda=16, cont_nlambda=10, nmu=3)
    base = rh_synth.chromosphere_column(ndep=82)
    info = _oracle(orc, base, atom).atom_info()
    c, nu = 2.99792458e8, info["nu0"]
    lam = np.array([c / nu[0] * (1 + 1e-4), c / nu[2], 9.0e-8])
    I = {}
    for M in (41, 82, 164, 328, 656):
        o = _oracle(orc, base, atom)
        o.regrid(M)
        o.iterate(maxiter=3000, tol=1e-10)
        assert np.all(o.populations()[2] == 0)
        I[M] = o.emergent_spectrum(1.0, lam)[0]
    Ms = sorted(I)
    d = np.array([np.abs(I[b] / I[a] - 1) for a, b in zip(Ms, Ms[1:])])
    assert np.all(np.diff(d, axis=0) < 0), d
    assert np.all(d[-1] < d[0] / 4), d
