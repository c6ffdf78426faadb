"""Pins of the oracle's untabulated transport (Oracle(..., exact=True)).

The stepping loop of the paper's method reads interpolated tables and samples
sampling tables (Sec. 3.5, Sec. 6.3).  The untabulated transport replaces
every tabulated quantity by its definition: cross sections from their
formulas at the track's own energy, the range and its inverse by quadrature
and root finding, and every final state by rejection from its differential
cross section.  Each piece is pinned here against a route independent of
it (scipy quadrature, chi-square against DCS bin integrals, a closed-form
transmission), no GPU needed.  The comparison of whole showers between the
tabulated and the untabulated transport is in test_tabulation.py.
"""
import math

import numpy as np
import pytest
from scipy import integrate, stats

from paper_2005_00949_gb300 import workloads as W

ME = 0.51099895
M_COMPTON, M_PAIR, M_BREM, M_MOLLER, M_BHABHA, M_ANNIH = range(6)


# ------------------------------------------------------------------ samplers
def _limits(model, E, cut):
    if model == M_MOLLER:
        return cut / E, 0.5, "inv"
    if model == M_BHABHA:
        return cut / E, 1.0, "inv"
    if model == M_ANNIH:
        g = E / ME + 1.0
        return 0.5 * (1.0 - math.sqrt((g - 1.0) / (g + 1.0))), 0.5, "log"
    if model == M_PAIR:
        return ME / E, 1.0 - ME / E, "lin"
    if model == M_BREM:
        return cut, E, "log"
    return 1.0 / (1.0 + 2.0 * E / ME), 1.0, "log"


def _edges(lo, hi, kind, n):
    t = np.linspace(0.0, 1.0, n + 1)
    if kind == "lin":
        return lo + t * (hi - lo)
    if kind == "log":
        return lo * (hi / lo) ** t
    return 1.0 / (1.0 / lo - t * (1.0 / lo - 1.0 / hi))  # equal steps in 1/eps


@pytest.mark.parametrize("model,E", [
    (M_MOLLER, 2.5), (M_MOLLER, 40.0), (M_MOLLER, 5e4),
    (M_BHABHA, 1.3), (M_BHABHA, 30.0), (M_BHABHA, 5e4),
    (M_ANNIH, 0.05), (M_ANNIH, 3.0), (M_ANNIH, 2e4),
    (M_COMPTON, 0.02), (M_PAIR, 3.0), (M_BREM, 2e3),
])
def test_exact_sampler_matches_dcs(oracle_mod, model, E):
    """Samples of the exact sampler against the bin integrals of the DCS
    (chi-square over 40 bins; e cut and gamma cut 1 MeV)."""
    o = oracle_mod.Oracle(W.pbps_electrons(1), exact=True)
    cut = {M_MOLLER: 1.0, M_BHABHA: 1.0, M_BREM: 1.0}.get(model, 0.0)
    n = 40_000
    v = np.empty(n)
    tr = np.empty(n)
    for i in range(n):
        v[i], _, tr[i] = o.exact_sample(model, E, (i, 3, 11, 0xBEEF, 0x5EED))
    lo, hi, kind = _limits(model, E, cut)
    assert v.min() >= lo * (1 - 1e-12) and v.max() <= hi * (1 + 1e-12)
    edges = _edges(lo, hi, kind, 40)
    want = np.array([integrate.quad(lambda x: oracle_mod.Oracle.dcs(model, E, x, cut), a, b,
                                    epsrel=1e-11, limit=200)[0] for a, b in zip(edges[:-1], edges[1:])])
    want = want / want.sum() * n
    got = np.histogram(v, edges)[0]
    ok = want > 20
    chi2 = ((got[ok] - want[ok]) ** 2 / want[ok]).sum()
    assert stats.chi2.sf(chi2, ok.sum() - 1) > 1e-3, (model, E, chi2)
    assert tr.max() < 200  # the acceptance never collapses


@pytest.mark.parametrize("model", [M_MOLLER, M_BHABHA, M_ANNIH])
def test_exact_acceptance_ratio_is_bounded(oracle_mod, model):
    """The acceptance ratio of the three new samplers (DCS in the proposal's
    variable over its bound) stays within [0, 1] on dense grids over the whole
    kinematic range, at energies from just above threshold to 1 TeV."""
    Oc = oracle_mod.Oracle
    cut = 1.0
    for E in 10.0 ** np.linspace(-2.9, 6, 60):
        g = E / ME + 1.0
        b2 = 1.0 - 1.0 / (g * g)
        if model == M_MOLLER:
            if E <= 2 * cut * 1.0001:
                continue
            xc = cut / E
            eps = xc / (1.0 - np.linspace(0, 1, 4001) * (1.0 - 2.0 * xc))
            C1 = ((g - 1) / g) ** 2
            r = np.array([e * e * Oc.dcs(model, E, e, cut) for e in eps]) / (2.0 + 0.25 * C1)
        elif model == M_BHABHA:
            if E <= cut * 1.0001:
                continue
            xc = cut / E
            eps = xc / (1.0 - np.linspace(0, 1, 4001) * (1.0 - xc))
            r = np.array([b2 * e * e * Oc.dcs(model, E, e, cut) for e in eps])
        else:
            lo, hi, _ = _limits(model, E, 0.0)
            eps = lo * (hi / lo) ** np.linspace(0, 1, 4001)
            r = np.array([e * Oc.dcs(model, E, e, 0.0) for e in eps]) / (1.5 * g * g + 5 * g - 2.5)
        assert r.max() <= 1.0 + 1e-12 and r.min() >= -1e-12, (model, E, r.min(), r.max())


# ------------------------------------------------------------------ range and loss
def _inv_S(o, ptype, mat):
    return lambda e: 1.0 / o.dedx(ptype, mat, e)


@pytest.mark.parametrize("ptype", [W.ELECTRON, W.POSITRON])
def test_exact_range_is_quadrature_of_inverse_stopping_power(oracle_mod, ptype):
    """R(E) = Emin/S(Emin) + int_{Emin}^{E} dE/S by scipy's adaptive
    quadrature, to 1e-10, for energies across the grid (kinks included)."""
    o = oracle_mod.Oracle(W.pbps_electrons(1), exact=True)
    Emin = 1e-3
    rng = np.random.default_rng(21)
    for mat in (0, 1):
        f = _inv_S(o, ptype, mat)
        R0 = Emin / o.dedx(ptype, mat, Emin)
        for E in list(10.0 ** rng.uniform(-2.9, 4.5, 12)) + [1.0, 2.0, 2.0000001, 7.3]:
            pts = [p for p in (1.0, 2.0) if Emin < p < E]
            want = R0 + integrate.quad(f, Emin, E, epsrel=1e-13, epsabs=0, limit=400, points=pts or None)[0]
            got = o.range_at(ptype, mat, E)
            assert abs(got / want - 1.0) < 1e-10, (mat, E, got, want)


@pytest.mark.parametrize("ptype", [W.ELECTRON, W.POSITRON])
def test_exact_eloss_solves_the_range_equation(oracle_mod, ptype):
    """The post-step energy E' satisfies int_{E'}^{E} dE/S = s (scipy
    quadrature) to 1e-9 of s, for steps from 1e-7 of the range to the whole
    range; a step of at least the range stops the track."""
    o = oracle_mod.Oracle(W.pbps_electrons(1), exact=True)
    rng = np.random.default_rng(22)
    for mat in (0, 1):
        f = _inv_S(o, ptype, mat)
        for _ in range(40):
            E = 10.0 ** rng.uniform(-2.5, 4.5)
            R = o.range_at(ptype, mat, E)
            s = R * 10.0 ** rng.uniform(-7, math.log10(0.999))
            Ep = o.eloss_exact(ptype, mat, E, s)
            assert 0.0 < Ep < E
            pts = [p for p in (1.0, 2.0) if Ep < p < E]
            got = integrate.quad(f, Ep, E, epsrel=1e-13, epsabs=0, limit=400, points=pts or None)[0]
            assert abs(got - s) < 1e-9 * s + 1e-15 * R, (mat, E, s, Ep, got)
        E = 50.0
        assert o.eloss_exact(ptype, mat, E, o.range_at(ptype, mat, E)) == 0.0
        assert o.eloss_exact(ptype, mat, E, 0.0) == E


def test_tabulated_range_error_is_the_interpolation_error(oracle_mod):
    """At mid-node energies the tabulated range (ln R linear in ln E between
    exact node values) differs from the untabulated one by the error of
    linear interpolation of ln R, ln(R_tab / R) = h^2/8 d2(ln R)/d(ln E)^2
    (h = ln 10 / 32), to within 5 % of itself: the tables carry no error
    beyond their discretisation.  The same discretisation moves the post-step
    energy of a step of 5 % of the range by at most 1 % of the energy lost
    (with R itself linear in ln E it was up to 3 %: the stopping power between
    nodes is the interval's mean, off by up to +-3.6 %)."""
    o = oracle_mod.Oracle(W.pbps_electrons(1), exact=True)
    g = o.grid()
    h = math.log(10.0) / 32
    for ptype, q in ((W.ELECTRON, 2), (W.POSITRON, 3)):
        for mat in (0, 1):
            for E in np.sqrt(g[:-1] * g[1:])[3:280:9]:
                R = o.range_at(ptype, mat, E)
                Lp = math.log(o.range_at(ptype, mat, E * math.exp(0.5 * h)))
                Lm = math.log(o.range_at(ptype, mat, E * math.exp(-0.5 * h)))
                want = h * h / 8.0 * (Lp - 2.0 * math.log(R) + Lm) / (0.5 * h) ** 2
                got = math.log(o.lookup(ptype, q, mat, E)[0] / R)
                assert abs(got - want) < 0.05 * abs(want) + 1e-12, (ptype, mat, E, got, want)
                s = 0.05 * R
                a = o.eloss_exact(ptype, mat, E, s)
                b = o.eloss(ptype, mat, E, s)[0]
                assert abs(a - b) < 0.01 * (E - a), (ptype, mat, E, a, b)


# ------------------------------------------------------------------ transport
def test_exact_transmission_is_exp_minus_mu_x(oracle_mod):
    """Untabulated transport: 1 MeV photons through 10 cm water-like leave
    unscattered with probability exp(-mu x) = 0.49359."""
    wl = W.photon_slab(100_000)
    o = oracle_mod.Oracle(wl, exact=True)
    r = o.transport(n_threads=8)
    f = r["counts"][:, 10].mean()
    T = 0.49359
    assert abs(f - T) < 3 * math.sqrt(T * (1 - T) / wl.n_events)


@pytest.mark.parametrize("make", [lambda: W.pbps_electrons(40, 2000.0),
                                  lambda: W.pbps_mixed(30).subset(30),
                                  lambda: W.with_msc(W.with_field(W.pblar_testem3(10, 1000.0), 4.0, 1))])
def test_exact_transport_conserves_energy_and_charge(oracle_mod, make):
    wl = make()
    if wl.name.startswith("mixed"):
        wl.primaries["E"] = np.minimum(wl.primaries["E"], 3000.0)
    r = oracle_mod.Oracle(wl, exact=True).transport(n_threads=8)
    c = r["counts"]
    T0 = np.zeros(wl.n_events)
    np.add.at(T0, wl.primaries["event"], wl.primaries["E"])
    npos = np.zeros(wl.n_events)
    np.add.at(npos, wl.primaries["event"], (wl.primaries["type"] == W.POSITRON).astype(float))
    resid = (r["edep"].sum(1) + r["escape"] - (T0 + 2 * ME * (c[:, 8] - c[:, 7]))) / T0
    assert np.abs(resid).max() < 1e-9
    assert np.all(c[:, 7] + npos == c[:, 8] + c[:, 9])


def test_exact_mode_refuses_the_integral_approach(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.Oracle(W.with_integral(W.pbps_electrons(1)), exact=True)
