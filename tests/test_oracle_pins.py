"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the printed
Cash-Karp table, Butcher order conditions, closed-form solutions of linear and
quadratic decay, the Chebyshev stability polynomial of RKC (evaluated with
numpy's Chebyshev module), the exact Gershgorin bound of a linear chain,
ideal-gas limits of the rate expressions, conservation laws, and a tight
scipy reference trajectory.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from numpy.polynomial import chebyshev as C

import oracle
from paper_1309_2710_gb300 import synth
from tests import mechs

R_GAS = 8.314462618
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_rkck():
    rows = []
    with open(os.path.join(GOLDEN, "rkck_table.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([Fraction(x) for x in line.split()[1:]])
    a = [r[0] for r in rows]
    b = [r[1:6] for r in rows]
    c = [r[6] for r in rows]
    cs = [r[7] for r in rows]
    return a, b, c, cs


# --------------------------------------------------------------- Table 1 ---
def test_rkck_table_is_the_printed_table():
    """Table 1 (T:rkck): every oracle coefficient is the nearest double of the
    printed rational."""
    a, b, c, cs = _golden_rkck()
    oa, ob, oc, ocs = oracle.rkck_table()
    for i in range(6):
        assert oa[i] == float(a[i])
        assert oc[i] == float(c[i])
        assert ocs[i] == float(cs[i])
        for j in range(5):
            assert ob[i, j] == float(b[i][j])


def _trees(order):
    """Rooted trees up to `order` as sorted tuples of children."""
    by_n = {1: [()]}
    for n in range(2, order + 1):
        out = set()

        def parts(remaining, minchild, acc):
            if remaining == 0:
                out.add(tuple(sorted(acc)))
                return
            for k in range(1, remaining + 1):
                for t in by_n[k]:
                    if (k, t) < minchild:
                        continue
                    parts(remaining - k, (k, t), acc + [t])

        parts(n - 1, (0, ()), [])
        by_n[n] = sorted(out)
    return by_n


def _size(t):
    return 1 + sum(_size(ch) for ch in t)


def _gamma(t):
    g = _size(t)
    for ch in t:
        g *= _gamma(ch)
    return g


def _phi(t, A):
    """Elementary weight vector of tree t for matrix A (exact Fractions)."""
    s = len(A)
    v = [Fraction(1)] * s
    for ch in t:
        pc = _phi(ch, A)
        w = [sum(A[i][j] * pc[j] for j in range(s)) for i in range(s)]
        v = [v[i] * w[i] for i in range(s)]
    return v


def test_rkck_order_conditions_from_oracle_table():
    """Butcher order conditions: the fifth-order weights satisfy all 17
    conditions up to order 5 and the embedded weights all 8 up to order 4
    (checked on the oracle's doubles), and row sums equal the nodes."""
    oa, ob, oc, ocs = oracle.rkck_table()
    A = [[Fraction(float(ob[i, j])) if j < i else Fraction(0) for j in range(6)] for i in range(6)]
    trees = _trees(5)
    ncond = {4: 0, 5: 0}
    for n, ts in trees.items():
        for t in ts:
            ph = _phi(t, A)
            lhs5 = sum(Fraction(float(oc[i])) * ph[i] for i in range(6))
            assert abs(float(lhs5) - 1.0 / _gamma(t)) < 1e-15, (n, t)
            ncond[5] += 1
            if n <= 4:
                lhs4 = sum(Fraction(float(ocs[i])) * ph[i] for i in range(6))
                assert abs(float(lhs4) - 1.0 / _gamma(t)) < 1e-15, (n, t)
                ncond[4] += 1
    assert ncond == {4: 8, 5: 17}
    for i in range(6):
        assert abs(sum(ob[i]) - oa[i]) < 1e-15
    # the embedded solution is not fifth order: some order-5 condition fails
    bad = 0
    for t in trees[5]:
        ph = _phi(t, A)
        if abs(float(sum(Fraction(float(ocs[i])) * ph[i] for i in range(6))) - 1 / _gamma(t)) > 1e-6:
            bad += 1
    assert bad > 0


# ----------------------------------------------------------- rate terms ---
def test_unimolecular_decay_closed_form():
    """A -> B with equal molar masses: dY_A/dt = -k Y_A, k from Eq. (E:rxn-const)
    evaluated here with A=3e5, beta=0.7, E=4e4 J/mol at 1234 K."""
    m = mechs.mech([28.0, 28.0], [dict(reac=[0], prod=[1], A=3e5, beta=0.7, Ea=4e4)])
    om = oracle.Mech(m)
    T = 1234.0
    k = 3e5 * T ** 0.7 * math.exp(-4e4 / (R_GAS * T))
    for p in (1e4, 101325.0, 2e6):
        y = np.array([0.3, 0.7])
        f = oracle.rates(om, T, p, y)
        assert f[0] == pytest.approx(-k * 0.3, rel=1e-14, abs=0)
        assert f[1] == pytest.approx(k * 0.3, rel=1e-14, abs=0)


def test_third_body_unit_efficiency_is_total_concentration():
    """With all efficiencies 1, [M] is the total concentration p/(RT) (ideal
    gas, mol/cm^3), whatever the composition."""
    W = [2.0, 32.0, 17.0, 17.0, 28.0]
    base = dict(reac=[0, 1], prod=[2, 3], A=1e12, beta=0.0, Ea=0.0)
    plain = mechs.mech(W, [base])
    tb = mechs.mech(W, [dict(base, type=1)], eff_rows=[[1.0] * 5])
    op, ot = oracle.Mech(plain), oracle.Mech(tb)
    rng = np.random.default_rng(5)
    for _ in range(4):
        y = rng.uniform(0.05, 1.0, 5)
        y /= y.sum()
        T = rng.uniform(800, 2000)
        p = rng.uniform(5e4, 2e6)
        ctot = p / (R_GAS * T) * 1e-6
        fp = oracle.rates(op, T, p, y)
        ft = oracle.rates(ot, T, p, y)
        np.testing.assert_allclose(ft, fp * ctot, rtol=1e-13)


def test_falloff_limits():
    """Lindemann falloff tends to the high-pressure rate when k0[M] >> k_inf and
    to a third-body rate with k0 when k0[M] << k_inf."""
    W = [2.0, 32.0, 17.0, 17.0, 28.0]
    eff = [[1.0, 2.0, 0.5, 1.5, 1.0]]
    hi = dict(reac=[0, 1], prod=[2, 3], A=1e11, type=2, A0=1e30)
    lo = dict(reac=[0, 1], prod=[2, 3], A=1e11, type=2, A0=1e-3)
    plain = oracle.Mech(mechs.mech(W, [dict(reac=[0, 1], prod=[2, 3], A=1e11)]))
    tb0 = oracle.Mech(mechs.mech(W, [dict(reac=[0, 1], prod=[2, 3], A=1e-3, type=1)], eff))
    fhi = oracle.Mech(mechs.mech(W, [hi], eff))
    flo = oracle.Mech(mechs.mech(W, [lo], eff))
    y = np.array([0.1, 0.3, 0.05, 0.05, 0.5])
    T, p = 1500.0, 101325.0
    np.testing.assert_allclose(oracle.rates(fhi, T, p, y), oracle.rates(plain, T, p, y), rtol=1e-9)
    np.testing.assert_allclose(oracle.rates(flo, T, p, y), oracle.rates(tb0, T, p, y), rtol=1e-9)


def test_pressure_order_and_density():
    """Bimolecular source terms scale with p (one power of density), the
    third-body ones with p^2; at fixed p and T they scale with the mean molar
    mass Wbar (ideal gas rho = p Wbar / RT)."""
    W = [2.0, 32.0, 17.0, 17.0, 28.0]
    r = dict(reac=[0, 1], prod=[2, 3], A=1e12)
    om = oracle.Mech(mechs.mech(W, [r]))
    ot = oracle.Mech(mechs.mech(W, [dict(r, type=1)], [[1, 1, 1, 1, 1]]))
    y = np.array([0.1, 0.3, 0.05, 0.05, 0.5])
    T = 1300.0
    f1 = oracle.rates(om, T, 1e5, y)
    f2 = oracle.rates(om, T, 3e5, y)
    np.testing.assert_allclose(f2, 3 * f1, rtol=1e-13)
    np.testing.assert_allclose(oracle.rates(ot, T, 3e5, y), 9 * oracle.rates(ot, T, 1e5, y), rtol=1e-13)
    # swap part of the inert diluent (W=28) for a heavier inert (same slot count):
    # reactant mass fractions fixed, Wbar changes, rates scale with Wbar.
    W2 = [2.0, 32.0, 17.0, 17.0, 56.0]
    om2 = oracle.Mech(mechs.mech(W2, [r]))
    wbar1 = 1.0 / np.sum(y / np.array(W))
    wbar2 = 1.0 / np.sum(y / np.array(W2))
    f3 = oracle.rates(om2, T, 1e5, y)
    np.testing.assert_allclose(f3[:4], f1[:4] * wbar2 / wbar1, rtol=1e-13)


def test_quadratic_decay_closed_form_rate():
    """A + A -> B + B: Omega = k C_A^2 and dC_A/dt = -2 k C_A^2."""
    W = 30.0
    om = oracle.Mech(mechs.mech([W, W], [dict(reac=[0, 0], prod=[1, 1], A=2e12)]))
    T, p = 1000.0, 101325.0
    y = np.array([0.4, 0.6])
    rho = p * W / (R_GAS * T) * 1e-6  # all molar masses equal: Wbar = W
    cA = rho * y[0] / W
    f = oracle.rates(om, T, p, y)
    assert f[0] == pytest.approx(W / rho * (-2 * 2e12 * cA * cA), rel=1e-13, abs=0)


@pytest.mark.parametrize("name", list(synth.WORKLOADS))
def test_source_terms_conserve_mass_and_elements(name):
    """Sum_i dY_i/dt = 0 and sum_i a_ei (dY_i/dt)/W_i = 0 for every element e
    (each reaction balances atoms), on the synthetic mechanisms."""
    m = synth.workload_mechanism(name)
    om = oracle.Mech(m)
    T, p, Y = synth.workload_states(name, m, cells=6)
    for c in range(6):
        f = oracle.rates(om, T[c], p[c], Y[:, c])
        scale = np.abs(f).sum()
        assert scale > 0
        assert abs(f.sum()) < 1e-13 * scale
        mol = f / m.W
        for e in range(len(m.elements)):
            assert abs((m.comp[:, e] * mol).sum()) < 1e-13 * (np.abs(mol) * m.comp[:, e]).sum() + 1e-300


# ------------------------------------------------------------------ RKCK ---
def test_rkck_local_order_on_linear_decay():
    """One Cash-Karp step on y' = -k y: the fifth-order local error scales as
    h^6 and the embedded fourth-order one as h^5 (Section 2.2)."""
    k = 1.0e6
    om = oracle.Mech(mechs.a_to_b(k))
    y0 = np.array([1.0, 0.0])
    e5, e4 = [], []
    for z in (0.08, 0.04, 0.02):
        y5, err = oracle.rkck_single(om, 1000.0, 1e5, y0, z / k)
        exact = math.exp(-z)
        e5.append(abs(y5[0] - exact))
        e4.append(abs(y5[0] - err[0] - exact))
    for i in range(2):
        assert 2 ** 5.6 < e5[i] / e5[i + 1] < 2 ** 6.4
        assert 2 ** 4.6 < e4[i] / e4[i + 1] < 2 ** 5.4


def test_rkck_step_matches_printed_table_exactly():
    """On y' = -k y one oracle step multiplies y by the stability function of
    the printed table, evaluated in exact rational arithmetic."""
    k = 1.0
    om = oracle.Mech(mechs.a_to_b(k))
    for z in (0.01, 0.3, 1.0, 2.5, 3.3):
        y5, err = oracle.rkck_single(om, 1000.0, 1e5, np.array([1.0, 0.0]), z / k)
        g5, g4 = _linear_rk_step(Fraction(-z))
        assert y5[0] == pytest.approx(float(g5), rel=1e-14, abs=1e-15)
        assert err[0] == pytest.approx(float(g5 - g4), rel=1e-10, abs=1e-16)


def _linear_rk_step(z):
    """Exact one-step factor and embedded factor of the printed table on
    y' = lambda y, z = h lambda (rational arithmetic on the golden table)."""
    a, b, c, cs = _golden_rkck()
    k = []
    for i in range(6):
        arg = 1 + sum(b[i][j] * k[j] for j in range(i))
        k.append(z * arg)
    y5 = 1 + sum(c[i] * k[i] for i in range(6))
    y4 = 1 + sum(cs[i] * k[i] for i in range(6))
    return y5, y4


def test_rkck_controller_trace_on_linear_decay():
    """Hand-worked trace on A -> B: first trial step = dt, error ratio from the
    exact linear step of the printed table, and the Eq. (E:hnew) rule with the
    5x/10x limits, for the first attempts."""
    k = 3.0e7
    om = oracle.Mech(mechs.a_to_b(k))
    dt, rtol, atol = 1e-7, 1e-6, 1e-10
    y = np.array([0.9, 0.1])
    _, st, tr = oracle.trace_cell(om, 1000.0, 1e5, y, dt, rtol, atol, method=0)
    assert st == 0
    t, h = Fraction(0), Fraction(dt)
    ya, yb = Fraction(0.9), Fraction(0.1)
    for n in range(min(6, len(tr["h"]))):
        hh = min(h, Fraction(dt) - t)
        assert float(hh) == pytest.approx(tr["h"][n], rel=1e-10, abs=0)
        hh = Fraction(float(tr["h"][n]))
        z = Fraction(-k) * hh
        g5, g4 = _linear_rk_step(z)
        da = (g5 - g4) * ya
        fa = -k * ya
        tol_a = rtol * (abs(ya) + abs(hh * fa)) + atol
        tol_b = rtol * (abs(yb) + abs(hh * (-fa))) + atol
        errmax = max(abs(float(da)) / float(tol_a), abs(float(da)) / float(tol_b))
        assert errmax == pytest.approx(tr["err"][n], rel=1e-9, abs=0)
        errmax = float(tr["err"][n])
        if errmax <= 1:
            ya, yb = g5 * ya, yb + (1 - g5) * ya
            t += hh
            h = min(5 * hh, Fraction(0.9 * float(hh) * errmax ** -0.2))
        else:
            h = max(hh / 10, Fraction(0.9 * float(hh) * errmax ** -0.25))


# ------------------------------------------------------------------- RKC ---
def _cheb_parts(s):
    """T_s, T_s', T_s'' as numpy Chebyshev series."""
    ts = np.zeros(s + 1)
    ts[s] = 1.0
    return ts, C.chebder(ts, 1), C.chebder(ts, 2)


def _stability_poly(s, z):
    """P_s(z) = a_s + b_s T_s(w0 + w1 z), Section 2.3 (kappa = 2/13)."""
    w0 = 1 + (2.0 / 13.0) / s ** 2
    t, d1, d2 = _cheb_parts(s)
    Td1, Td2 = C.chebval(w0, d1), C.chebval(w0, d2)
    w1 = Td1 / Td2
    bs = Td2 / Td1 ** 2
    a_s = 1 - bs * C.chebval(w0, t)
    return a_s + bs * C.chebval(w0 + w1 * z, t)


@pytest.mark.parametrize("s", [2, 3, 4, 7, 16, 40, 100, 250])
def test_rkc_step_is_chebyshev_stability_polynomial(s):
    """One s-stage step on y' = -k y multiplies y by P_s(-k h)."""
    k = 1.0
    om = oracle.Mech(mechs.a_to_b(k))
    beta = ((s - 1) ** 2 - 1) / 1.54
    for frac in (0.0, 0.01, 0.3, 0.77, 1.0):
        z = -frac * max(beta, 0.5)
        ys = oracle.rkc_single(om, 1000.0, 1e5, np.array([1.0, 0.0]), -z / k, s)
        ref = _stability_poly(s, z)
        assert ys[0] == pytest.approx(ref, abs=2e-13 * s, rel=1e-11)
        assert ys[0] + ys[1] == pytest.approx(1.0, abs=1e-12)


@pytest.mark.parametrize("s", [2, 3, 5, 10, 50, 250])
def test_rkc_stable_on_stage_rule_interval(s):
    """|P_s(z)| <= 1 on [-((s-1)^2-1)/1.54, 0], the interval the stage rule
    s = 1 + sqrt(1 + 1.54 h sigma) allows (Section 2.3)."""
    k = 1.0
    om = oracle.Mech(mechs.a_to_b(k))
    beta = ((s - 1) ** 2 - 1) / 1.54
    for z in np.linspace(-beta, 0.0, 41):
        ys = oracle.rkc_single(om, 1000.0, 1e5, np.array([1.0, 0.0]), -z / k, s)
        assert abs(ys[0]) <= 1.0 + 1e-12


def test_rkc_second_order_consistency_of_polynomial():
    """P_s(z) = 1 + z + z^2/2 + O(z^3): the oracle step on y' = -k y has local
    error O(h^3)."""
    om = oracle.Mech(mechs.a_to_b(1.0))
    for s in (2, 5, 20):
        errs = []
        for h in (1e-2, 5e-3, 2.5e-3):
            ys = oracle.rkc_single(om, 1000.0, 1e5, np.array([1.0, 0.0]), h, s)
            errs.append(abs(ys[0] - math.exp(-h)))
        assert 2 ** 2.8 < errs[0] / errs[1] < 2 ** 3.2
        assert 2 ** 2.8 < errs[1] / errs[2] < 2 ** 3.2


@pytest.mark.parametrize("s", [2, 3, 8, 30, 250])
def test_rkc_first_stage_abscissa(s):
    """mu~_1 is the first stage abscissa c_1, and the paper fixes
    c_1 = c_2 / T_2'(w0) with c_2 = w1 T_2''(w0)/T_2'(w0) (Section 2.3).
    This pins b_1 = b_2."""
    co = oracle.rkc_coeffs(s)
    w0 = 1 + (2.0 / 13.0) / s ** 2
    _, d1s, d2s = _cheb_parts(s)
    w1 = C.chebval(w0, d1s) / C.chebval(w0, d2s)
    _, d12, d22 = _cheb_parts(2)
    c2 = w1 * C.chebval(w0, d22) / C.chebval(w0, d12)
    c1 = c2 / C.chebval(w0, d12)
    assert co["w0"] == pytest.approx(w0, rel=1e-15, abs=0)
    assert co["w1"] == pytest.approx(w1, rel=1e-12, abs=0)
    assert co["mut"][1] == pytest.approx(c1, rel=1e-12, abs=0)
    # c_j ~ (j^2 - 1)/(s^2 - 1) for 2 <= j <= s-1, c_s = 1
    for j in range(2, s):
        assert co["c"][j] == pytest.approx((j * j - 1) / (s * s - 1), rel=0.05, abs=0.01)
    assert co["c"][s] == 1.0


def test_rkc_second_order_convergence_nonlinear():
    """Fixed-stage RKC on A + A -> B + B (closed form C_A = C0/(1 + 2 k C0 t))
    converges with order 2."""
    W = 30.0
    kf = 4e11
    om = oracle.Mech(mechs.mech([W, W], [dict(reac=[0, 0], prod=[1, 1], A=kf)]))
    T, p = 1000.0, 101325.0
    rho = p * W / (R_GAS * T) * 1e-6
    y0 = np.array([0.8, 0.2])
    c0 = rho * y0[0] / W
    tend = 2.0 / (2 * kf * c0)
    exact = c0 / (1 + 2 * kf * c0 * tend) * W / rho
    errs = []
    for nsteps in (40, 80, 160):
        y = y0.copy()
        for _ in range(nsteps):
            y = oracle.rkc_single(om, T, p, y, tend / nsteps, 4)
        errs.append(abs(y[0] - exact))
    assert 2 ** 1.8 < errs[0] / errs[1] < 2 ** 2.2
    assert 2 ** 1.8 < errs[1] / errs[2] < 2 ** 2.2


def test_gershgorin_on_linear_chain():
    """A_0 -> A_1 -> ... with rates k_i has Jacobian rows with |-k_i| + |k_{i-1}|:
    the Gershgorin bound is max_i (k_i + k_{i-1}); the finite-difference
    Jacobian of a linear f reproduces it to ~sqrt(eps)."""
    ks = [3e8, 1e9, 2.5e8, 7e9, 1e3]
    om = oracle.Mech(mechs.chain(ks))
    exact = max([ks[0]] + [ks[i] + ks[i - 1] for i in range(1, len(ks))] + [ks[-1]])
    y = np.array([0.3, 0.2, 0.1, 0.25, 0.1, 0.05])
    sig = oracle.sigma(om, 1500.0, 101325.0, y, 1e-10)
    assert sig == pytest.approx(exact, rel=1e-6, abs=0)


def _rkc_linear_decay_replay(k, dt, rtol, atol, ya, yb, tr):
    """Replay, by hand, RKC on A -> B (sigma = k exactly) against an oracle
    trace: initial step from h0 = 1/sigma and Delta_0 (both in closed form),
    the stage count rule with its cap at 250 stages and the step reset
    h = ((250 - 1)^2 - 1)/(1.54 sigma), the step factor P_s(-k h) from numpy
    Chebyshev, the error estimate, and the step factors (0.8/err^(1/3) first
    and after a rejection, the predictive form otherwise). Returns the
    attempts' stage counts."""
    sigma = k  # rows of J = [[-k, 0], [k, 0]] both sum to k
    h0 = min(1.0 / sigma, dt)
    # Delta_0 = h0 (f(y + h0 f0) - f0): A component = k h0 ya, B = -k h0 ya
    d = k * h0 * ya
    d0 = math.sqrt(0.5 * ((d / (atol + rtol * ya)) ** 2 + (d / (atol + rtol * yb)) ** 2))
    h = min(0.1 * h0 / math.sqrt(d0), dt)
    t = 0.0
    prev = None
    rejected = False
    n_att = len(tr["h"])
    stages = []
    for n in range(n_att):
        hh = min(h, dt - t)
        s = max(2, int(math.floor(1 + math.sqrt(1 + 1.54 * hh * sigma))))
        if s > 250:  # the cap: 250 stages and the longest step they keep stable
            s = 250
            hh = ((250 - 1.0) ** 2 - 1.0) / (1.54 * sigma)
        assert tr["h"][n] == pytest.approx(hh, rel=1e-9, abs=0), n
        hh = tr["h"][n]
        assert tr["s"][n] == s, n
        assert tr["sigma"][n] == pytest.approx(sigma, rel=1e-6, abs=0)
        stages.append(s)
        g = _stability_poly(s, -k * hh)
        na = g * ya
        nb = yb + (1 - g) * ya
        fa0, fa1 = -k * ya, -k * na
        da = 0.8 * (ya - na) + 0.4 * hh * (fa0 + fa1)
        db = -da
        ta = atol + rtol * max(abs(ya), abs(na))
        tb = atol + rtol * max(abs(yb), abs(nb))
        err = math.sqrt(0.5 * ((da / ta) ** 2 + (db / tb) ** 2))
        # the estimate cancels terms of size |y|: allow their rounding (and,
        # at the cap, that of a 250-stage recursion)
        cancel = (4e-16 if s < 250 else 1e-13) * (abs(ya) + abs(na) + abs(hh * fa0)) / min(ta, tb)
        assert tr["err"][n] == pytest.approx(err, rel=1e-8, abs=cancel), n
        err = tr["err"][n]
        assert tr["accepted"][n] == (err <= 1.0)
        if err <= 1.0:
            if err == 0:
                fac = 10.0
            elif prev is None or rejected:
                fac = 0.8 / err ** (1 / 3)
            else:
                fac = 0.8 * (hh / prev[0]) * prev[1] ** (1 / 3) / err ** (2 / 3)
            prev = (hh, err)
            rejected = False
            ya, yb = na, nb
            t += hh
        else:
            fac = 0.8 / err ** (1 / 3)
            rejected = True
        h = min(10.0, max(0.1, fac)) * hh
    assert t == pytest.approx(dt, rel=1e-12, abs=0)
    return stages


def test_rkc_controller_trace_on_linear_decay():
    """Hand-worked RKC trace on A -> B (k dt = 200), every attempt to the
    end of the flow step."""
    k = 2.0e8
    om = oracle.Mech(mechs.a_to_b(k))
    dt, rtol, atol = 1e-6, 1e-6, 1e-10
    _, st, tr = oracle.trace_cell(om, 1000.0, 1e5, np.array([0.7, 0.3]), dt, rtol, atol, method=1)
    assert st == 0
    stages = _rkc_linear_decay_replay(k, dt, rtol, atol, 0.7, 0.3, tr)
    assert len(stages) > 10
    assert max(stages) >= 10  # the stage rule is exercised beyond s = 2


def test_rkc_stage_cap_on_stiff_linear_decay():
    """k dt = 2e5: once the transient has decayed the stage rule asks for more
    than 250 stages. The cap (Section 2.3 gives the rule s = 1 + sqrt(1 +
    1.54 h sigma); the cap is this build's reading) keeps s = 250 and takes
    the step that 250 stages keep stable; the hand replay follows every
    attempt, including the capped ones and the rejection."""
    k = 2.0e11
    om = oracle.Mech(mechs.a_to_b(k))
    dt, rtol, atol = 1e-6, 1e-6, 1e-10
    _, st, tr = oracle.trace_cell(om, 1000.0, 1e5, np.array([0.7, 0.3]), dt, rtol, atol, method=1)
    assert st == 0
    stages = _rkc_linear_decay_replay(k, dt, rtol, atol, 0.7, 0.3, tr)
    assert stages.count(250) >= 2
    assert (~tr["accepted"]).sum() >= 1


def _autocatalytic(k, W=20.0):
    """A + B -> B + B with equal molar masses."""
    return mechs.mech([W, W], [dict(reac=[0, 1], prod=[1, 1], A=k)])


def _sigma_schedule(accepted):
    """Attempts before which the spectral radius is estimated, by the rule of
    Section 2.3 as read here: before the first attempt, before the attempt
    that follows 25 accepted steps since the last estimate, and before the
    attempt that follows a rejection when the last estimate was made at an
    earlier point (an estimate at the same point would repeat itself)."""
    est, since, fresh, after_reject = [], 0, False, False
    for n, acc in enumerate(accepted):
        if n == 0 or since >= 25 or (after_reject and not fresh):
            est.append(n)
            since, fresh = 0, True
        if acc:
            since, fresh, after_reject = since + 1, False, False
        else:
            after_reject = True
    return est


@pytest.mark.parametrize("kPdt,yb0", [(12.0, 1e-3), (40.0, 1e-16)])
def test_rkc_sigma_refresh_schedule(kPdt, yb0):
    """A + B -> B + B, equal molar masses. With Y_A + Y_B = 1 the density is
    p W/(R T), dY_B/dt = k P Y_A Y_B with P = p/(R T) [mol/cm^3] (a logistic
    curve), and the Jacobian of f with each Y_k perturbed alone (the density
    moves with it) has rows +-k P (Y_B^2, Y_A^2): its Gershgorin bound is
    sigma = k P (Y_A^2 + Y_B^2), which falls to half and rises again as B
    takes over. The spectral radius each attempt used must change exactly at
    the attempts the schedule names and equal the closed form at the exact
    state of that moment; the counters must equal the hand count.
    k P dt = 12 from Y_B = 1e-3 refreshes for age and after rejections; k P dt
    = 40 from Y_B = 1e-16 rejects the very first attempt (the initial-step
    probe sees almost no change, and the first step spans an e^40 growth), so
    no second estimate may follow at the same point. In that second case B
    stays below atol for most of the step, where the error test does not
    follow it, so the integrated state lags the exact curve: its estimates are
    checked against the bounds k P / 2 <= sigma <= k P instead of the closed
    form at the exact state."""
    T, p = 1000.0, 1e5
    P = p * 1e-6 / (R_GAS * T)
    dt, rtol, atol = 1e-6, 1e-6, 1e-10
    k = kPdt / (P * dt)
    r = k * P
    om = oracle.Mech(_autocatalytic(k))
    y, st, tr = oracle.trace_cell(om, T, p, np.array([1 - yb0, yb0]), dt, rtol, atol, method=oracle.RKC)
    assert st == 0
    acc, sig, h = tr["accepted"], tr["sigma"], tr["h"]
    est = _sigma_schedule(acc)
    since_counts = set()
    for n in range(1, len(acc)):
        if n in est:
            assert sig[n] != sig[n - 1], n
        else:
            assert sig[n] == sig[n - 1], n
    t = np.concatenate([[0.0], np.cumsum(np.where(acc, h, 0.0))])[:-1]  # start time of each attempt
    follows_exact = kPdt < 20
    for i, n in enumerate(est):
        if follows_exact:
            yb = 1.0 / (1.0 + (1.0 / yb0 - 1.0) * math.exp(-r * t[n]))
            exact = r * ((1.0 - yb) ** 2 + yb ** 2)
            assert sig[n] == pytest.approx(exact, rel=1e-4, abs=0), n
        else:
            assert 0.5 * r * (1 - 1e-6) <= sig[n] <= r * (1 + 1e-6), n
        if i:
            since_counts.add(int(acc[est[i - 1]:n].sum()))
    assert any(c < 25 for c in since_counts)  # refreshed after a rejection
    if follows_exact:
        assert 25 in since_counts  # ... and for age
        assert sig.max() / sig.min() > 1.8  # sigma does move along the trajectory
    else:
        assert not acc[0] and 1 not in est  # no second estimate at the same point
    nfe, nacc, nrej, nsig, nfs = tr["stats"]
    assert (nacc, nrej) == (int(acc.sum()), int((~acc).sum()))
    assert nsig == len(est)
    assert nfs == 2 * len(est)  # two Gershgorin columns per estimate
    # f(y0), the estimates, the initial-step probe, and s evaluations per attempt
    assert nfe == 1 + nfs + 1 + int(tr["s"].sum())
    if follows_exact:
        assert y[1] == pytest.approx(1.0 / (1.0 + (1.0 / yb0 - 1.0) * math.exp(-r * dt)), rel=1e-4)
    assert y[0] == pytest.approx(1.0 - y[1], abs=1e-12)


def test_status_step_size_underflow():
    """Status 2 (the step size fell below 1e-20 dt), with the state left at the
    last accepted one (here the initial one).
    RKCK on A -> B with k = 1e300: every trial step overflows, each rejection
    divides the step by 10, and the call stops at the first step below
    1e-20 dt: 21 attempts from dt, 1 + 5 evaluations of f each.
    RKC: sigma = k, h0 = 1/k, and the initial-step probe gives
    h1 = 0.1 h0/||Delta_0||^(1/2) (closed form) below 1e-20 dt for k = 1e23,
    so the call stops before any attempt; for k = 2.5e21, h1 lies above the
    bound and the call runs until its step limit."""
    dt, rtol, atol = 1e-6, 1e-6, 1e-10
    y0 = np.array([0.7, 0.3])
    om = oracle.Mech(mechs.a_to_b(1e300))
    y, st, tr = oracle.trace_cell(om, 1000.0, 1e5, y0, dt, rtol, atol, method=oracle.RKCK)
    h, n = dt, 0
    while True:  # the same IEEE operations as the integrator's
        n += 1
        h = 0.1 * h
        if h < 1e-20 * dt:
            break
    assert st == 2
    assert len(tr["h"]) == n == 21 and not tr["accepted"].any()
    assert list(tr["stats"]) == [1 + 5 * n, 0, n, 0, 0]
    assert np.array_equal(y, y0)

    def h1(k):  # closed form of the RKC initial step on A -> B (sigma = k)
        d0 = math.sqrt(0.5 * ((0.7 / (atol + rtol * 0.7)) ** 2 + (0.7 / (atol + rtol * 0.3)) ** 2))
        return 0.1 / k / math.sqrt(d0)

    assert h1(1e23) < 1e-20 * dt < h1(2.5e21)
    y, st, tr = oracle.trace_cell(oracle.Mech(mechs.a_to_b(1e23)), 1000.0, 1e5, y0, dt, rtol, atol,
                                  method=oracle.RKC)
    assert st == 2 and len(tr["h"]) == 0
    assert list(tr["stats"]) == [4, 0, 0, 1, 2]  # f(y0), two columns, the probe
    assert np.array_equal(y, y0)
    y, st, tr = oracle.trace_cell(oracle.Mech(mechs.a_to_b(2.5e21)), 1000.0, 1e5, y0, dt, rtol, atol,
                                  method=oracle.RKC, max_steps=5)
    assert st == 1 and len(tr["h"]) == 5
    assert tr["h"][0] == pytest.approx(h1(2.5e21), rel=1e-9)


# ------------------------------------------------------ whole integrator ---
def _tiny_mechanism(seed):
    return synth.make_mechanism(7, 16, ("H", "O"), tb_frac=0.2, fo_frac=0.1, seed=seed)


@pytest.mark.parametrize("method", [oracle.RKCK, oracle.RKC])
def test_integrator_against_tight_scipy_reference(method):
    """At rtol 1e-6 the integrated state is within a small multiple of the
    tolerance of a DOP853 trajectory at rtol 1e-13 using the same f."""
    integrate = pytest.importorskip("scipy.integrate")
    m = _tiny_mechanism(11)
    om = oracle.Mech(m)
    T, p, Y = synth.make_states(m, 4, T_range=(1000, 1600), seed=3)
    dt, rtol, atol = 1e-6, 1e-6, 1e-10
    Yn, st, stats, _ = oracle.integrate(om, T, p, Y, dt, rtol, atol, method)
    assert (st == 0).all()
    for c in range(4):
        sol = integrate.solve_ivp(lambda t, y: oracle.rates(om, T[c], p[c], y), (0, dt), Y[:, c],
                                  method="DOP853", rtol=1e-13, atol=1e-20)
        ref = sol.y[:, -1]
        rel = np.abs(Yn[:, c] - ref) / np.maximum(np.abs(ref), atol)
        assert rel.max() < 50 * rtol, rel.max()


@pytest.mark.parametrize("name", ["h2_9sp_rkck", "h2co_13sp_rkc", "ch4_53sp_rkc_mixed"])
def test_integrator_conserves_mass_and_elements(name):
    """Runge-Kutta methods keep linear invariants: sum Y = 1 and element totals
    stay at their initial values up to rounding."""
    m = synth.workload_mechanism(name)
    w = synth.WORKLOADS[name]
    om = oracle.Mech(m)
    T, p, Y = synth.workload_states(name, m, cells=8)
    Yn, st, stats, _ = oracle.integrate(om, T, p, Y, w["dt"], w["rtol"], w["atol"], w["method"])
    assert (st == 0).all()
    assert (stats[:, 1] > 0).all()
    np.testing.assert_allclose(Yn.sum(0), 1.0, atol=1e-13)
    el0 = m.comp.T @ (Y / m.W[:, None])
    el1 = m.comp.T @ (Yn / m.W[:, None])
    np.testing.assert_allclose(el1, el0, rtol=1e-12)
    assert np.abs(Yn - Y).max() > 1e-8  # something happened


def test_rkc_fewer_evaluations_when_stiff_and_rkck_when_not():
    """The qualitative stiffness split of Sections 3.1-3.2: on a stiff linear
    decay (k dt = 1e4) RKC needs far fewer f evaluations than RKCK; on a
    nonstiff one (k dt = 0.5) RKCK needs fewer."""
    for kdt, better in ((1e4, oracle.RKC), (0.5, oracle.RKCK)):
        om = oracle.Mech(mechs.a_to_b(kdt / 1e-6))
        Y = np.array([[0.9], [0.1]])
        nfe = {}
        for meth in (oracle.RKCK, oracle.RKC):
            _, st, stats, _ = oracle.integrate(om, [1000.0], [1e5], Y, 1e-6, 1e-6, 1e-10, meth)
            assert st[0] == 0
            nfe[meth] = stats[0, 0]
        other = oracle.RKC if better == oracle.RKCK else oracle.RKCK
        assert nfe[better] < nfe[other], (kdt, nfe)


def test_status_codes():
    """Step limit -> 1 with the last accepted state kept; non-finite input -> 3."""
    m = synth.workload_mechanism("h2co_13sp_rkc")
    om = oracle.Mech(m)
    T, p, Y = synth.workload_states("h2co_13sp_rkc", m, cells=2)
    Yn, st, stats, _ = oracle.integrate(om, T, p, Y, 1e-6, 1e-6, 1e-10, oracle.RKC, max_steps=3)
    assert (st == 1).all()
    assert (stats[:, 1] + stats[:, 2] == 3).all()
    np.testing.assert_allclose(Yn.sum(0), 1.0, atol=1e-13)
    Y2 = Y.copy()
    Y2[3, 1] = np.nan
    Yn, st, _, _ = oracle.integrate(om, T, p, Y2, 1e-6, 1e-6, 1e-10, oracle.RKCK)
    assert st[0] == 0 and st[1] == 3


# ------------------------------------------------------- power method ---
def test_power_method_on_linear_chain():
    """On A_0 -> A_1 -> ... (eigenvalues -k_i, 0) the nonlinear power method
    converges to |lambda_max| = max k_i; the estimate carries a 1.2 margin."""
    ks = [3e8, 1e9, 2.5e8, 7e9, 1e3]
    om = oracle.Mech(mechs.chain(ks))
    y = np.array([0.3, 0.2, 0.1, 0.25, 0.1, 0.05])
    sig, v, it = oracle.sigma_power(om, 1500.0, 101325.0, y)
    assert sig / 1.2 == pytest.approx(max(ks), rel=0.01, abs=0)
    assert 2 <= it <= 20
    # the direction is the dominant eigenvector: J v ~ -k_max v on species 3, 4
    u = v / np.linalg.norm(v)
    assert abs(u[3]) > 0.6 and abs(u[4]) > 0.6


def test_power_method_below_gershgorin_and_warm_start():
    """|lambda| <= Gershgorin bound: sigma/1.2 never exceeds it (up to the FD
    error); a warm start from the last direction needs at most as many
    products as the cold start from f(y)."""
    name = "ch4_53sp_rkc_mixed"
    m = synth.workload_mechanism(name)
    om = oracle.Mech(m)
    T, p, Y = synth.workload_states(name, m, cells=6)
    for c in range(6):
        g = oracle.sigma(om, T[c], p[c], Y[:, c], 1e-10)
        s1, v, it1 = oracle.sigma_power(om, T[c], p[c], Y[:, c])
        assert s1 / 1.2 <= g * (1 + 1e-6)
        s2, _, it2 = oracle.sigma_power(om, T[c], p[c], Y[:, c], v0=v)
        assert it2 <= it1
        assert s2 == pytest.approx(s1, rel=0.03, abs=0)


def test_power_method_diagonal_jacobian_exact():
    """Two independent decays A -> B (k1) and C -> D (k2): the Jacobian's
    eigenvalues are -k1, -k2, 0, 0; the power method finds max(k1, k2)."""
    W = 20.0
    m = mechs.mech([W] * 4, [dict(reac=[0], prod=[1], A=5e7), dict(reac=[2], prod=[3], A=2e6)])
    om = oracle.Mech(m)
    sig, _, it = oracle.sigma_power(om, 1000.0, 1e5, np.array([0.4, 0.1, 0.3, 0.2]))
    assert sig / 1.2 == pytest.approx(5e7, rel=0.01, abs=0)


@pytest.mark.parametrize("name", ["h2co_13sp_rkc", "ch4_53sp_rkc_mixed"])
def test_power_method_integration_accuracy(name):
    """RKC with the power-method spectral radius: conservation and agreement
    with the Gershgorin variant within the tolerance scale; fewer f evals."""
    m = synth.workload_mechanism(name)
    om = oracle.Mech(m)
    w = synth.WORKLOADS[name]
    T, p, Y = synth.workload_states(name, m, cells=8)
    Yg, sg, stg, _ = oracle.integrate(om, T, p, Y, w["dt"], w["rtol"], w["atol"], oracle.RKC)
    Yp, sp, stp, _ = oracle.integrate(om, T, p, Y, w["dt"], w["rtol"], w["atol"], oracle.RKC_POWER)
    assert (sp == 0).all()
    np.testing.assert_allclose(Yp.sum(0), 1.0, atol=1e-13)
    scale = np.maximum(np.abs(Yg), w["atol"] / w["rtol"])
    assert (np.abs(Yp - Yg) / scale).max() < 10 * w["rtol"]
    assert stp[:, 0].sum() < stg[:, 0].sum()


# ----------------------------------------------------- energy equation ---
def _thermo_mech(name, seed=4000):
    import dataclasses
    m = synth.workload_mechanism(name)
    cp, Hf = synth.make_thermo(m, seed)
    return dataclasses.replace(m, cp=cp, Hf=Hf)


def test_energy_f_conserves_mixture_enthalpy():
    """Adiabatic, constant pressure, closed: the mixture enthalpy
    h = sum_i Y_i H_i(T) / W_i is constant, so along f
    sum_i (dY_i/dt) H_i / W_i + cp (dT/dt) = 0 with cp = sum_i Y_i cp_i / W_i,
    H_i(T) = Hf_i + cp_i (T - 298.15) (the species model of the synthetic
    thermochemistry). Holds to rounding at random states."""
    m = _thermo_mech("h2co_13sp_rkc")
    om = oracle.Mech(m)
    T, p, Y = synth.workload_states("h2co_13sp_rkc", m, cells=16, seed_offset=77)
    for c in range(16):
        y = np.append(Y[:, c], T[c])
        f = oracle.rates_energy(om, p[c], y)
        H = m.Hf + m.cp * (T[c] - 298.15)
        terms = f[:-1] * H / m.W
        cpm = np.sum(Y[:, c] * m.cp / m.W)
        balance = terms.sum() + cpm * f[-1]
        assert abs(balance) <= 1e-11 * (np.abs(terms).sum() + abs(cpm * f[-1]))
        assert f[-1] != 0.0


def test_energy_species_part_is_the_isothermal_f_at_the_state_temperature():
    """The species rows of the coupled f are Eq. (E:mass) with k_j, rho and
    C_k at the state's own temperature (not the cell's initial one)."""
    m = _thermo_mech("ch4_53sp_rkc_mixed")
    om = oracle.Mech(m)
    T, p, Y = synth.workload_states("ch4_53sp_rkc_mixed", m, cells=6, seed_offset=78)
    for c in range(6):
        for Ts in (T[c], T[c] + 137.0):
            f = oracle.rates_energy(om, p[c], np.append(Y[:, c], Ts))
            np.testing.assert_array_equal(f[:-1], oracle.rates(om, Ts, p[c], Y[:, c]))


def _a_to_b_thermo(k, dH, cp=30.0, W=28.0):
    """A -> B with T-independent k (beta = 0, E = 0), equal W and cp, and an
    inert third species; B lies dH below A."""
    return mechs.mech([W, W, W], [dict(reac=[0], prod=[1], A=k)],
                      cp=[cp, cp, cp], Hf=[0.0, -dH, 0.0])


@pytest.mark.parametrize("method", [oracle.RKCK, oracle.RKC, oracle.RKC_POWER])
def test_energy_adiabatic_temperature_rise_closed_form(method):
    """With equal W and cp, enthalpy conservation gives
    T(t) = T0 + dH (Y_A0 - Y_A(t)) / cp and Y_A(t) = Y_A0 exp(-k t): the
    integrated temperature follows the released heat."""
    k, dH, cp = 1e6, 1e5, 30.0
    om = oracle.Mech(_a_to_b_thermo(k, dH, cp))
    T0, dt = 1000.0, 1e-6
    Y = np.array([[0.1], [0.0], [0.9]])
    Yn, st, sta, _, Tn = oracle.integrate(om, np.array([T0]), np.array([101325.0]), Y, dt,
                                          1e-10, 1e-14, method, energy=True)
    assert st[0] == 0
    ya = 0.1 * math.exp(-k * dt)
    assert Yn[0, 0] == pytest.approx(ya, rel=1e-7, abs=0)
    rise = dH * (0.1 - ya) / cp  # about 211 K
    assert Tn[0] - T0 == pytest.approx(rise, rel=1e-7, abs=0)


def test_energy_integration_against_tight_scipy_reference():
    """Thermal feedback on: RKC with the power-method sigma on the coupled
    (nS + 1)-vector against scipy's DOP853 on the oracle's own f."""
    from scipy.integrate import solve_ivp
    m = _thermo_mech("h2co_13sp_rkc")
    om = oracle.Mech(m)
    T, p, Y = synth.workload_states("h2co_13sp_rkc", m, cells=3, seed_offset=79)
    Yn, st, sta, _, Tn = oracle.integrate(om, T, p, Y, 1e-6, 1e-9, 1e-13, oracle.RKC_POWER,
                                          energy=True)
    assert (st == 0).all()
    for c in range(3):
        y0 = np.append(Y[:, c], T[c])
        ref = solve_ivp(lambda t, y: oracle.rates_energy(om, p[c], y), (0.0, 1e-6), y0,
                        method="DOP853", rtol=1e-12, atol=1e-16).y[:, -1]
        assert abs(Tn[c] - ref[-1]) <= 1e-6 * ref[-1]
        assert abs(Tn[c] - T[c]) > 1e-3  # the temperature moved
        np.testing.assert_allclose(Yn[:, c], ref[:-1], rtol=1e-5, atol=1e-12)


def test_energy_conserves_enthalpy_and_mass_over_a_flow_step():
    """Integrated over the flow step: sum Y = 1 and the mixture enthalpy stay
    at their initial values to the integration tolerance."""
    m = _thermo_mech("h2co_13sp_rkc")
    om = oracle.Mech(m)
    T, p, Y = synth.workload_states("h2co_13sp_rkc", m, cells=8, seed_offset=80)
    Yn, st, sta, _, Tn = oracle.integrate(om, T, p, Y, 1e-6, 1e-8, 1e-14, oracle.RKC_POWER,
                                          energy=True)

    def h(Y, T):
        return np.sum(Y * (m.Hf[:, None] + m.cp[:, None] * (T[None, :] - 298.15)) / m.W[:, None], axis=0)

    cpm = np.sum(Y * m.cp[:, None] / m.W[:, None], axis=0)
    assert np.abs(Yn.sum(0) - 1).max() < 1e-12
    assert np.all(np.abs(h(Yn, Tn) - h(Y, T)) < 1e-6 * cpm * T)
