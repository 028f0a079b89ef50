"""Pins of the FP64 oracle against what the mathematics fixes independently of it.

Each test checks the oracle against something it does not share code with:
four-vectors built from scratch, closed forms, a library routine
(scipy's natural cubic spline, scipy's adaptive quadrature), invariances of the
likelihood, or central finite differences. A dropped term, a wrong sign or a
transposed operand in the oracle fails one of them.
"""
import math

import numpy as np
import pytest

import oracle
import synth

RNG = np.random.default_rng(12345)


# --------------------------------------------------------------- four-vectors
def _two_body_k(M, ma, mb):
    """|momentum| of daughter a in the rest frame of M -> a b, from energies."""
    Ea = (M * M + ma * ma - mb * mb) / (2.0 * M)
    return math.sqrt(max(Ea * Ea - ma * ma, 0.0))


def _unit(rng):
    c = rng.uniform(-1.0, 1.0)
    ph = rng.uniform(0.0, 2.0 * math.pi)
    s = math.sqrt(1.0 - c * c)
    return np.array([s * math.cos(ph), s * math.sin(ph), c])


def _boost(p4, beta):
    """Lorentz boost of four-vector p4 = (E, px, py, pz) by velocity beta (3-vector)."""
    b2 = float(beta @ beta)
    if b2 == 0.0:
        return p4.copy()
    g = 1.0 / math.sqrt(1.0 - b2)
    bp = float(beta @ p4[1:])
    E = g * (p4[0] + bp)
    p = p4[1:] + ((g - 1.0) * bp / b2 + g * p4[0]) * beta
    return np.concatenate([[E], p])


def _m2(p4):
    return p4[0] ** 2 - float(p4[1:] @ p4[1:])


def _decay(spec, rng, m12=None, cos13=None):
    """D at rest -> R(12) + 3, R -> 1 + 2, built from explicit momenta.

    Returns the invariants from the four-vectors, plus q, p and cos(theta13)
    measured in the R rest frame."""
    M, m1, m2, m3 = spec.mD, spec.m1, spec.m2, spec.m2
    if m12 is None:
        m12 = rng.uniform(m1 + m2 + 1e-3, M - m3 - 1e-3)
    k = _two_body_k(M, m12, m3)
    n = _unit(rng)
    ER = math.sqrt(k * k + m12 * m12)
    p3 = np.concatenate([[math.sqrt(k * k + m3 * m3)], -k * n])
    q = _two_body_k(m12, m1, m2)
    beta = k * n / ER
    # direction of particle 3 in the R frame
    p3R = _boost(p3, -beta)
    d3 = p3R[1:] / np.linalg.norm(p3R[1:])
    if cos13 is None:
        u = _unit(rng)
    else:
        # build a direction at the requested angle to d3
        t = np.cross(d3, [1.0, 0.0, 0.0])
        if np.linalg.norm(t) < 1e-3:
            t = np.cross(d3, [0.0, 1.0, 0.0])
        t /= np.linalg.norm(t)
        u = cos13 * d3 + math.sqrt(max(1.0 - cos13 * cos13, 0.0)) * t
    p1R = np.concatenate([[math.sqrt(q * q + m1 * m1)], q * u])
    p2R = np.concatenate([[math.sqrt(q * q + m2 * m2)], -q * u])
    p1, p2 = _boost(p1R, beta), _boost(p2R, beta)
    s12, s13, s23 = _m2(p1 + p2), _m2(p1 + p3), _m2(p2 + p3)
    cos = float(u @ d3)
    return dict(s12=s12, s13=s13, s23=s23, q=q, p=float(np.linalg.norm(p3R[1:])), cos=cos,
                m12=m12)


SPECS = [synth.pipipi(10), synth.kpipi(40)]


@pytest.mark.parametrize("spec", SPECS, ids=lambda s: s.name)
def test_kinematics_from_four_vectors(spec):
    o = oracle.Oracle(spec)
    sigma = spec.mD ** 2 + spec.m1 ** 2 + 2 * spec.m2 ** 2
    for _ in range(200):
        d = _decay(spec, RNG)
        assert d["s12"] == pytest.approx(d["m12"] ** 2, rel=1e-12)
        assert d["s12"] + d["s13"] + d["s23"] == pytest.approx(sigma, rel=1e-13)
        assert o.q(d["s12"]) == pytest.approx(d["q"], rel=1e-10)
        assert o.p(d["s12"]) == pytest.approx(d["p"], rel=1e-10)
        lo, hi = o.s23_range(d["s12"])
        assert lo - 1e-12 <= d["s23"] <= hi + 1e-12
        assert o.inside([[d["s12"], d["s13"]]])[0] or abs(abs(d["cos"]) - 1) < 1e-9


@pytest.mark.parametrize("spec", SPECS, ids=lambda s: s.name)
def test_dalitz_boundary_at_cos_pm1(spec):
    o = oracle.Oracle(spec)
    for _ in range(50):
        for c in (-1.0, 1.0):
            d = _decay(spec, RNG, cos13=c)
            lo, hi = o.s23_range(d["s12"])
            # cos(theta13) = +1 puts particle 1 along 3: s13 is smallest, s23 largest
            target = hi if c > 0 else lo
            assert d["s23"] == pytest.approx(target, rel=1e-10, abs=1e-10)


@pytest.mark.parametrize("spec", SPECS, ids=lambda s: s.name)
def test_zemach_closed_forms(spec):
    """Z1 = -4 p q cos(theta13), Z2 = 16 p^2 q^2 (cos^2 - 1/3), from the R-frame angle."""
    o = oracle.Oracle(spec)
    for _ in range(200):
        d = _decay(spec, RNG)
        pq = d["p"] * d["q"]
        z1 = o.zemach(1, d["s12"], d["s13"])
        z2 = o.zemach(2, d["s12"], d["s13"])
        assert z1 == pytest.approx(-4.0 * pq * d["cos"], abs=1e-11 * (1 + 4 * pq))
        assert z2 == pytest.approx(16.0 * pq * pq * (d["cos"] ** 2 - 1.0 / 3.0),
                                   abs=1e-11 * (1 + 16 * pq * pq))
        assert o.zemach(0, d["s12"], d["s13"]) == 1.0


@pytest.mark.parametrize("spec", SPECS, ids=lambda s: s.name)
def test_inside_matches_cos_theta(spec):
    """Inside the plot <=> |cos(theta13)| <= 1, cos from R-frame energies."""
    o = oracle.Oracle(spec)
    M, m1, m3 = spec.mD, spec.m1, spec.m2
    lo, hi = spec.s_lo, spec.s_hi
    pts = lo + (hi - lo) * RNG.random((20000, 2))
    ins = o.inside(pts)
    for (s12, s13), got in zip(pts, ins):
        rs = math.sqrt(s12)
        q = _two_body_k(rs, m1, m3)
        E3 = (M * M - s12 - m3 * m3) / (2 * rs)
        p = math.sqrt(max(E3 * E3 - m3 * m3, 0.0))
        E1 = math.sqrt(q * q + m1 * m1)
        cos = (m1 * m1 + m3 * m3 + 2 * E1 * E3 - s13) / (2 * q * p)
        if abs(abs(cos) - 1.0) < 1e-9:
            continue
        assert bool(got) == (abs(cos) <= 1.0)


@pytest.mark.parametrize("spec,expect", [(synth.pipipi(10), 0.596), (synth.kpipi(40), 0.477)],
                         ids=["pipipi", "kpipi"])
def test_dalitz_area(spec, expect):
    """Area = integral of the s13 extent 4 p q over s12; the in-box fraction matches it."""
    from scipy.integrate import quad

    o = oracle.Oracle(spec)
    M, m1, m3 = spec.mD, spec.m1, spec.m2

    def width(s12):
        rs = math.sqrt(s12)
        q = _two_body_k(rs, m1, m3)
        E3 = (M * M - s12 - m3 * m3) / (2 * rs)
        p = math.sqrt(max(E3 * E3 - m3 * m3, 0.0))
        return 4.0 * p * q

    for s12 in np.linspace(spec.s_lo + 1e-4, spec.s_hi - 1e-4, 25):
        lo, hi = o.s23_range(s12)
        assert hi - lo == pytest.approx(width(s12), rel=1e-9, abs=1e-12)
    area, _ = quad(width, spec.s_lo, spec.s_hi, limit=200)
    box = (spec.s_hi - spec.s_lo) ** 2
    pts = spec.s_lo + (spec.s_hi - spec.s_lo) * RNG.random((400000, 2))
    frac = o.inside(pts).mean()
    assert frac == pytest.approx(area / box, abs=4 * math.sqrt(0.25 / len(pts)))
    assert area / box == pytest.approx(expect, abs=1e-3)


# --------------------------------------------------------------- Breit-Wigner
def test_barrier_special_values():
    for z0 in (0.0, 0.3, 2.0, 40.0):
        assert oracle.barrier(0, 1.7, z0) == 1.0
        for L in (1, 2):
            assert oracle.barrier(L, z0, z0) == pytest.approx(1.0, rel=1e-15)
        assert oracle.barrier(1, 0.0, z0) == pytest.approx(math.sqrt(1 + z0), rel=1e-15)
        assert oracle.barrier(2, 0.0, z0) == pytest.approx(
            math.sqrt((z0 * z0 + 3 * z0 + 9) / 9.0), rel=1e-15)
    # large-z fall-off: F1 ~ sqrt((1+z0)/z), F2 ~ sqrt(z0^2+3z0+9)/z
    z = 1e8
    assert oracle.barrier(1, z, 1.0) == pytest.approx(math.sqrt(2.0 / z), rel=1e-7)
    assert oracle.barrier(2, z, 1.0) == pytest.approx(math.sqrt(13.0) / z, rel=1e-7)


@pytest.mark.parametrize("spec", SPECS, ids=lambda s: s.name)
def test_bw_pole_value(spec):
    """At s = m^2: q = q0, Gamma = Gamma_r, F = 1, so T = i / (m Gamma)."""
    o = oracle.Oracle(spec)
    for r, (m, G, L) in enumerate(spec.resonances):
        T = o.propagator(r, m * m)
        assert T.real == pytest.approx(0.0, abs=1e-12 / (m * G))
        assert T.imag == pytest.approx(1.0 / (m * G), rel=1e-13)


def test_bw_fwhm_narrow_limit():
    """|T|^2 has full width 2 m Gamma in s as Gamma -> 0."""
    for L in (1, 2):
        m, G = 1.0, 1e-5
        spec = synth.ModelSpec(name="narrow", mD=synth.M_D, m1=synth.M_PI, m2=synth.M_PI,
                               resonances=((m, G, L),), knots=(0.1, 2.9))
        o = oracle.Oracle(spec)
        peak = abs(o.propagator(0, m * m)) ** 2

        def half(s):
            return abs(o.propagator(0, s)) ** 2 - 0.5 * peak

        def bisect(a, b):
            for _ in range(200):
                c = 0.5 * (a + b)
                if (half(a) > 0) == (half(c) > 0):
                    a = c
                else:
                    b = c
            return 0.5 * (a + b)

        lo = bisect(m * m - 10 * m * G, m * m)
        hi = bisect(m * m, m * m + 10 * m * G)
        assert (hi - lo) / (2 * m * G) == pytest.approx(1.0, rel=1e-3)


@pytest.mark.parametrize("spec", SPECS, ids=lambda s: s.name)
def test_resonance_at_pole_from_four_vectors(spec):
    """A_r(m^2, s13) = Z1 * i/(m Gamma) with Z1 = -4 p q cos(theta13) (L = 1), and
    16 p^2 q^2 (cos^2 - 1/3) (L = 2): barrier factors are 1 at the pole."""
    o = oracle.Oracle(spec)
    for r, (m, G, L) in enumerate(spec.resonances):
        for _ in range(20):
            d = _decay(spec, RNG, m12=m)
            pq = d["p"] * d["q"]
            z = -4 * pq * d["cos"] if L == 1 else 16 * pq * pq * (d["cos"] ** 2 - 1 / 3)
            A = o.resonance(r, d["s12"], d["s13"])
            scale = (4 * pq) ** L / (m * G)
            assert A.real == pytest.approx(0.0, abs=1e-9 * scale)
            assert A.imag == pytest.approx(z / (m * G), abs=1e-9 * scale)


# ---------------------------------------------------------------------- spline
def _random_knots(n, rng):
    x = np.sort(rng.uniform(0.0, 3.0, n))
    x[0], x[-1] = 0.05, 2.95
    return np.unique(x)


def test_spline_matches_scipy_natural():
    from scipy.interpolate import CubicSpline

    for n in (3, 4, 10, 30, 40):
        x = _random_knots(n, RNG) if n > 3 else np.array([0.1, 0.9, 2.5])
        y = RNG.normal(size=len(x))
        M = oracle.spline_second_derivs(x, y)
        ref = CubicSpline(x, y, bc_type="natural")
        s = np.concatenate([RNG.uniform(x[0] - 0.2, x[-1] + 0.2, 500), x])
        got = oracle.spline_eval(x, y, M, s)
        np.testing.assert_allclose(got, ref(s), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(M, ref(x, 2), rtol=1e-10, atol=1e-10)


def test_spline_interpolates_and_is_c2():
    x = np.linspace(0.078, 2.987, 10)
    y = 1 + 0.5 * np.sin(np.arange(10))
    M = oracle.spline_second_derivs(x, y)
    np.testing.assert_allclose(oracle.spline_eval(x, y, M, x), y, rtol=0, atol=1e-14)
    assert M[0] == 0.0 and M[-1] == 0.0
    h = 1e-5
    for xk in x[1:-1]:
        left = oracle.spline_eval(x, y, M, [xk - 2 * h, xk - h, xk])
        right = oracle.spline_eval(x, y, M, [xk, xk + h, xk + 2 * h])
        d1l = (3 * left[2] - 4 * left[1] + left[0]) / (2 * h)
        d1r = (-3 * right[0] + 4 * right[1] - right[2]) / (2 * h)
        assert d1l == pytest.approx(d1r, abs=1e-6)
        d2l = (left[2] - 2 * left[1] + left[0]) / h ** 2
        d2r = (right[2] - 2 * right[1] + right[0]) / h ** 2
        assert d2l == pytest.approx(d2r, abs=2e-3 * (1 + abs(d2l)))
    # natural ends: second derivative -> 0 at x0 and x_{N-1}
    for xe, sgn in ((x[0], 1), (x[-1], -1)):
        v = oracle.spline_eval(x, y, M, [xe, xe + sgn * h, xe + 2 * sgn * h])
        assert (v[2] - 2 * v[1] + v[0]) / h ** 2 == pytest.approx(0.0, abs=1e-3)


def test_spline_reproduces_linear_functions_everywhere():
    x = _random_knots(12, RNG)
    y = 0.7 - 1.3 * x
    M = oracle.spline_second_derivs(x, y)
    s = RNG.uniform(-1.0, 4.0, 1000)
    np.testing.assert_allclose(oracle.spline_eval(x, y, M, s), 0.7 - 1.3 * s, atol=1e-13)


# ------------------------------------------------------------------ amplitude
@pytest.mark.parametrize("spec", SPECS, ids=lambda s: s.name)
def test_bose_symmetry(spec):
    o = oracle.Oracle(spec)
    p = synth.perturbed_params(spec, 3)
    pts = spec.s_lo + (spec.s_hi - spec.s_lo) * RNG.random((5000, 2))
    pts = pts[o.inside(pts)]
    a = o.amp(p, pts)
    b = o.amp(p, pts[:, ::-1])
    np.testing.assert_allclose(b, a, rtol=1e-14, atol=0)


def test_swave_only_closed_form():
    """No resonances, constant magnitude, phase linear in s: the natural spline
    reproduces both exactly, so |A|^2 = 2 a^2 (1 + cos(beta (s12 - s13)))."""
    knots = synth.uniform_knots(0.078, 2.987, 10)
    spec = synth.ModelSpec(name="swave", mD=synth.M_D, m1=synth.M_PI, m2=synth.M_PI,
                           resonances=(), knots=knots)
    o = oracle.Oracle(spec)
    a, alpha, beta = 1.7, 0.4, 2.3
    params = np.array([a] * 10 + [alpha + beta * s for s in knots])
    pts = spec.s_lo + (spec.s_hi - spec.s_lo) * RNG.random((3000, 2))
    pts = pts[o.inside(pts)]
    got = o.amp2(params, pts)
    want = 2 * a * a * (1 + np.cos(beta * (pts[:, 0] - pts[:, 1])))
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)
    A = o.amp(params, pts)
    phase = np.exp(1j * (alpha + beta * pts[:, 0])) + np.exp(1j * (alpha + beta * pts[:, 1]))
    np.testing.assert_allclose(A, a * phase, rtol=1e-12, atol=1e-12)


def test_amplitude_is_linear_in_bw_coefficients():
    spec = synth.pipipi(10)
    o = oracle.Oracle(spec)
    p = synth.perturbed_params(spec, 5)
    pts = spec.s_lo + (spec.s_hi - spec.s_lo) * RNG.random((2000, 2))
    pts = pts[o.inside(pts)]
    B = o.basis(pts)
    q = p.copy()
    q[:4] = 0.0
    s_only = o.amp(q, pts)
    c = p[0:4:2] + 1j * p[1:4:2]
    np.testing.assert_allclose(o.amp(p, pts), s_only + B @ c, rtol=1e-12, atol=1e-13)


# ------------------------------------------------------------------ likelihood
def _small_problem(spec, n_data=400, seed=7):
    o = oracle.Oracle(spec)
    truth = synth.true_params(spec)
    dens = synth.numpy_density(lambda x: o.density(truth, x))
    ins = synth.numpy_density(lambda x: o.inside(x).astype(np.float64))
    data = synth.accept_reject(spec, n_data, dens, seed=seed).numpy()
    norm = synth.grid_in_plot(spec, 60, ins).numpy()
    return o, data, norm


def test_nll_zero_for_constant_amplitude():
    knots = synth.uniform_knots(0.078, 2.987, 6)
    spec = synth.ModelSpec(name="const", mD=synth.M_D, m1=synth.M_PI, m2=synth.M_PI,
                           resonances=(), knots=knots)
    o = oracle.Oracle(spec)
    ins = synth.numpy_density(lambda x: o.inside(x).astype(np.float64))
    norm = synth.grid_in_plot(spec, 40, ins).numpy()
    data = norm[::7]
    p = np.array([0.8] * 6 + [0.3] * 6)
    assert o.nll(p, data, norm) == pytest.approx(0.0, abs=1e-9)


@pytest.mark.parametrize("spec", [synth.pipipi(10), synth.kpipi(12)], ids=lambda s: s.name)
def test_nll_invariances(spec):
    """A -> lambda A (scale c and a) and A -> e^{i alpha} A (rotate c, shift phi)
    leave -2 ln L unchanged; the gradient is orthogonal to both directions."""
    o, data, norm = _small_problem(spec)
    p = synth.perturbed_params(spec, 11)
    R, N = spec.n_res, spec.n_knots
    v0, g = o.nll_grad(p, data, norm)
    scaled = p.copy()
    scaled[: 2 * R + N] *= 1.37
    assert o.nll(scaled, data, norm) == pytest.approx(v0, rel=1e-12, abs=1e-9)
    rot = p.copy()
    alpha = 0.61
    c = (p[0:2 * R:2] + 1j * p[1:2 * R:2]) * np.exp(1j * alpha)
    rot[0:2 * R:2], rot[1:2 * R:2] = c.real, c.imag
    rot[2 * R + N:] += alpha
    assert o.nll(rot, data, norm) == pytest.approx(v0, rel=1e-12, abs=1e-9)
    # directional derivatives
    d_scale = np.concatenate([p[: 2 * R + N], np.zeros(N)])
    d_phase = np.zeros_like(p)
    d_phase[0:2 * R:2] = -p[1:2 * R:2]
    d_phase[1:2 * R:2] = p[0:2 * R:2]
    d_phase[2 * R + N:] = 1.0
    gn = np.linalg.norm(g)
    assert abs(g @ d_scale) < 1e-9 * gn * np.linalg.norm(d_scale)
    assert abs(g @ d_phase) < 1e-9 * gn * np.linalg.norm(d_phase)


@pytest.mark.parametrize("spec", [synth.pipipi(10), synth.kpipi(12)], ids=lambda s: s.name)
def test_gradient_central_differences(spec):
    o, data, norm = _small_problem(spec)
    p = synth.perturbed_params(spec, 13)
    _, g = o.nll_grad(p, data, norm)
    h = 1e-6
    fd = np.empty_like(p)
    for k in range(len(p)):
        e = np.zeros_like(p)
        e[k] = h
        fd[k] = (o.nll(p + e, data, norm) - o.nll(p - e, data, norm)) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-5, atol=1e-5 * np.abs(g).max())


def test_nll_matches_direct_sum():
    """The oracle's compensated, chunked reduction equals a plain numpy sum of
    -2 ln|A|^2 + 2 N ln(mean |A|^2) over its own per-event amplitudes."""
    spec = synth.pipipi(10)
    o, data, norm = _small_problem(spec, n_data=9000)
    p = synth.perturbed_params(spec, 17)
    want = -2 * np.sum(np.log(o.amp2(p, data))) + 2 * len(data) * np.log(np.mean(o.amp2(p, norm)))
    assert o.nll(p, data, norm, threads=3) == pytest.approx(want, rel=1e-12)
    assert o.nll(p, data, norm, threads=1) == o.nll(p, data, norm, threads=4)


# ------------------------------------------------- weighted normalisation
# A weight per normalisation point makes the integral a weighted mean,
# I = sum w_j |A(y_j)|^2 / sum w_j. Integer weights are multiplicities, so they
# must give exactly the likelihood of the sample with each point repeated.
@pytest.mark.parametrize("spec", [synth.pipipi(10), synth.as_reim(synth.kpipi(12))],
                         ids=lambda s: s.name + "_" + s.swave_form)
def test_integer_weights_equal_repeated_points(spec):
    o, data, norm = _small_problem(spec)
    rng = np.random.default_rng(5)
    k = rng.integers(0, 4, len(norm))
    k[0] = max(k[0], 1)
    p = synth.perturbed_params(spec, 19)
    v, g = o.nll_grad(p, data, norm, norm_weights=k.astype(np.float64))
    vr, gr = o.nll_grad(p, data, np.repeat(norm, k, axis=0))
    assert v == pytest.approx(vr, rel=1e-13)
    np.testing.assert_allclose(g, gr, rtol=1e-11, atol=1e-11 * np.abs(gr).max())


def test_constant_weights_equal_unweighted_and_weighted_mean():
    spec = synth.pipipi(10)
    o, data, norm = _small_problem(spec, n_data=2000)
    p = synth.perturbed_params(spec, 23)
    v0, g0 = o.nll_grad(p, data, norm)
    v1, g1 = o.nll_grad(p, data, norm, norm_weights=np.full(len(norm), 0.37))
    assert v1 == pytest.approx(v0, rel=1e-14)
    np.testing.assert_allclose(g1, g0, rtol=1e-12, atol=1e-12 * np.abs(g0).max())
    # random weights: the direct numpy statement of the weighted mean
    w = np.random.default_rng(8).uniform(0.2, 3.0, len(norm))
    a2 = o.amp2(p, norm)
    want = -2 * np.sum(np.log(o.amp2(p, data))) + 2 * len(data) * np.log(np.sum(w * a2) / np.sum(w))
    assert o.nll(p, data, norm, norm_weights=w) == pytest.approx(want, rel=1e-12)
    with pytest.raises(ArithmeticError):  # no positive total weight
        o.nll(p, data, norm, norm_weights=np.zeros(len(norm)))


def test_weighted_gradient_central_differences():
    spec = synth.kpipi(12)
    o, data, norm = _small_problem(spec)
    w = np.random.default_rng(9).uniform(0.0, 2.0, len(norm))
    p = synth.perturbed_params(spec, 29)
    _, g = o.nll_grad(p, data, norm, norm_weights=w)
    h = 1e-6
    fd = np.empty_like(p)
    for k in range(len(p)):
        e = np.zeros_like(p)
        e[k] = h
        fd[k] = (o.nll(p + e, data, norm, norm_weights=w)
                 - o.nll(p - e, data, norm, norm_weights=w)) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-5, atol=1e-5 * np.abs(g).max())


def test_nll_rejects_nonpositive_amplitude():
    knots = synth.uniform_knots(0.078, 2.987, 6)
    spec = synth.ModelSpec(name="zero", mD=synth.M_D, m1=synth.M_PI, m2=synth.M_PI,
                           resonances=(), knots=knots)
    o = oracle.Oracle(spec)
    pts = np.array([[0.5, 1.0], [1.0, 0.5]])
    with pytest.raises(ArithmeticError):
        o.nll(np.zeros(12), pts, pts)


def test_normalisation_converges_to_quadrature():
    """Tiny model (4 knots, one resonance): the grid mean of |A|^2 approaches the
    adaptive 2-D quadrature of |A|^2 over the exact boundary divided by the area
    as the grid spacing shrinks (the grid refinement of Sec. 4, Fig. 2)."""
    from scipy.integrate import quad

    spec = synth.ModelSpec(name="tiny", mD=synth.M_D, m1=synth.M_PI, m2=synth.M_PI,
                           resonances=((0.77526, 0.1491, 1),),
                           knots=synth.uniform_knots(0.078, 2.987, 4))
    o = oracle.Oracle(spec)
    p = np.array([0.3, 0.1, 1.0, 1.4, 0.8, 1.2, 0.0, 0.9, 1.8, 2.4])
    sigma = spec.mD ** 2 + spec.m1 ** 2 + 2 * spec.m2 ** 2
    M, m1, m3 = spec.mD, spec.m1, spec.m2

    def s13_bounds(s12):
        rs = math.sqrt(s12)
        q = _two_body_k(rs, m1, m3)
        E3 = (M * M - s12 - m3 * m3) / (2 * rs)
        p_ = math.sqrt(max(E3 * E3 - m3 * m3, 0.0))
        E1 = math.sqrt(q * q + m1 * m1)
        mid = m1 * m1 + m3 * m3 + 2 * E1 * E3
        return mid - 2 * q * p_, mid + 2 * q * p_

    def inner(s12):
        lo, hi = s13_bounds(s12)
        f = lambda s13: float(o.amp2(p, [[s12, s13]])[0])
        return quad(f, lo, hi, epsabs=0, epsrel=1e-10, limit=200)[0]

    # split s12 at the resonance peak so the outer integral sees it
    edges = [spec.s_lo, 0.77526 ** 2 - 0.2, 0.77526 ** 2 + 0.2, spec.s_hi]
    integral = sum(quad(inner, a, b, epsabs=0, epsrel=1e-9, limit=200)[0]
                   for a, b in zip(edges[:-1], edges[1:]))
    area = sum(quad(lambda s: -np.subtract(*s13_bounds(s)), a, b, epsrel=1e-12, limit=200)[0]
               for a, b in zip(edges[:-1], edges[1:]))
    exact = integral / area
    ins = synth.numpy_density(lambda x: o.inside(x).astype(np.float64))
    x0 = np.array([[0.6, 1.5]])
    a0 = float(o.amp2(p, x0)[0])
    errs = []
    for n_side in (100, 300, 900):
        norm = synth.grid_in_plot(spec, n_side, ins).numpy()
        # ln I from the NLL of a single data event: NLL = -2 ln|A(x0)|^2 + 2 ln I
        I = math.exp(o.nll(p, x0, norm) / 2 + math.log(a0))
        errs.append(abs(I / exact - 1))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 2e-3
    assert sigma > 0


@pytest.mark.parametrize("spec", SPECS, ids=lambda s: s.name)
def test_running_width_scaling(spec):
    """Im T / |T|^2 = m Gamma(s) and Re T / |T|^2 = m^2 - s; the running width
    scales as q^(2L+1) F_R(q)^2 / sqrt(s), with q from four-vectors and F_R the
    (separately pinned) barrier factor, and equals Gamma_r at the pole."""
    o = oracle.Oracle(spec)
    for r, (m, G, L) in enumerate(spec.resonances):
        q0 = _two_body_k(m, spec.m1, spec.m2)
        z0 = (spec.r_res * q0) ** 2
        ratios = []
        for _ in range(40):
            d = _decay(spec, RNG)
            s = d["s12"]
            T = o.propagator(r, s)
            a2 = abs(T) ** 2
            assert T.real / a2 == pytest.approx(m * m - s, rel=1e-9, abs=1e-12)
            gam = T.imag / (m * a2)
            F2 = oracle.barrier(L, (spec.r_res * d["q"]) ** 2, z0) ** 2
            ratios.append(gam * math.sqrt(s) / (d["q"] ** (2 * L + 1) * F2))
        want = G * m / q0 ** (2 * L + 1)
        np.testing.assert_allclose(ratios, want, rtol=1e-9)


@pytest.mark.parametrize("spec", SPECS, ids=lambda s: s.name)
def test_resonance_factorisation_from_four_vectors(spec):
    """A_r = F_R(q) F_D(p) Z_L T: dividing out the (pinned) propagator and the
    Zemach factor leaves the product of the two barrier factors, evaluated at
    the breakup momentum q and the bachelor momentum p of the explicit decay,
    with radii r_res and r_D and the pole momenta q0, p0."""
    o = oracle.Oracle(spec)
    for r, (m, G, L) in enumerate(spec.resonances):
        q0 = _two_body_k(m, spec.m1, spec.m2)
        E3 = (spec.mD ** 2 - m * m - spec.m2 ** 2) / (2 * m)
        p0 = math.sqrt(E3 * E3 - spec.m2 ** 2)
        for _ in range(40):
            d = _decay(spec, RNG)
            if abs(d["cos"]) < 0.05:
                continue
            A = o.resonance(r, d["s12"], d["s13"])
            T = o.propagator(r, d["s12"])
            pq = d["p"] * d["q"]
            Z = -4 * pq * d["cos"] if L == 1 else 16 * pq * pq * (d["cos"] ** 2 - 1 / 3)
            FR = oracle.barrier(L, (spec.r_res * d["q"]) ** 2, (spec.r_res * q0) ** 2)
            FD = oracle.barrier(L, (spec.r_D * d["p"]) ** 2, (spec.r_D * p0) ** 2)
            ratio = A / (T * Z)
            assert ratio.imag == pytest.approx(0.0, abs=1e-9 * abs(ratio))
            assert ratio.real == pytest.approx(FR * FD, rel=1e-8)


def test_oracle_reproduces_frozen_values():
    """The oracle's output at fixed points, frozen by tests/golden/make_golden.py,
    is reproduced on this platform (guards against compiler/platform drift)."""
    import json
    import os

    path = os.path.join(os.path.dirname(__file__), "golden", "oracle_values.json")
    with open(path) as f:
        cases = json.load(f)
    specs = {s.name: s for s in (synth.pipipi(10), synth.pipipi(30), synth.kpipi(40),
                                 synth.kkk(40), synth.as_reim(synth.pipipi(10)))}
    for name, entry in cases.items():
        spec = specs[name]
        o = oracle.Oracle(spec)
        pts = np.array(entry["events"])
        data = np.array(entry["data"])
        n = entry["norm_side"]
        t = spec.s_lo + (spec.s_hi - spec.s_lo) * (np.arange(n) + 0.5) / n
        a, b = np.meshgrid(t, t, indexing="ij")
        norm = np.stack([a.ravel(), b.ravel()], 1)
        norm = norm[o.inside(norm)]
        for label in ("true", "perturbed"):
            e = entry[label]
            A = o.amp(np.array(e["params"]), pts)
            np.testing.assert_allclose(A.real, e["amp_re"], rtol=1e-12, atol=1e-13)
            np.testing.assert_allclose(A.imag, e["amp_im"], rtol=1e-12, atol=1e-13)
            v, g = o.nll_grad(np.array(e["params"]), data, norm, threads=2)
            assert v == pytest.approx(e["nll"], rel=1e-12)
            np.testing.assert_allclose(g, e["grad"], rtol=1e-9, atol=1e-9 * np.abs(g).max())


# ------------------------------------------------ Re/Im (complex-plane) spline
REIM_SPECS = [synth.as_reim(synth.pipipi(10)), synth.as_reim(synth.kpipi(12))]


@pytest.mark.parametrize("spec", [synth.pipipi(10), synth.kpipi(12)], ids=lambda s: s.name)
def test_reim_equals_magphase_on_knots(spec):
    """Both S-wave forms interpolate the same complex knot values: with
    x_k + i y_k = a_k e^{i phi_k} and both invariants on knots, the amplitudes
    agree exactly (to rounding)."""
    o_mp, o_ri = oracle.Oracle(spec), oracle.Oracle(synth.as_reim(spec))
    p = synth.perturbed_params(spec, 23)
    R, N = spec.n_res, spec.n_knots
    a, phi = p[2 * R:2 * R + N], p[2 * R + N:]
    q = np.concatenate([p[:2 * R], a * np.cos(phi), a * np.sin(phi)])
    k = np.asarray(spec.knots)
    pts = np.array([(x, y) for x in k for y in k])
    pts = pts[o_mp.inside(pts)]
    assert len(pts) > 10
    np.testing.assert_allclose(o_ri.amp(q, pts), o_mp.amp(p, pts), rtol=1e-13, atol=1e-13)
    # between knots the two forms differ (different interpolants)
    mid = np.array([[0.5 * (k[2] + k[3]), 0.5 * (k[4] + k[5])]])
    assert abs(o_ri.amp(q, mid)[0] - o_mp.amp(p, mid)[0]) > 1e-6


def test_reim_reproduces_complex_linear_function():
    """No resonances and knot values alpha + beta s_k (complex alpha, beta): the
    natural spline of each part is that line exactly, in every segment and
    beyond the end knots, so A = 2 alpha + beta (s12 + s13)."""
    knots = synth.uniform_knots(0.3, 2.6, 9)  # end knots inside the plot's range
    spec = synth.ModelSpec(name="lin", mD=synth.M_D, m1=synth.M_PI, m2=synth.M_PI,
                           resonances=(), knots=knots, swave_form="reim")
    o = oracle.Oracle(spec)
    alpha, beta = 0.7 - 0.2j, -0.35 + 1.1j
    z = alpha + beta * np.asarray(knots)
    pts = spec.s_lo + (spec.s_hi - spec.s_lo) * RNG.random((3000, 2))
    pts = pts[o.inside(pts)]
    assert (pts[:, 0] < knots[0]).any() and (pts[:, 0] > knots[-1]).any()
    got = o.amp(np.concatenate([z.real, z.imag]), pts)
    np.testing.assert_allclose(got, 2 * alpha + beta * (pts[:, 0] + pts[:, 1]), rtol=1e-12,
                               atol=1e-12)


@pytest.mark.parametrize("spec", REIM_SPECS, ids=lambda s: s.name)
def test_reim_amplitude_is_linear_in_all_parameters(spec):
    """A = sum_r c_r B_r + sum_k (x_k + i y_k) W_k with W_k the natural-spline
    cardinal function of knot k summed over both channels (scipy builds it):
    |A|^2 is then a Hermitian form in the complex parameters and the
    normalisation integral is theta^H M theta with M the mean of conj(b) b^T."""
    from scipy.interpolate import CubicSpline

    o = oracle.Oracle(spec)
    p = synth.perturbed_params(spec, 29)
    R, N = spec.n_res, spec.n_knots
    pts = spec.s_lo + (spec.s_hi - spec.s_lo) * RNG.random((4000, 2))
    pts = pts[o.inside(pts)]
    k = np.asarray(spec.knots)
    W = np.zeros((len(pts), N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        cs = CubicSpline(k, e, bc_type="natural", extrapolate=True)
        W[:, j] = cs(pts[:, 0]) + cs(pts[:, 1])
    b = np.concatenate([o.basis(pts), W.astype(complex)], axis=1)
    theta = np.concatenate([p[0:2 * R:2] + 1j * p[1:2 * R:2],
                            p[2 * R:2 * R + N] + 1j * p[2 * R + N:]])
    np.testing.assert_allclose(o.amp(p, pts), b @ theta, rtol=1e-10, atol=1e-12)
    M = (b.conj().T @ b) / len(pts)
    I_form = (theta.conj() @ M @ theta).real
    assert I_form == pytest.approx(np.mean(o.amp2(p, pts)), rel=1e-11)


@pytest.mark.parametrize("spec", REIM_SPECS, ids=lambda s: s.name)
def test_reim_nll_invariant_under_complex_scaling(spec):
    """A is linear in (c, x + i y): theta -> lambda theta scales A by lambda for
    any complex lambda, which leaves -2 ln L unchanged; the gradient is
    orthogonal to both the scale and the rotation direction."""
    o, data, norm = _small_problem(spec)
    p = synth.perturbed_params(spec, 31, 0.02)
    R, N = spec.n_res, spec.n_knots
    v0, g = o.nll_grad(p, data, norm)
    th = np.concatenate([p[0:2 * R:2] + 1j * p[1:2 * R:2], p[2 * R:2 * R + N] + 1j * p[2 * R + N:]])

    def to_params(t):
        q = np.empty_like(p)
        q[0:2 * R:2], q[1:2 * R:2] = t[:R].real, t[:R].imag
        q[2 * R:2 * R + N], q[2 * R + N:] = t[R:].real, t[R:].imag
        return q

    lam = 1.3 * np.exp(0.77j)
    assert o.nll(to_params(lam * th), data, norm) == pytest.approx(v0, rel=1e-12, abs=1e-9)
    gn = np.linalg.norm(g)
    for d in (to_params(th), to_params(1j * th)):
        assert abs(g @ d) < 1e-9 * gn * np.linalg.norm(d)


@pytest.mark.parametrize("spec", REIM_SPECS, ids=lambda s: s.name)
def test_reim_gradient_central_differences(spec):
    o, data, norm = _small_problem(spec)
    p = synth.perturbed_params(spec, 37, 0.02)
    _, g = o.nll_grad(p, data, norm)
    h = 1e-6
    fd = np.empty_like(p)
    for k in range(len(p)):
        e = np.zeros_like(p)
        e[k] = h
        fd[k] = (o.nll(p + e, data, norm) - o.nll(p - e, data, norm)) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-5, atol=1e-5 * np.abs(g).max())


# ------------------------------------------------ gradient in the local form
@pytest.mark.parametrize("spec", [synth.pipipi(10), synth.kpipi(12), synth.as_reim(synth.pipipi(10)),
                                  synth.kkk(40)], ids=lambda s: s.name)
def test_local_form_gradient_equals_dense(spec):
    """The adjoint summed in segment bins and mapped to the knots once (the
    local form the flop count follows) equals the dense per-event form."""
    o = oracle.Oracle(spec)
    truth = synth.true_params(spec)
    data = synth.accept_reject(spec, 3000, synth.numpy_density(lambda x: o.density(truth, x)),
                               seed=3).numpy()
    norm = synth.uniform_in_plot(spec, 4000, synth.numpy_density(
        lambda x: o.inside(x).astype(np.float64)), seed=4).numpy()
    p = synth.perturbed_params(spec, 8)
    w = 0.5 + np.random.default_rng(2).random(len(norm))
    for wts in (None, w):
        v, g = o.nll_grad(p, data, norm, norm_weights=wts)
        vl, gl = o.nll_grad_local(p, data, norm, norm_weights=wts)
        assert vl == pytest.approx(v, rel=1e-13)
        assert np.linalg.norm(gl - g) <= 1e-11 * np.linalg.norm(g)


# ------------------------------------------------------------- flop counting
def test_flop_counter_closed_form():
    """No resonances, two knots, Re/Im S-wave (a linear spline, M = 0): per
    channel A_ = s1 - s and B_ = s - s0 (2), x(s) = c0 A_ + c1 B_ (3), y(s) (3 more,
    A_ and B_ shared): 8; both channels and their sum 18; |A|^2 3; the running sum
    1; ln 1 (data). Gradient: w = 1/|A|^2 and 2w (data), Abar (2); per channel
    the four basis functions A_/h, B_/h, (A_^3/h - h A_)/6 and the same in B_
    (2 + 12) and 8 products and 8 bin sums: 30 per channel."""
    spec = synth.ModelSpec(name="count", mD=synth.M_D, m1=synth.M_PI, m2=synth.M_PI,
                           resonances=(), knots=(0.078, 2.987), swave_form="reim")
    o = oracle.Oracle(spec)
    p = np.array([1.0, 0.5, 0.3, -0.2])
    ev = np.array([[0.5, 1.2], [1.0, 0.9], [2.0, 0.4]])
    assert o.count_flops(p, ev, True, False)["total"] == 23
    assert o.count_flops(p, ev, False, False)["total"] == 22
    assert o.count_flops(p, ev, True, True)["total"] == 23 + 4 + 60
    assert o.count_flops(p, ev, False, True)["total"] == 22 + 2 + 60
    c = o.count_flops(p, ev, True, False)
    assert (c["add"], c["mul"], c["div"], c["sqrt"], c["func"]) == (12, 10, 0, 0, 1)


def test_flop_counter_cse_and_cached_basis():
    """Repeating the Breit-Wigner terms inside the gradient costs nothing (the
    same operations on the same operands), and a stored basis removes exactly
    the Breit-Wigner work: the cached count equals the direct count minus the
    symmetrised basis's own operations."""
    spec = synth.pipipi(10)
    o = oracle.Oracle(spec)
    p = synth.perturbed_params(spec, 3)
    ev = synth.uniform_in_plot(spec, 200, synth.numpy_density(
        lambda x: o.inside(x).astype(np.float64)), seed=9).numpy()
    d = o.count_flops(p, ev, False, False, cached=False)["total"]
    c = o.count_flops(p, ev, False, False, cached=True)["total"]
    dg = o.count_flops(p, ev, False, True, cached=False)["total"]
    cg = o.count_flops(p, ev, False, True, cached=True)["total"]
    assert d - c == pytest.approx(dg - cg, abs=1e-9)
    assert d - c > 100


def test_bench_flop_constants_are_the_oracle_counts():
    """The algorithmic flops per event that bench.py divides by are the
    oracle's counts on the benchmark's model and parameters, averaged over
    PDF-drawn data and uniform normalisation events in equal numbers."""
    import bench
    spec = synth.pipipi(40)
    o = oracle.Oracle(spec)
    truth = synth.true_params(spec)
    p = synth.perturbed_params(spec, 3)
    data = synth.accept_reject(spec, 20000, synth.numpy_density(lambda x: o.density(truth, x)),
                               seed=7).numpy()
    norm = synth.uniform_in_plot(spec, 20000, synth.numpy_density(
        lambda x: o.inside(x).astype(np.float64)), seed=8).numpy()

    def mean(grad, cached, sp=spec):
        oo = oracle.Oracle(sp)
        return 0.5 * (oo.count_flops(p, data, True, grad, cached)["total"] +
                      oo.count_flops(p, norm, False, grad, cached)["total"])
    assert bench.FLOPS_PER_EVENT_FWD == pytest.approx(mean(False, False), abs=0.5)
    assert bench.FLOPS_PER_EVENT_GRAD == pytest.approx(mean(True, False), abs=0.5)
    assert bench.FLOPS_PER_EVENT_GRAD_CACHED == pytest.approx(mean(True, True), abs=0.5)
    reim = synth.as_reim(spec)
    assert bench.FLOPS_PER_EVENT_GRAD_REIM == pytest.approx(mean(True, False, reim), abs=0.5)
    assert bench.FLOPS_PER_EVENT_GRAD_REIM_CACHED == pytest.approx(mean(True, True, reim), abs=0.5)
