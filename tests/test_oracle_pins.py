"""Pins of the CPU oracle to facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself or with the CUDA library.  Each
test checks the oracle against something independent: a library routine
(numpy's Gauss-Legendre, scipy's adaptive quadrature), an exact symbolic
derivation of the integral definitions (sympy), closed forms and textbook
special cases, exact invariants (integer shifts are permutations, mass), the
exact solution of eq. (advection) (translation), the convergence order k+1
of the projection (Sec. II-A), and a brute-force projection that never forms
the update matrices.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_1603_07008_gb300 import workloads as W


# ---------------------------------------------------------------- quadrature

@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 12, 20])
def test_gauss_legendre_matches_numpy(n):
    x, w = O.gauss_legendre(n)
    X, Wt = np.polynomial.legendre.leggauss(n)
    assert np.max(np.abs(x - X)) < 1e-15
    assert np.max(np.abs(w - Wt)) < 1e-14


@pytest.mark.parametrize("n", [2, 4, 5, 12])
def test_gauss_legendre_exact_on_monomials(n):
    x, w = O.gauss_legendre(n)
    for p in range(2 * n):
        exact = 0.0 if p % 2 else 2.0 / (p + 1)
        assert abs(np.dot(w, x ** p) - exact) < 1e-14


def test_legendre_matches_numpy():
    xs = np.linspace(-1, 1, 17)
    for j in range(7):
        c = np.zeros(j + 1)
        c[j] = 1
        ref = np.polynomial.legendre.legval(xs, c)
        got = np.array([O.legendre(j, v) for v in xs])
        assert np.max(np.abs(got - ref)) < 1e-14


# ---------------------------------------------------------------- A and B

def _sympy_ab(k, alpha):
    """A, B from their integral definitions, integrated exactly by sympy."""
    sp = pytest.importorskip("sympy")
    xi = sp.Symbol("xi")
    a = sp.Rational(alpha.numerator, alpha.denominator)
    o = k + 1
    A = [[None] * o for _ in range(o)]
    B = [[None] * o for _ in range(o)]
    for j in range(o):
        for l in range(o):
            Pj = sp.legendre(j, xi)
            A[j][l] = sp.Rational(2 * j + 1, 2) * sp.integrate(Pj * sp.legendre(l, xi - 2 * a), (xi, 2 * a - 1, 1))
            B[j][l] = sp.Rational(2 * j + 1, 2) * sp.integrate(Pj * sp.legendre(l, xi + 2 - 2 * a), (xi, -1, 2 * a - 1))
    return A, B


@pytest.mark.parametrize("k", [0, 1, 2, 3])
@pytest.mark.parametrize("alpha", [Fraction(3, 8), Fraction(1, 3), Fraction(1, 2), Fraction(37, 100),
                                   Fraction(1, 1024), Fraction(1023, 1024)])
def test_ab_matches_exact_symbolic_integrals(k, alpha):
    A, B = O.ab_matrices(k, float(alpha))
    As, Bs = _sympy_ab(k, alpha)
    o = k + 1
    for j in range(o):
        for l in range(o):
            assert abs(A[j, l] - float(As[j][l])) < 4e-15, (j, l)
            assert abs(B[j, l] - float(Bs[j][l])) < 4e-15, (j, l)


def test_ab_dyadic_alpha_three_eighths_k2():
    """At alpha = 3/8 every entry is a dyadic rational; check them exactly
    (values from the symbolic integrals, compared with the rational itself)."""
    As, Bs = _sympy_ab(2, Fraction(3, 8))
    A, B = O.ab_matrices(2, 0.375)
    for j in range(3):
        for l in range(3):
            qa, qb = Fraction(str(As[j][l])), Fraction(str(Bs[j][l]))
            assert qa.denominator & (qa.denominator - 1) == 0   # power of two
            assert abs(A[j, l] - float(qa)) <= 2 * np.finfo(float).eps * max(1, abs(float(qa)))
            assert abs(B[j, l] - float(qb)) <= 2 * np.finfo(float).eps * max(1, abs(float(qb)))


@pytest.mark.parametrize("alpha", [0.0, 0.1, 0.37, 0.5, 0.9])
def test_k0_is_donor_cell(alpha):
    """k = 0 is first-order upwind: u_i <- u_i - alpha (u_i - u_{i-1})."""
    A, B = O.ab_matrices(0, alpha)
    u = np.array([0.3, -1.2, 2.5, 0.7, 1.1])
    upwind = u - alpha * (u - np.roll(u, 1))
    got = O.sweep(u.reshape(-1, 1), [5], 0, 0, -1, alpha)[:, 0]
    assert np.max(np.abs(got - upwind)) < 1e-15
    assert abs(A[0, 0] - (1 - alpha)) < 1e-15 and abs(B[0, 0] - alpha) < 1e-15


@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_ab_identities(k):
    o = k + 1
    A0, B0 = O.ab_matrices(k, 0.0)
    assert np.array_equal(A0, np.eye(o)) and np.array_equal(B0, np.zeros((o, o)))
    sign = np.array([[(-1) ** (j + l) for l in range(o)] for j in range(o)])
    for a in [0.013, 0.25, 0.37, 0.5, 0.81]:
        A, B = O.ab_matrices(k, a)
        Ar, _ = O.ab_matrices(k, 1.0 - a)
        # reflection: B(a) = S A(1-a) S
        assert np.max(np.abs(B - sign * Ar)) < 1e-14
        # row 0: mass conservation; column 0: constants are preserved
        assert np.max(np.abs((A + B)[0, :] - np.eye(o)[0])) < 1e-15
        assert np.max(np.abs((A + B)[:, 0] - np.eye(o)[:, 0])) < 1e-15
    # alpha -> 1 is the pure neighbour copy
    A, B = O.ab_matrices(k, 1.0 - 2.0 ** -40)
    assert np.max(np.abs(B - np.eye(o))) < 1e-10 and np.max(np.abs(A)) < 1e-10


def test_shift_split():
    assert O.shift_split(0.37) == (0, 0.37)
    assert O.shift_split(2.0) == (2, 0.0)
    assert O.shift_split(-0.25) == (-1, 0.75)
    sg, a = O.shift_split(-1e-20)      # s - floor(s) rounds to 1 -> next integer
    assert sg == 0 and a == 0.0
    assert O.shift_split(-3.0) == (-3, 0.0)


# ---------------------------------------------------------------- sweeps

def _rand(n, k, seed):
    return W.random_coefficients(int(np.prod(n)), k, len(n), seed)


@pytest.mark.parametrize("n,dim,shift_dim", [((7,), 0, -1), ((5, 3), 0, 1), ((5, 3), 1, 0),
                                             ((3, 4, 2), 2, 0), ((3, 4, 2), 1, -1)])
@pytest.mark.parametrize("k", [0, 1, 2])
def test_integer_shift_is_bit_exact_roll(n, dim, shift_dim, k):
    u = _rand(n, k, 11)
    ncls = 1 if shift_dim < 0 else n[shift_dim]
    shifts = np.array([(-1) ** c * (c * 3 + 2) for c in range(ncls)], dtype=float)
    got = O.sweep(u, n, k, dim, shift_dim, shifts)
    ref = np.empty_like(u)
    # reshape to [n_{d-1}, ..., n_0, ncoef] and roll each line by its shift
    shp = tuple(reversed(n)) + (u.shape[1],)
    U = u.reshape(shp)
    R = ref.reshape(shp)
    ax = len(n) - 1 - dim
    for c in range(ncls):
        s = int(shifts[c])
        if shift_dim < 0:
            R[...] = np.roll(U, s, axis=ax)
        else:
            sl = [slice(None)] * (len(n) + 1)
            sl[len(n) - 1 - shift_dim] = c
            R[tuple(sl)] = np.roll(U, s, axis=ax)[tuple(sl)]
    assert np.array_equal(got, ref)


def test_full_period_shift_returns_bit_exactly():
    n = (6, 4)
    u = _rand(n, 2, 3)
    assert np.array_equal(O.sweep(u, n, 2, 0, -1, 6.0), u)
    assert np.array_equal(O.sweep(u, n, 2, 1, -1, -8.0), u)


@pytest.mark.parametrize("n,k", [((8,), 1), ((8,), 3), ((5, 4), 2), ((3, 3, 2), 1)])
def test_bruteforce_projection_agrees(n, k):
    u = _rand(n, k, 5)
    rng = np.random.default_rng(1)
    for dim in range(len(n)):
        for shift_dim in [-1] + [m for m in range(len(n)) if m != dim]:
            ncls = 1 if shift_dim < 0 else n[shift_dim]
            shifts = rng.uniform(-2.5 * n[dim], 2.5 * n[dim], size=ncls)
            a = O.sweep(u, n, k, dim, shift_dim, shifts)
            b = O.bruteforce_sweep(u, n, k, dim, shift_dim, shifts, nq=12)
            assert np.max(np.abs(a - b)) < 1e-13 * max(1.0, np.max(np.abs(u)))


def test_mass_conserved_and_l2_nonincreasing():
    n = (16, 8)
    k = 2
    g = W.Grid(n=n, lo=(0.0, -1.0), hi=(2.0, 3.0), pair=(1, -1))
    u = _rand(n, k, 7)
    m0 = O.mass(u, g, k)
    wts = O.l2_weights(k, 2)
    norm = lambda v: math.sqrt(float(np.sum(v * v * wts)))
    rng = np.random.default_rng(2)
    for it in range(20):
        dim = it % 2
        s = rng.uniform(-3, 3, size=n[1 - dim])
        v = O.sweep(u, n, k, dim, 1 - dim, s)
        assert norm(v) <= norm(u) * (1 + 1e-15)
        u = v
    assert abs(O.mass(u, g, k) - m0) <= 1e-14 * np.sum(np.abs(u[:, 0])) * 0.5


def test_one_full_period_in_fractional_steps():
    """Translating by one period in fractional steps returns to the start up
    to the projection error, which shrinks at order k+1."""
    errs = []
    for N in (32, 64):
        g = W.Grid(n=(N,), lo=(0.0,), hi=(1.0,), pair=(-1,))
        u0 = O.project(g, 2, 8, np.array([1.0]), np.array([[[100.0, 0.5, 0.0, 0.0]]]))
        u = u0
        steps = 4 * N // 3 + 1
        s = N / steps
        for _ in range(steps):
            u = O.sweep(u, (N,), 2, 0, -1, s)
        errs.append(O.rel_l2(u, u0, 2, 1))
    assert errs[1] < errs[0] / 6 and errs[1] < 2e-3


def _periodic_gauss(T):
    return np.ones(3), np.array([[[100.0, 0.5 + T + d, 0.0, 0.0]] for d in (-1, 0, 1)])


@pytest.mark.parametrize("k,lo_order", [(0, 0.8), (1, 1.9), (2, 2.9), (3, 3.8)])
def test_convergence_order_vs_exact_translation(k, lo_order):
    """Against the projected exact solution u0(x - aT) of eq. (advection)."""
    errs = []
    for N in (64, 128, 256):
        g = W.Grid(n=(N,), lo=(0.0,), hi=(1.0,), pair=(-1,))
        u = O.project(g, k, 8, *_periodic_gauss(0.0))
        s = 0.37
        steps = int(round(0.25 * N / s))
        for _ in range(steps):
            u = O.sweep(u, g.n, k, 0, -1, s)
        T = steps * s / N
        errs.append(O.rel_l2(u, O.project(g, k, 8, *_periodic_gauss(T)), k, 1))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) > lo_order, orders


def test_config1_close_to_exact_solution():
    p = W.config1()
    g = p.grid
    u = O.project(g, p.k, p.nq, p.weights, p.params)
    h = (g.hi[0] - g.lo[0]) / g.n[0]
    s = p.velocity * p.dt / h
    for _ in range(p.steps):
        u = O.sweep(u, g.n, p.k, 0, -1, s)
    T = p.steps * p.velocity * p.dt
    w, prm = _periodic_gauss(T)
    ex = O.project(g, p.k, p.nq, w, prm)
    assert O.rel_l2(u, ex, p.k, 1) < 1e-7


# ---------------------------------------------------------------- projection

def test_projection_of_polynomials_is_exact():
    """eq. (cj) reproduces a polynomial's own Legendre coefficients.  On a cell
    with centre x_c and width h, x = x_c + h xi / 2, so the linear function has
    c0 = x_c, c1 = h/2 and nothing else.  The factor family holds
    sin(eps x)/eps = x - eps^2 x^3/6 + ..., close enough to x for eps = 1e-5."""
    g = W.Grid(n=(5,), lo=(-1.0,), hi=(2.0,), pair=(-1,))
    eps = 1e-5
    c = O.project(g, 2, 5, np.array([1.0 / eps]), np.array([[[0.0, 0.0, eps, -math.pi / 2]]]))
    h = 3.0 / 5
    xc = -1.0 + (np.arange(5) + 0.5) * h
    assert np.max(np.abs(c[:, 0] - xc)) < 1e-9
    assert np.max(np.abs(c[:, 1] - h / 2)) < 1e-9
    assert np.max(np.abs(c[:, 2])) < 1e-9
    one = O.project(g, 3, 2, np.array([2.5]), np.array([[[0.0, 0.0, 0.0, 0.0]]]))
    assert np.max(np.abs(one[:, 0] - 2.5)) < 1e-15 and np.max(np.abs(one[:, 1:])) < 1e-15


def test_projection_tensor_order_in_several_dimensions():
    """In d dimensions coefficient J = sum_m j_m o^m belongs to P_{j_0}(xi_0)
    P_{j_1}(xi_1) ...: the product of a linear function of x_m (the factor
    sin(eps x)/eps) and constants in the other dimensions has c_0 = x_c, the
    coefficient with j_m = 1 equal to h_m / 2, and no other."""
    eps = 1e-5
    for ndim in (2, 3):
        n = (3, 4, 2)[:ndim]
        g = W.Grid(n=n, lo=(-1.0, 0.5, 2.0)[:ndim], hi=(2.0, 1.5, 3.0)[:ndim], pair=(-1,) * ndim)
        k, o = 2, 3
        for m in range(ndim):
            prm = [[0.0, 0.0, 0.0, 0.0] for _ in range(ndim)]
            prm[m] = [0.0, 0.0, eps, -math.pi / 2]
            c = O.project(g, k, 5, np.array([1.0 / eps]), np.array([prm]))
            h = (g.hi[m] - g.lo[m]) / g.n[m]
            J1 = o ** m
            assert np.max(np.abs(c[:, J1] - h / 2)) < 1e-9, (ndim, m)
            others = [J for J in range(o ** ndim) if J not in (0, J1)]
            assert np.max(np.abs(c[:, others])) < 1e-9, (ndim, m)


def test_projection_matches_adaptive_quadrature():
    scipy_integrate = pytest.importorskip("scipy.integrate")
    p = W.config1()
    g = p.grid
    c = O.project(g, p.k, p.nq, p.weights, p.params)
    h = 1.0 / 1024
    for i in (0, 300, 511, 512, 700):
        xc = (i + 0.5) * h
        for j in range(3):
            f = lambda xi: math.exp(-100 * (xc + h * xi / 2 - 0.5) ** 2) * np.polynomial.legendre.legval(xi, [0] * j + [1])
            ref = (2 * j + 1) / 2 * scipy_integrate.quad(f, -1, 1, epsabs=1e-16, epsrel=1e-14)[0]
            assert abs(c[i, j] - ref) < 1e-14


def test_mass_of_maxwellian_workload_closed_form():
    """int_0^{4pi} int_{-6}^{6} M(v)(1 + 0.01 cos(x/2)) dv dx = 4 pi erf(6/sqrt 2)."""
    p = W.config2(n=64, steps=1)
    u = O.project(p.grid, p.k, p.nq, p.weights, p.params)
    ref = 4 * math.pi * math.erf(6 / math.sqrt(2))
    assert abs(O.mass(u, p.grid, p.k) - ref) / ref < 1e-12


# ---------------------------------------------------------------- bookkeeping

def test_sample_after_matches_full_grid():
    p = W.config3(n=6, steps=1)
    g = p.grid
    u = O.project(g, p.k, p.nq, p.weights, p.params)
    sched = O.schedule(g, "strang", p.dt, p.field_list())
    full = u
    for dim, sd, s in sched:
        full = O.sweep(full, g.n, p.k, dim, sd, s)
    cells = [0, 17, 433, g.cells - 1]
    got = O.sample_after(g, p.k, p.nq, p.weights, p.params, sched, cells)
    assert np.array_equal(got, full[cells])


def test_schedule_structure():
    p = W.config3(n=4, steps=1)
    sched = O.schedule(p.grid, "strang", 0.1, p.field_list())
    assert [d for d, _, _ in sched] == [0, 1, 2, 3, 0, 1]
    assert [sd for _, sd, _ in sched] == [2, 3, 0, 1, 2, 3]
    lie = O.schedule(p.grid, "lie", 0.1, p.field_list())
    assert [d for d, _, _ in lie] == [0, 1, 2, 3]
    # the x-sweep shift is v * tau / h_x with v at the v-cell centres
    h_x = 4 * math.pi / 4
    h_v = 12.0 / 4
    v = -6 + (np.arange(4) + 0.5) * h_v
    assert np.allclose(sched[0][2], v * 0.05 / h_x, rtol=1e-15, atol=0)
    E = p.field_list()[0]
    assert np.allclose(sched[2][2], E * 0.1 / h_v, rtol=1e-15, atol=0)


# ---------------------------------------------------------------- self-consistent field (Vlasov-Poisson)

def _landau_grid(nx, nv):
    p = W.config2(n=8, steps=1)
    return p, W.Grid(n=(nx, nv), lo=p.grid.lo, hi=p.grid.hi, pair=p.grid.pair)


def test_poisson_field_of_a_cosine_density_converges_at_second_order():
    """f0 = M(v)(1 + a cos(k x)) has rho = e (1 + a cos(k x)) with
    e = erf(6 / sqrt 2) on v in [-6, 6]; d_x E = rho - rho_bar gives
    E = e (a / k) sin(k x).  The cell-centre field converges at order 2."""
    errs = []
    for nx in (16, 32, 64):
        p, g = _landau_grid(nx, 64)
        u = O.project(g, 2, p.nq, p.weights, p.params)
        E = O.poisson_field(u, g, 2)
        h = 4 * math.pi / nx
        xc = (np.arange(nx) + 0.5) * h
        ex = math.erf(6 / math.sqrt(2)) * (0.01 / 0.5) * np.sin(0.5 * xc)
        errs.append(np.max(np.abs(E - ex)) / np.max(np.abs(ex)))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) > 1.9 and errs[-1] < 2e-3, (errs, orders)
    # a density constant in x has no field; the sign: E grows where rho > rho_bar
    p, g = _landau_grid(8, 16)
    u = np.zeros((g.cells, 9))
    u[:, 0] = 0.7
    assert np.all(O.poisson_field(u, g, 2) == 0.0)
    u[0, 0] += 1.0        # extra density in cell 0 (v-row 0)
    E = O.poisson_field(u, g, 2)
    assert E[1] - E[0] > 0 and abs(np.mean(E)) < 1e-15


def test_linear_landau_damping_rate():
    """The self-consistent split step damps the field energy of
    f0 = M(v)(1 + 0.01 cos(x / 2)) at twice the linear Landau rate
    gamma = -0.1533 (wave number 1/2), and it oscillates at omega = 1.4156:
    textbook linear theory, independent of the paper."""
    p, g = _landau_grid(64, 128)
    u = O.project(g, 2, p.nq, p.weights, p.params)
    en = [O.field_energy(O.poisson_field(u, g, 2), g)]
    O.vp_step(u, g, 2, "strang", 0.1, 200, en)
    t = np.arange(len(en)) * 0.1
    le = np.log(np.array(en))
    peaks = [i for i in range(1, len(le) - 1) if le[i] > le[i - 1] and le[i] >= le[i + 1] and t[i] < 20]
    gamma = np.polyfit(t[peaks], le[peaks], 1)[0] / 2
    assert abs(gamma + 0.1533) < 0.003, gamma
    omega = math.pi / np.mean(np.diff(t[peaks]))
    assert abs(omega - 1.4156) < 0.05, omega


# ---------------------------------------------------------------- split storage ("# double", Sec. III-A)

def _golden_memorydown():
    rows = []
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "memory_reduction.txt")):
        if line.strip() and not line.startswith("#"):
            d, o, nd, red, src = line.split()
            rows.append((int(d), int(o), int(nd), float(red), src))
    return rows


def test_storage_bytes_reproduce_the_printed_memory_reductions():
    """The memorydown columns of Tables III-VI (one dimension, "# double" =
    0..o) and the 2D / 3D figures of Sec. III-A (c_0 only) follow from which
    coefficients the oracle keeps in FP64."""
    rows = _golden_memorydown()
    for d, o, nd, red, src in rows:
        q = o if nd == o ** d else nd
        assert d == 1 or q in (1, o), src
        r = O.storage_bytes(o - 1, d, o) / O.storage_bytes(o - 1, d, q)
        digits = len(str(red).split(".")[1])
        assert abs(r - red) <= 10 ** -digits + 1e-12, (d, o, nd, r, red, src)
    assert len(rows) == 12


@pytest.mark.parametrize("k,ndim", [(1, 1), (3, 1), (2, 2), (3, 3), (1, 6)])
def test_fp64_coefficients_structure(k, ndim):
    o = k + 1
    for q in range(o + 1):
        m = O.fp64_coefficients(k, ndim, q)
        assert m.sum() == q ** ndim
        # tensor structure: J is FP64 iff each of its digits is
        one = np.arange(o) < q
        full = one
        for _ in range(ndim - 1):
            full = np.logical_and.outer(one, full).reshape(-1)
        assert np.array_equal(m, full)
    assert not O.fp64_coefficients(k, ndim, 0).any()
    assert np.flatnonzero(O.fp64_coefficients(k, ndim, 1)).tolist() == [0]
    assert O.fp64_coefficients(k, ndim, o).all()


def test_round_storage_and_stored_sweeps():
    rng = np.random.default_rng(5)
    n, k = (6, 5), 2
    u = rng.standard_normal((30, 9))
    assert np.array_equal(O.round_storage(u, k, 2, 3), u)
    assert np.array_equal(O.round_storage(u, k, 2, 0), u.astype(np.float32).astype(np.float64))
    r = O.round_storage(u, k, 2, 2)
    assert np.array_equal(O.round_storage(r, k, 2, 2), r)
    m = O.fp64_coefficients(k, 2, 2)
    assert np.array_equal(r[:, m], u[:, m]) and not np.array_equal(r[:, ~m], u[:, ~m])
    # with every coefficient in FP64 the stored sweeps are the plain sweeps
    sw = [(0, 1, rng.uniform(-2, 2, n[1])), (1, -1, [0.37])]
    plain = O.sweep(O.sweep(u, n, k, *sw[0]), n, k, *sw[1])
    assert np.array_equal(O.stored_sweeps(u, n, k, 3, sw), plain)
    # an integer shift moves the stored values unchanged
    for q in (0, 1, 2):
        got = O.stored_sweeps(u, n, k, q, [(1, -1, [2.0])])
        want = np.roll(O.round_storage(u, k, 2, q).reshape(5, 6, 9), 2, axis=0).reshape(30, 9)
        assert np.array_equal(got, want)


# ---------------------------------------------------------------- nodal-in-velocity x-sweep

def _xv(n, lo=(0.0, -1.0), hi=(1.0, 1.0)):
    return W.Grid(n=tuple(n), lo=lo, hi=hi, pair=(1, -1))


@pytest.mark.parametrize("n,k", [((5, 4), 1), ((6, 3), 2), ((4, 3), 3)])
def test_nodal_sweep_agrees_with_bruteforce(n, k):
    """Per node, the update rule equals translating the node's values and
    projecting them back by quadrature (no A, B), for shifts of several cells
    either way."""
    rng = np.random.default_rng(11)
    u = rng.standard_normal((n[0] * n[1], (k + 1) ** 2))
    g = _xv(n, lo=(0.0, -3.0), hi=(1.0, 2.0))
    for tau in (0.37, -0.91, 1.3):
        a = O.sweep_nodal(u, g, k, 0, tau)
        b = O.bruteforce_nodal(u, g, k, 0, tau)
        assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(a))


def test_nodal_sweep_in_three_dimensions_acts_fibre_by_fibre():
    """With a third, unpaired dimension the sweep acts on each of its
    coefficient indices separately: a state that depends on that index only
    through a factor gives the 2D result times the factor."""
    rng = np.random.default_rng(12)
    k, o = 1, 2
    n2 = (4, 3)
    u2 = rng.standard_normal((12, o * o))
    f = rng.standard_normal((2, o))            # the third dimension: 2 cells, o coefficients
    u3 = np.einsum("cj,dk->dckj", u2, f).reshape(2 * 12, o * o * o)   # J = j0 + o j1 + o^2 j2
    g2 = _xv(n2)
    g3 = W.Grid(n=(4, 3, 2), lo=(0.0, -1.0, 0.0), hi=(1.0, 1.0, 1.0), pair=(1, -1, -1))
    a2 = O.sweep_nodal(u2, g2, k, 0, 0.41)
    a3 = O.sweep_nodal(u3, g3, k, 0, 0.41)
    want = np.einsum("cj,dk->dckj", a2, f).reshape(2 * 12, o * o * o)
    assert np.max(np.abs(a3 - want)) <= 1e-14 * np.max(np.abs(want))


def test_nodal_round_trip_and_mass():
    """tau = 0: values at the o Gauss nodes and back reproduce every
    polynomial of degree k in v (the o-point rule is exact to degree 2o - 1);
    and the sweep conserves the mass (sum of cell means)."""
    rng = np.random.default_rng(13)
    for k in (1, 2, 3):
        g = _xv((5, 4))
        u = rng.standard_normal((20, (k + 1) ** 2))
        assert np.max(np.abs(O.sweep_nodal(u, g, k, 0, 0.0) - u)) <= 1e-14 * np.max(np.abs(u))
        a = O.sweep_nodal(u, g, k, 0, 0.73)
        assert abs(O.mass(a, g, k) - O.mass(u, g, k)) <= 1e-14 * np.sum(np.abs(u[:, 0]))


def _free_streaming_terms(T):
    """f(x, v, T) = e^{-v^2} (1 + cos(2 pi (x - v T)) / 2), a sum of three
    separable products: the exact solution of d_t f + v d_x f = 0."""
    w = np.array([1.0, 0.5, 0.5])
    p = np.array([[[0, 0, 0, 0], [1, 0, 0, 0]],
                  [[0, 0, 2 * math.pi, 0], [1, 0, 2 * math.pi * T, 0]],
                  [[0, 0, 2 * math.pi, -math.pi / 2], [1, 0, 2 * math.pi * T, -math.pi / 2]]], dtype=float)
    return w, p


@pytest.mark.parametrize("k", [1, 2])
def test_nodal_sweep_converges_to_free_streaming(k):
    """Free streaming d_t f + v d_x f = 0 over T = 1/2 in 8 x-sweeps: the
    nodal-in-v sweep converges at order k + 1 under refinement in x and v,
    while one velocity per v-cell (the centre) stays first order."""
    T, steps = 0.5, 8
    errs, errc = [], []
    for N in (16, 32):
        g = _xv((N, N))
        u0 = O.project(g, k, k + 3, *_free_streaming_terms(0.0))
        ue = O.project(g, k, k + 3, *_free_streaming_terms(T))
        un, uc = u0, u0
        v = -1.0 + (np.arange(N) + 0.5) * (2.0 / N)
        for _ in range(steps):
            un = O.sweep_nodal(un, g, k, 0, T / steps)
            uc = O.sweep(uc, g.n, k, 0, 1, v * (T / steps) * N)
        errs.append(O.rel_l2(un, ue, k, 2))
        errc.append(O.rel_l2(uc, ue, k, 2))
    order = math.log2(errs[0] / errs[1])
    assert order >= k + 0.8, (errs, order)
    assert errs[1] < errc[1] / 10, (errs, errc)
    assert math.log2(errc[0] / errc[1]) < 1.2


# ---------------------------------------------------------------- error norm

def test_l2_norm_of_projected_data():
    """The function-space L2 norm of the expansion: 1 for the constant 1 on
    the unit box in 1D and 2D (only c_0 = 1), the closed form
    (pi / 200)^(1/4) for exp(-100 (x - 1/2)^2) on [0, 1) to projection
    accuracy, and sqrt(2 / (2j + 1) * h / 2) for a single Legendre mode P_j
    on one cell of width h (Parseval on [-1, 1])."""
    from paper_1603_07008_gb300 import workloads as W
    g1 = W.Grid(n=(16,), lo=(0.0,), hi=(1.0,), pair=(-1,))
    one = O.project(g1, 2, 5, [1.0], [[[0.0, 0.0, 0.0, 0.0]]])
    assert abs(O.l2_norm(one, g1, 2) - 1.0) < 1e-14
    g2 = W.Grid(n=(4, 8), lo=(0.0, -1.0), hi=(2.0, 0.0), pair=(1, -1))
    one2 = O.project(g2, 1, 5, [1.0], [[[0.0, 0.0, 0.0, 0.0], [0.0, 0.0, 0.0, 0.0]]])
    assert abs(O.l2_norm(one2, g2, 1) - np.sqrt(2.0)) < 1e-14   # area 2
    g = W.Grid(n=(512,), lo=(0.0,), hi=(1.0,), pair=(-1,))
    u = O.project(g, 3, 8, [1.0], [[[100.0, 0.5, 0.0, 0.0]]])
    # int_0^1 exp(-200 (x - 1/2)^2) dx = sqrt(pi / 200) erf(sqrt(200) / 2)
    import math
    want = math.sqrt(math.sqrt(math.pi / 200) * math.erf(math.sqrt(200) / 2))
    assert abs(O.l2_norm(u, g, 3) - want) < 1e-9
    h = 0.25
    gc = W.Grid(n=(1,), lo=(0.0,), hi=(h,), pair=(-1,))
    for j in range(4):
        c = np.zeros((1, 4))
        c[0, j] = 1.0
        assert abs(O.l2_norm(c, gc, 3) - math.sqrt(2.0 / (2 * j + 1) * h / 2)) < 1e-15


@pytest.mark.parametrize("dt", [0.1, 2.3])
def test_sample_after_with_nodal_sweeps_equals_the_full_grid(dt):
    """The dependency cones of sampled cells include nodal x-sweeps: two
    Strang steps with nodal x-sweeps, evaluated cell by cell from each target's
    node source cells (apply_cell_nodal), equal the full-grid step bit for bit.
    Odd v-extents put v = 0 inside a v-cell, so some v-cells have nodes on both
    sides of it (different sigma per node); dt = 2.3 shifts by several cells."""
    from paper_1603_07008_gb300 import workloads as W
    for p in (W.config3(n=5, steps=1), W.config2(n=9, steps=1)):
        g = p.grid
        u0 = O.project(g, p.k, p.nq, p.weights, p.params)
        full = O.step(u0, g, p.k, "strang", dt, 2, p.field_list(), nodal_v=True)
        sched = O.schedule_nodal(g, "strang", dt, p.field_list())
        x0 = g.x_dims()[0]
        vd = g.pair[x0]
        sigs = [O.node_sigma(g, p.k, x0, 0.5 * dt, j) for j in range(g.n[vd])]
        assert any(len(set(s)) > 1 for s in sigs)            # nodes of one v-cell that differ in sigma
        if dt > 1:
            assert max(abs(x) for s in sigs for x in s) >= 2   # shifts of several cells
        cells = np.arange(0, g.cells, 3)
        got = O.sample_after(g, p.k, p.nq, p.weights, p.params, sched * 2, cells)
        assert np.array_equal(got, full[cells])
