"""Pins of the FP64 oracle against mathematics, not against itself.

Each test ties one part of the oracle (Section 2 of the paper: kernel, density
Eq. (rho), smoothing-length root, Omega, Eqs. (dvdt)/(dudt); Section 3.1:
integrator) to a closed form, an identity, a symmetry, an independent
enumeration or a limit, so that a dropped term, a wrong sign or index, or a
transposed operand in the oracle fails at least one of them.
"""
import os

import numpy as np
import pytest
from scipy import integrate
from scipy.spatial import cKDTree

import oracle
from paper_1606_02738_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- kernel

def test_cubic_spline_golden_values(oracle_lib):
    """w, w' at dyadic q equal the exact rationals derived by hand."""
    tab = np.loadtxt(os.path.join(GOLDEN, "cubic_spline_values.txt"))
    w, dw = oracle.w_hat(tab[:, 0])
    np.testing.assert_array_equal(w, tab[:, 1])
    np.testing.assert_array_equal(dw, tab[:, 2])


@pytest.mark.parametrize("h", [0.37, 1.0, 2.9])
def test_kernel_normalisation_by_quadrature(oracle_lib, h):
    """int W dV over R^3 = 1 (quadrature on both spline pieces)."""
    f = lambda r: 4 * np.pi * r * r * oracle.W(r, h)
    tot = integrate.quad(f, 0, h / 2, epsabs=0, epsrel=1e-13)[0] + \
        integrate.quad(f, h / 2, h, epsabs=0, epsrel=1e-13)[0]
    assert abs(tot - 1.0) < 1e-12
    assert oracle.W(0.0, h) == pytest.approx(8.0 / (np.pi * h ** 3), rel=1e-15)
    assert oracle.W(h, h) == 0.0 and oracle.W(1.3 * h, h) == 0.0


def test_kernel_derivatives_match_finite_differences(oracle_lib):
    """dW/dr and dW/dh against central differences of W; w' against w; the
    spline and its first derivative are continuous at q = 1/2 and q = 1."""
    h = 0.8
    for r in np.linspace(0.013, 0.987, 37) * h:
        e = 1e-6 * h
        fd_r = (oracle.W(r + e, h) - oracle.W(r - e, h)) / (2 * e)
        fd_h = (oracle.W(r, h + e) - oracle.W(r, h - e)) / (2 * e)
        assert oracle.dWdr(r, h) == pytest.approx(fd_r, rel=1e-7, abs=1e-9)
        assert oracle.dWdh(r, h) == pytest.approx(fd_h, rel=1e-7, abs=1e-9)
    for q0 in (0.5, 1.0):
        e = 1e-9
        w, dw = oracle.w_hat([q0 - e, q0 + e])
        assert abs(w[0] - w[1]) < 1e-8 and abs(dw[0] - dw[1]) < 1e-7
    q = np.linspace(0.001, 0.999, 501)
    e = 1e-7
    wp, _ = oracle.w_hat(q + e)
    wm, _ = oracle.w_hat(q - e)
    _, dw = oracle.w_hat(q)
    np.testing.assert_allclose(dw, (wp - wm) / (2 * e), rtol=1e-6, atol=1e-7)


# ----------------------------------------------------- neighbour search

def _ckdtree_sets(x, L, R):
    t = cKDTree(x, boxsize=L)
    out = []
    for i in range(x.shape[0]):
        js = np.array(sorted(j for j in t.query_ball_point(x[i], R[i]) if j != i), dtype=np.int64)
        out.append(js)
    return out


def test_neighbour_sets_tree_brute_scipy(oracle_lib):
    """k-d tree enumeration == O(N^2) scan == scipy's periodic cKDTree, in a
    non-cubic periodic box with a spread of radii."""
    rng = np.random.default_rng(7)
    L = np.array([1.0, 0.7, 1.3])
    x = rng.random((1500, 3)) * L
    R = rng.uniform(0.03, 0.22, 1500)
    a = oracle.neighbours(x, L, R, use_tree=True)
    b = oracle.neighbours(x, L, R, use_tree=False)
    c = _ckdtree_sets(x, L, R)
    for i in range(len(a)):
        np.testing.assert_array_equal(a[i], b[i])
        np.testing.assert_array_equal(a[i], c[i])
    assert sum(len(s) for s in a) > 20 * 1500


def test_neighbour_sets_on_faces_and_edges(oracle_lib):
    """Particles exactly on the box faces, edges and corner (a lattice through
    the origin) plus tiny offsets across the periodic seam."""
    n = 9
    a = 1.0 / n
    g = np.arange(n) * a
    x = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    x = np.concatenate([x, [[1 - 1e-12, 0.0, 0.0], [1e-12, 1 - 1e-12, 0.5]]])
    L = np.ones(3)
    R = np.full(x.shape[0], 1.5 * a)
    ta = oracle.neighbours(x, L, R, use_tree=True)
    tb = oracle.neighbours(x, L, R, use_tree=False)
    for i in range(len(ta)):
        np.testing.assert_array_equal(ta[i], tb[i])
    # a lattice site has 6 face neighbours and 12 edge neighbours within 1.5 a
    counts = np.array([len(s) for s in ta[:n ** 3]])
    assert np.all(counts >= 18)
    assert np.sum(counts == 18) > n ** 3 // 2


def test_force_pair_sets_tree_brute_scipy(oracle_lib):
    """The force enumerates the pairs r_ij < max(h_i, h_j), reached from either
    side: the k-d tree (which widens each node's reach to its largest h),
    the O(N^2) scan and scipy's periodic cKDTree (the union of i's sphere
    and of every j's sphere that holds i) give the same count per particle,
    on clumps with a 30x spread of h, and the tree and the scan give the
    same a and du/dt."""
    rng = np.random.default_rng(19)
    L = np.array([1.0, 0.8, 1.2])
    centres = rng.random((4, 3)) * L
    x = np.concatenate([
        (centres[rng.integers(0, 4, 1200)] + rng.normal(0.0, 0.04, (1200, 3))) % L,
        rng.random((600, 3)) * L])
    n = x.shape[0]
    h = np.exp(rng.uniform(np.log(0.006), np.log(0.18), n))
    v = rng.normal(0.0, 0.3, (n, 3))
    m = np.full(n, 1.0 / n)
    u = rng.uniform(0.5, 1.5, n)
    rho = rng.uniform(0.5, 2.0, n)
    omega = rng.uniform(0.8, 1.2, n)
    ft = oracle.force(x, v, m, u, h, rho, omega, L, 5.0 / 3.0, use_tree=True)
    fb = oracle.force(x, v, m, u, h, rho, omega, L, 5.0 / 3.0, use_tree=False)
    t = cKDTree(x, boxsize=L)
    reach = [set(t.query_ball_point(x[i], h[i])) - {i} for i in range(n)]
    for j in range(n):
        for i in t.query_ball_point(x[j], h[j]):
            if i != j:
                reach[i].add(j)
    want = np.array([len(r) for r in reach])
    np.testing.assert_array_equal(ft["count"], want)
    np.testing.assert_array_equal(fb["count"], want)
    # pairs reached only through j's larger h are a real share of the set
    own = np.array([len(t.query_ball_point(x[i], h[i])) - 1 for i in range(n)])
    assert (want - own).sum() > 0.2 * want.sum()
    amax = np.abs(fb["a"]).max()
    np.testing.assert_allclose(ft["a"], fb["a"], rtol=0, atol=1e-12 * amax)
    dmax = np.abs(fb["dudt"]).max()
    np.testing.assert_allclose(ft["dudt"], fb["dudt"], rtol=0, atol=1e-12 * dmax)


# --------------------------------------------------- h root and density

@pytest.fixture(scope="module")
def uniform_state(oracle_lib):
    p = inputs.uniform(4096, seed=11, sigma_v=0.3)
    s = oracle.State.from_particles(p)
    oracle.evaluate(s)
    return s


def test_h_root_and_uniqueness(uniform_state):
    """N_i(h_i) = 48 to 1e-12 (re-evaluated at fixed h) and the same root from
    very different starting guesses."""
    s = uniform_state
    d = oracle.density_fixed_h(s.x, s.m, s.box[0], s.h)
    assert np.max(np.abs(d["n_w"] - 48.0)) < 48.0 * 1e-12
    for f in (0.2, 3.0):
        r = oracle.density(s.x, s.m, s.box[0], s.h * f)
        np.testing.assert_allclose(r["h"], s.h, rtol=1e-12)
    np.testing.assert_array_equal(d["count"], s.n_dens)
    nb = oracle.neighbours(s.x, s.box[0], s.h, use_tree=False)
    np.testing.assert_array_equal([len(v) for v in nb], s.n_dens)


def test_density_equals_neighbour_number_relation(uniform_state):
    """Equal masses: rho_i = m (3 / (4 pi h_i^3)) N_i, linking Eq. (rho)
    (constant 8/pi) to the neighbour-number definition (constant 32/3)."""
    s = uniform_state
    expect = s.m * 3.0 / (4 * np.pi * s.h ** 3) * 48.0
    np.testing.assert_allclose(s.rho, expect, rtol=1e-11)


def test_omega_and_dn_dh_by_finite_differences(uniform_state):
    """Omega_i = 1 + h/(3 rho) drho/dh with drho/dh from a central difference
    of rho(h) at fixed positions; dN/dh likewise."""
    s = uniform_state
    idx = np.arange(0, s.x.shape[0], 17)
    e = 1e-6
    up = oracle.density_fixed_h(s.x, s.m, s.box[0], s.h * (1 + e))
    dn = oracle.density_fixed_h(s.x, s.m, s.box[0], s.h * (1 - e))
    fd = (up["rho"] - dn["rho"]) / (2 * e * s.h)
    omega_fd = 1 + s.h / (3 * s.rho) * fd
    np.testing.assert_allclose(s.omega[idx], omega_fd[idx], rtol=2e-6, atol=2e-6)
    base = oracle.density_fixed_h(s.x, s.m, s.box[0], s.h)
    fdn = (up["n_w"] - dn["n_w"]) / (2 * e * s.h)
    np.testing.assert_allclose(base["dn_w_dh"][idx], fdn[idx], rtol=2e-6)


def _lattice_n_w(h_over_a, kmax=8):
    """Weighted neighbour number of a simple-cubic lattice site, summed over
    lattice vectors (no neighbour search) with the oracle's w(q)."""
    k = np.arange(-kmax, kmax + 1)
    n = np.stack(np.meshgrid(k, k, k, indexing="ij"), -1).reshape(-1, 3)
    q = np.linalg.norm(n, axis=1) / h_over_a
    w, _ = oracle.w_hat(q)
    return 32.0 / 3.0 * w.sum()


@pytest.mark.parametrize("n_ngb", [48.0, 100.0, 200.0])
def test_lattice_symmetry_and_limit(oracle_lib, n_ngb):
    """Perfect periodic lattice: every site has the same h, h solves the
    lattice-vector sum, rho is uniform and close to m/a^3, a = 0 and
    du/dt = 0 (v = 0), and a uniform drift leaves both at zero."""
    p = inputs.lattice(14, h_factor=2.0)
    s = oracle.State.from_particles(p)
    s.n_ngb = n_ngb
    oracle.evaluate(s)
    a = p.meta["spacing"]
    assert np.ptp(s.h) <= 1e-12 * s.h[0]
    assert _lattice_n_w(s.h[0] / a) == pytest.approx(n_ngb, rel=1e-12)
    assert np.ptp(s.rho) <= 1e-12 * s.rho[0]
    assert abs(s.rho[0] * a ** 3 / s.m[0] - 1) < (5e-3 if n_ngb < 50 else 1e-3)
    scale = s.m[0] * np.abs(s.omega).max() * s.rho[0] ** -2 * s.u[0] * s.rho[0] / s.h[0] ** 4
    assert np.abs(s.a).max() < 1e-10 * scale * s.m[0] * 100
    assert np.abs(s.dudt).max() == 0.0
    s.v[:] = [0.3, -0.2, 0.7]
    oracle.compute_force(s)
    assert np.abs(s.dudt).max() < 1e-12 * scale
    assert np.abs(s.a).max() < 1e-10 * scale * s.m[0] * 100


# ------------------------------------------------------------- force

def test_momentum_conservation(oracle_lib):
    """sum_i m_i a_i = 0 to round-off: Eq. (dvdt) is antisymmetric in i, j
    once both the h_i and the h_j terms are present (clustered, h spread)."""
    p = inputs.clustered(6000, n_spheres=4, seed=5, sigma_v=0.2)
    s = oracle.State.from_particles(p)
    oracle.evaluate(s)
    assert s.h.max() / s.h.min() > 10
    tot = (s.m[:, None] * s.a).sum(axis=0)
    mag = (s.m[:, None] * np.abs(s.a)).sum()
    assert np.abs(tot).max() < 1e-13 * mag


def test_energy_identity(uniform_state):
    """sum_i m_i (v_i . a_i + du_i/dt) = 0 for any velocities: relabelling
    i <-> j in the h_j term of Eq. (dvdt) cancels Eq. (dudt) exactly."""
    s = uniform_state
    pw = (s.m * (s.v * s.a).sum(axis=1)).sum()
    du = (s.m * s.dudt).sum()
    mag = (s.m * np.abs((s.v * s.a).sum(axis=1))).sum()
    assert mag > 0
    assert abs(pw + du) < 1e-12 * mag


def test_galilean_invariance(uniform_state):
    s = uniform_state
    v2 = s.v + np.array([1.5, -0.4, 2.0])
    t = oracle.State(**{k: getattr(s, k) for k in ("x", "v", "m", "u", "h", "box",
                                                    "box_offsets", "gamma", "n_ngb",
                                                    "rho", "drho_dh", "omega")})
    oracle.compute_force(t, v=v2)
    np.testing.assert_allclose(t.dudt, s.dudt, rtol=1e-9, atol=1e-9 * np.abs(s.dudt).max())
    np.testing.assert_array_equal(t.a, s.a)


def test_force_is_gradient_of_thermal_energy(oracle_lib):
    """Variational pin of Eq. (dvdt) with the Omega term: at fixed entropies
    K_i = P_i / rho_i^gamma the thermal energy U(x) = sum_i m_i K_i
    rho_i^(gamma-1) / (gamma-1), with every h_i re-solved at each position,
    satisfies m_k a_k = -dU/dx_k (equal masses: the neighbour-number and
    mass-density constraints coincide)."""
    p = inputs.uniform(700, seed=23)
    rng = np.random.default_rng(3)
    p.u[:] = np.exp(rng.normal(0, 0.3, p.n)).astype(np.float32)
    s = oracle.State.from_particles(p)
    oracle.evaluate(s, use_tree=False)
    g = s.gamma
    K = (g - 1) * s.u / s.rho ** (g - 1)

    def U(x):
        d = oracle.density(x, s.m, s.box[0], s.h, s.n_ngb, use_tree=False)
        return float((s.m * K * d["rho"] ** (g - 1) / (g - 1)).sum())

    eps = 2e-6
    for k in (0, 101, 333):
        for dim in range(3):
            xp = s.x.copy()
            xm = s.x.copy()
            xp[k, dim] += eps
            xm[k, dim] -= eps
            grad = (U(xp) - U(xm)) / (2 * eps)
            assert -grad / s.m[k] == pytest.approx(s.a[k, dim], rel=2e-5,
                                                   abs=2e-5 * np.abs(s.a[k]).max())


def test_sod_plateau_densities(oracle_lib):
    """The shock-tube set-up: rho ~ 1 on the left, ~0.125 on the right, away
    from the two contact planes (x = 0 and x = 1)."""
    p = inputs.sod(nx_left=96, n_yz_left=24, nx_right=48, n_yz_right=12)
    s = oracle.State.from_particles(p)
    oracle.compute_density(s)
    x0 = s.x[:, 0]
    left = (x0 > 0.3) & (x0 < 0.7)
    right = (x0 > 1.3) & (x0 < 1.7)
    assert abs(np.median(s.rho[left]) - 1.0) < 0.02
    assert abs(np.median(s.rho[right]) - 0.125) < 0.02 * 0.125


# --------------------------------------------------------- integrator

def _energy_error(dt, t_end, p):
    s = oracle.State.from_particles(p)
    oracle.evaluate(s)
    e0 = oracle.diagnostics(s)["energy"]
    mom0 = oracle.diagnostics(s)["momentum"]
    for _ in range(int(round(t_end / dt))):
        oracle.kdk_step(s, dt)
    d = oracle.diagnostics(s)
    return d["energy"] - e0, d["momentum"] - mom0


def test_kdk_second_order_energy_and_momentum(oracle_lib):
    """KDK with a global step: energy error at fixed end time falls as dt^2
    (ratio ~4 when dt halves); total momentum stays at round-off."""
    p = inputs.lattice(10, jitter=0.1, sigma_v=0.05, h_factor=2.3)
    t_end = 0.04
    e1, m1 = _energy_error(0.0025, t_end, p)
    e2, m2 = _energy_error(0.00125, t_end, p)
    assert abs(e1) > 1e-12
    ratio = e1 / e2
    assert 3.0 < ratio < 5.0, (e1, e2, ratio)
    assert np.abs(m1).max() < 1e-14 and np.abs(m2).max() < 1e-14


def _reversal_error(dt, t_end, p):
    """Run to t_end, reverse v (and du/dt, which is odd in v), run back: the
    distance from the starting x, -v and u."""
    s = oracle.State.from_particles(p)
    oracle.evaluate(s)
    x0, v0, u0 = s.x.copy(), s.v.copy(), s.u.copy()
    n = int(round(t_end / dt))
    for _ in range(n):
        oracle.kdk_step(s, dt)
    s.v = -s.v
    s.dudt = -s.dudt
    for _ in range(n):
        oracle.kdk_step(s, dt)
    d = s.x - x0
    d -= s.box[0] * np.round(d / s.box[0])
    return np.abs(d).max(), np.abs(s.v + v0).max(), np.abs(s.u - u0).max()


def test_kdk_time_reversal(oracle_lib):
    """Kick-drift-kick retraces its path when the velocities are reversed: the
    half kicks and the drift are symmetric in time, and only the prediction
    of v and u for the mid-step force (with the rates of the step's start)
    breaks the symmetry, by an amount that falls as dt^3 over a fixed time.
    A drift with the old v, a closing kick with the old a, or a one-sided
    energy update returns with an error of lower order."""
    p = inputs.lattice(10, jitter=0.1, sigma_v=0.05, h_factor=2.3)
    e1 = _reversal_error(0.0025, 0.04, p)
    e2 = _reversal_error(0.00125, 0.04, p)
    for a, b in zip(e1, e2):
        assert 6.0 < a / b < 10.0, (e1, e2)
    assert e1[0] < 1e-8 and e1[1] < 1e-6 and e1[2] < 1e-5


# ------------------------------------------------------------ errors

def test_box_too_small_error(oracle_lib):
    p = inputs.uniform(20, seed=1)
    with pytest.raises(oracle.OracleError) as e:
        oracle.density(p.x, p.m, p.box[0], p.h)
    assert e.value.code == oracle.EBOXTOOSMALL
