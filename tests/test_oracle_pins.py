"""Pins for the FP64 oracle against what the model itself fixes.

Nothing here compares the oracle with itself: every check is a closed form,
an invariant, an independent formulation or a hand-expanded neighbour list,
chosen so that a dropped term, a wrong sign, a wrong index or a transposed
axis in the oracle fails at least one test.
"""
import json
import os

import numpy as np
import pytest

import rdcnn_inputs as inp

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# A second gene with no special values, so that terms cannot cancel by accident.
ODD_GENE = {"dt": 0.05, "a": 0.2, "b": 0.7, "eps": 0.3, "c": 0.5, "Du": 0.11, "Dv": 0.37}


def homogeneous_equilibrium(p):
    """Real solutions of f1 = f2 = 0 (Eq. 2-3) for a uniform field.

    f2 = 0  =>  v = (u + a) / b;  f1 = 0  =>  -u^3/3 + (c - 1/b) u - a/b = 0.
    """
    roots = np.roots([-1.0 / 3.0, 0.0, p["c"] - 1.0 / p["b"], -p["a"] / p["b"]])
    real = sorted(r.real for r in roots if abs(r.imag) < 1e-12)
    return [(u, (u + p["a"]) / p["b"]) for u in real]


def jacobian(p, u):
    """d(f1, f2)/d(u, v) at (u, v), differentiated from Eq. 2-3 by hand."""
    return np.array([[p["c"] - u * u, -1.0], [-p["eps"], p["eps"] * p["b"]]])


@pytest.mark.parametrize("gene", [inp.default_params(), ODD_GENE], ids=["default", "odd"])
def test_fixed_point_is_stationary(oracle_mod, gene):
    eqs = homogeneous_equilibrium(gene)
    assert eqs, "the cubic always has a real root"
    for us, vs in eqs:
        u = np.full((5, 7), us)
        v = np.full((5, 7), vs)
        ut, vt = oracle_mod.run(u, v, gene, 400)
        assert np.max(np.abs(ut - us)) < 1e-12
        assert np.max(np.abs(vt - vs)) < 1e-12


def test_default_equilibrium_value():
    # Derived from Eq. 2-3 with the Sec. II.A defaults (a=-0.3, b=1.3, c=1): a single real
    # equilibrium near (1.139998, 0.646153), a stable focus.
    (us, vs), = homogeneous_equilibrium(inp.default_params())
    assert abs(us - 1.139998) < 1e-6 and abs(vs - 0.646153) < 1e-6
    ev = np.linalg.eigvals(jacobian(inp.default_params(), us))
    assert np.all(ev.real < 0) and np.all(np.abs(ev.imag) > 0.3)


@pytest.mark.parametrize("gene", [inp.default_params(), ODD_GENE], ids=["default", "odd"])
def test_linearisation_about_equilibrium(oracle_mod, gene):
    """A small uniform perturbation evolves by (I + dt J)^t to first order.

    Pins dt and all four partial derivatives of the reaction (Eq. 2-3).
    """
    us, vs = homogeneous_equilibrium(gene)[-1]
    d0 = np.array([1e-7, -0.6e-7])
    u = np.full((3, 4), us + d0[0])
    v = np.full((3, 4), vs + d0[1])
    T = 60
    ut, vt = oracle_mod.run(u, v, gene, T)
    M = np.eye(2) + gene["dt"] * jacobian(gene, us)
    pred = np.linalg.matrix_power(M, T) @ d0
    got = np.array([ut[1, 2] - us, vt[1, 2] - vs])
    assert np.linalg.norm(got - pred) <= 1e-5 * np.linalg.norm(pred) + 1e-15


@pytest.mark.parametrize("shape,p,q", [((12, 20), 1, 3), ((16, 16), 2, 5), ((9, 7), 4, 1)])
def test_fourier_mode_decay(oracle_mod, shape, p, q):
    """Pure diffusion: a Fourier mode decays by 1 - dt D (4 - 2 cos kx - 2 cos ky) per step."""
    nn, nm = shape
    par = dict(ODD_GENE)
    u0 = inp.fourier_mode(nn, nm, p, q)
    v0 = inp.fourier_mode(nn, nm, q % nn, p % nm)
    T = 25
    ut, vt = oracle_mod.run(u0, v0, par, T, reaction=oracle_mod.NONE)

    def gain(D, pp, qq):
        return 1.0 - par["dt"] * D * (4.0 - 2.0 * np.cos(2 * np.pi * pp / nn) - 2.0 * np.cos(2 * np.pi * qq / nm))

    np.testing.assert_allclose(ut, gain(par["Du"], p, q) ** T * u0, rtol=0, atol=1e-12)
    np.testing.assert_allclose(vt, gain(par["Dv"], q % nn, p % nm) ** T * v0, rtol=0, atol=1e-12)


def test_mass_conserved_without_reaction(oracle_mod):
    x = inp.uniform_field(3, 13, 17)
    y = inp.uniform_field(4, 13, 17)
    ut, vt = oracle_mod.run(x, y, ODD_GENE, 40, reaction=oracle_mod.NONE)
    assert abs(ut.sum() - x.sum()) < 1e-11
    assert abs(vt.sum() - y.sum()) < 1e-11


def test_uniform_stays_uniform_and_follows_cell_map(oracle_mod):
    gene = inp.default_params()
    u = np.full((6, 9), 0.37)
    v = np.full((6, 9), -0.21)
    ut, vt = oracle_mod.run(u, v, gene, 300)
    assert np.all(ut == ut[0, 0]) and np.all(vt == vt[0, 0])
    su, sv = oracle_mod.scalar_map(0.37, -0.21, gene, 300)
    assert ut[0, 0] == su[-1] and vt[0, 0] == sv[-1]


# u = v = k_a x (Eq. 1, first line) on a 2 x 3 image, the products worked by hand
# (every factor and product is a short binary fraction, so FP64 holds them exactly).
INIT_X = [[1.0, -2.0, 0.5], [4.0, -0.25, 3.0]]
INIT_CASES = {
    0.75: [[0.75, -1.5, 0.375], [3.0, -0.1875, 2.25]],
    -2.5: [[-2.5, 5.0, -1.25], [-10.0, 0.625, -7.5]],
}


@pytest.mark.parametrize("ka", sorted(INIT_CASES))
def test_init_state_scales_both_fields_by_ka(oracle_mod, ka):
    x = np.array(INIT_X)
    u, v = oracle_mod.init_state(x, ka)
    want = np.array(INIT_CASES[ka])
    assert u.dtype == np.float64 and v.dtype == np.float64
    assert u.shape == (2, 3) and v.shape == (2, 3)
    assert np.array_equal(u, want) and np.array_equal(v, want)
    # two independent planes, neither of them the input image
    assert not np.shares_memory(u, v)
    assert not np.shares_memory(u, x) and not np.shares_memory(v, x)
    u[0, 0] = 99.0
    assert v[0, 0] == want[0, 0] and x[0, 0] == INIT_X[0][0]


@pytest.mark.parametrize("ka", [1.0, 0.6])
def test_no_diffusion_means_independent_cells(oracle_mod, ka):
    gene = inp.default_params(Du=0.0, Dv=0.0)
    x = inp.uniform_field(0, 5, 6)
    u, v = oracle_mod.init_state(x, ka)
    ut, vt = oracle_mod.run(u, v, gene, 100)
    for i in range(5):
        for j in range(6):
            su, sv = oracle_mod.scalar_map(ka * x[i, j], ka * x[i, j], gene, 100)
            assert ut[i, j] == su[-1] and vt[i, j] == sv[-1]


def test_one_by_one_grid_is_the_cell_map(oracle_mod):
    """On a 1 x 1 torus every neighbour is the cell itself: the Laplacian is exactly 0."""
    gene = inp.default_params()
    ut, vt = oracle_mod.run(np.array([[0.8]]), np.array([[-0.4]]), gene, 200)
    su, sv = oracle_mod.scalar_map(0.8, -0.4, gene, 200)
    assert ut[0, 0] == su[-1] and vt[0, 0] == sv[-1]


def test_scalar_map_closed_form_special_case(oracle_mod):
    """With c = 0, v = 0, eps = 0 the cell map is u <- u - dt u^3 / 3, v fixed.

    For a single step from u0 that is u0 (1 - dt u0^2 / 3); check against this
    and against the known monotone decay toward 0 for |u0| < sqrt(3/dt).
    """
    p = {"dt": 0.1, "a": 0.0, "b": 1.0, "eps": 0.0, "c": 0.0, "Du": 0.0, "Dv": 0.0}
    tu, tv = oracle_mod.scalar_map(1.5, 0.0, p, 50)
    assert abs(tu[1] - 1.5 * (1 - 0.1 * 1.5 ** 2 / 3.0)) < 1e-15
    assert np.all(np.diff(tu) < 0) and np.all(tu > 0) and np.all(tv == 0.0)


# Neighbour lists written out by hand (N, S, W, E) for small tori, cell = (row, col).
HAND_NEIGHBOURS = {
    (2, 2): {
        (0, 0): [(1, 0), (1, 0), (0, 1), (0, 1)],
        (0, 1): [(1, 1), (1, 1), (0, 0), (0, 0)],
        (1, 0): [(0, 0), (0, 0), (1, 1), (1, 1)],
        (1, 1): [(0, 1), (0, 1), (1, 0), (1, 0)],
    },
    (2, 3): {
        (0, 0): [(1, 0), (1, 0), (0, 2), (0, 1)],
        (0, 1): [(1, 1), (1, 1), (0, 0), (0, 2)],
        (0, 2): [(1, 2), (1, 2), (0, 1), (0, 0)],
        (1, 0): [(0, 0), (0, 0), (1, 2), (1, 1)],
        (1, 1): [(0, 1), (0, 1), (1, 0), (1, 2)],
        (1, 2): [(0, 2), (0, 2), (1, 1), (1, 0)],
    },
    (3, 3): {
        (0, 0): [(2, 0), (1, 0), (0, 2), (0, 1)],
        (0, 1): [(2, 1), (1, 1), (0, 0), (0, 2)],
        (0, 2): [(2, 2), (1, 2), (0, 1), (0, 0)],
        (1, 0): [(0, 0), (2, 0), (1, 2), (1, 1)],
        (1, 1): [(0, 1), (2, 1), (1, 0), (1, 2)],
        (1, 2): [(0, 2), (2, 2), (1, 1), (1, 0)],
        (2, 0): [(1, 0), (0, 0), (2, 2), (2, 1)],
        (2, 1): [(1, 1), (0, 1), (2, 0), (2, 2)],
        (2, 2): [(1, 2), (0, 2), (2, 1), (2, 0)],
    },
    (3, 4): {
        (0, 0): [(2, 0), (1, 0), (0, 3), (0, 1)],
        (0, 1): [(2, 1), (1, 1), (0, 0), (0, 2)],
        (0, 2): [(2, 2), (1, 2), (0, 1), (0, 3)],
        (0, 3): [(2, 3), (1, 3), (0, 2), (0, 0)],
        (1, 0): [(0, 0), (2, 0), (1, 3), (1, 1)],
        (1, 1): [(0, 1), (2, 1), (1, 0), (1, 2)],
        (1, 2): [(0, 2), (2, 2), (1, 1), (1, 3)],
        (1, 3): [(0, 3), (2, 3), (1, 2), (1, 0)],
        (2, 0): [(1, 0), (0, 0), (2, 3), (2, 1)],
        (2, 1): [(1, 1), (0, 1), (2, 0), (2, 2)],
        (2, 2): [(1, 2), (0, 2), (2, 1), (2, 3)],
        (2, 3): [(1, 3), (0, 3), (2, 2), (2, 0)],
    },
}


@pytest.mark.parametrize("shape", sorted(HAND_NEIGHBOURS))
def test_tiny_grids_hand_expanded(oracle_mod, shape):
    nb = HAND_NEIGHBOURS[shape]
    gene = ODD_GENE
    u = inp.uniform_field(11, *shape)
    v = inp.uniform_field(12, *shape)
    un, vn = oracle_mod.step(u, v, gene)
    dt, a, b, eps, c, Du, Dv = (gene[k] for k in ("dt", "a", "b", "eps", "c", "Du", "Dv"))
    for cell, nbrs in nb.items():
        lu = sum(u[r] for r in nbrs) - 4 * u[cell]
        lv = sum(v[r] for r in nbrs) - 4 * v[cell]
        eu = u[cell] + dt * (c * u[cell] - u[cell] ** 3 / 3 - v[cell] + Du * lu)
        ev = v[cell] + dt * (-eps * (u[cell] - b * v[cell] + a) + Dv * lv)
        assert abs(un[cell] - eu) < 1e-14 and abs(vn[cell] - ev) < 1e-14


def test_c_loops_agree_with_numpy_formulation(oracle_mod):
    gene = inp.default_params()
    x = inp.uniform_field(0, 17, 23)
    u, v = oracle_mod.init_state(x, 1.0)
    uc, vc = oracle_mod.run(u, v, gene, 60)
    un, vn = oracle_mod.run_numpy(u, v, gene, 60)
    assert np.linalg.norm(uc - un) <= 1e-13 * np.linalg.norm(un)
    assert np.linalg.norm(vc - vn) <= 1e-13 * np.linalg.norm(vn)


def test_threads_do_not_change_results(oracle_mod):
    x = inp.uniform_field(5, 33, 20)
    u1, v1 = oracle_mod.run(x, x, inp.default_params(), 20, nthreads=1)
    u4, v4 = oracle_mod.run(x, x, inp.default_params(), 20, nthreads=4)
    assert np.array_equal(u1, u4) and np.array_equal(v1, v4)


def test_shift_and_d4_symmetry_bitwise(oracle_mod):
    gene = inp.default_params()
    x = inp.uniform_field(7, 16, 16)
    u, v = oracle_mod.run(x, -x, gene, 30)
    us, vs = oracle_mod.run(np.roll(x, (3, -5), (0, 1)), np.roll(-x, (3, -5), (0, 1)), gene, 30)
    assert np.array_equal(us, np.roll(u, (3, -5), (0, 1))) and np.array_equal(vs, np.roll(v, (3, -5), (0, 1)))
    ut, vt = oracle_mod.run(x.T, -x.T, gene, 30)
    assert np.array_equal(ut, u.T) and np.array_equal(vt, v.T)
    uf, vf = oracle_mod.run(x[::-1, :], -x[::-1, :], gene, 30)
    assert np.array_equal(uf, u[::-1, :]) and np.array_equal(vf, v[::-1, :])
    ug, vg = oracle_mod.run(x[:, ::-1], -x[:, ::-1], gene, 30)
    assert np.array_equal(ug, u[:, ::-1]) and np.array_equal(vg, v[:, ::-1])


def test_light_cone_embedding(oracle_mod):
    """A centred patch evolves identically on any torus large enough to hold its light cone;
    outside the cone every cell follows the cell map started from (0, 0)."""
    gene = inp.default_params()
    T = 12
    small = inp.mid_patch(0, 48, 48)
    big = inp.mid_patch(0, 80, 80)
    us, vs = oracle_mod.run(small, small, gene, T)
    ub, vb = oracle_mod.run(big, big, gene, T)
    off = 16  # patch origin moves from 16 to 32
    assert np.array_equal(ub[off:off + 48, off:off + 48], us)
    assert np.array_equal(vb[off:off + 48, off:off + 48], vs)
    bu, bv = oracle_mod.scalar_map(0.0, 0.0, gene, T)
    r0, c0 = inp.patch_origin(80, 80)
    far = np.ones((80, 80), bool)
    far[r0 - T:r0 + 16 + T, c0 - T:c0 + 16 + T] = False
    assert np.all(ub[far] == bu[-1]) and np.all(vb[far] == bv[-1])


def test_zero_steps_is_identity(oracle_mod):
    x = inp.uniform_field(1, 4, 5)
    u, v = oracle_mod.run(x, 2 * x, inp.default_params(), 0)
    assert np.array_equal(u, x) and np.array_equal(v, 2 * x)


def test_golden_small_run(oracle_mod):
    """Regression fixture written by tests/golden/make_golden.py (oracle only)."""
    with open(os.path.join(GOLDEN, "oracle_4x5_T10.json")) as f:
        g = json.load(f)
    x = inp.uniform_field(g["seed"], 4, 5)
    u, v = oracle_mod.run(x, x, g["params"], g["T"])
    np.testing.assert_allclose(u, np.array(g["u"]), rtol=0, atol=1e-15)
    np.testing.assert_allclose(v, np.array(g["v"]), rtol=0, atol=1e-15)


# ----------------------------------------------------------------------------- adjoint pins

def _loss(u, v, wu, wv):
    return float(np.sum(wu * u) + np.sum(wv * v))


CENN_ADJ_GENE = {"dt": 0.1, "a": 0.0, "b": 0.0, "eps": 0.0, "c": 1.3, "Du": -0.2, "Dv": 0.0}
ADJ_CASES = [(inp.default_params(), "fhn", "periodic", (7, 9)), (ODD_GENE, "fhn", "periodic", (7, 9)),
             (inp.default_params(), "fhn", "zeroflux", (7, 9)), (ODD_GENE, "fhn", "zeroflux", (2, 5)),
             (CENN_ADJ_GENE, "cenn", "periodic", (7, 9)), (CENN_ADJ_GENE, "cenn", "zeroflux", (6, 5))]


@pytest.mark.parametrize("gene,reaction,boundary,shape", ADJ_CASES,
                         ids=["default-torus", "odd-torus", "default-zeroflux", "odd-zeroflux-2x5",
                              "cenn-torus", "cenn-zeroflux-6x5"])
def test_adjoint_matches_central_differences(oracle_mod, gene, reaction, boundary, shape):
    """Linear loss L = <wu, u_T> + <wv, v_T>; FD of the forward map in every gene entry and
    along random directions of the start state (the forward map is pinned on its own).  The
    CeNN start state spans both saturated arms (no cell sits within the FD step of a corner
    of the output function along these seeded trajectories)."""
    nn, nm = shape
    T = 25
    bc = oracle_mod.ZEROFLUX if boundary == "zeroflux" else oracle_mod.PERIODIC
    rx = oracle_mod.CENN if reaction == "cenn" else oracle_mod.FHN
    scale = 1.7 if reaction == "cenn" else 1.0
    x = scale * inp.uniform_field(21, nn, nm)
    y = inp.uniform_field(22, nn, nm)
    wu = inp.uniform_field(23, nn, nm)
    wv = inp.uniform_field(24, nn, nm)
    run = lambda a, b, g: oracle_mod.run(a, b, g, T, reaction=rx, boundary=bc)
    lu0, lv0, g = oracle_mod.adjoint(x, y, gene, T, wu, wv, n_checkpoints=4, reaction=rx, boundary=bc)
    names = ["Du", "Dv", "a", "b", "eps", "c"]
    for k, name in enumerate(names):
        h = 1e-5 * max(1.0, abs(gene[name]))
        pp = dict(gene); pp[name] += h
        pm = dict(gene); pm[name] -= h
        fd = (_loss(*run(x, y, pp), wu, wv) - _loss(*run(x, y, pm), wu, wv)) / (2 * h)
        assert abs(g[k] - fd) <= 1e-7 * max(1.0, abs(fd)), (name, g[k], fd)
    du = inp.uniform_field(25, nn, nm)
    dv = inp.uniform_field(26, nn, nm)
    h = 1e-5
    fd = (_loss(*run(x + h * du, y + h * dv, gene), wu, wv)
          - _loss(*run(x - h * du, y - h * dv, gene), wu, wv)) / (2 * h)
    ad = float(np.sum(lu0 * du) + np.sum(lv0 * dv))
    assert abs(ad - fd) <= 1e-7 * max(1.0, abs(fd))


def test_adjoint_checkpoint_count_does_not_matter(oracle_mod):
    gene = inp.default_params()
    x = inp.uniform_field(31, 6, 8)
    wu = inp.uniform_field(32, 6, 8)
    ref = oracle_mod.adjoint(x, x, gene, 17, wu, 0 * wu, n_checkpoints=17)
    for nck in (1, 3, 5, 0):
        got = oracle_mod.adjoint(x, x, gene, 17, wu, 0 * wu, n_checkpoints=nck)
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
        np.testing.assert_allclose(got[2], ref[2], rtol=1e-14, atol=1e-300)


@pytest.mark.parametrize("boundary", ["periodic", "zeroflux"])
def test_adjoint_of_pure_diffusion_is_diffusion(oracle_mod, boundary):
    """The 5-point Laplacian is symmetric (on the torus, and under zero flux, where a missing
    neighbour adds to the diagonal), so with no reaction the adjoint sweep is the forward
    sweep applied to the co-state, and the gene gradients of the reaction vanish."""
    bc = oracle_mod.ZEROFLUX if boundary == "zeroflux" else oracle_mod.PERIODIC
    gene = ODD_GENE
    x = inp.uniform_field(41, 8, 11)
    wu = inp.uniform_field(42, 8, 11)
    wv = inp.uniform_field(43, 8, 11)
    lu0, lv0, g = oracle_mod.adjoint(x, x, gene, 13, wu, wv, reaction=oracle_mod.NONE, boundary=bc)
    fu, fv = oracle_mod.run(wu, wv, gene, 13, reaction=oracle_mod.NONE, boundary=bc)
    assert np.array_equal(lu0, fu) and np.array_equal(lv0, fv)
    assert np.all(g[2:] == 0.0)


@pytest.mark.parametrize("boundary", ["periodic", "zeroflux"])
def test_cenn_adjoint_without_feedback_is_a_closed_form(oracle_mod, boundary):
    """CeNN cell with c = Du = 0: u+ = (1 - dt) u + dt v, v+ = v, a linear map whose transpose
    gives lu_0 = (1 - dt)^T lu_T and lv_0 = lv_T + (1 - (1 - dt)^T) lu_T; only the c and Du
    entries of the gene gradient can be non-zero."""
    bc = oracle_mod.ZEROFLUX if boundary == "zeroflux" else oracle_mod.PERIODIC
    gene = {"dt": 0.07, "a": 0.0, "b": 0.0, "eps": 0.0, "c": 0.0, "Du": 0.0, "Dv": 0.0}
    T = 19
    x = 1.5 * inp.uniform_field(44, 5, 6)
    y = inp.uniform_field(45, 5, 6)
    wu = inp.uniform_field(46, 5, 6)
    wv = inp.uniform_field(47, 5, 6)
    lu0, lv0, g = oracle_mod.adjoint(x, y, gene, T, wu, wv, reaction=oracle_mod.CENN, boundary=bc)
    q = (1.0 - gene["dt"]) ** T
    np.testing.assert_allclose(lu0, q * wu, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(lv0, wv + (1.0 - q) * wu, rtol=1e-13, atol=1e-15)
    assert np.all(g[1:5] == 0.0)


def test_adjoint_zero_steps(oracle_mod):
    x = inp.uniform_field(1, 3, 3)
    lu0, lv0, g = oracle_mod.adjoint(x, x, inp.default_params(), 0, x, 2 * x)
    assert np.array_equal(lu0, x) and np.array_equal(lv0, 2 * x) and np.all(g == 0)


# ----------------------------------------------------------------------------- search statistics

def test_summary_uniform_field(oracle_mod):
    s = oracle_mod.summary(np.full((6, 9), 0.25), np.full((6, 9), -2.0), 0.01)
    np.testing.assert_array_equal(s, [0.25, 0.0, 0.25, 0.25, -2.0, 0.0, 0.0, 0.0])


def test_summary_checkerboard_closed_form(oracle_mod):
    """+-1 checkerboard of period 2 on an even torus: every cell differs from both forward
    neighbours by 2, so the gradient sum is 4 everywhere; mean 0, variance 1."""
    i, j = np.meshgrid(np.arange(8), np.arange(10), indexing="ij")
    u = np.where((i + j) % 2 == 0, 1.0, -1.0)
    s = oracle_mod.summary(u, 0.5 * u, 3.9)
    np.testing.assert_allclose(s, [0.0, 1.0, -1.0, 1.0, 0.0, 0.25, 4.0, 1.0], atol=1e-15)
    assert oracle_mod.summary(u, u, 4.0)[7] == 0.0  # strict inequality


def test_summary_single_bump_wraps(oracle_mod):
    """One cell of height h at the corner of a 5 x 4 torus: the gradient sum is 2h at the
    bump and h at the two cells whose forward neighbour (wrapping) is the bump."""
    h = 0.7
    u = np.zeros((5, 4))
    u[0, 0] = h
    s = oracle_mod.summary(u, u, 0.5)
    assert abs(s[6] - (2 * h + h + h) / 20) < 1e-15
    assert s[7] == 3 / 20
    assert abs(s[1] - (h * h / 20 - (h / 20) ** 2)) < 1e-15


# ---------------------------------------------------------------------------
# Zero-flux boundary and the CeNN cell (the framework-as-template variants of
# Sec. I / Sec. II.A; the readings are stated in rdcnn_oracle.c).
# ---------------------------------------------------------------------------

# Chua-Yang cell gene: feedback centre c, arms Du; a, b, eps, Dv unused.
CENN_GENE = {"dt": 0.1, "a": 0.0, "b": 0.0, "eps": 0.0, "c": 0.2, "Du": 0.05, "Dv": 0.0}


def _mirror_extend(f):
    """Even extension of an N x M plane to a 2N x 2M torus (reflection about the cell faces)."""
    top = np.concatenate([f, f[:, ::-1]], axis=1)
    return np.concatenate([top, top[::-1, :]], axis=0)


@pytest.mark.parametrize("reaction", ["FHN", "NONE", "CENN"])
def test_zero_flux_is_the_mirrored_torus_bitwise(oracle_mod, reaction):
    """A zero-flux N x M grid evolves exactly as the first quadrant of the 2N x 2M torus holding
    the mirror image: the face between the edge cell and its ghost is a mirror plane, and the
    periodic model (pinned above) keeps a mirror-symmetric state mirror-symmetric, so the edge
    cell's outside neighbour is the edge cell itself in both.  Sums are formed in the same order,
    so equality is bitwise."""
    rx = getattr(oracle_mod, reaction)
    gene = CENN_GENE if reaction == "CENN" else ODD_GENE
    x = 1.6 * inp.uniform_field(21, 7, 10)
    w = 0.3 * inp.uniform_field(22, 7, 10)
    ut, vt = oracle_mod.run(x, w, gene, 15, reaction=rx, boundary=oracle_mod.ZEROFLUX)
    ue, ve = oracle_mod.run(_mirror_extend(x), _mirror_extend(w), gene, 15, reaction=rx)
    assert np.array_equal(ut, ue[:7, :10]) and np.array_equal(vt, ve[:7, :10])
    # and the zero-flux answer is not the small torus's
    up, _ = oracle_mod.run(x, w, gene, 15, reaction=rx)
    assert not np.allclose(up, ut)


@pytest.mark.parametrize("shape,k,l", [((12, 20), 1, 3), ((9, 7), 4, 2), ((16, 5), 0, 1)])
def test_zero_flux_cosine_mode_decay(oracle_mod, shape, k, l):
    """Pure diffusion with zero flux: cos(pi k (i + 1/2) / N) cos(pi l (j + 1/2) / M) is an
    eigenvector of the Neumann 5-point Laplacian with eigenvalue
    2 cos(pi k / N) - 2 + 2 cos(pi l / M) - 2."""
    nn, nm = shape
    i, j = np.meshgrid(np.arange(nn), np.arange(nm), indexing="ij")
    mode = np.cos(np.pi * k * (i + 0.5) / nn) * np.cos(np.pi * l * (j + 0.5) / nm)
    par = dict(ODD_GENE)
    T = 30
    ut, vt = oracle_mod.run(mode, 0.5 * mode, par, T, reaction=oracle_mod.NONE,
                            boundary=oracle_mod.ZEROFLUX)
    lam = 2 * np.cos(np.pi * k / nn) - 2 + 2 * np.cos(np.pi * l / nm) - 2
    np.testing.assert_allclose(ut, (1 + par["dt"] * par["Du"] * lam) ** T * mode, rtol=0, atol=1e-12)
    np.testing.assert_allclose(vt, (1 + par["dt"] * par["Dv"] * lam) ** T * 0.5 * mode, rtol=0, atol=1e-12)


def test_zero_flux_conserves_mass_without_reaction(oracle_mod):
    x = inp.uniform_field(5, 11, 14)
    ut, vt = oracle_mod.run(x, -x, ODD_GENE, 40, reaction=oracle_mod.NONE, boundary=oracle_mod.ZEROFLUX)
    assert abs(ut.sum() - x.sum()) < 1e-11 and abs(vt.sum() + x.sum()) < 1e-11


def test_zero_flux_uniform_field_follows_cell_map(oracle_mod):
    gene = inp.default_params()
    ut, vt = oracle_mod.run(np.full((5, 8), 0.37), np.full((5, 8), -0.21), gene, 200,
                            boundary=oracle_mod.ZEROFLUX)
    su, sv = oracle_mod.scalar_map(0.37, -0.21, gene, 200)
    assert np.all(ut == su[-1]) and np.all(vt == sv[-1])


@pytest.mark.parametrize("boundary", ["PERIODIC", "ZEROFLUX"])
def test_cenn_uniform_linear_region_closed_form(oracle_mod, boundary):
    """|x| < 1 throughout: y(x) = x, so a uniform state obeys x+ = x + dt (-x + (c + 4 Du) x + w):
    x_T = x* + (x0 - x*) r^T with r = 1 - dt (1 - c - 4 Du), x* = w / (1 - c - 4 Du)."""
    g = CENN_GENE
    x0, w = 0.3, 0.2
    T = 60
    ut, vt = oracle_mod.run(np.full((6, 5), x0), np.full((6, 5), w), g, T, reaction=oracle_mod.CENN,
                            boundary=getattr(oracle_mod, boundary))
    k = 1 - g["c"] - 4 * g["Du"]
    xs = w / k
    np.testing.assert_allclose(ut, xs + (x0 - xs) * (1 - g["dt"] * k) ** T, rtol=0, atol=1e-14)
    assert np.all(vt == w)


@pytest.mark.parametrize("x0,expect_star", [(3.0, 3.5), (-3.0, -2.5)])
def test_cenn_uniform_saturated_closed_form(oracle_mod, x0, expect_star):
    """|x| > 1 throughout: every output is sign(x), so x+ = x + dt (-x + (c + 4 Du) sign(x) + w)
    with fixed point x* = (c + 4 Du) sign(x) + w; here c = 2, Du = 0.25, w = 0.5."""
    g = dict(CENN_GENE, c=2.0, Du=0.25)
    T = 50
    ut, _ = oracle_mod.run(np.full((4, 7), x0), np.full((4, 7), 0.5), g, T, reaction=oracle_mod.CENN)
    np.testing.assert_allclose(ut, expect_star + (x0 - expect_star) * (1 - g["dt"]) ** T, rtol=0, atol=1e-13)


@pytest.mark.parametrize("shape,p,q", [((12, 20), 1, 3), ((9, 7), 4, 1)])
def test_cenn_fourier_mode_linear_region(oracle_mod, shape, p, q):
    """About the uniform fixed point xbar (|x| < 1), a periodic mode of amplitude d evolves as
    d_T = d mu^T, mu = 1 + dt (-1 + c + 2 Du (cos(2 pi p / N) + cos(2 pi q / M)))."""
    nn, nm = shape
    g = CENN_GENE
    xbar = 0.2
    w = xbar * (1 - g["c"] - 4 * g["Du"])
    mode = inp.fourier_mode(nn, nm, p, q)
    T = 40
    ut, _ = oracle_mod.run(xbar + 0.1 * mode, np.full(shape, w), g, T, reaction=oracle_mod.CENN)
    mu = 1 + g["dt"] * (-1 + g["c"] + 2 * g["Du"] * (np.cos(2 * np.pi * p / nn) + np.cos(2 * np.pi * q / nm)))
    np.testing.assert_allclose(ut, xbar + 0.1 * mu ** T * mode, rtol=0, atol=1e-13)


def test_cenn_uncoupled_bistable_cells_saturate_to_their_sign(oracle_mod):
    """Du = 0, w = 0, c = 2: each cell is x+ = x + dt (-x + 2 y(x)), whose stable fixed points
    are +-2 (outputs +-1); a cell starting at x0 != 0 ends at 2 sign(x0)."""
    g = dict(CENN_GENE, c=2.0, Du=0.0)
    rng = np.random.default_rng(5)
    x = rng.uniform(0.1, 1.5, (6, 9)) * rng.choice([-1.0, 1.0], (6, 9))
    ut, _ = oracle_mod.run(x, np.zeros_like(x), g, 400, reaction=oracle_mod.CENN,
                           boundary=oracle_mod.ZEROFLUX)
    np.testing.assert_allclose(ut, 2.0 * np.sign(x), rtol=0, atol=1e-12)


def test_cenn_numpy_formulation_agrees(oracle_mod):
    """The C loops (|x+1| - |x-1| form) against the numpy clamp form, both boundaries."""
    x = 2.0 * inp.uniform_field(31, 9, 12)
    w = 0.4 * inp.uniform_field(32, 9, 12)
    g = dict(CENN_GENE, c=1.7, Du=0.4)
    for b in (oracle_mod.PERIODIC, oracle_mod.ZEROFLUX):
        a = oracle_mod.run(x, w, g, 25, reaction=oracle_mod.CENN, boundary=b)
        n = oracle_mod.run_numpy(x, w, g, 25, reaction=oracle_mod.CENN, boundary=b)
        np.testing.assert_allclose(a[0], n[0], rtol=0, atol=1e-12)
        assert np.array_equal(a[1], w)


# ---------------------------------------------------------------------------
# Reduced-precision storage (16-bit planes, FP32 arithmetic, rounding after
# every k-step block).
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("storage,cases", [
    ("bf16", [(1.0, 1.0), (1 + 2**-8, 1.0), (1 + 3 * 2**-8, 1 + 2**-6), (1 + 2**-8 + 2**-20, 1 + 2**-7),
              (-(1 + 2**-8 + 2**-20), -(1 + 2**-7)), (3.0, 3.0), (0.1, 0.10009765625), (2.0**-130, 2.0**-130)]),
    ("f16", [(1.0, 1.0), (1 + 2**-11, 1.0), (1 + 3 * 2**-11, 1 + 2**-9), (65504.0, 65504.0),
             (2.0**-24, 2.0**-24), (0.1, 0.0999755859375), (-0.1, -0.0999755859375)]),
])
def test_round_to_storage_known_values(oracle_mod, storage, cases):
    """Nearest representable value, ties to the even significand (values worked by hand)."""
    got = oracle_mod.round_to_storage(np.array([c[0] for c in cases], dtype=np.float32), storage)
    np.testing.assert_array_equal(got, np.array([c[1] for c in cases], dtype=np.float32))


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_round_to_storage_matches_torch_conversion(oracle_mod, storage):
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(11).uniform(-5, 5, 20000).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16 if storage == "bf16" else torch.float16).float().numpy()
    np.testing.assert_array_equal(oracle_mod.round_to_storage(x, storage), ref)


@pytest.mark.parametrize("reaction,boundary", [("FHN", "PERIODIC"), ("NONE", "ZEROFLUX"), ("CENN", "ZEROFLUX")])
def test_step_f32_is_one_rounded_step(oracle_mod, reaction, boundary):
    """The FP32 step stays within a few single-precision rounding units of the FP64 step."""
    rx, bc = getattr(oracle_mod, reaction), getattr(oracle_mod, boundary)
    gene = CENN_GENE if reaction == "CENN" else ODD_GENE
    x = (1.5 * inp.uniform_field(80, 13, 21)).astype(np.float32).astype(np.float64)
    y = (0.4 * inp.uniform_field(81, 13, 21)).astype(np.float32).astype(np.float64)
    u32, v32 = oracle_mod.step_f32(x, y, gene, rx, bc)
    u64, v64 = oracle_mod.step(x, y, gene, rx, boundary=bc)
    assert u32.dtype == np.float32
    scale = max(np.abs(u64).max(), np.abs(v64).max())
    assert np.abs(u32 - u64).max() <= 1e-6 * scale and np.abs(v32 - v64).max() <= 1e-6 * scale


def test_run_storage_f32_follows_fp64(oracle_mod):
    x = inp.uniform_field(82, 32, 40)
    u, v = oracle_mod.run_storage(x, x, inp.default_params(), 60, 7, "f32")
    ru, rv = oracle_mod.run(x.astype(np.float32).astype(np.float64), x.astype(np.float32).astype(np.float64),
                            inp.default_params(), 60)
    assert np.linalg.norm(u - ru) / np.linalg.norm(ru) < 1e-5
    assert np.linalg.norm(v - rv) / np.linalg.norm(rv) < 1e-5


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_run_storage_returns_representable_values(oracle_mod, storage):
    x = inp.uniform_field(83, 24, 24)
    u, v = oracle_mod.run_storage(x, 0.5 * x, inp.default_params(), 30, 4, storage)
    assert np.array_equal(oracle_mod.round_to_storage(u, storage), u)
    assert np.array_equal(oracle_mod.round_to_storage(v, storage), v)


def test_bf16_storage_freezes_sub_half_ulp_increments(oracle_mod):
    """Pure diffusion of one bump of one bf16 unit (2^-7) on a field of ones, dt Du = 0.006:
    rounded every step (k = 1) the bump keeps its value (its loss, 0.024 units, is below half a
    unit) and every neighbour's gain (0.006 units) rounds away, so the state never changes;
    rounded once after 50 steps, the FP32 increments accumulate and the bump decays."""
    u = np.ones((9, 9))
    u[4, 4] = 1 + 2**-7
    par = inp.default_params()
    uk1, _ = oracle_mod.run_storage(u, u, par, 50, 1, "bf16", reaction=oracle_mod.NONE)
    assert np.array_equal(uk1, u.astype(np.float32))
    uk50, _ = oracle_mod.run_storage(u, u, par, 50, 50, "bf16", reaction=oracle_mod.NONE)
    assert uk50[4, 4] == 1.0 and not np.array_equal(uk50, u.astype(np.float32))


def test_fewer_roundings_mean_smaller_storage_error(oracle_mod):
    x = inp.uniform_field(84, 48, 48)
    ref, _ = oracle_mod.run(x.astype(np.float32).astype(np.float64), x.astype(np.float32).astype(np.float64),
                            inp.default_params(), 96)
    err = {}
    for k in (1, 8, 96):
        u, _ = oracle_mod.run_storage(x, x, inp.default_params(), 96, k, "bf16")
        err[k] = np.linalg.norm(u - ref) / np.linalg.norm(ref)
    assert err[96] < err[8] < err[1]
