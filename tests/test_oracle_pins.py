"""Pins of the FP64 oracle against what the paper and mathematics fix.

Nothing here compares the oracle with itself: every expected value is a
closed form (hydrogenic energies, Kato-cusp two-electron wave functions
differentiated symbolically with sympy), a brute-force computation
(Leibniz determinants), a finite difference, an exact invariance of the
ansatz (antisymmetry Eq. 3, equivariance Eq. 9, rigid motions), a sampling
statement with its batch-means error bar (Eq. 35), a published known-answer
vector, or a hand-computable special case of the network with one-hot
weights (which pins every layout and index convention).
"""
import dataclasses
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from paper_2307_14123_gb300 import fixtures as fx

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def setp(theta, system, cfg, name, value):
    o, shape = fx.param_offsets(system, cfg)[name]
    theta[o:o + int(np.prod(shape))] = np.broadcast_to(np.asarray(value, dtype=np.float64), shape).reshape(-1)


def pidx(system, cfg, name, flat=0):
    return fx.param_offsets(system, cfg)[name][0] + flat


def rand_rotation(rng, reflect=False):
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    if reflect:
        q = q @ np.diag([1.0, 1.0, -1.0])
    return q


def small_system():
    return fx.System(Z=np.array([2.0, 1.0]), R=np.array([[0.0, 0.0, 0.0], [0.3, -0.2, 1.4]]), n_up=2, n_down=1)


# ----------------------------------------------------------------------------
# Inputs: Philox, Box-Muller, parameter count
# ----------------------------------------------------------------------------
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    for row in rows:
        v = [int(x, 16) for x in row]
        out = fx.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_box_muller_moments():
    z = fx.walker_normals(7, np.arange(2000), 3, fx.TAG_PROPOSE, 64).ravel()
    n = z.size
    assert abs(z.mean()) < 5 / math.sqrt(n)
    assert abs(z.var() - 1) < 5 * math.sqrt(2 / n)
    assert abs(np.mean(z ** 4) - 3) < 5 * math.sqrt(96 / n)


@pytest.mark.parametrize("name,P", [("lih_fp64", 19285), ("n2_fp32", 412656), ("c4h4_bf16", 2210720)])
def test_param_count(name, P):
    wl = fx.workload(name)
    assert fx.param_count(wl.system, wl.cfg) == P
    assert oracle.Oracle(wl.system, wl.cfg).P == P


# ----------------------------------------------------------------------------
# Closed-form wave functions (network switched off)
# ----------------------------------------------------------------------------
def test_hydrogen_network_off_exact():
    """psi = exp(-r): E_loc = -1/2 at every r (Sec. 2.2: hydrogenic atoms are solvable)."""
    H = fx.molecule("H")
    cfg = fx.AnsatzCfg(8, 2, 1, use_cusp=0)
    o = oracle.Oracle(H, cfg)
    th = fx.network_off_params(H, cfg, 1.0)
    r = fx.init_walkers(H, 64, 11, sigma=2.0)
    out = o.local_energy(th, r)
    rr = np.linalg.norm(r[:, 0], axis=1)
    np.testing.assert_allclose(out["logabs"], -rr, rtol=0, atol=1e-13)
    assert np.all(np.abs(out["e_loc"] + 0.5) <= 1e-12 * np.maximum(1, 1 / rr))
    assert np.all(out["sign"] == 1)


@pytest.mark.parametrize("Z", [2.0, 3.0])
def test_hydrogenic_ion(Z):
    sys_ = fx.System(Z=np.array([Z]), R=np.array([[0.1, -0.3, 0.2]]), n_up=1, n_down=0)
    cfg = fx.AnsatzCfg(8, 1, 1, use_cusp=0)
    o = oracle.Oracle(sys_, cfg)
    th = fx.network_off_params(sys_, cfg, Z)
    r = fx.init_walkers(sys_, 32, 5)
    e = o.local_energy(th, r)["e_loc"]
    np.testing.assert_allclose(e, -Z * Z / 2, rtol=0, atol=1e-11)


def test_two_electron_product_no_cusp():
    """psi = exp(-Z r1 - Z r2): E_loc = -Z^2 + 1/r12 (V_ee and the spin split)."""
    Z = 2.0
    sys_ = fx.System(Z=np.array([Z]), R=np.zeros((1, 3)), n_up=1, n_down=1)
    cfg = fx.AnsatzCfg(8, 2, 1, use_cusp=0)
    o = oracle.Oracle(sys_, cfg)
    th = fx.network_off_params(sys_, cfg, Z)
    r = fx.init_walkers(sys_, 32, 9)
    e = o.local_energy(th, r)["e_loc"]
    r12 = np.linalg.norm(r[:, 0] - r[:, 1], axis=1)
    np.testing.assert_allclose(e, -Z * Z + 1 / r12, rtol=1e-12, atol=1e-11)


def _sympy_eloc(psi_fn, n_elec, Zs, Rs):
    """E_loc = -1/2 (Lap psi)/psi + V from a closed-form psi, by sympy."""
    sp = pytest.importorskip("sympy")
    xs = sp.symbols(" ".join(f"x{i}_{k}" for i in range(n_elec) for k in range(3)), real=True)
    pos = [sp.Matrix(xs[3 * i:3 * i + 3]) for i in range(n_elec)]
    psi = psi_fn(sp, pos)
    lap = sum(sp.diff(psi, x, 2) for x in xs)
    V = 0
    for i in range(n_elec):
        for j in range(i + 1, n_elec):
            V += 1 / (pos[i] - pos[j]).norm()
        for Z, R in zip(Zs, Rs):
            V -= Z / (pos[i] - sp.Matrix(R)).norm()
    eloc = -sp.Rational(1, 2) * lap / psi + V
    return sp.lambdify(xs, eloc, "math"), sp.lambdify(xs, sp.log(sp.Abs(psi)), "math"), sp.lambdify(xs, psi, "math")


def test_opposite_spin_cusp_closed_form():
    """exp(-Z r1 - Z r2) times the electron cusp of Eq. (25) with c = 1/2, alpha = 1."""
    Z = 2.0
    sys_ = fx.System(Z=np.array([Z]), R=np.zeros((1, 3)), n_up=1, n_down=1)
    cfg = fx.AnsatzCfg(8, 2, 1, use_cusp=1, cusp_alpha=1.0)
    o = oracle.Oracle(sys_, cfg)
    th = fx.network_off_params(sys_, cfg, Z)

    def psi(sp, p):
        r1, r2, r12 = p[0].norm(), p[1].norm(), (p[0] - p[1]).norm()
        return sp.exp(-Z * r1 - Z * r2) * sp.exp(-sp.Rational(1, 2) / (1 + r12))

    f_e, f_l, _ = _sympy_eloc(psi, 2, [Z], [[0, 0, 0]])
    r = fx.init_walkers(sys_, 12, 21)
    out = o.local_energy(th, r)
    for b in range(r.shape[0]):
        args = r[b].ravel()
        assert out["e_loc"][b] == pytest.approx(f_e(*args), rel=1e-10, abs=1e-10)
        assert out["logabs"][b] == pytest.approx(f_l(*args), rel=1e-12, abs=1e-12)


def test_same_spin_pair_determinant_and_cusp():
    """Two same-spin electrons, orbitals exp(-a r), exp(-b r):
    psi = (e^{-a r1 - b r2} - e^{-b r1 - a r2}) exp(-1/4 / (1 + r12))."""
    a, b = 1.7, 0.6
    sys_ = fx.System(Z=np.array([2.0]), R=np.zeros((1, 3)), n_up=2, n_down=0)
    cfg = fx.AnsatzCfg(8, 2, 1, use_cusp=1, cusp_alpha=1.0)
    o = oracle.Oracle(sys_, cfg)
    th = fx.network_off_params(sys_, cfg, 1.0)
    setp(th, sys_, cfg, "zeta_up", [[a], [b]])

    def psi(sp, p):
        r1, r2, r12 = p[0].norm(), p[1].norm(), (p[0] - p[1]).norm()
        return (sp.exp(-a * r1 - b * r2) - sp.exp(-b * r1 - a * r2)) * sp.exp(-sp.Rational(1, 4) / (1 + r12))

    f_e, f_l, f_p = _sympy_eloc(psi, 2, [2.0], [[0, 0, 0]])
    r = fx.init_walkers(sys_, 12, 4)
    out = o.local_energy(th, r)
    for k in range(r.shape[0]):
        args = r[k].ravel()
        assert out["e_loc"][k] == pytest.approx(f_e(*args), rel=1e-9, abs=1e-9)
        assert out["logabs"][k] == pytest.approx(f_l(*args), rel=1e-12, abs=1e-12)
        assert out["sign"][k] == np.sign(f_p(*args))


# ----------------------------------------------------------------------------
# Determinants against the Leibniz formula; envelope layout
# ----------------------------------------------------------------------------
def _leibniz(A):
    n = A.shape[0]
    tot = 0.0
    for perm in itertools.permutations(range(n)):
        inv = sum(1 for i in range(n) for j in range(i + 1, n) if perm[i] > perm[j])
        tot += (-1) ** inv * np.prod([A[i, perm[i]] for i in range(n)])
    return tot


@pytest.mark.parametrize("n_up", [1, 3, 4])
def test_multi_determinant_leibniz(n_up):
    """psi = sum_p c_p det A^p with A^p_ik = sum_I omega exp(-zeta d_iI) (Eqs. 20-21), brute force."""
    rng = np.random.default_rng(n_up)
    sys_ = fx.System(Z=np.array([3.0, 1.0]), R=np.array([[0, 0, 0], [0.2, 0.5, 1.9]]), n_up=n_up, n_down=0)
    K = 3
    cfg = fx.AnsatzCfg(8, 1, K, use_cusp=0)
    o = oracle.Oracle(sys_, cfg)
    th = fx.network_off_params(sys_, cfg, 1.0)
    om = rng.normal(size=(K * n_up, 2))
    ze = rng.uniform(0.5, 2.0, size=(K * n_up, 2))
    c = np.array([1.0, -0.7, 0.4])
    setp(th, sys_, cfg, "omega_up", om)
    setp(th, sys_, cfg, "zeta_up", ze)
    setp(th, sys_, cfg, "c", c)
    r = fx.init_walkers(sys_, 16, 8)
    la, sg = o.evaluate(th, r)
    for b in range(r.shape[0]):
        d = np.linalg.norm(r[b][:, None, :] - sys_.R[None], axis=-1)  # [i][I]
        psi = 0.0
        for p in range(K):
            A = np.array([[sum(om[p * n_up + k, I] * math.exp(-ze[p * n_up + k, I] * d[i, I]) for I in range(2))
                           for k in range(n_up)] for i in range(n_up)])
            if b == 0:
                _, Ao = o.intermediates(th, r[b:b + 1])
                np.testing.assert_allclose(Ao[0, p, :n_up, :n_up], A, rtol=1e-13)
            psi += c[p] * _leibniz(A)
        assert la[b] == pytest.approx(math.log(abs(psi)), rel=1e-12, abs=1e-12)
        assert sg[b] == np.sign(psi)


def mirrored_pair_walkers(B, seed):
    """Two same-spin electrons mirrored through the nucleus at the origin:
    (r1, r2) -> (R r1, R r2) with R the reflection x -> -x swaps them, so a
    distance-only ansatz gives psi = -psi = 0 exactly (Eq. 3)."""
    r = fx.init_walkers(fx.System(Z=np.array([2.0]), R=np.zeros((1, 3)), n_up=2, n_down=0), B, seed)
    r[:, 1] = r[:, 0] * np.array([-1.0, 1.0, 1.0])
    return r


def test_singular_determinant():
    """psi = 0 exactly: sign 0, log|psi| = -inf, E_loc NaN (full random-weight network)."""
    sys_ = fx.System(Z=np.array([2.0]), R=np.zeros((1, 3)), n_up=2, n_down=0)
    cfg = fx.AnsatzCfg(8, 2, 2)
    o = oracle.Oracle(sys_, cfg)
    th = fx.init_params(sys_, cfg, 1)
    out = o.local_energy(th, mirrored_pair_walkers(4, 1))
    assert np.all(out["sign"] == 0) and np.all(np.isneginf(out["logabs"])) and np.all(np.isnan(out["e_loc"]))


# ----------------------------------------------------------------------------
# Coulomb terms
# ----------------------------------------------------------------------------
def test_potential_hand_placed():
    sys_ = fx.System(Z=np.array([1.0, 1.0]), R=np.array([[0, 0, 0], [0, 0, 2.0]]), n_up=1, n_down=1)
    o = oracle.Oracle(sys_, fx.AnsatzCfg(8, 1, 1))
    r = np.array([[[1.0, 0, 0], [-1.0, 0, 0]]])
    expect = 1 / 2.0 - 2 * (1.0 + 1 / math.sqrt(5.0)) + 1 / 2.0
    assert o.potential(r)[0] == pytest.approx(expect, rel=1e-15)


@pytest.mark.parametrize("name,vnn", [("N2", 49 / 2.068), ("LiH", 3 / 3.015)])
def test_nuclear_repulsion(name, vnn):
    sys_ = fx.molecule(name)
    o = oracle.Oracle(sys_, fx.AnsatzCfg(8, 1, 1))
    N = sys_.n_elec
    far = 1e16 * (np.arange(N)[:, None] + 1) * np.array([[1.0, 2.0, 3.0]])
    assert o.potential(far[None])[0] == pytest.approx(vnn, rel=1e-12)


# ----------------------------------------------------------------------------
# Symmetries of the full random-weight ansatz
# ----------------------------------------------------------------------------
def _random_case(name):
    if name.startswith("small"):
        sys_, cfg = small_system(), fx.AnsatzCfg(8, 2, 2)
    else:
        wl = fx.workload("lih_fp64")
        sys_, cfg = wl.system, wl.cfg
    if name.endswith("_full"):
        cfg = dataclasses.replace(cfg, full_det=1)
    if name.endswith("_eu"):
        cfg = dataclasses.replace(cfg, edge_update=1)
    if name.endswith("_ei"):
        cfg = dataclasses.replace(cfg, el_init=1)
    th = fx.init_params(sys_, cfg, 3)
    r = fx.init_walkers(sys_, 6, 3)
    return sys_, cfg, th, r


@pytest.mark.parametrize("name", ["small", "lih", "small_full", "lih_full", "small_eu", "small_ei", "lih_ei"])
def test_antisymmetry(name):
    """Exchange of two same-spin electrons flips the sign only (Eqs. 3, 9)."""
    sys_, cfg, th, r = _random_case(name)
    o = oracle.Oracle(sys_, cfg)
    a = o.local_energy(th, r)
    rs = r.copy()
    rs[:, [0, 1]] = rs[:, [1, 0]]
    b = o.local_energy(th, rs)
    np.testing.assert_allclose(b["logabs"], a["logabs"], rtol=1e-12, atol=1e-12)
    assert np.all(b["sign"] == -a["sign"])
    np.testing.assert_allclose(b["e_loc"], a["e_loc"], rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("name", ["small", "small_full", "small_ei"])
def test_opposite_spin_exchange_is_not_a_symmetry(name):
    """Spins are fixed (Sec. 2.2): exchanging an up and a down electron changes psi; the full
    determinant (Eq. 22) is not antisymmetric under it either (Sec. 3.3)."""
    sys_, cfg, th, r = _random_case(name)
    o = oracle.Oracle(sys_, cfg)
    la, _ = o.evaluate(th, r)
    rs = r.copy()
    rs[:, [0, 2]] = rs[:, [2, 0]]
    lb, _ = o.evaluate(th, rs)
    assert np.all(np.abs(la - lb) > 1e-6)


@pytest.mark.parametrize("reflect", [False, True])
@pytest.mark.parametrize("name", ["small", "small_full", "small_eu"])
def test_rigid_motion_invariance(reflect, name):
    sys_, cfg, th, r = _random_case(name)
    o = oracle.Oracle(sys_, cfg)
    a = o.local_energy(th, r)
    rng = np.random.default_rng(5)
    Q, t = rand_rotation(rng, reflect), rng.normal(size=3)
    sys2 = fx.System(Z=sys_.Z, R=sys_.R @ Q.T + t, n_up=sys_.n_up, n_down=sys_.n_down)
    b = oracle.Oracle(sys2, cfg).local_energy(th, r @ Q.T + t)
    np.testing.assert_allclose(b["logabs"], a["logabs"], rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(b["e_loc"], a["e_loc"], rtol=1e-9, atol=1e-9)
    assert np.all(a["sign"] == b["sign"])


def test_orbital_equivariance():
    """Permuting same-spin electrons permutes rows of A and of the embeddings (Eq. 9)."""
    sys_ = fx.molecule("N2")
    cfg = fx.AnsatzCfg(16, 2, 2)
    o = oracle.Oracle(sys_, cfg)
    th = fx.init_params(sys_, cfg, 1)
    r = fx.init_walkers(sys_, 1, 1)
    perm_up = np.array([3, 0, 6, 1, 5, 2, 4])
    perm_dn = np.array([2, 4, 0, 6, 1, 3, 5])
    order = np.concatenate([perm_up, 7 + perm_dn])
    f, A = o.intermediates(th, r)
    f2, A2 = o.intermediates(th, r[:, order])
    np.testing.assert_allclose(f2, f[order], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(A2[0], A[0][:, perm_up], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(A2[1], A[1][:, perm_dn], rtol=1e-12, atol=1e-14)


def _embed_factorised(sys_, cfg, th):
    """Full-determinant parameters whose N x N matrices are block diagonal, diag(A^up, A^down):
    orbital k < n_up of spin up and orbital k >= n_up of spin down copy the factorised orbitals,
    the others are zero (W_o and b_o rows 0, so phi = 0)."""
    cfg_f = dataclasses.replace(cfg, full_det=1)
    off, off_f = fx.param_offsets(sys_, cfg), fx.param_offsets(sys_, cfg_f)
    th_f = np.zeros(fx.param_count(sys_, cfg_f))
    for nm in ("omega_up", "zeta_up", "omega_dn", "zeta_dn"):
        setp(th_f, sys_, cfg_f, nm, 1.0)
    for name, (o, shape) in off.items():
        if name in off_f and off_f[name][1] == shape:
            th_f[off_f[name][0]:off_f[name][0] + int(np.prod(shape))] = th[o:o + int(np.prod(shape))]
    N, K, nu = sys_.n_elec, cfg.n_det, sys_.n_up
    for sname, ns, k0 in (("up", nu, 0), ("dn", sys_.n_down, nu)):
        for blk in ("W_o", "b_o", "omega", "zeta"):
            o, shape = off[f"{blk}_{sname}"]
            src = th[o:o + int(np.prod(shape))].reshape(shape[0], -1)
            of, shape_f = off_f[f"{blk}_{sname}"]
            dst = th_f[of:of + int(np.prod(shape_f))].reshape(shape_f[0], -1)
            for p in range(K):
                dst[p * N + k0:p * N + k0 + ns] = src[p * ns:(p + 1) * ns]
    return cfg_f, th_f


@pytest.mark.parametrize("name", ["small", "lih"])
def test_full_determinant_block_diagonal_reduces_to_factorised(name):
    """With block-diagonal matrices the generalised Laplace expansion (Eq. 23) keeps one term, so
    the full determinant (Eq. 22) equals det A^up det A^down (Eq. 21): log|psi|, sign and E_loc
    agree with the factorised ansatz."""
    sys_, cfg, th, r = _random_case(name)
    cfg_f, th_f = _embed_factorised(sys_, cfg, th)
    a = oracle.Oracle(sys_, cfg).local_energy(th, r)
    b = oracle.Oracle(sys_, cfg_f).local_energy(th_f, r)
    np.testing.assert_allclose(b["logabs"], a["logabs"], rtol=1e-12, atol=1e-12)
    assert np.array_equal(b["sign"], a["sign"])
    np.testing.assert_allclose(b["e_loc"], a["e_loc"], rtol=1e-10, atol=1e-10)
    _, A = oracle.Oracle(sys_, cfg_f).intermediates(th_f, r[:1])
    assert A.shape == (1, cfg.n_det, sys_.n_elec, sys_.n_elec)
    nu = sys_.n_up
    assert np.all(A[0, :, :nu, nu:] == 0) and np.all(A[0, :, nu:, :nu] == 0)


def test_full_determinant_laplace_expansion():
    """Eq. (23) by brute force on the oracle's own full matrices: det A^p = sum over n_up-subsets S of
    the orbitals of eps_S det A^{up,S} det A^{down,S-bar} (Leibniz determinants); with the Jastrow
    factor and cusp off, log|psi| = log|sum_p c_p det A^p|.  Each matrix row is the orbital network
    of that electron's spin, checked against the embeddings."""
    sys_ = fx.System(Z=np.array([3.0, 1.0]), R=np.array([[0, 0, 0], [0.2, 0.5, 1.9]]), n_up=3, n_down=2)
    cfg = fx.AnsatzCfg(8, 2, 3, use_jastrow=0, use_cusp=0, full_det=1)
    o = oracle.Oracle(sys_, cfg)
    th = fx.init_params(sys_, cfg, 4)
    setp(th, sys_, cfg, "c", [1.0, -0.6, 0.3])
    r = fx.init_walkers(sys_, 4, 2)
    la, sg = o.evaluate(th, r)
    N, K, nu = 5, 3, 3
    off = fx.param_offsets(sys_, cfg)
    get = lambda nm: th[off[nm][0]:off[nm][0] + int(np.prod(off[nm][1]))].reshape(off[nm][1])
    for b in range(r.shape[0]):
        f, A = o.intermediates(th, r[b:b + 1])
        d = np.linalg.norm(r[b][:, None, :] - sys_.R[None], axis=-1)
        psi = 0.0
        for p in range(K):
            for i in range(N):
                s = "up" if i < nu else "dn"
                phi = get(f"W_o_{s}") @ f[i] + get(f"b_o_{s}")
                env = (get(f"omega_{s}") * np.exp(-get(f"zeta_{s}") * d[i][None, :])).sum(axis=1)
                np.testing.assert_allclose(A[0, p, i], (phi * env)[p * N:(p + 1) * N], rtol=1e-12, atol=1e-14)
            Ap = A[0, p]
            lap = 0.0
            for S in itertools.combinations(range(N), nu):
                Sb = [k for k in range(N) if k not in S]
                perm = list(S) + Sb
                eps = (-1) ** sum(1 for i in range(N) for j in range(i + 1, N) if perm[i] > perm[j])
                lap += eps * _leibniz(Ap[:nu][:, list(S)]) * _leibniz(Ap[nu:][:, Sb])
            assert lap == pytest.approx(_leibniz(Ap), rel=1e-12, abs=1e-300)
            psi += get("c")[p] * lap
        assert la[b] == pytest.approx(math.log(abs(psi)), rel=1e-12, abs=1e-12)
        assert sg[b] == np.sign(psi)


# ----------------------------------------------------------------------------
# Derivatives against finite differences
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["small", "lih", "small_full", "lih_full", "small_eu", "lih_eu", "small_ei",
                                  "lih_ei"])
def test_coordinate_derivatives_finite_differences(name):
    sys_, cfg, th, r = _random_case(name)
    o = oracle.Oracle(sys_, cfg)
    r = r[:3]
    out = o.local_energy(th, r, with_grad=True)
    N3 = 3 * sys_.n_elec
    for b in range(r.shape[0]):
        # steps scaled to the walker's smallest e-e / e-n distance and to its distance from the
        # nodal surface, about 1 / |grad log|psi|| (the stencil's truncation error grows like
        # (h / distance)^4 near a coalescence or a node)
        pts = np.concatenate([r[b], sys_.R])
        dd = np.linalg.norm(pts[:, None] - pts[None], axis=-1)[:sys_.n_elec]
        d_min = min(np.min(dd[dd > 0]), 1.0 / np.max(np.abs(out["grad"][b])))
        h1, h2 = 1e-5, min(2e-3, 0.02 * d_min)
        lap_fd = 0.0
        for x in range(N3):
            def f(dx):
                rr = r[b].ravel().copy()
                rr[x] += dx
                return o.evaluate(th, rr[None])[0][0]
            f0 = f(0.0)
            g = (f(h1) - f(-h1)) / (2 * h1)
            d2 = (-f(2 * h2) + 16 * f(h2) - 30 * f0 + 16 * f(-h2) - f(-2 * h2)) / (12 * h2 * h2)
            assert out["grad"][b, x] == pytest.approx(g, rel=1e-6, abs=1e-6)
            lap_fd += d2
        assert out["lap"][b] == pytest.approx(lap_fd, rel=1e-5, abs=1e-5)
        V = o.potential(r[b:b + 1])[0]
        e_fd = -0.5 * (lap_fd + np.sum(out["grad"][b] ** 2)) + V
        # E_loc inherits the Laplacian's finite-difference error, which near a node (large |lap|,
        # cancelled by |grad|^2) is far above 1e-5 |E_loc|.
        tol = 0.5 * 1e-5 * max(1.0, abs(lap_fd)) + 1e-5 * max(1.0, abs(e_fd))
        assert abs(out["e_loc"][b] - e_fd) <= tol, (out["e_loc"][b], e_fd, tol)


@pytest.mark.parametrize("edge_update,el_init", [(0, 0), (1, 0), (0, 1)])
def test_parameter_gradient_finite_differences(edge_update, el_init):
    """d log|psi| / d theta by dual numbers vs central differences (h = 1e-4... 1e-5, FP64)."""
    wl = fx.workload("lih_fp64")
    sys_, cfg = wl.system, dataclasses.replace(wl.cfg, edge_update=edge_update, el_init=el_init)
    o = oracle.Oracle(sys_, cfg)
    th = fx.init_params(sys_, cfg, 0)
    r = fx.init_walkers(sys_, 2, 0)
    rng = np.random.default_rng(0)
    idx = []
    for name, (off, shape) in fx.param_offsets(sys_, cfg).items():
        n = int(np.prod(shape))
        idx += list(off + rng.choice(n, size=min(n, 4), replace=False))
    idx = np.array(sorted(set(idx)))
    g = o.grad_index(th, r, idx)
    h = 1e-5
    for k, p in enumerate(idx):
        tp, tm = th.copy(), th.copy()
        tp[p] += h
        tm[p] -= h
        fd = (o.evaluate(tp, r)[0] - o.evaluate(tm, r)[0]) / (2 * h)
        np.testing.assert_allclose(g[:, k], fd, rtol=1e-6, atol=1e-7)
    # directional derivatives agree with the sum of partials
    dirs = np.zeros((2, o.P))
    dirs[0, idx] = rng.normal(size=idx.size)
    dirs[1] = rng.normal(size=o.P) * 1e-2
    jv = o.grad_jvp(th, r, dirs)
    np.testing.assert_allclose(jv[:, 0], g @ dirs[0, idx], rtol=1e-10, atol=1e-12)
    fd = (o.evaluate(th + h * dirs[1], r)[0] - o.evaluate(th - h * dirs[1], r)[0]) / (2 * h)
    np.testing.assert_allclose(jv[:, 1], fd, rtol=1e-6, atol=1e-7)


def test_envelope_exponent_gradient_closed_form():
    """For psi = exp(-zeta r), d log|psi| / d zeta = -r exactly."""
    H = fx.molecule("H")
    cfg = fx.AnsatzCfg(8, 1, 1, use_cusp=0)
    o = oracle.Oracle(H, cfg)
    th = fx.network_off_params(H, cfg, 1.3)
    r = fx.init_walkers(H, 16, 2)
    g = o.grad_index(th, r, [pidx(H, cfg, "zeta_up")])[:, 0]
    np.testing.assert_allclose(g, -np.linalg.norm(r[:, 0], axis=1), rtol=1e-14)


# ----------------------------------------------------------------------------
# Network structure pinned by one-hot weights (layouts, normalisations, order)
# ----------------------------------------------------------------------------
def test_embedding_update_layout():
    """W_h = I, constant edge filters (W2 = 0, b2 = beta_t): messages are
    beta_t times the normalised sums of Eq. (17); W_g acts on [m_par; m_anti; m_nuc]."""
    sys_ = small_system()  # 2 up, 1 down, 2 nuclei
    D = 2
    cfg = fx.AnsatzCfg(D, 1, 1, use_cusp=0)
    rng = np.random.default_rng(1)
    th = fx.init_params(sys_, cfg, 4)
    setp(th, sys_, cfg, "W_h0", np.eye(D))
    beta = {"par": np.array([0.7, -1.1]), "anti": np.array([1.3, 0.4]), "nuc": np.array([-0.5, 0.9])}
    for t in beta:
        setp(th, sys_, cfg, f"W2_{t}0", 0.0)
        setp(th, sys_, cfg, f"b2_{t}0", beta[t])
    Wg = rng.normal(size=(D, 3 * D))
    bg = rng.normal(size=D)
    setp(th, sys_, cfg, "W_g0", Wg)
    setp(th, sys_, cfg, "b_g0", bg)
    E = th[pidx(sys_, cfg, "E_spin"):][:2 * D].reshape(2, D)
    Y = th[pidx(sys_, cfg, "Y0"):][:2 * D].reshape(2, D)
    o = oracle.Oracle(sys_, cfg)
    f, _ = o.intermediates(th, fx.init_walkers(sys_, 1, 0))
    spins = [0, 0, 1]
    for i in range(3):
        same = [j for j in range(3) if j != i and spins[j] == spins[i]]
        opp = [j for j in range(3) if spins[j] != spins[i]]
        m_par = beta["par"] * sum((E[spins[j]] for j in same), np.zeros(D)) / max(1, len(same))
        m_anti = beta["anti"] * sum((E[spins[j]] for j in opp), np.zeros(D)) / max(1, len(opp))
        m_nuc = beta["nuc"] * (Y[0] + Y[1]) / 2
        expect = E[spins[i]] + np.tanh(Wg @ np.concatenate([m_par, m_anti, m_nuc]) + bg)
        np.testing.assert_allclose(f[i], expect, rtol=1e-13)


def test_edge_filter_and_gaussian_features():
    """One up and one down electron; W1 one-hot on Gaussian features 3 and 5,
    W2 = I: w_anti(d) = tanh(e_{3,5}(d)), e_q(d) = exp(-(d - q rc/15)^2 / (2 (rc/15)^2))."""
    sys_ = fx.System(Z=np.array([1.0]), R=np.array([[0.0, 0.0, 0.0]]), n_up=1, n_down=1)
    D, Q, rc = 2, 16, 10.0
    cfg = fx.AnsatzCfg(D, 1, 1, n_rbf=Q, rbf_cutoff=rc, use_cusp=0)
    th = fx.init_params(sys_, cfg, 2)
    Hm = np.array([[0.3, -1.2], [0.8, 0.5]])
    G = np.array([[1.1, 0.2], [-0.4, 0.9]])
    W1 = np.zeros((D, Q))
    W1[0, 3] = 1.0
    W1[1, 5] = 1.0
    setp(th, sys_, cfg, "W_h0", Hm)
    setp(th, sys_, cfg, "W1_anti0", W1)
    setp(th, sys_, cfg, "b1_anti0", 0.0)
    setp(th, sys_, cfg, "W2_anti0", np.eye(D))
    setp(th, sys_, cfg, "b2_anti0", 0.0)
    setp(th, sys_, cfg, "W2_nuc0", 0.0)
    setp(th, sys_, cfg, "b2_nuc0", 0.0)
    Wg = np.zeros((D, 3 * D))
    Wg[:, D:2 * D] = G
    setp(th, sys_, cfg, "W_g0", Wg)
    setp(th, sys_, cfg, "b_g0", 0.0)
    E = th[pidx(sys_, cfg, "E_spin"):][:2 * D].reshape(2, D)
    r = np.array([[[0.4, -0.3, 1.0], [-1.2, 0.9, 2.1]]])
    d = np.linalg.norm(r[0, 0] - r[0, 1])
    s = rc / (Q - 1)
    e = np.exp(-(d - np.arange(Q) * s) ** 2 / (2 * s * s))
    w = np.tanh(np.array([e[3], e[5]]))
    f, _ = oracle.Oracle(sys_, cfg).intermediates(th, r)
    np.testing.assert_allclose(f[0], E[0] + np.tanh(G @ (w * (Hm @ E[1]))), rtol=1e-13)
    np.testing.assert_allclose(f[1], E[1] + np.tanh(G @ (w * (Hm @ E[0]))), rtol=1e-13)


def test_iterated_edge_embedding_closed_form():
    """Eq. (16), second case, on one up and one down electron: layer 0 switched off (W_g = 0,
    b_g = 0 keep f^1 = E_spin); in layer 1 the opposite-spin edge embedding is
    e + tanh(U e + c) and W1 one-hot on its components 3 and 5, W2 = I: the messages are
    tanh of those two components times W_h f of the other electron."""
    sys_ = fx.System(Z=np.array([1.0]), R=np.array([[0.0, 0.0, 0.0]]), n_up=1, n_down=1)
    D, Q, rc = 2, 16, 10.0
    cfg = fx.AnsatzCfg(D, 2, 1, n_rbf=Q, rbf_cutoff=rc, use_cusp=0, edge_update=1)
    th = fx.init_params(sys_, cfg, 2)
    rng = np.random.default_rng(7)
    U, c = rng.normal(size=(Q, Q)) * 0.5, rng.normal(size=Q) * 0.3
    Hm = np.array([[0.3, -1.2], [0.8, 0.5]])
    G = np.array([[1.1, 0.2], [-0.4, 0.9]])
    W1 = np.zeros((D, Q))
    W1[0, 3] = 1.0
    W1[1, 5] = 1.0
    setp(th, sys_, cfg, "W_g0", 0.0)
    setp(th, sys_, cfg, "b_g0", 0.0)
    setp(th, sys_, cfg, "U_anti1", U)
    setp(th, sys_, cfg, "c_anti1", c)
    setp(th, sys_, cfg, "W_h1", Hm)
    setp(th, sys_, cfg, "W1_anti1", W1)
    setp(th, sys_, cfg, "b1_anti1", 0.0)
    setp(th, sys_, cfg, "W2_anti1", np.eye(D))
    setp(th, sys_, cfg, "b2_anti1", 0.0)
    setp(th, sys_, cfg, "W2_nuc1", 0.0)
    setp(th, sys_, cfg, "b2_nuc1", 0.0)
    Wg = np.zeros((D, 3 * D))
    Wg[:, D:2 * D] = G
    setp(th, sys_, cfg, "W_g1", Wg)
    setp(th, sys_, cfg, "b_g1", 0.0)
    E = th[pidx(sys_, cfg, "E_spin"):][:2 * D].reshape(2, D)
    r = np.array([[[0.4, -0.3, 1.0], [-1.2, 0.9, 2.1]]])
    d = np.linalg.norm(r[0, 0] - r[0, 1])
    s = rc / (Q - 1)
    e = np.exp(-(d - np.arange(Q) * s) ** 2 / (2 * s * s))
    fe = e + np.tanh(U @ e + c)
    w = np.tanh(np.array([fe[3], fe[5]]))
    f, _ = oracle.Oracle(sys_, cfg).intermediates(th, r)
    np.testing.assert_allclose(f[0], E[0] + np.tanh(G @ (w * (Hm @ E[1]))), rtol=1e-13)
    np.testing.assert_allclose(f[1], E[1] + np.tanh(G @ (w * (Hm @ E[0]))), rtol=1e-13)


@pytest.mark.parametrize("name", ["small", "lih"])
def test_iterated_edge_embedding_zero_update_reduces(name):
    """U = 0 and c = 0 make every edge-embedding update the identity (f + tanh 0), so the
    iterated ansatz equals the one with fixed Gaussian edge features."""
    sys_, cfg, th, r = _random_case(name)
    cfg_u = dataclasses.replace(cfg, edge_update=1)
    off, off_u = fx.param_offsets(sys_, cfg), fx.param_offsets(sys_, cfg_u)
    th_u = np.zeros(fx.param_count(sys_, cfg_u))
    for nm, (o, shape) in off.items():
        th_u[off_u[nm][0]:off_u[nm][0] + int(np.prod(shape))] = th[o:o + int(np.prod(shape))]
    assert set(off_u) - set(off) == {f"{k}_{t}{l}" for k in "Uc" for t in ("par", "anti", "nuc")
                                      for l in range(1, cfg.n_layers)}
    a = oracle.Oracle(sys_, cfg).local_energy(th, r)
    b = oracle.Oracle(sys_, cfg_u).local_energy(th_u, r)
    np.testing.assert_allclose(b["logabs"], a["logabs"], rtol=1e-13, atol=1e-13)
    assert np.array_equal(b["sign"], a["sign"])
    np.testing.assert_allclose(b["e_loc"], a["e_loc"], rtol=1e-11, atol=1e-11)
    th_u[pidx(sys_, cfg_u, "U_anti1")] = 0.5  # and a non-zero update changes psi
    assert np.all(np.abs(oracle.Oracle(sys_, cfg_u).evaluate(th_u, r)[0] - a["logabs"]) > 1e-9)


def test_electron_nucleus_initial_embedding_closed_form():
    """Eq. (13), second case, with one-hot weights: W_e1 rows pick single components of the
    difference vectors r_i - R_I, W_e2 = diag(g); with one layer whose update is switched off
    (W_g = 0, b_g = 0) the final embeddings are f_i = g * tanh(x_i[k] + beta) + b_e2."""
    sys_ = small_system()  # 2 up, 1 down, nuclei at R_0, R_1
    D = 4
    cfg = fx.AnsatzCfg(D, 1, 1, use_cusp=0, el_init=1)
    th = fx.init_params(sys_, cfg, 5)
    picks = [(0, 0), (1, 2), (0, 1), (1, 0)]  # feature a <- (nucleus I, component c)
    W1 = np.zeros((D, 6))
    for a, (I, c) in enumerate(picks):
        W1[a, 3 * I + c] = 1.0
    beta, g, b2 = np.array([0.3, -0.2, 0.0, 0.5]), np.array([1.5, -0.7, 2.0, 0.4]), np.array([0.1, 0, -0.3, 0.2])
    setp(th, sys_, cfg, "W_e1", W1)
    setp(th, sys_, cfg, "b_e1", beta)
    setp(th, sys_, cfg, "W_e2", np.diag(g))
    setp(th, sys_, cfg, "b_e2", b2)
    setp(th, sys_, cfg, "W_g0", 0.0)
    setp(th, sys_, cfg, "b_g0", 0.0)
    r = fx.init_walkers(sys_, 1, 4)
    f, _ = oracle.Oracle(sys_, cfg).intermediates(th, r)
    for i in range(3):
        for a, (I, c) in enumerate(picks):
            x = r[0, i, c] - sys_.R[I, c]
            assert f[i, a] == pytest.approx(g[a] * math.tanh(x + beta[a]) + b2[a], rel=1e-14, abs=1e-15)


def test_electron_nucleus_initial_embedding_frame():
    """Difference vectors are translation invariant but turn with the molecule: a common shift of
    electrons and nuclei leaves psi unchanged, a common rotation does not (with the spin-only
    embedding it does, see the rigid-motion test)."""
    sys_, cfg, th, r = _random_case("small_ei")
    a = oracle.Oracle(sys_, cfg).local_energy(th, r)
    t = np.array([0.7, -1.3, 0.4])
    sys_t = fx.System(Z=sys_.Z, R=sys_.R + t, n_up=sys_.n_up, n_down=sys_.n_down)
    b = oracle.Oracle(sys_t, cfg).local_energy(th, r + t)
    np.testing.assert_allclose(b["logabs"], a["logabs"], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(b["e_loc"], a["e_loc"], rtol=1e-9, atol=1e-9)
    Q = rand_rotation(np.random.default_rng(8))
    sys_q = fx.System(Z=sys_.Z, R=sys_.R @ Q.T, n_up=sys_.n_up, n_down=sys_.n_down)
    lq, _ = oracle.Oracle(sys_q, cfg).evaluate(th, r @ Q.T)
    assert np.all(np.abs(lq - a["logabs"]) > 1e-8)


def test_orbital_head_and_jastrow_layout():
    """W_g = 0 keeps f^L = E_spin; then A_ik = (W_o f_i + b_o)_{p n + k} env and
    J = w_J2 . tanh(W_J1 sum_i f_i + b_J1) (Eqs. 19, 24)."""
    sys_ = small_system()
    D, K = 4, 2
    cfg = fx.AnsatzCfg(D, 2, K, use_cusp=0)
    th = fx.init_params(sys_, cfg, 6)
    for l in range(2):
        setp(th, sys_, cfg, f"W_g{l}", 0.0)
        setp(th, sys_, cfg, f"b_g{l}", 0.0)
    rng = np.random.default_rng(3)
    setp(th, sys_, cfg, "b_o_up", rng.normal(size=K * 2))
    setp(th, sys_, cfg, "b_J1", rng.normal(size=D))
    E = th[pidx(sys_, cfg, "E_spin"):][:2 * D].reshape(2, D)
    off = fx.param_offsets(sys_, cfg)

    def get(name):
        o_, shape = off[name]
        return th[o_:o_ + int(np.prod(shape))].reshape(shape)

    o = oracle.Oracle(sys_, cfg)
    r = fx.init_walkers(sys_, 1, 2)
    f, A = o.intermediates(th, r)
    np.testing.assert_allclose(f, E[[0, 0, 1]], rtol=1e-15)
    Wo, bo, om, ze = get("W_o_up"), get("b_o_up"), get("omega_up"), get("zeta_up")
    d = np.linalg.norm(r[0][:, None, :] - sys_.R[None], axis=-1)
    for p in range(K):
        for i in range(2):
            for k in range(2):
                row = p * 2 + k
                env = np.sum(om[row] * np.exp(-ze[row] * d[i]))
                assert A[0, p, i, k] == pytest.approx((Wo[row] @ E[0] + bo[row]) * env, rel=1e-13)
    J = get("w_J2")[0] @ np.tanh(get("W_J1") @ (2 * E[0] + E[1]) + get("b_J1"))
    la_on, _ = o.evaluate(th, r)
    th_off = th.copy()
    setp(th_off, sys_, cfg, "w_J2", 0.0)
    la_off, _ = o.evaluate(th_off, r)
    assert la_on[0] - la_off[0] == pytest.approx(J, rel=1e-12, abs=1e-13)


# ----------------------------------------------------------------------------
# Sampling statements (Sec. 5, Eq. 35) and the gradient estimator (Eq. 30)
# ----------------------------------------------------------------------------
def _sample_hydrogen(zeta, B, n_burn, n_keep, step, seed):
    H = fx.molecule("H")
    cfg = fx.AnsatzCfg(4, 1, 1, use_cusp=0)
    o = oracle.Oracle(H, cfg)
    th = fx.network_off_params(H, cfg, zeta)
    r = fx.init_walkers(H, B, seed)
    la, _ = o.evaluate(th, r)
    rs, acc_tot = [], 0
    for t in range(n_burn + n_keep):
        xi, u = fx.metropolis_draws(seed, B, 1, t)
        r, la, acc = o.metropolis_step(th, r, la, xi, u, step)
        if t >= n_burn:
            rs.append(r.copy())
            acc_tot += acc.sum()
    return o, th, H, cfg, np.stack(rs, axis=1), acc_tot / (B * n_keep)


def test_metropolis_zero_variance_and_mean_radius():
    """psi = exp(-r): E_loc has zero variance; <r> under |psi|^2 is 3/2 (within the Eq. 35 error bar)."""
    o, th, H, cfg, rs, acc = _sample_hydrogen(1.0, 256, 100, 300, 0.6, 12)
    e = o.local_energy(th, rs[:, -1])["e_loc"]
    assert np.all(np.abs(e + 0.5) < 1e-11)
    rad = np.linalg.norm(rs[:, :, 0], axis=-1)  # [B][steps]
    mean, err = oracle.energy_estimate(rad)
    assert 0.2 < acc < 0.95
    assert abs(mean - 1.5) < 5 * err, (mean, err)


def test_gradient_estimator_hydrogen():
    """psi = exp(-zeta r): E(zeta) = zeta^2/2 - zeta, so dE/dzeta = zeta - 1; the
    estimator 2 E[(E_loc - E) d log|psi|/d zeta] of Eq. (30) agrees within its error bar."""
    zeta = 1.3
    o, th, H, cfg, rs, _ = _sample_hydrogen(zeta, 256, 100, 200, 0.6, 13)
    B, S = rs.shape[:2]
    flat = rs.reshape(B * S, 1, 3)
    e = o.local_energy(th, flat)["e_loc"].reshape(B, S)
    g = o.grad_index(th, flat, [pidx(H, cfg, "zeta_up")])[:, 0].reshape(B, S)
    contrib = np.empty((B, S))
    for t in range(S):
        w, _, _, _ = oracle.clipped_loss_weights(e[:, t], k=1e12)
        contrib[:, t] = B * w * g[:, t]
    est, err = oracle.energy_estimate(contrib)
    assert abs(est - (zeta - 1)) < 5 * err + 1e-3, (est, err)
    mean_e, err_e = oracle.energy_estimate(e)
    assert abs(mean_e - (zeta ** 2 / 2 - zeta)) < 5 * err_e, (mean_e, err_e)


def test_clipping_rule():
    """Median / mean-absolute-deviation window (Sec. 4.4); brute force on a small batch."""
    rng = np.random.default_rng(0)
    for B in (7, 8):
        e = rng.standard_cauchy(B)
        w, c, med, hw = oracle.clipped_loss_weights(e, k=5.0)
        s = sorted(e)
        m = s[B // 2] if B % 2 else (s[B // 2 - 1] + s[B // 2]) / 2
        assert med == m
        assert hw == pytest.approx(5 * sum(abs(x - m) for x in e) / B)
        assert np.all(c >= m - hw - 1e-15) and np.all(c <= m + hw + 1e-15)
        assert np.allclose(w, 2 / B * (c - c.mean()))
        assert abs(w.sum()) < 1e-14


def test_log_clipping_properties():
    """Logarithmic soft clipping (Sec. 4.4): the identity inside the window, value and slope
    continuous at its edges (slope 1 on both sides), odd about the centre, strictly increasing,
    between the hard clamp and the raw value, and logarithmic outside: equal ratios of distance
    beyond the edge give equal steps, sigma * ln(ratio)."""
    mu, sig = -3.7, 0.8
    inside = mu + sig * np.linspace(-1, 1, 41)
    assert np.array_equal(oracle.log_clip(inside, mu, sig), inside)
    for side in (1, -1):
        edge = mu + side * sig
        for h in (1e-4, 1e-6):
            out = oracle.log_clip(np.array([edge + side * h]), mu, sig)[0]
            assert abs((out - edge) / (side * h) - 1) < 2 * h / sig
    u = np.geomspace(1e-3, 1e4, 200) * sig
    up, dn = oracle.log_clip(mu + u, mu, sig) - mu, oracle.log_clip(mu - u, mu, sig) - mu
    assert np.allclose(up, -dn, rtol=0, atol=1e-12)
    assert np.all(np.diff(up) > 0)
    assert np.all(up <= u + 1e-12) and np.all(up >= np.minimum(u, sig) - 1e-12)
    for t in (1.0, 2.5, 40.0):
        for ratio in (np.e, 10.0, 1e3):
            a, b = oracle.log_clip(np.array([mu + sig * t, mu + sig * t * ratio]), mu, sig)
            assert abs((b - a) - sig * np.log(ratio)) < 1e-12 * max(1, abs(mu) + sig * np.log(ratio))


def test_soft_clipped_weights():
    """Soft-clipped weights: same centre and half-width as the hard rule, clipped energies between
    the hard clamp and the raw values, weights summing to zero, and no clipping as k grows."""
    rng = np.random.default_rng(3)
    e = rng.standard_cauchy(33) - 5
    wh, ch, medh, hwh = oracle.clipped_loss_weights(e, k=2.0)
    ws, cs, meds, hws = oracle.clipped_loss_weights(e, k=2.0, soft=True)
    assert meds == medh and hws == hwh
    assert np.all(np.abs(ch - medh) <= np.abs(cs - meds) + 1e-12)
    assert np.all(np.abs(cs - meds) <= np.abs(e - meds) + 1e-12)
    assert np.any(np.abs(cs - meds) > hws)
    assert abs(ws.sum()) < 1e-14
    w_inf, c_inf, _, _ = oracle.clipped_loss_weights(e, k=1e9, soft=True)
    assert np.array_equal(c_inf, e)
    with pytest.raises(ValueError):
        oracle.clipped_loss_weights(e, k=0.0, soft=True)


# ----------------------------------------------------------------------------
# Langevin (MALA) sampler, Sec. 5
# ----------------------------------------------------------------------------
def _drift_limited(g, tau):
    """Per-electron drift limiting (Umrigar, Nightingale, Runge 1993, a = 1)."""
    v2 = np.sum(g * g, axis=-1, keepdims=True)
    s = tau * v2
    f = np.where(s > 0, (np.sqrt(1 + 2 * s) - 1) / np.where(s > 0, s, 1), 1.0)
    return f * g


def test_mala_hydrogen_closed_form():
    """psi = exp(-r): grad log|psi| = -r/|r|, so proposal and acceptance ratio
    follow in closed form; the oracle gets its gradient from the network
    (switched off) by hyper-dual numbers."""
    H = fx.molecule("H")
    cfg = fx.AnsatzCfg(8, 1, 1, use_cusp=0)
    o = oracle.Oracle(H, cfg)
    th = fx.network_off_params(H, cfg, 1.0)
    B, tau = 64, 0.3
    r = fx.init_walkers(H, B, 21, sigma=1.5)
    la = -np.linalg.norm(r[:, 0], axis=1)
    g = -r / np.linalg.norm(r, axis=-1, keepdims=True)
    xi, u = fx.metropolis_draws(5, B, 1, 0)
    rn, lan, gn, acc, lal = o.mala_step(th, r, la, g, xi, u, tau)
    rp = r + tau * _drift_limited(g, tau) + np.sqrt(tau) * xi
    rpn = np.linalg.norm(rp[:, 0], axis=1)
    gp = -rp / rpn[:, None, None]
    back = r - rp - tau * _drift_limited(gp, tau)
    want = 2 * (-rpn - la) + 0.5 * np.sum(xi ** 2, axis=(1, 2)) - np.sum(back ** 2, axis=(1, 2)) / (2 * tau)
    np.testing.assert_allclose(lal, want, rtol=0, atol=1e-11)
    want_acc = np.log(u) < want
    assert np.array_equal(acc.astype(bool), want_acc)
    assert 0 < want_acc.sum() < B
    np.testing.assert_allclose(rn[want_acc], rp[want_acc], rtol=0, atol=1e-14)
    np.testing.assert_allclose(rn[~want_acc], r[~want_acc], rtol=0, atol=0)
    np.testing.assert_allclose(gn[want_acc], gp[want_acc], rtol=0, atol=1e-12)
    np.testing.assert_allclose(lan[want_acc], -rpn[want_acc], rtol=0, atol=1e-13)


def test_mala_detailed_balance():
    """The acceptance ratio of the move r -> r' and of the reverse move r' -> r
    multiply to one, log alpha(r -> r') + log alpha(r' -> r) = 0, for the
    network switched on (checks the asymmetric-proposal correction)."""
    sys_, cfg = small_system(), fx.AnsatzCfg(8, 2, 2)
    o = oracle.Oracle(sys_, cfg)
    th = fx.init_params(sys_, cfg, 4)
    B, tau = 6, 0.05
    r = fx.init_walkers(sys_, B, 8)
    out = o.local_energy(th, r, with_grad=True)
    g = out["grad"].reshape(r.shape)
    xi, _ = fx.metropolis_draws(9, B, sys_.n_elec, 0)
    tiny = np.full(B, 1e-300)
    r1, la1, g1, acc1, lal1 = o.mala_step(th, r, out["logabs"], g, xi, tiny, tau)
    assert acc1.all()
    xi_back = (r - r1 - tau * _drift_limited(g1, tau)) / np.sqrt(tau)
    r2, la2, g2, acc2, lal2 = o.mala_step(th, r1, la1, g1, xi_back, tiny, tau)
    assert acc2.all()
    np.testing.assert_allclose(r2, r, rtol=0, atol=1e-12)
    np.testing.assert_allclose(lal1 + lal2, 0.0, rtol=0, atol=1e-9)
    # the gradient carried along is the oracle's own gradient at the new positions
    np.testing.assert_allclose(g1, o.local_energy(th, r1, with_grad=True)["grad"].reshape(r.shape), rtol=0,
                               atol=1e-12)


def test_mala_stationarity_hydrogen():
    """MALA samples |psi|^2: psi = exp(-r) gives <r> = 3/2 (within the Eq. 35 error
    bar) and zero-variance local energies."""
    H = fx.molecule("H")
    cfg = fx.AnsatzCfg(4, 1, 1, use_cusp=0)
    o = oracle.Oracle(H, cfg)
    th = fx.network_off_params(H, cfg, 1.0)
    B, tau = 256, 0.4
    r = fx.init_walkers(H, B, 31)
    out = o.local_energy(th, r, with_grad=True)
    la, g = out["logabs"], out["grad"].reshape(r.shape)
    rs, acc_tot = [], 0
    for t in range(400):
        xi, u = fx.metropolis_draws(31, B, 1, t)
        r, la, g, acc, _ = o.mala_step(th, r, la, g, xi, u, tau)
        if t >= 100:
            rs.append(r.copy())
            acc_tot += acc.sum()
    rad = np.linalg.norm(np.stack(rs, axis=1)[:, :, 0], axis=-1)
    mean, err = oracle.energy_estimate(rad)
    assert 0.5 < acc_tot / (B * 300) < 1.0
    assert abs(mean - 1.5) < 5 * err, (mean, err)
    assert np.all(np.abs(o.local_energy(th, r)["e_loc"] + 0.5) < 1e-11)


# ----------------------------------------------------------------------------
# Natural-gradient direction (Sec. 4, "Optimizer")
# ----------------------------------------------------------------------------
def _natgrad_inputs(B, P, seed):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((B, P)) * rng.uniform(0.1, 3.0, P) + rng.standard_normal(P)
    e = rng.standard_normal(B)
    w = (2.0 / B) * (e - e.mean())
    return G, w


def test_param_update_step_length_limit():
    """The parameter step moves along -delta by lr ||delta|| when that is within max_norm (or
    max_norm <= 0), and by exactly max_norm otherwise."""
    rng = np.random.default_rng(3)
    th, d = rng.normal(size=50), rng.normal(size=50)
    lr, nrm = 0.1, np.linalg.norm(d)
    for max_norm, length in ((0.0, lr * nrm), (-1.0, lr * nrm), (10.0, lr * nrm), (0.05, 0.05)):
        new, n_out, s = oracle.param_update(th, d, lr, max_norm)
        step = th - new
        assert n_out == pytest.approx(nrm, rel=1e-14)
        assert np.linalg.norm(step) == pytest.approx(length, rel=1e-12)
        np.testing.assert_allclose(step / np.linalg.norm(step), d / nrm, rtol=1e-12, atol=1e-14)
        assert s == pytest.approx(length / (lr * nrm), rel=1e-12)


@pytest.mark.parametrize("B,P", [(40, 13), (12, 30)])
def test_natural_gradient_push_through(B, P):
    """Sample-space (B x B) and parameter-space (P x P) forms agree."""
    G, w = _natgrad_inputs(B, P, 1)
    a = oracle.natural_gradient(G, w, 0.3, "sample")
    b = oracle.natural_gradient(G, w, 0.3, "parameter")
    np.testing.assert_allclose(a, b, rtol=1e-10, atol=1e-12)


def test_natural_gradient_limits():
    """Large damping: delta -> g / lam; centring: a constant added to every walker's
    gradient changes nothing; the sample-space result solves the damped normal
    equations (F + lam I) delta = g of parameter space."""
    G, w = _natgrad_inputs(50, 7, 2)
    g = G.T @ w
    lam = 1e9  # the deviation from g / lam is of relative order ||F|| / lam (||F|| ~ 10 here)
    np.testing.assert_allclose(oracle.natural_gradient(G, w, lam) * lam, g, rtol=1e-6, atol=1e-12)
    shift = np.random.default_rng(3).standard_normal(7) * 10
    np.testing.assert_allclose(oracle.natural_gradient(G + shift, w, 0.1), oracle.natural_gradient(G, w, 0.1),
                               rtol=1e-9, atol=1e-12)
    Gc = G - G.mean(axis=0)
    d = oracle.natural_gradient(G, w, 1e-3)
    np.testing.assert_allclose(Gc.T @ Gc / 50 @ d + 1e-3 * d, g, rtol=1e-8, atol=1e-12)


# ----------------------------------------------------------------------------
# Pseudopotential quadrature (Eqs. 11, 12)
# ----------------------------------------------------------------------------
def test_icosahedral_rule_and_legendre():
    """The 12-point rule integrates P_l(u . v) exactly for l = 1..5 (mean 0) and is exact for
    the constant; the Legendre polynomials and the Gaussian radial form as defined."""
    from scipy.special import eval_legendre
    ico = oracle.icosahedron()
    assert ico.shape == (12, 3) and np.allclose(np.linalg.norm(ico, axis=1), 1.0)
    rng = np.random.default_rng(0)
    for _ in range(5):
        v = rng.standard_normal(3)
        v /= np.linalg.norm(v)
        x = ico @ v
        for l in range(1, 6):
            assert abs(np.mean(eval_legendre(l, x))) < 1e-12
        for l in range(4):
            np.testing.assert_allclose([oracle.legendre(l, t) for t in x], eval_legendre(l, x), atol=1e-14)
    coef = [(2.0, 2, 0.7), (-1.5, 1, 1.3), (0.5, 3, 0.2)]
    rr = 0.83
    direct = 2.0 * np.exp(-0.7 * rr * rr) - 1.5 / rr * np.exp(-1.3 * rr * rr) + 0.5 * rr * np.exp(-0.2 * rr * rr)
    assert oracle.pp_radial(coef, rr) == pytest.approx(direct, rel=1e-14)


def test_pseudopotential_hydrogen_closed_form():
    """psi = exp(-r) (network off) and the pseudopotential on the nucleus: every rotated point
    keeps r, so every psi ratio is 1 and the quadrature leaves V_NL = W_0(r) exactly (the
    l >= 1 channels average P_l over the icosahedron to zero); V_loc = V(r)."""
    H = fx.molecule("H")
    cfg = fx.AnsatzCfg(32, 1, 1, use_jastrow=0, use_cusp=0)
    th = fx.network_off_params(H, cfg, 1.0)
    o = oracle.Oracle(H, cfg)
    r = np.random.default_rng(4).normal(size=(6, 1, 3)) * 1.2
    coef = np.array([[(1.0, 1, 0.5), (0.3, 2, 1.1)],    # V
                     [(2.0, 2, 0.8), (-0.4, 3, 0.3)],   # W_0
                     [(1.5, 2, 0.6), (0.2, 2, 2.0)],    # W_1
                     [(-0.7, 2, 0.4), (0.1, 4, 0.9)]])  # W_2
    rng = np.random.default_rng(5)
    rot = [np.linalg.qr(rng.standard_normal((3, 3)))[0] for _ in range(6)]
    v_loc, v_nl = oracle.pseudopotential(o, th, r, [(0, coef)], rot)
    for b in range(6):
        rr = float(np.linalg.norm(r[b, 0]))
        assert v_loc[b] == pytest.approx(oracle.pp_radial(coef[0], rr), rel=1e-13)
        assert v_nl[b] == pytest.approx(oracle.pp_radial(coef[1], rr), rel=1e-12, abs=1e-14)


def test_pseudopotential_icosahedral_symmetry():
    """A rotation that maps the icosahedron onto itself (a fivefold turn about a vertex) leaves
    the quadrature unchanged: LiH with the network on, pseudopotential on Li."""
    wl = fx.workload("lih_fp64")
    o = oracle.Oracle(wl.system, wl.cfg)
    th = fx.init_params(wl.system, wl.cfg, wl.param_seed)
    r = fx.init_walkers(wl.system, 2, wl.walker_seed)
    coef = np.array([[(0.5, 2, 0.9)], [(1.0, 2, 0.7)], [(0.6, 2, 0.5)]])
    ico = oracle.icosahedron()
    a = ico[0]
    ang = 2 * np.pi / 5
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    Rsym = np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * K @ K
    mapped = ico @ Rsym.T
    assert all(np.min(np.linalg.norm(ico - m, axis=1)) < 1e-12 for m in mapped)
    _, v1 = oracle.pseudopotential(o, th, r, [(0, coef)], [np.eye(3)] * 2)
    _, v2 = oracle.pseudopotential(o, th, r, [(0, coef)], [Rsym] * 2)
    np.testing.assert_allclose(v1, v2, rtol=1e-11, atol=1e-13)
