"""Initial electron embeddings from the electron-nucleus difference vectors
(Eq. 13, second case): f_i^0 = W_e2 tanh(W_e1 x_i + b_e1) + b_e2 with
x_i = (r_i - R_1, ..., r_i - R_M), through the C ABI against the oracle.  Layer
0 then runs the general path (node map, messages of non-constant embeddings,
residual update), in every precision mode.

Tolerances as for the base ansatz: FP64 1e-10 relative per walker (log|psi|,
E_loc), signs equal; FP32 the contract of tests/fp32_contract.py (log|psi| 1e-5
relative, E_loc within max(1e-4, 1e-5 S), S = (|lap| + |grad|^2) / 2, exceptions only
at listed near-nodal walkers); BF16 (embedding GEMMs with
8-bit mantissas) E_loc within max(1e-2, 2e-2 S); gradients 1e-8 relative per
parameter (FP64) and directional derivatives within 1e-3 of sum |g v| (FP32).
"""
import dataclasses
import os

import numpy as np
import pytest
import torch

import oracle
from fp32_contract import check_fp32_oracle
from paper_2307_14123_gb300 import fixtures as fx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2307_14123_gb300 import _build
    _build.build()
    oracle.build()
    oracle.Oracle.set_threads(os.cpu_count() or 1)


def _case(name, **kw):
    if name == "small":
        sys_ = fx.System(Z=np.array([2.0, 1.0]), R=np.array([[0.0, 0, 0], [0.3, -0.2, 1.4]]), n_up=2, n_down=1)
        cfg, seed = fx.AnsatzCfg(32, 2, 2), 2
    else:
        wl = fx.workload({"lih": "lih_fp64", "n2": "n2_fp32"}[name])
        sys_, cfg, seed = wl.system, wl.cfg, wl.param_seed
    return sys_, dataclasses.replace(cfg, el_init=1, **kw), seed


def _handle(system, cfg, precision):
    from paper_2307_14123_gb300 import Ansatz
    return Ansatz(system, cfg, precision, device="cuda:0")


def _inputs(sys_, cfg, precision, B, pseed, wseed):
    theta = fx.init_params(sys_, cfg, pseed)
    r = fx.init_walkers(sys_, B, wseed)
    dt = torch.float64 if precision == "fp64" else torch.float32
    if precision != "fp64":
        theta = theta.astype(np.float32).astype(np.float64)
        r = r.astype(np.float32).astype(np.float64)
    return theta, r, torch.tensor(theta, dtype=dt, device="cuda:0"), torch.tensor(r, dtype=dt, device="cuda:0")


def _np(*ts):
    return [t.detach().cpu().numpy().astype(np.float64) if t.dtype != torch.int8 else t.cpu().numpy() for t in ts]


def test_parameter_count_matches_layout():
    sys_, cfg, _ = _case("n2")
    h = _handle(sys_, cfg, "fp32")
    D, M = cfg.width, 2
    assert h.P == fx.param_count(sys_, cfg)
    assert h.P - fx.param_count(sys_, dataclasses.replace(cfg, el_init=0)) == D * 3 * M + D + D * D + D - 2 * D


@pytest.mark.parametrize("name,B,kw", [("small", 40, {}), ("lih", 64, {}), ("n2", 12, {}),
                                       ("lih", 48, {"full_det": 1, "edge_update": 1})])
def test_el_init_fp64_vs_oracle(name, B, kw):
    sys_, cfg, seed = _case(name, **kw)
    h = _handle(sys_, cfg, "fp64")
    theta, r, th_t, r_t = _inputs(sys_, cfg, "fp64", B, seed, 7)
    la, sg, el = _np(*h.local_energy(th_t, r_t))
    ref = oracle.Oracle(sys_, cfg).local_energy(theta, r)
    assert np.array_equal(sg, ref["sign"])
    e1, e2 = np.abs(la - ref["logabs"]), np.abs(el - ref["e_loc"])
    print(f"{name} el init {kw} FP64: max |dlogabs| {e1.max():.2e}, max |dE| {e2.max():.2e}")
    assert np.all(e1 <= 1e-10 * np.maximum(1, np.abs(ref["logabs"])))
    assert np.all(e2 <= 1e-10 * np.maximum(1, np.abs(ref["e_loc"])))
    la2, sg2 = _np(*h.ansatz_eval(th_t, r_t))
    assert np.array_equal(sg2, ref["sign"])
    assert np.all(np.abs(la2 - ref["logabs"]) <= 1e-10 * np.maximum(1, np.abs(ref["logabs"])))


@pytest.mark.parametrize("name,B,prec", [("lih", 64, "fp32"), ("n2", 24, "fp32"), ("n2", 24, "bf16")])
def test_el_init_fp32_bf16_vs_oracle(name, B, prec):
    sys_, cfg, seed = _case(name)
    h = _handle(sys_, cfg, prec)
    theta, r, th_t, r_t = _inputs(sys_, cfg, "fp32", B, seed, 8)
    la, sg, el = _np(*h.local_energy(th_t, r_t))
    ref = oracle.Oracle(sys_, cfg).local_energy(theta, r, with_grad=True)
    S = 0.5 * (np.abs(ref["lap"]) + np.sum(ref["grad"] ** 2, axis=1))
    e_la, e_el = np.abs(la - ref["logabs"]), np.abs(el - ref["e_loc"])
    print(f"{name} el init {prec}: max |dlogabs| {e_la.max():.2e}, |dE|/S max {np.max(e_el / S):.2e}")
    if prec == "fp32":
        check_fp32_oracle(f"{name} el init FP32", la, sg, el, oracle.Oracle(sys_, cfg), theta, r, ref=ref)
    else:
        ok = sg == ref["sign"]
        assert ok.mean() >= 0.95
        assert np.all(e_el[ok] <= np.maximum(1e-2, 2e-2 * S[ok]))


@pytest.mark.parametrize("name,kw", [("small", {}), ("lih", {}), ("lih", {"full_det": 1, "edge_update": 1})])
def test_el_init_gradient_fp64(name, kw):
    sys_, cfg, seed = _case(name, **kw)
    h = _handle(sys_, cfg, "fp64")
    theta = fx.init_params(sys_, cfg, seed)
    r = fx.init_walkers(sys_, 6, 3)
    G = h.grad_logpsi(torch.tensor(theta, device="cuda:0"), torch.tensor(r, device="cuda:0"), mode=1).cpu().numpy()
    o = oracle.Oracle(sys_, cfg)
    off = fx.param_offsets(sys_, cfg)
    rng = np.random.default_rng(0)
    idx = set()
    for nm, (o_, sh) in off.items():
        n = int(np.prod(sh))
        if nm in ("W_e1", "b_e1", "b_e2") or nm.startswith("W_h0"):
            idx |= set(range(o_, o_ + n))  # every entry of the embedding MLP's small blocks and W_h^0
        elif n:
            idx |= {o_ + int(k) for k in rng.choice(n, size=min(n, 6), replace=False)}
    idx = np.array(sorted(idx))
    ref = o.grad_index(theta, r, idx)
    err = np.abs(G[:, idx] - ref)
    print(f"{name} el init {kw}: max |dg| {err.max():.3e} over {idx.size} parameters")
    assert np.all(err <= 1e-8 * np.maximum(1, np.abs(ref)))
    dirs = np.random.default_rng(1).normal(size=(3, o.P))
    assert np.all(np.abs(G @ dirs.T - o.grad_jvp(theta, r, dirs)) <= 1e-10 * np.maximum(1, np.abs(G) @ np.abs(dirs.T)))


def test_el_init_gradient_n2_fp32_directions():
    sys_, cfg, seed = _case("n2")
    h = _handle(sys_, cfg, "fp32")
    theta, r, th_t, r_t = _inputs(sys_, cfg, "fp32", 6, seed, 4)
    G = h.grad_logpsi(th_t, r_t, mode=1).cpu().numpy().astype(np.float64)
    o = oracle.Oracle(sys_, cfg)
    dirs = np.random.default_rng(2).normal(size=(3, o.P))
    rel = np.abs(G @ dirs.T - o.grad_jvp(theta, r, dirs)) / (np.abs(G) @ np.abs(dirs.T))
    print("N2 el init FP32 |g.v - ref| / sum|g v|: max %.2e" % rel.max())
    assert np.all(rel <= 1e-3)


def test_el_init_metropolis_and_langevin_consistent():
    """Samplers on this ansatz: the log|psi| carried by a Metropolis and a Langevin step equals the
    oracle's at the final positions."""
    sys_, cfg, seed = _case("lih")
    h = _handle(sys_, cfg, "fp64")
    theta, r, th_t, r_t = _inputs(sys_, cfg, "fp64", 96, seed, 9)
    la_t, _ = h.ansatz_eval(th_t, r_t)
    h.mcmc_step(th_t, r_t, la_t, 3, 0.2, 11, 0)
    ref, _ = oracle.Oracle(sys_, cfg).evaluate(theta, r_t.cpu().numpy())
    assert np.all(np.abs(la_t.cpu().numpy() - ref) <= 1e-10 * np.maximum(1, np.abs(ref)))
    g = torch.empty_like(r_t)
    h.mala_step(th_t, r_t, la_t, g, n_steps=2, tau=0.05, seed=5, step_counter=0, grad_valid=False)
    ref, _ = oracle.Oracle(sys_, cfg).evaluate(theta, r_t.cpu().numpy())
    assert np.all(np.abs(la_t.cpu().numpy() - ref) <= 1e-10 * np.maximum(1, np.abs(ref)))


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_el_init_in_a_batch_equals_single(prec):
    """A batch mixing an electron-nucleus-embedding molecule with a spin-embedding one (layer 0
    on the general path for the first only, in the same grouped launches) gives each molecule's
    single-handle results bit for bit; the FP32 results match the oracle."""
    from paper_2307_14123_gb300 import Ansatz, AnsatzBatch
    small = _case("small")
    lih = _case("lih")
    mols = [lih, (small[0], dataclasses.replace(small[1], el_init=0), small[2]),
            (small[0], small[1], small[2])]
    if prec == "bf16":  # the BF16 GEMMs need D % 64 == 0
        mols = [(m[0], dataclasses.replace(m[1], width=64), m[2]) for m in mols]
    batch = AnsatzBatch([m[0] for m in mols], [m[1] for m in mols], prec, device="cuda:0")
    th, r, ths, rs = [], [], [], []
    for k, (sys_, cfg, seed) in enumerate(mols):
        a, b, c, d = _inputs(sys_, cfg, "fp32", 24 + 8 * k, seed, 5 + k)
        th.append(c), r.append(d), ths.append(a), rs.append(b)
    la, sg, el = batch.local_energy(th, r)
    for k, (sys_, cfg, _) in enumerate(mols):
        la1, sg1, el1 = Ansatz(sys_, cfg, prec, device="cuda:0").local_energy(th[k], r[k])
        assert torch.equal(la[k], la1) and torch.equal(sg[k], sg1) and torch.equal(el[k], el1)
        if prec != "fp32":
            continue
        lan, sgn, eln = _np(la[k], sg[k], el[k])
        check_fp32_oracle(f"batch molecule {k}", lan, sgn, eln, oracle.Oracle(sys_, cfg), ths[k], rs[k])
