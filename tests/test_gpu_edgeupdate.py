"""Iterated edge embeddings (Eq. 16, second case): before the filters of layer
l >= 1, f^l = f^{l-1} + tanh(U^{l,t} f^{l-1} + c^{l,t}) per edge type, through
the C ABI against the oracle; also combined with the full determinant (the
PauliNet2-style ansatz) and in a batch of molecules.

Tolerances as for the base ansatz: FP64 1e-10 relative per walker (log|psi|,
E_loc), signs equal; FP32 the contract of tests/fp32_contract.py (log|psi| 1e-5
relative, E_loc within max(1e-4, 1e-5 S), S = (|lap| + |grad|^2) / 2, exceptions only
at listed near-nodal walkers); gradients 1e-8 relative per
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
        cfg, seed = fx.AnsatzCfg(32, 3, 2), 2
    else:
        wl = fx.workload({"lih": "lih_fp64", "n2": "n2_fp32"}[name])
        sys_, cfg, seed = wl.system, wl.cfg, wl.param_seed
    return sys_, dataclasses.replace(cfg, edge_update=1, **kw), seed


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


def _check_fp64(la, sg, el, ref, label):
    assert np.array_equal(sg, ref["sign"])
    e1 = np.abs(la - ref["logabs"])
    assert np.all(e1 <= 1e-10 * np.maximum(1, np.abs(ref["logabs"])))
    if el is not None:
        e2 = np.abs(el - ref["e_loc"])
        print(f"{label}: max |dlogabs| {e1.max():.2e}, max |dE| {e2.max():.2e}")
        assert np.all(e2 <= 1e-10 * np.maximum(1, np.abs(ref["e_loc"])))


def test_parameter_count_matches_layout():
    sys_, cfg, _ = _case("n2")
    h = _handle(sys_, cfg, "fp32")
    Q, L = cfg.n_rbf, cfg.n_layers
    assert h.P == fx.param_count(sys_, cfg)
    assert h.P - fx.param_count(sys_, dataclasses.replace(cfg, edge_update=0)) == (L - 1) * 3 * (Q * Q + Q)


@pytest.mark.parametrize("name,B,full", [("small", 40, 0), ("lih", 64, 0), ("n2", 12, 0), ("lih", 48, 1)])
def test_edge_update_fp64_vs_oracle(name, B, full):
    sys_, cfg, seed = _case(name, full_det=full)
    h = _handle(sys_, cfg, "fp64")
    theta, r, th_t, r_t = _inputs(sys_, cfg, "fp64", B, seed, 7)
    la, sg, el = _np(*h.local_energy(th_t, r_t))
    ref = oracle.Oracle(sys_, cfg).local_energy(theta, r)
    _check_fp64(la, sg, el, ref, f"{name} edge update{' + full det' if full else ''} FP64")
    la2, sg2 = _np(*h.ansatz_eval(th_t, r_t))
    _check_fp64(la2, sg2, None, ref, "")


@pytest.mark.parametrize("name,B", [("lih", 64), ("n2", 24)])
def test_edge_update_fp32_vs_oracle(name, B):
    sys_, cfg, seed = _case(name)
    h = _handle(sys_, cfg, "fp32")
    theta, r, th_t, r_t = _inputs(sys_, cfg, "fp32", B, seed, 8)
    la, sg, el = _np(*h.local_energy(th_t, r_t))
    check_fp32_oracle(f"{name} edge update FP32", la, sg, el, oracle.Oracle(sys_, cfg), theta, r)


@pytest.mark.parametrize("name,full", [("small", 0), ("lih", 0), ("lih", 1)])
def test_edge_update_gradient_fp64(name, full):
    sys_, cfg, seed = _case(name, full_det=full)
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
        if nm.startswith(("U_", "c_")):
            idx |= set(range(o_, o_ + n))  # every entry of the edge-embedding maps
        elif n:
            idx |= {o_ + int(k) for k in rng.choice(n, size=min(n, 6), replace=False)}
    idx = np.array(sorted(idx))
    ref = o.grad_index(theta, r, idx)
    err = np.abs(G[:, idx] - ref)
    print(f"{name} edge update: max |dg| {err.max():.3e} over {idx.size} parameters")
    assert np.all(err <= 1e-8 * np.maximum(1, np.abs(ref)))
    w = np.random.default_rng(3).normal(size=r.shape[0])
    g0 = h.grad_logpsi(torch.tensor(theta, device="cuda:0"), torch.tensor(r, device="cuda:0"),
                       torch.tensor(w, device="cuda:0"), mode=0).cpu().numpy()
    np.testing.assert_allclose(g0, w @ G, rtol=1e-9, atol=1e-11)


def test_edge_update_gradient_n2_fp32_directions():
    sys_, cfg, seed = _case("n2")
    h = _handle(sys_, cfg, "fp32")
    theta, r, th_t, r_t = _inputs(sys_, cfg, "fp32", 6, seed, 4)
    G = h.grad_logpsi(th_t, r_t, mode=1).cpu().numpy().astype(np.float64)
    o = oracle.Oracle(sys_, cfg)
    dirs = np.random.default_rng(2).normal(size=(3, o.P))
    rel = np.abs(G @ dirs.T - o.grad_jvp(theta, r, dirs)) / (np.abs(G) @ np.abs(dirs.T))
    print("N2 edge update FP32 |g.v - ref| / sum|g v|: max %.2e" % rel.max())
    assert np.all(rel <= 1e-3)


def test_edge_update_in_a_batch_equals_single():
    """Two molecules with iterated edge embeddings in one grouped call (FP32; batches share the
    layer count) give the single-molecule results bit for bit, and those match the oracle."""
    from paper_2307_14123_gb300 import Ansatz, AnsatzBatch
    small = _case("small")
    mols = [_case("lih"), (small[0], dataclasses.replace(small[1], n_layers=2), small[2])]
    batch = AnsatzBatch([m[0] for m in mols], [m[1] for m in mols], "fp32", device="cuda:0")
    th, r, ths, rs = [], [], [], []
    for k, (sys_, cfg, seed) in enumerate(mols):
        a, b, c, d = _inputs(sys_, cfg, "fp32", 24 + 8 * k, seed, 5 + k)
        th.append(c), r.append(d), ths.append(a), rs.append(b)
    la, sg, el = batch.local_energy(th, r)
    for k, (sys_, cfg, _) in enumerate(mols):
        la1, sg1, el1 = Ansatz(sys_, cfg, "fp32", device="cuda:0").local_energy(th[k], r[k])
        assert torch.equal(la[k], la1) and torch.equal(sg[k], sg1) and torch.equal(el[k], el1)
        lan, sgn, eln = _np(la[k], sg[k], el[k])
        check_fp32_oracle(f"batch molecule {k}", lan, sgn, eln, oracle.Oracle(sys_, cfg), ths[k], rs[k])
