"""The full-determinant ansatz (Eq. 22): one N x N determinant per p whose rows
come from the orbital network and envelopes of each electron's spin, through
the C ABI against the oracle.

Tolerances as for the factorised ansatz: FP64 1e-10 relative per walker for
log|psi| and E_loc, signs equal; FP32 the contract of tests/fp32_contract.py
(log|psi| within 1e-5 relative, E_loc within max(1e-4, 1e-5 S) with S = (|lap| +
|grad|^2) / 2 the size of the kinetic terms that cancel, exceptions only at listed
near-nodal walkers); gradients
1e-8 relative per parameter in FP64, directional derivatives within 1e-3 of
sum |g v| in FP32.
"""
import dataclasses
import os

import numpy as np
import pytest
import torch

import oracle
from fp32_contract import check_fp32_oracle, near_nodal
from paper_2307_14123_gb300 import fixtures as fx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2307_14123_gb300 import _build
    _build.build()
    oracle.build()
    oracle.Oracle.set_threads(os.cpu_count() or 1)


def _case(name):
    if name == "small":
        sys_ = fx.System(Z=np.array([2.0, 1.0]), R=np.array([[0.0, 0, 0], [0.3, -0.2, 1.4]]), n_up=2, n_down=1)
        cfg = fx.AnsatzCfg(32, 2, 3)
        seed = 2
    else:
        wl = fx.workload({"lih": "lih_fp64", "n2": "n2_fp32"}[name])
        sys_, cfg, seed = wl.system, wl.cfg, wl.param_seed
    return sys_, dataclasses.replace(cfg, full_det=1), seed


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
    assert h.P == fx.param_count(sys_, cfg)
    N, K, D, M = 14, cfg.n_det, cfg.width, 2
    assert h.P - fx.param_count(sys_, dataclasses.replace(cfg, full_det=0)) == 2 * K * 7 * (D + 1 + 2 * M)


@pytest.mark.parametrize("name,B", [("small", 40), ("lih", 64), ("n2", 12)])
def test_full_det_fp64_vs_oracle(name, B):
    sys_, cfg, seed = _case(name)
    h = _handle(sys_, cfg, "fp64")
    theta, r, th_t, r_t = _inputs(sys_, cfg, "fp64", B, seed, 7)
    la, sg, el = _np(*h.local_energy(th_t, r_t))
    ref = oracle.Oracle(sys_, cfg).local_energy(theta, r)
    assert np.array_equal(sg, ref["sign"])
    e1, e2 = np.abs(la - ref["logabs"]), np.abs(el - ref["e_loc"])
    print(f"{name} full det FP64: max |dlogabs| {e1.max():.2e}, max |dE| {e2.max():.2e}")
    assert np.all(e1 <= 1e-10 * np.maximum(1, np.abs(ref["logabs"])))
    assert np.all(e2 <= 1e-10 * np.maximum(1, np.abs(ref["e_loc"])))
    la2, sg2 = _np(*h.ansatz_eval(th_t, r_t))  # value-only path (the Metropolis proposal)
    assert np.array_equal(sg2, ref["sign"])
    assert np.all(np.abs(la2 - ref["logabs"]) <= 1e-10 * np.maximum(1, np.abs(ref["logabs"])))


@pytest.mark.parametrize("name,B", [("lih", 64), ("n2", 24)])
def test_full_det_fp32_vs_oracle(name, B):
    sys_, cfg, seed = _case(name)
    h = _handle(sys_, cfg, "fp32")
    theta, r, th_t, r_t = _inputs(sys_, cfg, "fp32", B, seed, 8)
    la, sg, el = _np(*h.local_energy(th_t, r_t))
    o = oracle.Oracle(sys_, cfg)
    ref = o.local_energy(theta, r, with_grad=True)
    check_fp32_oracle(f"{name} full det FP32", la, sg, el, o, theta, r, ref=ref)
    la2, sg2 = _np(*h.ansatz_eval(th_t, r_t))  # value-only path: the log|psi| bounds of the contract
    nodal = near_nodal(o, theta, r, ref["logabs"])
    tol = 1e-5 * np.maximum(1, np.abs(ref["logabs"])) * np.where(nodal, 10, 1)
    assert np.array_equal(sg2[~nodal], ref["sign"][~nodal])
    assert np.all(np.abs(la2 - ref["logabs"]) <= tol)


@pytest.mark.parametrize("name", ["small", "lih"])
def test_full_det_gradient_fp64(name):
    sys_, cfg, seed = _case(name)
    h = _handle(sys_, cfg, "fp64")
    theta = fx.init_params(sys_, cfg, seed)
    r = fx.init_walkers(sys_, 6, 3)
    G = h.grad_logpsi(torch.tensor(theta, device="cuda:0"), torch.tensor(r, device="cuda:0"), mode=1).cpu().numpy()
    o = oracle.Oracle(sys_, cfg)
    off = fx.param_offsets(sys_, cfg)
    rng = np.random.default_rng(0)
    idx = sorted({o_ + int(rng.integers(int(np.prod(sh)))) for _, (o_, sh) in off.items() if int(np.prod(sh))
                  for _ in range(8)})
    # every orbital-network and envelope entry of both spins
    for nm in ("b_o_up", "b_o_dn", "omega_up", "omega_dn", "zeta_up", "zeta_dn"):
        o_, sh = off[nm]
        idx += list(range(o_, o_ + int(np.prod(sh))))
    idx = np.array(sorted(set(idx)))
    ref = o.grad_index(theta, r, idx)
    err = np.abs(G[:, idx] - ref)
    print(f"{name} full det: max |dg| {err.max():.3e} over {idx.size} parameters")
    assert np.all(err <= 1e-8 * np.maximum(1, np.abs(ref)))
    dirs = np.random.default_rng(1).normal(size=(3, o.P))
    jv = o.grad_jvp(theta, r, dirs)
    assert np.all(np.abs(G @ dirs.T - jv) <= 1e-10 * np.maximum(1, np.abs(G) @ np.abs(dirs.T)))


def test_full_det_gradient_n2_fp32_directions():
    sys_, cfg, seed = _case("n2")
    h = _handle(sys_, cfg, "fp32")
    theta, r, th_t, r_t = _inputs(sys_, cfg, "fp32", 6, seed, 4)
    G = h.grad_logpsi(th_t, r_t, mode=1).cpu().numpy().astype(np.float64)
    o = oracle.Oracle(sys_, cfg)
    dirs = np.random.default_rng(2).normal(size=(3, o.P))
    rel = np.abs(G @ dirs.T - o.grad_jvp(theta, r, dirs)) / (np.abs(G) @ np.abs(dirs.T))
    print("N2 full det FP32 |g.v - ref| / sum|g v|: max %.2e" % rel.max())
    assert np.all(rel <= 1e-3)


def test_full_det_metropolis_consistent():
    """Metropolis steps on the full-determinant ansatz: the carried log|psi| equals the oracle's
    at the final positions, and some moves are accepted."""
    sys_, cfg, seed = _case("lih")
    h = _handle(sys_, cfg, "fp64")
    theta, r, th_t, r_t = _inputs(sys_, cfg, "fp64", 128, seed, 9)
    la_t, _ = h.ansatz_eval(th_t, r_t)
    r0 = r_t.clone()
    n_acc = h.mcmc_step(th_t, r_t, la_t, 5, 0.2, 11, 0)
    rr = r_t.cpu().numpy()
    ref_la, _ = oracle.Oracle(sys_, cfg).evaluate(theta, rr)
    assert np.all(np.abs(la_t.cpu().numpy() - ref_la) <= 1e-10 * np.maximum(1, np.abs(ref_la)))
    moved = (r_t != r0).any(dim=2).any(dim=1).float().mean().item()
    assert 0.05 < moved <= 1.0
    assert int(n_acc) > 0
