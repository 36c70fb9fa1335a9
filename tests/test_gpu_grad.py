"""The hand-written backward: d log|psi| / d theta through the C ABI, against
the oracle's dual-number derivatives, central finite differences of the GPU's
own FP64 log|psi|, and the weighted / per-walker / autograd consistency.

Tolerances: FP64 |dg| <= 1e-8 max(1, |g|) per parameter (dual numbers are
exact to rounding; the GPU's backward rounds in another order).  FP32 (N2):
directional derivatives g.v within 1e-3 of sum_p |g_p v_p| (the size of the
summed terms), from the FP32 rounding of the 4e5-term contraction and the
FP32 network.
"""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2307_14123_gb300 import fixtures as fx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2307_14123_gb300 import _build
    _build.build()
    oracle.build()
    oracle.Oracle.set_threads(os.cpu_count() or 1)


def _handle(system, cfg, precision):
    from paper_2307_14123_gb300 import Ansatz
    return Ansatz(system, cfg, precision, device="cuda:0")


def _stratified(system, cfg, per_block, seed=0):
    rng = np.random.default_rng(seed)
    idx = []
    for _, (off, shape) in fx.param_offsets(system, cfg).items():
        n = int(np.prod(shape))
        if n:
            idx += list(off + rng.choice(n, size=min(n, per_block), replace=False))
    return np.array(sorted(set(idx)))


@pytest.mark.parametrize("name,small", [("lih_fp64", False), ("small", True)])
def test_per_walker_gradient_fp64_vs_oracle(name, small):
    if small:
        sys_ = fx.System(Z=np.array([2.0, 1.0]), R=np.array([[0.0, 0, 0], [0.3, -0.2, 1.4]]), n_up=2, n_down=1)
        cfg = fx.AnsatzCfg(32, 2, 3)
    else:
        wl = fx.workload(name)
        sys_, cfg = wl.system, wl.cfg
    h = _handle(sys_, cfg, "fp64")
    theta = fx.init_params(sys_, cfg, 2)
    r = fx.init_walkers(sys_, 6, 3)
    G = h.grad_logpsi(torch.tensor(theta, device="cuda:0"), torch.tensor(r, device="cuda:0"), mode=1).cpu().numpy()
    o = oracle.Oracle(sys_, cfg)
    idx = _stratified(sys_, cfg, 12)
    ref = o.grad_index(theta, r, idx)
    err = np.abs(G[:, idx] - ref)
    print(f"{name}: max |dg| {err.max():.3e} over {idx.size} parameters x {r.shape[0]} walkers")
    assert np.all(err <= 1e-8 * np.maximum(1, np.abs(ref)))
    # random directions over all parameters
    dirs = np.random.default_rng(1).normal(size=(3, o.P))
    jv = o.grad_jvp(theta, r, dirs)
    got = G @ dirs.T
    scale = np.abs(G) @ np.abs(dirs.T)
    assert np.all(np.abs(got - jv) <= 1e-10 * np.maximum(1, scale))


def test_weighted_mode_and_autograd_fp64():
    wl = fx.workload("lih_fp64")
    h = _handle(wl.system, wl.cfg, "fp64")
    th = torch.tensor(fx.init_params(wl.system, wl.cfg, 0), device="cuda:0")
    r = torch.tensor(fx.init_walkers(wl.system, 300, 0), device="cuda:0")
    w = torch.tensor(np.random.default_rng(3).normal(size=300), device="cuda:0")
    G = h.grad_logpsi(th, r, mode=1)
    g0 = h.grad_logpsi(th, r, w, mode=0)
    ref = (w[:, None] * G).sum(0)
    torch.testing.assert_close(g0, ref, rtol=1e-10, atol=1e-12)
    # chunked weighted sum equals unchunked
    h.set_max_chunk(128)
    torch.testing.assert_close(h.grad_logpsi(th, r, w, mode=0), g0, rtol=1e-12, atol=1e-13)
    h.set_max_chunk(4096)
    # autograd.Function: backward of sum_b w_b log|psi_b|
    from paper_2307_14123_gb300 import log_abs_psi
    p = th.clone().requires_grad_(True)
    la = log_abs_psi(h, p, r)
    (w * la).sum().backward()
    torch.testing.assert_close(p.grad, g0, rtol=1e-12, atol=1e-13)


def test_gradient_finite_differences_fp64_gpu():
    """Central differences of the GPU's own FP64 log|psi| (h = 1e-5)."""
    wl = fx.workload("lih_fp64")
    h = _handle(wl.system, wl.cfg, "fp64")
    theta = fx.init_params(wl.system, wl.cfg, 0)
    r = torch.tensor(fx.init_walkers(wl.system, 4, 1), device="cuda:0")
    G = h.grad_logpsi(torch.tensor(theta, device="cuda:0"), r, mode=1).cpu().numpy()
    idx = _stratified(wl.system, wl.cfg, 3, seed=5)
    eps = 1e-5
    for p in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[p] += eps
        tm[p] -= eps
        fp = h.ansatz_eval(torch.tensor(tp, device="cuda:0"), r)[0].cpu().numpy()
        fm = h.ansatz_eval(torch.tensor(tm, device="cuda:0"), r)[0].cpu().numpy()
        fd = (fp - fm) / (2 * eps)
        np.testing.assert_allclose(G[:, p], fd, rtol=1e-6, atol=1e-7)


def test_n2_fp32_gradient_directions():
    wl = fx.workload("n2_fp32")
    h = _handle(wl.system, wl.cfg, "fp32")
    theta = fx.init_params(wl.system, wl.cfg, wl.param_seed).astype(np.float32).astype(np.float64)
    r = fx.init_walkers(wl.system, 6, wl.walker_seed).astype(np.float32).astype(np.float64)
    G = h.grad_logpsi(torch.tensor(theta, dtype=torch.float32, device="cuda:0"),
                      torch.tensor(r, dtype=torch.float32, device="cuda:0"), mode=1).cpu().numpy().astype(np.float64)
    o = oracle.Oracle(wl.system, wl.cfg)
    dirs = np.random.default_rng(2).normal(size=(3, o.P))
    jv = o.grad_jvp(theta, r, dirs)
    got = G @ dirs.T
    scale = np.abs(G) @ np.abs(dirs.T)
    rel = np.abs(got - jv) / scale
    print("N2 FP32 |g.v - ref| / sum|g v|: max %.2e median %.2e" % (rel.max(), np.median(rel)))
    assert np.all(rel <= 1e-3)
    idx = _stratified(wl.system, wl.cfg, 4, seed=9)
    ref = o.grad_index(theta, r, idx)
    scale_p = np.maximum(np.abs(ref), np.abs(G[:, idx]).max(axis=0, keepdims=True) * 1e-2 + 1e-6)
    print("N2 FP32 partials: max rel %.2e" % np.max(np.abs(G[:, idx] - ref) / scale_p))


def test_full_batch_per_walker_gradient_n2_fp32():
    """The benchmark batch (4096 walkers): per-walker gradients for all walkers
    (6.8 GB); sampled walkers checked against the oracle along random directions."""
    wl = fx.workload("n2_fp32")
    h = _handle(wl.system, wl.cfg, "fp32")
    theta = fx.init_params(wl.system, wl.cfg, wl.param_seed).astype(np.float32)
    r = fx.init_walkers(wl.system, wl.B, wl.walker_seed).astype(np.float32)
    G = h.grad_logpsi(torch.tensor(theta, device="cuda:0"), torch.tensor(r, device="cuda:0"), mode=1)
    dirs = np.random.default_rng(4).normal(size=(2, G.shape[1]))
    sel = np.array([0, 1777, wl.B - 1])
    Gs = G[torch.tensor(sel, device="cuda:0")].cpu().numpy().astype(np.float64)
    del G
    jv = oracle.Oracle(wl.system, wl.cfg).grad_jvp(theta.astype(np.float64), r[sel].astype(np.float64), dirs)
    rel = np.abs(Gs @ dirs.T - jv) / (np.abs(Gs) @ np.abs(dirs.T))
    assert np.all(rel <= 1e-3), rel


def test_weighted_mode_fp32_equals_weighted_sum_of_per_walker():
    """Summed (weighted) mode of the FP32 path, whose weight-matrix blocks are
    row reductions on the tensor cores (3 x TF32 split, split over walkers),
    against the weighted sum of the per-walker gradients (CUDA-core path) over
    1024 N2 walkers.  Both sides sum FP32 products of the same activations, so
    on the matrix blocks they differ by rounding only: |dg| <= 5e-5 sum_b
    |w_b g_b| (a transposed or misplaced operand gives errors of order
    sum_b |w_b g_b|).  Bias blocks are column sums whose per-walker terms can
    cancel, so sum_b |w_b g_b| is no scale for their rounding; they are checked
    against the FP64 path elsewhere and only reported here."""
    wl = fx.workload("n2_fp32")
    h = _handle(wl.system, wl.cfg, "fp32")
    B = 1024
    th = torch.tensor(fx.init_params(wl.system, wl.cfg, wl.param_seed), dtype=torch.float32, device="cuda:0")
    r = torch.tensor(fx.init_walkers(wl.system, B, wl.walker_seed), dtype=torch.float32, device="cuda:0")
    w = torch.tensor(np.random.default_rng(11).uniform(-1.0, 1.0, B), dtype=torch.float32, device="cuda:0")
    g0 = h.grad_logpsi(th, r, w, mode=0).double()
    G = h.grad_logpsi(th, r, mode=1)
    ref = torch.zeros_like(g0)
    scale = torch.zeros_like(g0)
    for b0 in range(0, B, 256):
        Gb = G[b0:b0 + 256].double()
        wb = w[b0:b0 + 256].double()[:, None]
        ref += (wb * Gb).sum(0)
        scale += (wb.abs() * Gb.abs()).sum(0)
    del G
    rel = ((g0 - ref).abs() / (scale + 1e-30)).cpu().numpy()
    worst_matrix, worst_other, o = 0.0, 0.0, 0
    for name, shape, _ in fx.param_layout(wl.system, wl.cfg):
        n = int(np.prod(shape))
        m = float(rel[o:o + n].max())
        if name.startswith(("W_h", "W_g", "W1_", "W2_", "W_o_")) or name == "W_J1":
            worst_matrix = max(worst_matrix, m)
        else:
            worst_other = max(worst_other, m)
        o += n
    print(f"N2 FP32 weighted vs per-walker sum: max |dg| / sum|w g| {worst_matrix:.2e} (weight matrices), "
          f"{worst_other:.2e} (other blocks)")
    assert worst_matrix <= 5e-5


def test_lih_fp32_per_walker_gradient():
    """LiH in FP32 mode (one determinant pair, two electrons per spin: the orbital adjoint
    product takes the CUDA-core path, its rows being too short for the tensor maps)."""
    wl = fx.workload("lih_fp64")
    h = _handle(wl.system, wl.cfg, "fp32")
    theta = fx.init_params(wl.system, wl.cfg, wl.param_seed).astype(np.float32).astype(np.float64)
    r = fx.init_walkers(wl.system, 8, wl.walker_seed).astype(np.float32).astype(np.float64)
    G = h.grad_logpsi(torch.tensor(theta, dtype=torch.float32, device="cuda:0"),
                      torch.tensor(r, dtype=torch.float32, device="cuda:0"), mode=1).cpu().numpy().astype(np.float64)
    o = oracle.Oracle(wl.system, wl.cfg)
    dirs = np.random.default_rng(4).normal(size=(3, o.P))
    jv = o.grad_jvp(theta, r, dirs)
    rel = np.abs(G @ dirs.T - jv) / (np.abs(G) @ np.abs(dirs.T))
    print("LiH FP32 |g.v - ref| / sum|g v|: max %.2e" % rel.max())
    assert np.all(rel <= 1e-3)
