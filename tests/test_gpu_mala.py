"""Langevin (MALA) sampler on the GPU against the oracle's MALA step,
teacher-forced: at every step both sides start from the GPU's state
(positions, log|psi|, d log|psi| / d r) and use the same Philox draws.

Accept decisions may differ only where log u sits within the rounding band
of log alpha (1e-8 in FP64, 1e-3 in FP32); elsewhere positions, log|psi| and
the carried gradient match the oracle."""
import os

import numpy as np
import pytest
import torch

import oracle
from fp32_contract import near_nodal
from paper_2307_14123_gb300 import fixtures as fx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2307_14123_gb300 import _build
    _build.build()
    oracle.build()
    oracle.Oracle.set_threads(os.cpu_count() or 1)


def _setup(name, precision, B):
    from paper_2307_14123_gb300 import Ansatz
    wl = fx.workload(name)
    h = Ansatz(wl.system, wl.cfg, precision, device="cuda:0")
    theta = fx.init_params(wl.system, wl.cfg, wl.param_seed)
    r = fx.init_walkers(wl.system, B, wl.walker_seed)
    if precision != "fp64":
        theta = theta.astype(np.float32).astype(np.float64)
        r = r.astype(np.float32).astype(np.float64)
    dt = torch.float64 if precision == "fp64" else torch.float32
    th_t = torch.tensor(theta, dtype=dt, device="cuda:0")
    r_t = torch.tensor(r, dtype=dt, device="cuda:0")
    return wl, h, theta, r, th_t, r_t


def _np(t):
    return t.detach().cpu().numpy().astype(np.float64)


def _teacher_forced(name, precision, B, steps, tau, pos_tol, la_tol, g_tol, band):
    wl, h, theta, r, th_t, r_t = _setup(name, precision, B)
    o = oracle.Oracle(wl.system, wl.cfg)
    la_t = torch.empty(B, dtype=th_t.dtype, device="cuda:0")
    g_t = torch.empty_like(r_t)
    e_t = torch.empty_like(la_t)
    # n_steps = 0, grad_valid = False: log|psi|, d log|psi| / d r and E_loc at the starting positions only
    n = h.mala_step(th_t, r_t, la_t, g_t, n_steps=0, tau=tau, grad_valid=False, e_loc=e_t)
    assert int(n.item()) == 0 and torch.equal(r_t, torch.tensor(r, dtype=th_t.dtype, device="cuda:0"))
    ref0 = o.local_energy(theta, r, with_grad=True)
    loose0 = near_nodal(o, theta, r, ref0["logabs"]) if precision != "fp64" else np.zeros(B, bool)
    _check_state(_np(la_t), _np(g_t), ref0["logabs"], ref0["grad"].reshape(r.shape), np.ones(B, bool), la_tol, g_tol,
                 loose0)
    _check_eloc(_np(e_t), ref0, np.ones(B, bool), precision, loose0)
    flips = rejected = 0
    for t in range(steps):
        r_prev, la_prev, g_prev, e_prev = _np(r_t), _np(la_t), _np(g_t), _np(e_t)
        n = h.mala_step(th_t, r_t, la_t, g_t, n_steps=1, tau=tau, seed=wl.walker_seed, step_counter=t, e_loc=e_t)
        r_new, la_new, g_new, e_new = _np(r_t), _np(la_t), _np(g_t), _np(e_t)
        xi, u = fx.metropolis_draws(wl.walker_seed, B, wl.system.n_elec, t)
        ro, lo, go, acc, lal = o.mala_step(theta, r_prev, la_prev, g_prev, xi, u, tau)
        gpu_acc = np.any(r_new != r_prev, axis=(1, 2))
        assert int(n.item()) == int(gpu_acc.sum())
        diff = gpu_acc != acc.astype(bool)
        if diff.any():  # only where log u sits on the rounding band of log alpha
            margin = np.abs(np.log(u[diff]) - lal[diff])
            assert np.all(margin < band), margin
            flips += int(diff.sum())
        same = ~diff
        np.testing.assert_allclose(r_new[same], ro[same], rtol=0, atol=pos_tol)
        ref_new = o.local_energy(theta, r_new, with_grad=True)
        loose = near_nodal(o, theta, r_new, ref_new["logabs"]) if precision != "fp64" else np.zeros(B, bool)
        _check_state(la_new, g_new, lo, go, same & gpu_acc, la_tol, g_tol, loose)
        assert np.array_equal(la_new[~gpu_acc], la_prev[~gpu_acc]) and np.array_equal(g_new[~gpu_acc], g_prev[~gpu_acc])
        assert np.array_equal(e_new[~gpu_acc], e_prev[~gpu_acc])
        # the carried E_loc of moved walkers is the local energy at their new positions
        _check_eloc(e_new, ref_new, gpu_acc, precision, loose)
        assert gpu_acc.sum() > 0
        rejected += int(B - gpu_acc.sum())
    print(f"{name} MALA: {flips} near-threshold flips, {rejected} rejections over {steps} steps of {B} walkers")
    return rejected


def _check_eloc(e, ref, mask, precision, loose):
    """FP64: 1e-10 max(1, |E_loc|); FP32: the contract's max(1e-4 Ha, 1e-5 S_b), S_b the size of the
    kinetic terms, ten times looser at near-nodal walkers (tests/fp32_contract.py)."""
    er = ref["e_loc"][mask]
    err = np.abs(e[mask] - er)
    if precision == "fp64":
        assert np.all(err <= 1e-10 * np.maximum(1, np.abs(er))), float(err.max())
    else:
        S = 0.5 * (np.abs(ref["lap"][mask]) + np.sum(ref["grad"][mask] ** 2, axis=1))
        tol = np.maximum(1e-4, 1e-5 * S) * np.where(loose[mask], 10, 1)
        assert np.all(err <= tol), float((err / S).max())


def _check_state(la, g, la_ref, g_ref, mask, la_tol, g_tol, loose):
    """log|psi| within la_tol max(1, |log|psi||) and each walker's drift within g_tol of its largest
    component; both ten times looser at near-nodal walkers."""
    f = np.where(loose[mask], 10, 1)
    assert np.all(np.abs(la[mask] - la_ref[mask]) <= la_tol * np.maximum(1, np.abs(la_ref[mask])) * f)
    scale = np.abs(g_ref[mask]).max(axis=(1, 2), keepdims=True)
    gerr = np.abs(g[mask] - g_ref[mask]) / np.maximum(scale, 1.0)
    assert np.all(gerr <= g_tol * f[:, None, None]), float(gerr.max())


def test_mala_lih_fp64_teacher_forced():
    # FP64: positions to 1e-12 bohr, log|psi| and drift to 1e-10; flips only within 1e-8 of the threshold
    assert _teacher_forced("lih_fp64", "fp64", 128, 5, 0.05, 1e-12, 1e-10, 1e-10, 1e-8) > 0


def test_mala_n2_fp32_teacher_forced():
    # FP32 state: the position is stored in FP32 (|r| <= ~10 bohr: 1e-6 rounding) after a
    # drift step of tau * vbar with vbar computed from the FP32 drift; log|psi| to the FP32
    # contract's 1e-5 relative, the drift to the FP32 rounding floor of the jets; flips within
    # 1e-3 of the threshold
    _teacher_forced("n2_fp32", "fp32", 32, 2, 0.02, 2e-5, 1e-5, 1e-3, 1e-3)


def test_mala_multi_step_and_device_counter():
    """n steps in one call equal n single-step calls; the device counter form equals the host one."""
    wl, h, theta, r, th_t, r_t = _setup("lih_fp64", "fp64", 96)
    la = torch.empty(96, dtype=torch.float64, device="cuda:0")
    g = torch.empty_like(r_t)
    r1, la1, g1 = r_t.clone(), la.clone(), g.clone()
    n4 = h.mala_step(th_t, r1, la1, g1, n_steps=4, tau=0.05, seed=3, step_counter=10, grad_valid=False)
    r2, la2, g2 = r_t.clone(), la.clone(), g.clone()
    tot = 0
    for k in range(4):
        tot += int(h.mala_step(th_t, r2, la2, g2, n_steps=1, tau=0.05, seed=3, step_counter=10 + k,
                               grad_valid=(k > 0)).item())
    assert torch.equal(r1, r2) and torch.equal(la1, la2) and torch.equal(g1, g2)
    assert int(n4.item()) == tot
    ctr = torch.tensor([10], dtype=torch.int64, device="cuda:0")
    r3, la3, g3 = r_t.clone(), la.clone(), g.clone()
    h.mala_step(th_t, r3, la3, g3, n_steps=4, tau=0.05, seed=3, step_counter=ctr, grad_valid=False)
    assert torch.equal(r1, r3) and torch.equal(g1, g3)
    assert int(ctr.item()) == 14
