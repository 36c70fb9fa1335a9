"""Natural-gradient direction (Sec. 4, "Optimizer") on the GPU against the FP64
oracle's dense solve.

Parity inputs are seeded synthetic per-walker gradients (the oracle takes no
input from the CUDA path); their column scales and offsets vary, like those of
real gradients.  Bound: the Gram matrix is formed from 3 x TF32 products
accumulated in FP32 over chunks of 8192 parameters and added in FP64 (relative
error about 2^-21 of sum |g||g| per chunk), and the conjugate gradients stop at a
relative residual of 1e-9, so delta carries a relative (norm-wise) error of order
kappa 2^-21 for a system of condition kappa; the damping below keeps kappa under
1e3, and the bound is 2e-3 (norm-wise; element-wise the bound of each element
follows from it by Cauchy-Schwarz).  Real N2 per-walker gradients are
checked through the damped normal equations they must satisfy."""
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


def _handle(name):
    from paper_2307_14123_gb300 import Ansatz
    wl = fx.workload(name)
    return wl, Ansatz(wl.system, wl.cfg, "fp32", device="cuda:0")


def _synthetic(B, P, seed):
    rng = np.random.default_rng(seed)
    G = (rng.standard_normal((B, P)) * rng.uniform(0.05, 2.0, P) + rng.standard_normal(P)).astype(np.float32)
    e = rng.standard_normal(B)
    w = ((2.0 / B) * (e - e.mean())).astype(np.float32)
    return G.astype(np.float64), w.astype(np.float64)


def _damping(G, rel):
    Gc = G - G.mean(axis=0)
    return rel * float(np.sum(Gc * Gc)) / G.shape[0] / G.shape[0]  # rel x mean eigenvalue of Gc Gc^T / B


@pytest.mark.parametrize("B", [96, 256])
def test_natural_gradient_matches_oracle(B):
    wl, h = _handle("lih_fp64")  # LiH ansatz in FP32 mode: P = 19285, not a multiple of 4 (padded rows)
    G, w = _synthetic(B, h.P, 11 + B)
    lam = _damping(G, 1e-2)
    d, st = h.natural_gradient(torch.tensor(G, dtype=torch.float32, device="cuda:0"),
                               torch.tensor(w, dtype=torch.float32, device="cuda:0"), lam, max_iter=400, tol=1e-9)
    ref = oracle.natural_gradient(G, w, lam)
    got = d.cpu().numpy().astype(np.float64)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    st = st.cpu().numpy()
    print(f"B={B}: CG iterations {st[0]:.0f}, residual {st[1]:.2e}, relative error {err:.2e}")
    assert st[1] <= 1e-9 and err <= 2e-3
    # element by element: delta_p = sum_b Gc_bp x_b with x the sample-space solution, so an error
    # dx of the solve moves delta_p by at most ||Gc[:, p]|| ||dx|| (Cauchy-Schwarz); with
    # ||dx|| <= 2e-3 ||x|| as above, plus the FP32 rounding of the final product
    Gc = G - G.mean(axis=0)
    x = np.linalg.solve(Gc @ Gc.T / B + lam * np.eye(B), w)
    tol = 2e-3 * np.linalg.norm(Gc, axis=0) * np.linalg.norm(x) + 1e-5 * (np.abs(Gc).T @ np.abs(x))
    print(f"B={B}: max element error / bound {np.max(np.abs(got - ref) / tol):.2e}")
    assert np.all(np.abs(got - ref) <= tol)


def test_natural_gradient_deterministic_and_zero_iterations():
    wl, h = _handle("lih_fp64")
    G, w = _synthetic(64, h.P, 5)
    Gt = torch.tensor(G, dtype=torch.float32, device="cuda:0")
    wt = torch.tensor(w, dtype=torch.float32, device="cuda:0")
    lam = _damping(G, 1e-2)
    a, _ = h.natural_gradient(Gt, wt, lam)
    b, _ = h.natural_gradient(Gt, wt, lam)
    assert torch.equal(a, b)
    z, st = h.natural_gradient(Gt, wt, lam, max_iter=0)
    assert float(z.abs().max()) == 0.0 and float(st[0]) == 0.0


def test_natural_gradient_real_gradients_normal_equations():
    """N2 (P = 412656): per-walker gradients from grad_logpsi(mode 1), clipped-energy weights;
    (Gc^T Gc / B + lam I) delta = Gc^T w checked in FP64 with torch, at a damping of 1e-2 of
    the mean eigenvalue (a much worse conditioned system than the synthetic ones)."""
    wl, h = _handle("n2_fp32")
    B = 128
    th = torch.tensor(fx.init_params(wl.system, wl.cfg, wl.param_seed), dtype=torch.float32, device="cuda:0")
    r = torch.tensor(fx.init_walkers(wl.system, B, wl.walker_seed), dtype=torch.float32, device="cuda:0")
    G = h.grad_logpsi(th, r, mode=1)
    _, _, el = h.local_energy(th, r)
    w, _ = h.vmc_loss_weights(el, 5.0)
    Gd = G.double()
    Gc = Gd - Gd.mean(dim=0, keepdim=True)
    lam = 1e-2 * float((Gc * Gc).sum()) / B / B
    d, st = h.natural_gradient(G, w, lam, max_iter=400, tol=1e-9)
    g = Gc.t() @ w.double()
    lhs = Gc.t() @ (Gc @ d.double()) / B + lam * d.double()
    rel = float((lhs - g).norm() / g.norm())
    print(f"N2 B={B}: CG iterations {float(st[0]):.0f}, residual {float(st[1]):.2e}, normal-equation residual {rel:.2e}")
    assert rel <= 2e-3


def test_relative_damping_matches_absolute():
    """lambda < 0 means |lambda| x tr(Gc Gc^T) / B^2; against the oracle at that absolute damping."""
    wl, h = _handle("lih_fp64")
    G, w = _synthetic(128, h.P, 21)
    Gc = G - G.mean(axis=0)
    lam = 0.05 * float(np.sum(Gc * Gc)) / 128 / 128
    d, st = h.natural_gradient(torch.tensor(G, dtype=torch.float32, device="cuda:0"),
                               torch.tensor(w, dtype=torch.float32, device="cuda:0"), -0.05, max_iter=400, tol=1e-9)
    # the Gram diagonal sums positive squares in FP32 over chunks of 8192: at most 8192 x 2^-24 relative
    assert abs(float(st[3]) - lam) <= 5e-4 * lam
    ref = oracle.natural_gradient(G, w, lam)
    assert np.linalg.norm(d.cpu().numpy() - ref) <= 2e-3 * np.linalg.norm(ref)


@pytest.mark.parametrize("max_norm", [0.0, 1e-3])
def test_param_update_against_oracle(max_norm):
    """theta <- theta - lr s delta against oracle.param_update: the GPU forms the step in FP64 and
    rounds the new parameters to FP32 once, so every element equals the oracle's FP64 value
    rounded to FP32 (up to the last bit of lr s, a fixed-order FP64 norm)."""
    wl, h = _handle("lih_fp64")
    rng = np.random.default_rng(7)
    th = rng.standard_normal(h.P).astype(np.float32)
    dl = rng.standard_normal(h.P).astype(np.float32)
    lr = 0.05
    t = torch.tensor(th, device="cuda:0")
    st = h.param_update(t, torch.tensor(dl, device="cuda:0"), lr, max_norm).cpu().numpy()
    ref, nrm, s = oracle.param_update(th, dl, lr, max_norm)
    assert st[0] == pytest.approx(nrm, rel=1e-12) and st[1] == pytest.approx(s, rel=1e-12)
    got = t.cpu().numpy().astype(np.float64)
    ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
    assert np.all(np.abs(got - ref) <= 0.5 * ulp + 1e-12 * np.abs(ref))


def test_vmc_train_step_runs_and_is_reproducible():
    """Three training steps (sampler, local energies, weights, per-walker gradients, natural
    gradient, update) on LiH: finite statistics, parameters move, and a second run from the
    same state gives the same bits."""
    from paper_2307_14123_gb300 import vmc_train_step
    wl, h = _handle("lih_fp64")
    th0 = torch.tensor(fx.init_params(wl.system, wl.cfg, wl.param_seed), dtype=torch.float32, device="cuda:0")
    r0 = torch.tensor(fx.init_walkers(wl.system, 256, wl.walker_seed), dtype=torch.float32, device="cuda:0")
    runs = []
    for _ in range(2):
        th, r = th0.clone(), r0.clone()
        la, _ = h.ansatz_eval(th, r)
        for t in range(3):
            out = vmc_train_step(h, th, r, la, lr=0.02, damping=-0.1, max_norm=0.05, seed=1, step_counter=t)
            e2 = out["e_sum2"].cpu().numpy()
            assert np.all(np.isfinite(e2)) and np.all(np.isfinite(out["natural_gradient"].cpu().numpy()))
            assert float(out["update"][1]) <= 1.0
        runs.append((th.clone(), r.clone()))
    assert not torch.equal(runs[0][0], th0)
    assert torch.equal(runs[0][0], runs[1][0]) and torch.equal(runs[0][1], runs[1][1])
