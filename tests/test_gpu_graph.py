"""A VMC step (Metropolis sweep with the step counter on the device,
local_energy, clipped loss weights, weighted gradient) captured as one CUDA
graph and replayed: the replays reproduce eager steps from the same state
bit for bit (same kernels on the same inputs), and the device counter
advances as mcmc_step's host counter would."""
import pytest
import torch

from paper_2307_14123_gb300 import Ansatz
from paper_2307_14123_gb300 import fixtures as fx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2307_14123_gb300 import _build
    _build.build()


def _setup(B):
    wl = fx.workload("n2_fp32")
    h = Ansatz(wl.system, wl.cfg, "fp32", device="cuda:0")
    th = torch.tensor(fx.init_params(wl.system, wl.cfg, wl.param_seed), dtype=torch.float32, device="cuda:0")
    r = torch.tensor(fx.init_walkers(wl.system, B, wl.walker_seed), dtype=torch.float32, device="cuda:0")
    la, _ = h.ansatz_eval(th, r)
    return wl, h, th, r, la


def test_graph_replay_matches_eager_steps():
    B, steps = 256, 3
    wl, h, th, r0, la0 = _setup(B)

    def step(rr, la, ctr):
        h.mcmc_step(th, rr, la, 1, 0.2, wl.walker_seed, ctr)
        _, _, el, e2 = h.local_energy(th, rr, sums=True)
        w, _ = h.vmc_loss_weights(el, 5.0)
        g = h.grad_logpsi(th, rr, w, 0)
        return el, e2, g

    # eager reference with the host counter
    r_e, la_e = r0.clone(), la0.clone()
    ref = []
    for k in range(steps):
        el, e2, g = step(r_e, la_e, 5 + k)
        ref.append((r_e.clone(), la_e.clone(), el.clone(), e2.clone(), g.clone()))

    # graph: warm up on scratch copies (workspaces), capture, then replay from the initial state
    r_g, la_g = r0.clone(), la0.clone()
    ctr = torch.tensor([5], dtype=torch.int64, device="cuda:0")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        rs, ls, cs = r0.clone(), la0.clone(), ctr.clone()
        step(rs, ls, cs)
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        out = step(r_g, la_g, ctr)
    # capture records the work without running it: restore the state, then replay
    r_g.copy_(r0)
    la_g.copy_(la0)
    ctr.fill_(5)
    for k in range(steps):
        graph.replay()
        torch.cuda.synchronize()
        rr, ll, el, e2, g = ref[k]
        assert torch.equal(r_g, rr)
        assert torch.equal(la_g, ll)
        assert torch.equal(out[0], el)
        assert torch.equal(out[1], e2)
        assert torch.equal(out[2], g)
    assert int(ctr.item()) == 5 + steps
