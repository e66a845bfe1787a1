"""Failure detection without a GPU fault.  Every wait of a kernel on an asynchronous unit is
bounded: the apply kernel's waits for its bulk copies (MS_DEV_TIMEOUT) and the tcgen05
training kernel's waits for its MMAs (the error word of its scratch).  Test entry points
withhold what such a wait waits for (no copy, no MMA issued), so that it runs out after a
short limit; the failure must come back as an error, and the context must stay usable."""
import numpy as np
import pytest

from oracle import mlp as ref
from paper_2405_12520_b300 import learned, moss, synth

pytestmark = pytest.mark.gpu
P = synth.default_params()
DEV_TIMEOUT = 16


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    assert torch.cuda.is_available(), "needs a CUDA device"
    return torch


def test_tc_training_wait_timeout_is_reported(torch_mod):
    torch = torch_mod
    rng = np.random.default_rng(3)
    n = 1000
    X = torch.tensor(rng.normal(size=(n, 16)), dtype=torch.bfloat16, device="cuda")
    y = torch.tensor(rng.integers(0, 3, size=n), dtype=torch.int32, device="cuda")
    idx = torch.arange(n, dtype=torch.int32, device="cuda")
    theta = learned.init_params(4)
    th = torch.tensor(theta, device="cuda")
    cw = np.array([1.0, 2.0, 2.0], np.float32)
    work = torch.zeros(moss.MLP_WORK_FLOATS, device="cuda")
    assert moss.test_tc_timeout(X, y, idx, th, cw, work) == moss.MS_ERR_DEVICE
    # the context is usable: the same gradient with the MMAs issued, against the reference
    g = torch.zeros(moss.MLP_NPARAM, device="cuda")
    moss.mlp_grad(X, y, idx, th, cw, work, g, tc=True)
    torch.cuda.synchronize()
    assert work[moss.MLP_NPARAM + 2:moss.MLP_NPARAM + 3].view(torch.int32).item() == 0
    gr = ref.grad_bf16(theta.astype(np.float64), X.float().cpu().double().numpy(), y.cpu().numpy(),
                       cw.astype(np.float64))
    gg = g.cpu().double().numpy()
    assert np.linalg.norm(gg - gr) <= 1e-2 * np.linalg.norm(gr)


def test_apply_copy_wait_timeout_is_reported(torch_mod):
    net, dem = synth.small_grid_workload(3)
    sim = moss.Sim(P)
    sim.load_network(net)
    sim.add_vehicles(dem)
    sim.step(60)
    sim.sync()
    m = sim.read_metrics(lanes=False)
    assert m["err"] == 0 and m["n_active"] > 0   # the apply kernel has tiles to wait for
    sim.test_withhold_copies(True)
    sim.step(1)
    with pytest.raises(moss.MossError) as e:
        sim.sync()
    assert e.value.code == moss.MS_ERR_DEVICE
    assert sim.read_metrics(lanes=False)["err"] & DEV_TIMEOUT
    sim.destroy()
    # the context is usable: a fresh simulation of the same workload steps cleanly
    sim2 = moss.Sim(P)
    sim2.load_network(net)
    sim2.add_vehicles(dem)
    sim2.step(20)
    sim2.sync()
    m = sim2.read_metrics(lanes=False)
    assert m["err"] == 0 and m["n_active"] > 0
    sim2.destroy()
