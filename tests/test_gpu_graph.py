"""A whole RK3 step captured into a CUDA graph through the public API (torch.cuda.graph around
three hyp_rk_stage calls) and replayed gives the state of the same step run eagerly, bit for bit:
on a two-dimensional shock / boundary-layer case and on the three-dimensional jet (whose
velocity-gradient phases fork onto the grid's second stream and join back inside the step)."""
import numpy as np
import pytest

from paper_2210_05547_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _zoom(cfg):
    cfg.update(x0=50.0, x1=55.0, z0=0.0, z1=3.0, jet_x=52.5, jet_z=1.5, sponge_in=0.5,
               sponge_out=0.5)
    return cfg


CASES = {"sbli_96x40": I.sbli_case(96, 40, seed=3),
         "jet_40x24x12": _zoom(I.jet_case(40, 24, 12, seed=1))}


def _state(A, cfg):
    import torch
    gas = A.gas_model_load(cfg)
    n = A.state_size(gas, cfg)
    U = torch.empty(n, dtype=torch.float64, device="cuda")
    dQ = torch.empty_like(U)
    return gas, A.state_init(gas, cfg, U, dQ, I.state_noise(n, cfg["seed"]))


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_graph_replay_equals_eager_step(name, precision):
    import torch
    from paper_2210_05547_gb300 import abi as A
    cfg = CASES[name]
    dt = cfg["dt"]
    _, eager = _state(A, cfg)
    _, graphed = _state(A, cfg)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for st in (eager, graphed):          # one eager step each: the closure caches are warm
            for k in range(3):
                A.rk_stage(st, k, dt, precision=precision)
        for k in range(3):
            A.rk_stage(eager, k, dt, precision=precision)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for k in range(3):
            A.rk_stage(graphed, k, dt, precision=precision)
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(graphed.U.cpu().numpy(), eager.U.cpu().numpy())
    assert np.array_equal(graphed.dQ.cpu().numpy(), eager.dQ.cpu().numpy())
    assert A.grid_status(graphed.grid) == 0
