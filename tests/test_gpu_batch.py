"""Batched execution (hyp_batch_*): independent solves of different sizes, freestreams, cases and
time steps stepped together in shared launches. Each member's state after any sequence of joins
and leaves is bit-identical to the same member stepped alone with hyp_rk_stage, with and without
CUDA-graph replay and in both precisions."""
import numpy as np
import pytest

from gpu_util import gpu_state
from paper_2210_05547_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _cases():
    a = I.bl_case(96, 32, seed=3)
    b = I.sbli_case(160, 48, seed=1)          # artificial diffusivity and the state filter on
    c = I.bl_case(64, 24, seed=4)
    c.update(mach=6.0, T_wall=700.0, dt=1.5e-4)
    d = I.sbli_case(200, 40, seed=2)
    d["dt"] = 1.0e-3
    return [a, b, c, d]


def _alone(cfg, nsteps, precision):
    from paper_2210_05547_gb300 import abi as A
    gas, st = gpu_state(cfg)
    for _ in range(nsteps):
        for k in range(3):
            A.rk_stage(st, k, cfg["dt"], precision=precision)
    return st.U.cpu().numpy(), A.grid_status(st.grid)


@pytest.mark.parametrize("precision,use_graph", [(0, False), (0, True), (1, True)],
                         ids=["fp64", "fp64_graph", "mixed_graph"])
def test_members_identical_alone_and_in_the_mix(precision, use_graph):
    import torch
    from paper_2210_05547_gb300 import abi as A
    cfgs = _cases()
    # schedule: a and b from the start, c joins after 2 steps, a leaves after 4, d joins after 4
    steps = {0: 4, 1: 6, 2: 4, 3: 2}
    states = [gpu_state(c) for c in cfgs]
    batch = A.Batch(precision, use_graph=use_graph, tile=1024)
    batch.add(states[0][1], cfgs[0]["dt"])
    batch.add(states[1][1], cfgs[1]["dt"])
    batch.step(2)
    batch.add(states[2][1], cfgs[2]["dt"])
    batch.step(2)
    batch.remove(states[0][1])
    batch.add(states[3][1], cfgs[3]["dt"])
    assert batch.size() == 3
    batch.step(2)
    torch.cuda.synchronize()
    for k, cfg in enumerate(cfgs):
        ref, status = _alone(cfg, steps[k], precision)
        got = states[k][1].U.cpu().numpy()
        assert status == 0
        assert np.array_equal(got, ref), (k, float(np.abs(got - ref).max()))


def test_batch_rejects_a_different_gas_kind():
    from paper_2210_05547_gb300 import abi as A
    batch = A.Batch()
    _, st = gpu_state(I.bl_case(48, 32))
    _, st_cpg = gpu_state(I.bl_case(48, 32, kind="cpg"))
    batch.add(st, 2e-4)
    with pytest.raises(A.HypError, match="share one gas table"):
        batch.add(st_cpg, 2e-4)
    with pytest.raises(A.HypError, match="already in the batch"):
        batch.add(st, 2e-4)
    batch.remove(st)
    with pytest.raises(A.HypError, match="not in the batch"):
        batch.remove(st)
    batch.step(3)                              # empty batch: nothing to do
