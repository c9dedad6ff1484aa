"""Run-to-run determinism of the stepping paths: the same case stepped twice from two fresh grids
gives bitwise the same state, alone (hyp_rk_stage, with its second stream beside the closure) and
in a batch (hyp_batch_step), for the five-species, eleven-species and equilibrium gases in both
precisions. A race between launches that share scratch would show here as differing runs."""
import pytest

from gpu_util import gpu_state
from paper_2210_05547_gb300 import inputs as I

pytestmark = pytest.mark.gpu

CASES = {"sbli_160x48": I.sbli_case(160, 48, seed=1),
         "sbli_160x48_air11": I.with_species(I.sbli_case(160, 48, seed=16)),
         "sbli_160x48_lte": I.sbli_case(160, 48, seed=3, kind="lte")}


def _alone(cfg, precision, nsteps=3):
    from paper_2210_05547_gb300 import abi as A
    _, st = gpu_state(cfg)
    for _ in range(nsteps):
        for k in range(3):
            A.rk_stage(st, k, cfg["dt"], precision=precision)
    return st.U.clone()


def _batched(cfg, precision, nsteps=3):
    from paper_2210_05547_gb300 import abi as A
    _, st = gpu_state(cfg)
    species = 11 if "air11" in cfg["name"] else 5
    batch = A.Batch(precision, use_graph=False, tile=1024, species=species)
    batch.add(st, cfg["dt"])
    batch.step(nsteps)
    return st.U.clone()


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("name", list(CASES))
def test_alone_runs_are_bitwise_equal(name, precision):
    import torch
    a = _alone(CASES[name], precision)
    b = _alone(CASES[name], precision)
    torch.cuda.synchronize()
    assert torch.equal(a, b), float((a - b).abs().max())


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("name", list(CASES))
def test_batched_runs_are_bitwise_equal(name, precision):
    import torch
    a = _batched(CASES[name], precision)
    b = _batched(CASES[name], precision)
    torch.cuda.synchronize()
    assert torch.equal(a, b), float((a - b).abs().max())


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("name", list(CASES))
def test_alone_equals_batched(name, precision):
    import torch
    a = _alone(CASES[name], precision)
    b = _batched(CASES[name], precision)
    torch.cuda.synchronize()
    assert torch.equal(a, b), float((a - b).abs().max())
