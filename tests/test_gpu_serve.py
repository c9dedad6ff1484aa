"""Serving (hyp_server_*): continuous batching of independent solves. Requests submitted while
others run join the batch at a step boundary; each result is bit-identical to the same request
stepped alone with hyp_rk_stage; admission waits for device memory and never over-commits;
a request that can never fit is reported, not left waiting."""
import time

import numpy as np
import pytest

from gpu_util import gpu_state
from paper_2210_05547_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _alone(cfg, nsteps, precision):
    from paper_2210_05547_gb300 import abi as A
    gas, st = gpu_state(cfg)
    for _ in range(nsteps):
        for k in range(3):
            A.rk_stage(st, k, cfg["dt"], precision=precision)
    return st.U.cpu().numpy()


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_results_identical_alone_and_in_the_mix(precision):
    from paper_2210_05547_gb300 import abi as A
    reqs = I.serving_requests(7, seed=11, steps=(6, 30))
    sv = A.Server(precision=precision, max_members=16)
    ids = []
    for k, (cfg, nsteps, gap) in enumerate(reqs):
        noise = I.state_noise(A.state_len(cfg), cfg["seed"])
        ids.append(sv.submit(cfg, nsteps, noise=noise, keep_result=True))
        time.sleep(0.02 * gap)                 # later requests arrive while earlier ones run
    sv.wait(timeout=600)
    for rid, (cfg, nsteps, _) in zip(ids, reqs):
        st = sv.stats(rid)
        assert st["done"] == 1 and st["error"] == 0, st
        assert 0.0 <= st["t_submit"] <= st["t_admit"] < st["t_finish"], st
        got = sv.result(rid, cfg)
        ref = _alone(cfg, nsteps, precision)
        assert np.array_equal(got, ref), (cfg["name"], float(np.abs(got - ref).max()))
    c = sv.counters()
    assert c["max_members"] >= 2                # requests really shared launches
    sv.close()


def test_eleven_species_requests_identical_alone_and_in_the_mix():
    from paper_2210_05547_gb300 import abi as A
    reqs = I.serving_requests(4, seed=13, steps=(4, 12), air11=1.0)
    assert all(c["table"] == "air11" for c, _, _ in reqs)
    sv = A.Server(precision=0, max_members=8, path=A.TABLE_AIR11)
    with pytest.raises(ValueError):
        sv.submit(I.bl_case(128, 32), 2)                # a five-species request
    ids = []
    for cfg, nsteps, gap in reqs:
        noise = I.state_noise(A.state_len(cfg), cfg["seed"])
        ids.append(sv.submit(cfg, nsteps, noise=noise, keep_result=True))
        time.sleep(0.02 * gap)
    sv.wait(timeout=600)
    for rid, (cfg, nsteps, _) in zip(ids, reqs):
        st = sv.stats(rid)
        assert st["done"] == 1 and st["error"] == 0 and st["status"] == 0, st
        got = sv.result(rid, cfg)
        assert np.array_equal(got, _alone(cfg, nsteps, 0)), cfg["name"]
    sv.close()


def test_admission_waits_for_memory():
    import torch
    from paper_2210_05547_gb300 import abi as A
    cfg = I.bl_case(512, 128, seed=1)
    need = 2400 * 512 * 128 + (4 << 20)
    free, _ = torch.cuda.mem_get_info()
    # room for one member at a time
    sv = A.Server(reserve_bytes=free - int(1.5 * need), max_members=8)
    ids = [sv.submit(cfg, 3) for _ in range(3)]
    sv.wait(timeout=600)
    for rid in ids:
        st = sv.stats(rid)
        assert st["done"] == 1 and st["error"] == 0, st
    assert sv.counters()["max_members"] == 1
    s = [sv.stats(r) for r in ids]
    assert s[1]["t_admit"] >= s[0]["t_finish"] and s[2]["t_admit"] >= s[1]["t_finish"]
    sv.close()


def test_request_that_can_never_fit_is_reported():
    import torch
    from paper_2210_05547_gb300 import abi as A
    free, _ = torch.cuda.mem_get_info()
    sv = A.Server(reserve_bytes=free, max_members=4)
    rid = sv.submit(I.bl_case(128, 32), 2)
    sv.wait(rid, timeout=60)
    st = sv.stats(rid)
    assert st["done"] == 1 and st["error"] == -4       # HYP_ERR_OOM
    with pytest.raises(A.HypError):
        sv.submit(I.bl_case(128, 32), 0)               # no steps: rejected at submission
    sv.close()
