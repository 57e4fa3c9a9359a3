"""Batched plans (one persistent launch captured in a CUDA graph) and the
launch-shape autotuner, against the CPU oracle: bit-exact, replay after replay."""
import numpy as np
import pytest

import oracle
from paper_2108_05038_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2108_05038_gb300 import fim  # noqa: E402


def odict(res):
    so, si, sp = res
    return {tuple(int(v) for v in si[so[k]:so[k + 1]]): int(sp[k]) for k in range(len(sp))}


@pytest.mark.parametrize("name,D", [("dense_deep", 50_000), ("tiny", 10_000), ("sparse_mid", 40_000)])
def test_plan_replays_match_oracle(name, D):
    w = synth.make_workload(name, D=D)
    ms = synth.abs_minsup(w["rel_minsup"], D)
    want = odict(oracle.eclat(w["offsets"], w["items"], w["N"], ms))
    db = fim.build_vertical_db(w["offsets"], w["items"], w["N"])
    db.estimate_class_costs(0.02 if D >= 40_000 else 0.1, w["rel_minsup"], 11)
    plan = db.plan(ms)
    for _ in range(3):
        plan.launch()
        res = plan.result()
        assert res.as_dict() == want
    for _ in range(4):  # back-to-back replays, one result at the end
        plan.launch()
    assert plan.result().as_dict() == want
    plan.free()
    db.free()


def test_plan_on_torch_stream_and_device_result():
    w = synth.make_workload("dense_deep", D=20_000)
    ms = 12_000
    want = odict(oracle.eclat(w["offsets"], w["items"], w["N"], ms))
    s = torch.cuda.Stream()
    db = fim.build_vertical_db(w["offsets"], w["items"], w["N"], stream=s)
    plan = db.plan(ms, result_on_device=True)
    assert plan.stream == s.cuda_stream
    plan.launch()
    res = plan.result(result_on_device=True)
    assert res.on_device and res.n_sets == len(want)
    plan.free()
    db.free()


def test_autotune_shape_is_valid_and_output_unchanged():
    w = synth.make_workload("dense_deep", D=30_000)
    ms = 18_000
    want = odict(oracle.eclat(w["offsets"], w["items"], w["N"], ms))
    db = fim.build_vertical_db(w["offsets"], w["items"], w["N"])
    shape, best_ms = db.autotune(ms)
    assert shape["threads_per_cta"] in (128, 256, 512) and shape["vec_per_lane"] in (1, 2, 4, 8)
    assert best_ms > 0
    again, ms2 = db.autotune(ms)  # cached
    assert again == shape and ms2 == best_ms
    assert db.mine(ms, shape=shape).as_dict() == want
    plan = db.plan(ms, shape=shape)
    plan.launch()
    assert plan.result().as_dict() == want
    plan.free()
    db.free()


def test_launch_counter_counts_graph_kernels_per_replay():
    """fim_kernel_launches: a mine adds its kernels; each plan replay adds the kernels of its graph."""
    w = synth.make_workload("dense_deep", D=20_000)
    ms = 12_000
    db = fim.build_vertical_db(w["offsets"], w["items"], w["N"])
    c0 = fim.kernel_launches()
    db.mine(ms).free()
    c1 = fim.kernel_launches()
    assert c1 - c0 >= 5  # pair counts, survivor count, level-2 scan and fill, DFS
    plan = db.plan(ms)
    c2 = fim.kernel_launches()
    plan.launch()
    c3 = fim.kernel_launches()
    plan.launch()
    plan.launch()
    c4 = fim.kernel_launches()
    assert c3 - c2 >= 5 and c4 - c3 == 2 * (c3 - c2)
    plan.result().free()
    plan.free()
    db.free()
