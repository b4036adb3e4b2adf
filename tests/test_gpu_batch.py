"""Batched uneven arrays (grouped launches replayed from a CUDA graph) and the shape autotuner."""
import os

import numpy as np
import pytest

import oracle as O
from synth import configs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_08887_gb300.build import build
    build()


def _plans(insts, stage2="auto"):
    import paper_2512_08887_gb300 as fb
    return [fb.Plan(fb.make_geometry("ula", d["M"]), d["N"], fb.make_band(d["frac_bw"], stage2=stage2, max_blocks=1))
            for d in insts]


def _nan(shape):
    return torch.full(shape, complex(np.nan, np.nan), dtype=torch.complex64, device="cuda")


def test_batch_equals_per_plan_execution_and_replays():
    import paper_2512_08887_gb300 as fb
    insts = configs.c4_instances(count=10)
    plans = _plans(insts)
    ys = [torch.from_numpy(d["y"]).cuda() for d in insts]
    ref = [_nan((1, d["B"], d["N"])) for d in insts]
    for p, y, r in zip(plans, ys, ref):
        p.execute(y, r, 1)
    batch = fb.Batch(plans)
    outs = [_nan((1, d["B"], d["N"])) for d in insts]
    batch.execute(ys, outs, [1] * len(insts))      # eager run + capture
    torch.cuda.synchronize()
    for o, r in zip(outs, ref):
        assert torch.equal(o, r)
    launches = batch.launch_count()
    assert 0 < launches < 3 * len(insts)
    for o in outs:
        o.fill_(complex(np.nan, np.nan))
    batch.execute(ys, outs, [1] * len(insts))      # graph replay
    torch.cuda.synchronize()
    for o, r in zip(outs, ref):
        assert torch.equal(o, r)
    # A different block-count pattern (one instance skipped) is a new configuration.
    outs2 = [_nan((1, d["B"], d["N"])) for d in insts]
    batch.execute(ys, outs2, [1] * (len(insts) - 1) + [0])
    torch.cuda.synchronize()
    for o, r in zip(outs2[:-1], ref[:-1]):
        assert torch.equal(o, r)
    assert torch.isnan(outs2[-1].real).all()
    # Against the FP64 oracle on a few beams of two instances.
    for k in (0, len(insts) - 1):
        d, i = insts[k], plans[k].info
        pb = O.make_problem("ula", d["M"], 1, d["M"], 1, d["N"], frac_bw=i.fb_num / i.fb_den,
                            epsilon=i.eps_num / i.eps_den, delta=i.delta, L=i.L)
        beams = np.array([0, d["M"] // 3, d["M"] - 1])
        got = outs[k].cpu().numpy()[:, beams]
        assert O.rel_l2(got, O.fbst(pb, d["y"], beams=beams)) < 1e-5
    batch.close()


def test_autotune_picks_a_compiled_shape_and_keeps_results(tmp_path):
    import paper_2512_08887_gb300 as fb
    from paper_2512_08887_gb300 import autotune
    rng = np.random.default_rng(5)
    plan = fb.Plan(fb.make_geometry("ula", 96, 1, 80, 1), 128, fb.make_band(0.45, max_blocks=8))
    y = torch.from_numpy((rng.standard_normal((8, 96, 128)) + 1j * rng.standard_normal((8, 96, 128)))
                         .astype(np.complex64)).cuda()
    ref, out = _nan((8, 80, 128)), _nan((8, 80, 128))
    plan.execute(y, ref, 8)
    cache = str(tmp_path / "tune.json")
    shapes = autotune.tune(plan, 8, path=cache)
    assert os.path.exists(cache) and plan.shapes() == tuple(shapes)
    plan.execute(y, out, 8)
    torch.cuda.synchronize()
    a, b = out.cpu().numpy(), ref.cpu().numpy()
    # Another radix changes the FFT rounding; both results stay within the suite's 1e-5 bar.
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-5
    plan.set_shapes(0, 0, 0, 0)
    assert autotune.tune(plan, 8, path=cache) == tuple(shapes)   # cache hit
    with pytest.raises(fb.FBSTError):
        plan.set_shapes(8, 3, 0, 0)


def test_all_64_uneven_arrays_of_the_workload_in_one_batch():
    # The whole uneven-array workload (64 ULAs, M = 2^U{5..10}, N from 128..1024, B = M, fb in
    # [0.2, 0.6]): the batch equals the per-plan execution bitwise for every array, and the FP64
    # oracle agrees on sampled beams of arrays spread over the set (every M and N present).
    import paper_2512_08887_gb300 as fb
    insts = configs.c4_instances(count=64)
    plans = _plans(insts)
    ys = [torch.from_numpy(d["y"]).cuda() for d in insts]
    ref = [_nan((1, d["B"], d["N"])) for d in insts]
    for p, y, r in zip(plans, ys, ref):
        p.execute(y, r, 1)
    batch = fb.Batch(plans)
    outs = [_nan((1, d["B"], d["N"])) for d in insts]
    batch.execute(ys, outs, [1] * 64)
    batch.execute(ys, outs, [1] * 64)              # graph replay
    torch.cuda.synchronize()
    for k, (o, r) in enumerate(zip(outs, ref)):
        assert torch.equal(o, r), k
    picked = {}
    for k, d in enumerate(insts):
        picked.setdefault((d["M"], d["N"]), k)
    for k in sorted(picked.values())[::2]:
        d, i = insts[k], plans[k].info
        pb = O.make_problem("ula", d["M"], 1, d["M"], 1, d["N"], frac_bw=i.fb_num / i.fb_den,
                            epsilon=i.eps_num / i.eps_den, delta=i.delta, L=i.L)
        beams = np.unique(np.array([0, d["M"] // 2, d["M"] - 1]))
        assert O.rel_l2(outs[k].cpu().numpy()[:, beams], O.fbst(pb, d["y"], beams=beams)) < 1e-5, (k, d["M"], d["N"])
    batch.close()
