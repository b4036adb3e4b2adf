"""The server on the GPU: each result is the same alone and in the continuous-batching mix."""
import numpy as np
import pytest

import oracle as O
from synth import configs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_results_are_the_same_alone_and_in_the_mix():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_08887_gb300.build import build
    build()
    import paper_2512_08887_gb300 as fb
    from paper_2512_08887_gb300 import serve

    insts = [d for d in configs.c4_instances(count=16) if d["M"] * d["N"] <= 256 * 512][:6]
    plans = [fb.Plan(fb.make_geometry("ula", d["M"]), d["N"], fb.make_band(d["frac_bw"], max_blocks=4))
             for d in insts]
    rng = np.random.default_rng(11)
    pools = []
    for d in insts:
        blocks = []
        for _ in range(3):
            y = d["y"] + 0.1 * (rng.standard_normal(d["y"].shape) + 1j * rng.standard_normal(d["y"].shape))
            blocks.append(torch.from_numpy(y.astype(np.complex64)).pin_memory())
        pools.append(blocks)
    reqs = serve.poisson_requests(2e4, 60, pools, seed=5)
    ex = serve.GPUExecutor(plans, n_streams=3, keep_outputs=True)
    sched = serve.Scheduler([ex.request_bytes(a) for a in range(len(plans))], ex.device_budget, max_per_array=4,
                            max_batch_bytes=ex.arena_bytes)
    stats = serve.run_loop(reqs, sched, ex)
    ex.close()
    assert stats["requests"] == 60 and stats["mean_batch"] > 1
    # Alone: the same block through fbst_execute on its own.
    for r in reqs:
        p = plans[r.array]
        y = r.y.cuda()
        out = torch.empty((1, p.B, p.N), dtype=torch.complex64, device="cuda")
        p.execute(y, out, 1)
        torch.cuda.synchronize()
        a, b = r.out.numpy(), out.cpu().numpy()
        assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b), r.rid
    # And two requests against the FP64 oracle.
    for r in reqs[:2]:
        d, i = insts[r.array], plans[r.array].info
        pb = O.make_problem("ula", d["M"], 1, d["M"], 1, d["N"], frac_bw=i.fb_num / i.fb_den,
                            epsilon=i.eps_num / i.eps_den, delta=i.delta, L=i.L)
        beams = np.array([0, d["M"] // 2, d["M"] - 1])
        assert O.rel_l2(r.out.numpy()[:, beams], O.fbst(pb, r.y.numpy(), beams=beams)) < 1e-5
