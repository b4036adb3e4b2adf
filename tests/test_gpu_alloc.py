"""The plan's allocator hook (fbst_plan's alloc / free) on the GPU, with failures injected on the
host: an allocator that returns NULL on its n-th call.

Every device block of a plan goes through the caller's allocator: its tables and workspace, the
plan-time temporaries, the staging of the host-buffer path, the test input of fbst_autotune and the
memory of nulling objects. An allocation that fails must surface as FBST_ERR_OOM from the entry
point that needed it, with every block obtained so far given back (nothing leaks), and the process
must go on working: a later plan computes the right result.
"""
import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OOM = -2


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_08887_gb300.build import build
    build()


class Counting:
    """Backed by PyTorch's caching allocator; counts calls, records live blocks and their sizes,
    and returns NULL on the call numbers in `fail_on`."""

    def __init__(self, fail_on=()):
        import paper_2512_08887_gb300 as fb
        self.calls, self.fail_on, self.live, self.mismatch = 0, set(fail_on), {}, 0
        self.streams = set()

        def alloc(nbytes, stream):
            self.calls += 1
            self.streams.add(stream)
            if self.calls in self.fail_on:
                return 0
            ptr = torch.cuda.caching_allocator_alloc(nbytes, stream=stream)
            self.live[ptr] = nbytes
            return ptr

        def free(ptr, nbytes, stream):
            if self.live.pop(ptr, None) != nbytes:
                self.mismatch += 1
            torch.cuda.caching_allocator_delete(ptr)

        self.allocator = fb.Allocator(alloc, free)


def _plan(stage2, alloc, M=24, N=64, max_blocks=4):
    import paper_2512_08887_gb300 as fb
    return fb.Plan(fb.make_geometry("ula", M), N, fb.make_band(0.5, stage2=stage2, max_blocks=max_blocks),
                   allocator=alloc.allocator if isinstance(alloc, Counting) else alloc)


def _check_result(plan, rng, nblk=3):
    i = plan.info
    pb = O.make_problem("ula", plan.M, 1, plan.B, 1, plan.N, frac_bw=i.fb_num / i.fb_den,
                        epsilon=i.eps_num / i.eps_den, delta=i.delta, L=i.L)
    y = (rng.standard_normal((nblk, plan.M, plan.N)) + 1j * rng.standard_normal((nblk, plan.M, plan.N))).astype(np.complex64)
    out = torch.full((nblk, plan.B, plan.N), complex(np.nan, np.nan), dtype=torch.complex64, device="cuda")
    plan.execute(torch.from_numpy(y).cuda(), out, nblk)
    assert plan.sync_status() == 0
    assert O.rel_l2(out.cpu().numpy(), O.fbst(pb, y)) < 1e-5


@pytest.mark.parametrize("stage2", ["gs_ir1", "dense_tf32x3", "dense_fp32"])
def test_every_block_comes_from_the_allocator_and_goes_back(rng, stage2):
    c = Counting()
    plan = _plan(stage2, c)
    n_alloc = c.calls
    assert n_alloc > 5 and c.live, "the plan took no memory from the allocator"
    # Temporaries are already back; what is live is the plan's tables and workspace.
    i = plan.info
    live = sum(c.live.values())
    assert i.table_bytes + i.workspace_bytes <= live <= i.table_bytes + i.workspace_bytes + 256, \
        (live, i.table_bytes, i.workspace_bytes)
    assert c.streams == {int(torch.cuda.current_stream().cuda_stream)}
    _check_result(plan, rng)
    # The host path allocates its staging through the same allocator, on first use.
    y = np.zeros((2, plan.M, plan.N), dtype=np.complex64)
    out = np.empty((2, plan.B, plan.N), dtype=np.complex64)
    plan.execute_host(y, out, 2)
    assert c.calls == n_alloc + 2
    plan.close()
    assert c.live == {} and c.mismatch == 0


@pytest.mark.parametrize("stage2", ["gs_ir1", "dense_tf32x3"])
def test_a_failing_allocation_is_oom_and_leaks_nothing(rng, stage2):
    import paper_2512_08887_gb300 as fb
    n_alloc = Counting()
    _plan(stage2, n_alloc).close()
    total = n_alloc.calls
    for k in range(1, total + 1):
        c = Counting(fail_on=(k,))
        with pytest.raises(fb.FBSTError) as e:
            _plan(stage2, c)
        assert e.value.status == OOM, f"allocation {k} of {total}"
        torch.cuda.synchronize()
        assert c.live == {} and c.mismatch == 0, f"allocation {k} of {total} leaked {len(c.live)} blocks"
    # The device and the library are still in order: a plan built afterwards is correct.
    plan = _plan(stage2, Counting())
    _check_result(plan, rng)
    plan.close()


def test_failures_after_the_plan_leave_it_usable(rng):
    import paper_2512_08887_gb300 as fb
    c = Counting()
    plan = _plan("gs_ir1", c)
    base = c.calls
    # Host-path staging: its second block fails.
    c.fail_on = {base + 2}
    y = np.zeros((2, plan.M, plan.N), dtype=np.complex64)
    out = np.empty((2, plan.B, plan.N), dtype=np.complex64)
    with pytest.raises(fb.FBSTError) as e:
        plan.execute_host(y, out, 2)
    assert e.value.status == OOM
    # A nulling object whose third block fails.
    c.fail_on = {c.calls + 3}
    with pytest.raises(fb.FBSTError) as e:
        fb.Nulling(plan, [3, 7])
    assert e.value.status == OOM
    # Autotune's test input fails.
    c.fail_on = {c.calls + 1}
    with pytest.raises(fb.FBSTError) as e:
        plan.autotune(2)
    assert e.value.status == OOM
    c.fail_on = set()
    _check_result(plan, rng)
    plan.execute_host(y, out, 2)            # staging now allocated and the host path works
    nl = fb.Nulling(plan, [3, 7])
    nl.close()
    plan.close()
    assert c.live == {} and c.mismatch == 0


def test_default_allocator_paths_match(rng):
    # allocator=None: the library's cudaMallocAsync / cudaFreeAsync path.
    plan = _plan("gs_ir1", None)
    _check_result(plan, rng)
    plan.close()


def test_server_reports_a_malformed_request_and_keeps_serving():
    import paper_2512_08887_gb300 as fb
    from paper_2512_08887_gb300 import serve
    from synth import configs
    insts = [d for d in configs.c4_instances(count=12) if d["M"] * d["N"] <= 128 * 512][:3]
    plans = [fb.Plan(fb.make_geometry("ula", d["M"]), d["N"], fb.make_band(d["frac_bw"], max_blocks=4))
             for d in insts]
    pools = [[torch.from_numpy(d["y"]).pin_memory()] for d in insts]
    reqs = serve.poisson_requests(2e3, 40, pools, seed=3)
    bad = reqs[7]
    bad.y = torch.zeros((1, 3, 5), dtype=torch.complex64).pin_memory()   # wrong shape for its array
    ex = serve.GPUExecutor(plans, n_streams=2, keep_outputs=True, arena_bytes=64 << 20)
    sched = serve.Scheduler([ex.request_bytes(a) for a in range(len(plans))], ex.device_budget, 4,
                            max_batch_bytes=ex.arena_bytes)
    stats = serve.run_loop(reqs, sched, ex)
    ex.close()
    assert bad.error is not None and "does not fit" in bad.error
    served = [r for r in reqs if r.error is None]
    assert stats["failed"] >= 1 and len(served) >= 30
    assert any(r.t_arrival > bad.t_done for r in served)     # requests after the failure were served
    for r in served:
        p = plans[r.array]
        out = torch.empty((1, p.B, p.N), dtype=torch.complex64, device="cuda")
        p.execute(r.y.cuda(), out, 1)
        torch.cuda.synchronize()
        assert np.linalg.norm(r.out.numpy() - out.cpu().numpy()) <= 1e-5 * np.linalg.norm(out.cpu().numpy())
