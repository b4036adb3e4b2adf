"""The library's stage trace (fbst_trace_stages / fbst_trace_read; no counterpart in the paper):
CUDA events around the three stages of each fbst_execute call on its own stream. Checks that the
stage times of a traced call add up to the call's own event-timed duration, that the ring keeps
the newest calls, that a read clears the record, that tracing leaves the output bitwise unchanged,
and that a chunked call (nblk > max_blocks) traces its first chunk."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_08887_gb300.build import build
    build()


def test_stage_trace_of_execute_calls():
    import paper_2512_08887_gb300 as fb
    plan = fb.Plan(fb.make_geometry("ula", 256), 256, fb.make_band(0.5, stage2="dense_f16x3", max_blocks=16))
    rng = np.random.default_rng(2)
    y = torch.from_numpy((rng.standard_normal((40, 256, 256)) + 1j * rng.standard_normal((40, 256, 256)))
                         .astype(np.complex64)).cuda()
    ref = torch.empty((16, 256, 256), dtype=torch.complex64, device="cuda")
    out = torch.empty((40, 256, 256), dtype=torch.complex64, device="cuda")
    plan.execute(y, ref, 16)
    s = torch.cuda.current_stream()
    plan.trace_stages(3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
    for a, b in ev:
        a.record(s)
        plan.execute(y, out, 16)
        b.record(s)
    torch.cuda.synchronize()
    assert torch.equal(out[:16], ref)
    tr = plan.trace_read(8)
    assert len(tr) == 3                                   # the ring keeps the newest three calls
    for (k1, k2, k3), (a, b) in zip(tr, ev[2:]):
        total = a.elapsed_time(b)
        assert min(k1, k2, k3) > 0
        assert abs((k1 + k2 + k3) - total) < 0.05 * total + 0.02
    assert plan.trace_read(8) == []                       # read clears
    plan.execute(y, out, 40)                              # 3 chunks: the first one is traced
    torch.cuda.synchronize()
    (c,) = plan.trace_read(8)
    assert all(v > 0 for v in c)
    plan.trace_stages(0)
    plan.execute(y, out, 16)
    assert plan.trace_read(8) == []
