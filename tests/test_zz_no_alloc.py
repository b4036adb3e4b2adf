"""fbst_execute_noalloc: the transform for callers that cannot allocate device memory at run time.

A real-time receive loop that must not block in the allocator, or a process whose device-memory
budget is fixed at start-up, cannot call cudaMalloc while it runs the transform.
fbst_execute_noalloc keeps the intermediates in the library's static 64 MiB device array instead.
This test calls it through the C ABI twice in a row (on different inputs) and checks each result
against fbst_execute within the suite's FP32 tolerance, and checks that an oversized request is
refused before anything runs. It builds what it needs, so it passes alone in a fresh process as
well as after the rest of the suite (this file is collected last).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def test_noalloc_matches_execute_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_08887_gb300.build import build
    build()
    import paper_2512_08887_gb300 as fb

    M, B, N, nblk = 48, 40, 64, 6
    rng = np.random.default_rng(99)
    plan = fb.Plan(fb.make_geometry("ula", M, 1, B, 1), N, fb.make_band(0.5, max_blocks=nblk))
    for call in range(2):
        y = torch.from_numpy((rng.standard_normal((nblk, M, N)) + 1j * rng.standard_normal((nblk, M, N)))
                             .astype(np.complex64)).cuda()
        ref = torch.full((nblk, B, N), complex(np.nan, np.nan), dtype=torch.complex64, device="cuda")
        out = torch.full_like(ref, complex(np.nan, np.nan))
        plan.execute(y, ref, nblk)
        plan.execute_noalloc(y, out, nblk)
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.isfinite(a).all(), f"call {call}: unwritten output"
        assert _rel(a, b) < TOL, f"call {call}"

    # 8*nblk*(L*M + B*L) bytes above 64 MiB must be refused up front.
    big = 64 * 1024 * 1024 // (8 * (plan.L * M + B * plan.L)) + 1
    with pytest.raises(fb.FBSTError) as e:
        plan.execute_noalloc(y.data_ptr(), out.data_ptr(), big)
    assert e.value.status == -1
    plan.close()
