"""Streaming over contiguous, overlapping blocks (Sec. III-A) through the C ABI: fbst_execute_stream
against the oracle's fbst_stream (blocks every `hop` samples, each contributing its central hop
samples), at the transform's FP32 bar 1e-5. Blocks are read in place from the record; chunks of
max_blocks and a ragged last chunk are covered. Outputs are poisoned with NaN first."""
import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_08887_gb300.build import build
    build()


def _plan(M, B, N, fbw, stage2="auto", max_blocks=4):
    import paper_2512_08887_gb300 as fb
    plan = fb.Plan(fb.make_geometry("ula", M, 1, B, 1), N, fb.make_band(fbw, stage2=stage2, max_blocks=max_blocks))
    i = plan.info
    pb = O.make_problem("ula", M, 1, B, 1, N, frac_bw=i.fb_num / i.fb_den, epsilon=i.eps_num / i.eps_den,
                        delta=i.delta, L=i.L)
    return plan, pb


@pytest.mark.parametrize("M,B,N,hop,stage2", [(16, 16, 64, 32, "auto"), (40, 24, 96, 96, "auto"),
                                              (33, 20, 64, 48, "dense_tf32x3"), (64, 64, 128, 96, "gs_ir1")])
def test_stream_matches_oracle(rng, M, B, N, hop, stage2):
    plan, pb = _plan(M, B, N, 0.5, stage2=stage2, max_blocks=4)
    nblk = 9                                                   # chunks of 4, 4 and 1
    T = (nblk - 1) * hop + N + 5                               # a few samples past the last block
    rec = (rng.standard_normal((M, T)) + 1j * rng.standard_normal((M, T))).astype(np.complex64)
    out = torch.full((B, nblk * hop), complex(np.nan, np.nan), dtype=torch.complex64, device="cuda")
    plan.execute_stream(torch.from_numpy(rec).cuda(), T, hop, out, nblk)
    assert plan.sync_status() == 0
    got = out.cpu().numpy()
    ref = O.fbst_stream(pb, rec, hop, nblk)
    assert np.isfinite(got).all()
    assert O.rel_l2(got, ref) < 1e-5


def test_hop_n_equals_execute_on_cut_blocks(rng):
    plan, pb = _plan(24, 24, 64, 0.5)
    nblk, N = 5, 64
    rec = (rng.standard_normal((24, nblk * N)) + 1j * rng.standard_normal((24, nblk * N))).astype(np.complex64)
    out = torch.empty((24, nblk * N), dtype=torch.complex64, device="cuda")
    plan.execute_stream(torch.from_numpy(rec).cuda(), nblk * N, N, out, nblk)
    blocks = torch.from_numpy(np.ascontiguousarray(O.stream_blocks(rec, N, N, nblk))).cuda()
    ref = torch.empty((nblk, 24, N), dtype=torch.complex64, device="cuda")
    plan.execute(blocks, ref, nblk)
    torch.cuda.synchronize()
    assert torch.equal(out, ref.permute(1, 0, 2).reshape(24, nblk * N))     # bitwise: same kernels


def test_stream_invalid_arguments():
    import paper_2512_08887_gb300 as fb
    plan, pb = _plan(16, 16, 64, 0.5)
    rec = torch.zeros((16, 256), dtype=torch.complex64, device="cuda")
    out = torch.zeros((16, 256), dtype=torch.complex64, device="cuda")
    for T, hop, nblk in ((256, 33, 2), (256, 0, 2), (256, 66, 2), (100, 32, 3)):
        with pytest.raises(fb.FBSTError) as e:
            plan.execute_stream(rec, T, hop, out, nblk)
        assert e.value.status == -1
    plan.execute_stream(rec, 256, 32, out, 0)                 # an empty call is a no-op
    assert plan.sync_status() == 0
