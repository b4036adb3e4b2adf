"""FP64 CPU oracle of the fast broadband beamspace transform.

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by the CPU-baseline
leg of bench.py. The CUDA library and its Python binding never import it.

Parity status of each function is stated in fbst_oracle's docstrings; every function is pinned by
the tests in tests/test_oracle_pins.py except the size of the noise-free bias of a plane wave,
which the paper gives no number for ("parity unpinned": only a sanity bound is checked). The
beamspace interference nulling of Eq. (14) is pinned by tests/test_oracle_nulling.py, and the
non-uniform arrays of Sec. IX (make_problem(..., offsets=...)) by tests/test_oracle_nonuniform.py,
the off-grid beams of Sec. VIII-A by tests/test_oracle_offgrid.py, and the time-domain nulling of
Eq. (15) by tests/test_oracle_nulling_time.py.
"""
from .fbst_oracle import (  # noqa: F401
    Problem,
    Stage2Factors,
    make_problem,
    F_theta,
    F_u,
    stage1_time,
    stage1_space,
    fan_coefficients,
    gram,
    gram_direction,
    natural_spline_weights,
    interp_window,
    offgrid_terms,
    OffGridFactors,
    fbst_offgrid,
    stream_blocks,
    fbst_stream,
    fbst,
    dense_operator,
    cross_gram,
    cross_gram_direction,
    OffGridNullingFactors,
    fbst_nulled_offgrid,
    NullingFactors,
    fbst_nulled,
    F_u_interval,
    time_interval,
    TimeNullingFactors,
    fbst_nulled_time,
    lstsq_augmented,
    noise_power_trace,
    delay_and_sum_exact,
    delay_and_sum_exact_record,
    rel_l2,
)
