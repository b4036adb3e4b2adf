"""GB300 (sm_103a) fast broadband beamspace transform: CUDA library + thin Python binding."""
from ._native import (  # noqa: F401
    Allocator,
    FBSTError,
    Band,
    Batch,
    Geometry,
    Info,
    Nulling,
    Plan,
    STAGE2,
    STAGE2_NAMES,
    derive,
    fp32_fma_peak,
    load_library,
    make_band,
    make_geometry,
    torch_allocator,
)
