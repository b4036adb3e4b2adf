"""The four synthetic workloads (array, sizes, signal recipe, seed). Data only, no transform maths.

C1  linear array M=16, N=64, B=16, fb=0.5; K=3 plane waves, 20 dB; one block; seed 1001.
C2  linear array M=256, N=256, B=256, fb=0.5; K=8 plane waves, 10 dB; one continuous record cut
    into 64 blocks of 256 snapshots; seed 1002.
C3  32x32 rectangular array (M=1024), N=512, 32x32 beam grid (B=1024), fb=0.3; K=16 plane waves
    from the unit disk, 10 dB; nblk blocks of one record; seed 1003.
C4  64 independent linear arrays, M = 2^U{5..10}, N from {128,256,512,1024}, B=M, fb ~ U[0.2,0.6]
    rounded to 1e-3, K=4 plane waves, 15 dB, one block each, per-instance child seeds of 1004.
ULA1024 linear array M=1024, N=512, B=1024, fb=0.5 (L=1024); K=8 plane waves, 10 dB; one continuous
    record cut into 64 blocks of 512 snapshots; Q=64 sinusoids per waveform; seed 2024. The large
    array (M = B = 1024) at which the transform's roofline is stated.
NU1024 the ULA1024 signal on the same array with every element but the first moved by N(0, 0.2^2)
    half wavelengths along the axis (position seed 11): a non-uniform array (Sec. IX).
NUC3 the C3 signal on the same 32x32 array with every element but the first moved by N(0, 0.2^2)
    half wavelengths in both coordinates (position seed 12): a non-uniform rectangular array.
C2N the C2 array and grid with one unit-power source on grid beam 160 and two interferers on grid
    beams 64 and 96 at 20 dB above it, 10 dB SNR, 64 blocks; seed 1005. Workload of the beamspace
    interference nulling (Sec. VIII-B), which removes beams 64 and 96.
Every waveform is a sum of Q sinusoids with CN(0, 1/Q) weights and uniform in-band frequencies.
"""
from __future__ import annotations

from .planewave import interference_config, ula_config, ura_config, uneven_ula_instances

CONFIGS = {
    "C1": dict(kind="ula", mx=16, my=1, bx=16, by=1, N=64, frac_bw=0.5, K=3, snr_db=20.0, seed=1001, nblk=1),
    "C2": dict(kind="ula", mx=256, my=1, bx=256, by=1, N=256, frac_bw=0.5, K=8, snr_db=10.0, seed=1002, nblk=64),
    "C3": dict(kind="ura", mx=32, my=32, bx=32, by=32, N=512, frac_bw=0.3, K=16, snr_db=10.0, seed=1003, nblk=16),
    "ULA1024": dict(kind="ula", mx=1024, my=1, bx=1024, by=1, N=512, frac_bw=0.5, K=8, snr_db=10.0, seed=2024,
                    nblk=64, Q=64),
    "NU1024": dict(kind="ula", mx=1024, my=1, bx=1024, by=1, N=512, frac_bw=0.5, K=8, snr_db=10.0, seed=2024,
                   nblk=64, Q=64, sigma=0.2, pos_seed=11),
    "NUC3": dict(kind="ura", mx=32, my=32, bx=32, by=32, N=512, frac_bw=0.3, K=16, snr_db=10.0, seed=1003,
                 nblk=16, sigma=0.2, pos_seed=12),
}


def config_geometry(name: str):
    """The array of a workload: the grid, or for a non-uniform workload the perturbed positions."""
    from .planewave import ArrayGeometry, perturbed_geometry
    c = CONFIGS[name]
    if "sigma" in c:
        return perturbed_geometry(c["kind"], c["mx"], c["my"], c["sigma"], c["pos_seed"])
    return ArrayGeometry(c["kind"], c["mx"], c["my"])


def config_data(name: str, nblk: int | None = None, Q: int | None = None, first_block: int = 0) -> dict:
    """Generate the seeded data of C1..C3 and ULA1024 (nblk overrides the block count). A linear
    array's record may start at block `first_block` of the same continuous signal (a replica's share
    of the stream; the sources are the same, the noise of a later segment has its own seed)."""
    c = dict(CONFIGS[name])
    Q = Q if Q is not None else c.pop("Q", 256)
    c.pop("Q", None)
    if nblk is not None:
        c["nblk"] = nblk
    if c["kind"] == "ula":
        d = ula_config(c["mx"], c["N"], c["nblk"], c["frac_bw"], c["K"], c["snr_db"], c["seed"], Q=Q,
                       first_block=first_block, geom=config_geometry(name))
    else:
        d = ura_config(c["mx"], c["my"], c["N"], c["nblk"], c["frac_bw"], c["K"], c["snr_db"], c["seed"], Q=Q,
                       geom=config_geometry(name))
    d.update(c)
    return d


NULLING = {
    "C2N": dict(kind="ula", mx=256, my=1, bx=256, by=1, N=256, frac_bw=0.5, source_beams=[160],
                interferers=[64, 96], inr_db=20.0, snr_db=10.0, seed=1005, nblk=64),
}


def nulling_data(name: str, nblk: int | None = None, Q: int = 256) -> dict:
    """Seeded data of a nulling workload. Grid beam b of a linear array looks at u = -1 + 2b/B, so
    the sources and interferers sit exactly on grid beams."""
    c = dict(NULLING[name])
    if nblk is not None:
        c["nblk"] = nblk
    grid = lambda b: (-1.0 + 2.0 * b / c["bx"], 0.0)
    d = interference_config(c["kind"], c["mx"], c["my"], c["N"], c["nblk"], c["frac_bw"],
                            [grid(b) for b in c["source_beams"]], [grid(b) for b in c["interferers"]],
                            c["inr_db"], c["snr_db"], c["seed"], Q=Q)
    d.update(c)
    return d


def c4_instances(count: int = 64, with_data: bool = True) -> list[dict]:
    return uneven_ula_instances(1004, count=count, with_data=with_data)
