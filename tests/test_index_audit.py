"""The stream-collide kernels' addressing, audited on the host (lbm_debug_index_audit; no
GPU): for every computed cell, every gather must read the element the pull-stream
definition names (population i of the cell (x, y, z) - c_i: periodic by modulo, clamped at
open x ends, ghost rows beyond walls), every store the cell's own element, all inside the
buffer, the paired kernel's 32-bit accesses word-aligned.  It covers every lattice,
boundary, kernel variant and extents from 1 (modulo wrap) past the paired kernel's
256-cell blocks.  A wrong wrap threshold must be caught (the audit is not vacuous)."""
import pytest

from paper_1611_02409_gb300 import lbm as L

DIRECT, PAIRED, TWOPASS = 1, 3, 4


@pytest.fixture(scope="module")
def audit():
    L.lib()

    def run(lat, storage="fp32", walls=False, open_x=False, nx=8, ny=8, nz=1, variant=DIRECT, wrap=0):
        p = L.make_params(lattice=lat, storage=storage, nx=nx, ny=ny, nz=nz, bc_y=1 if walls else 0,
                          bc_x=2 if open_x else 0, tau=0.8)
        return L.lbm_debug_index_audit(p, variant, wrap)
    return run


@pytest.mark.parametrize("lat", [L.LBM_D2Q37, L.LBM_D2Q33, L.LBM_D2Q77])
@pytest.mark.parametrize("open_x", [False, True])
def test_2d_periodic_and_open(audit, lat, open_x):
    for storage in ("fp32", "fp16"):
        for nx in (1, 2, 3, 4, 5, 6, 7, 11, 12, 37, 262):
            for ny in (1, 2, 3, 4, 5, 6, 9):
                for v in (DIRECT, TWOPASS):
                    assert audit(lat, storage, False, open_x, nx, ny, 1, v) == 0, (storage, nx, ny, v)
                if lat == L.LBM_D2Q37 and storage != "fp32" and not open_x and nx % 2 == 0:
                    assert audit(lat, storage, False, False, nx, ny, 1, PAIRED) == 0, (nx, ny)


def test_2d_walls(audit):
    for storage in ("fp32", "bf16"):
        for nx in (1, 2, 3, 4, 6, 130, 520):
            for ny in (5, 6, 7, 23):
                for v in (DIRECT, TWOPASS):
                    assert audit(L.LBM_D2Q37, storage, True, False, nx, ny, 1, v) == 0, (storage, nx, ny, v)
                if storage != "fp32" and nx % 2 == 0:
                    assert audit(L.LBM_D2Q37, storage, True, False, nx, ny, 1, PAIRED) == 0, (nx, ny)


@pytest.mark.parametrize("walls", [False, True])
def test_3d(audit, walls):
    for nx, ny, nz in ((1, 5, 1), (2, 6, 3), (3, 7, 4), (5, 9, 5), (8, 8, 8)):
        for v in (DIRECT, TWOPASS):
            assert audit(L.LBM_D3Q103, "fp32", walls, False, nx, ny, nz, v) == 0, (nx, ny, nz, v)


def test_staged_kernel_copies(audit):
    # the staged kernel's bulk copies (in the buffer, 16-byte aligned at both ends, sizes
    # multiples of 16) and its shared-memory reads against the definition
    for storage in ("fp32", "fp16", "bf16"):
        for walls in (False, True):
            for nx in (128, 256, 384):
                for ny in ((5, 6, 9) if walls else (1, 2, 3, 4, 9)):
                    assert audit(L.LBM_D2Q37, storage, walls, False, nx, ny, 1, L.LBM_KERNEL_STAGED) == 0
    with pytest.raises(L.LbmError):
        audit(L.LBM_D2Q37, "fp32", nx=130, variant=L.LBM_KERNEL_STAGED)   # nx not a multiple of 128


def test_batched_step(audit):
    # one instance of the batched step (D2Q37, FP32): same definition, 32-bit offsets
    for walls in (False, True):
        for nx in (1, 2, 3, 4, 5, 64, 130):
            for ny in ((5, 6, 9, 64) if walls else (1, 2, 3, 4, 5, 64)):
                assert audit(L.LBM_D2Q37, "fp32", walls, False, nx, ny, 1, L.LBM_AUDIT_BATCH) == 0, (walls, nx, ny)
    # the largest instance lbm_batch_create admits (29,020,049 cells per plane) still fits
    assert audit(L.LBM_D2Q37, "fp32", False, False, 29020049, 1, 1, L.LBM_AUDIT_BATCH) == 0
    with pytest.raises(L.LbmError):                          # one cell more does not
        audit(L.LBM_D2Q37, "fp32", False, False, 450, 64489, 1, L.LBM_AUDIT_BATCH)


def test_wrong_wrap_threshold_is_caught(audit):
    # one add cannot wrap x - 5 into [0, 4): with threshold 4 (reach-3 lattices' value) an
    # extent-4 D2Q77 row would read the neighbouring row's cells; the launch uses 5
    assert audit(L.LBM_D2Q77, nx=4, ny=6, variant=TWOPASS) == 0
    assert audit(L.LBM_D2Q77, nx=4, ny=6, variant=TWOPASS, wrap=4) > 0
    assert audit(L.LBM_D2Q77, nx=4, ny=6, variant=DIRECT, wrap=4) > 0
    assert audit(L.LBM_D2Q37, nx=2, ny=6, variant=DIRECT, wrap=1) > 0


def test_inadmissible_variants_rejected(audit):
    with pytest.raises(L.LbmError):
        audit(L.LBM_D2Q37, "fp32", nx=8, variant=PAIRED)        # paired needs 16-bit storage
    with pytest.raises(L.LbmError):
        audit(L.LBM_D2Q37, "fp16", nx=7, variant=PAIRED)        # ... and an even row
    with pytest.raises(L.LbmError):
        audit(L.LBM_D2Q77, walls=True, ny=16)                   # no walls on D2Q77


def test_fp64_storage_two_pass(audit):
    # FP64 storage (8-byte values, two-pass kernel only): the byte offsets of the stores
    # are tabulated at 8 bytes per value; the other variants are refused
    for walls in (False, True):
        for nx in (1, 2, 3, 4, 6, 37):
            for ny in ((5, 6, 9) if walls else (1, 2, 3, 4, 9)):
                assert audit(L.LBM_D2Q37, "fp64", walls, False, nx, ny, 1, TWOPASS) == 0, (walls, nx, ny)
        for nx, ny, nz in ((1, 5, 1), (3, 7, 4), (8, 8, 8)):
            assert audit(L.LBM_D3Q103, "fp64", walls, False, nx, ny, nz, TWOPASS) == 0, (walls, nx, ny, nz)
    for v in (DIRECT, PAIRED, L.LBM_KERNEL_STAGED):
        with pytest.raises(L.LbmError):
            audit(L.LBM_D2Q37, "fp64", nx=128, variant=v)
    with pytest.raises(L.LbmError):
        audit(L.LBM_D2Q33, "fp64", nx=8, variant=TWOPASS)     # FP64 storage: D2Q37 and D3Q103

