"""Host arithmetic of the benchmark line, on CPU: the algorithmic bytes per
cell each roofline fraction divides by, the launch count it claims, and the
consistency of the ncu tables it quotes traffic and instructions from."""
import re

import bench


def test_step_bytes_per_cell():
    # 2 (15 + 27) S populations + phi write; FP16S adds the h-shift read (4 B)
    # and the g-shift write and read (2 + 2 B)
    assert bench.step_kernel_bytes("fp64") == 2 * 42 * 8 + 8 == 680
    assert bench.step_kernel_bytes("fp32") == 2 * 42 * 4 + 4 == 340
    assert bench.step_kernel_bytes("fp16s") == 2 * 42 * 2 + 4 + 4 + 4 == 180
    # the D3Q27 phase field: 2 (27 + 27) S
    assert bench.step_kernel_bytes("fp32", qh=27) == 2 * 54 * 4 + 4 == 436
    assert bench.step_kernel_bytes("fp16s", qh=27) == 2 * 54 * 2 + 12 == 228
    # the whole step's ideal adds the phi read
    assert bench.ideal_step_bytes("fp32") == 344 and bench.ideal_step_bytes("fp16s") == 176


def test_launch_count():
    # graph replays of 32 steps plus one step-count kernel each
    assert bench.step_launches(100, 0) == 100 + 3 + 1
    assert bench.step_launches(64, 0) == 64 + 2
    assert bench.step_launches(5, 1) == 10


def test_mlups():
    assert bench.mlups(100_663_296, 100, 0.626) == 100_663_296 * 100 / 0.626 / 1e6


def test_ncu_tables_one_version_and_plausible():
    keys = set(bench.NCU_TRAFFIC) | set(bench.NCU_INST)
    versions = {k[2] for k in keys}
    assert len(versions) == 1 and all(re.fullmatch(r"[0-9a-f]{16}", v) for v in versions)
    assert re.fullmatch(r"[0-9a-f]{16}", bench.kernel_hash())
    cells = 512 * 384 * 512
    for (wl, prec, _), traffic in bench.NCU_TRAFFIC.items():
        assert wl == "drop_impact"
        per_cell = traffic / cells
        # DRAM bytes within a few per cent above the algorithmic bytes: no re-reads
        algo = bench.step_kernel_bytes(prec)
        assert algo * 0.97 <= per_cell <= algo * 1.06, (prec, per_cell, algo)
