"""Host-side pieces of bench.py's roofline: the byte models and the source hash
that keeps a recorded DRAM traffic figure tied to the sources it was taken on."""
import os
import shutil

import bench


def test_design_bytes_worked_example():
    # Batched form, width 128 (W = 4 mask words), FP32 theta, u32 path counts:
    #   10 scanned arcs x (4 + 6*4)   = 280
    #    3 entries      x (32 + 20*4) = 336
    #    5 DAG pairs    x (4 + 4)     =  40
    #    4 reached      x (2*4 + 4)   =  48
    #    7 vertices     x 8           =  56     -> 760
    st = {"scanned_arcs": 10, "entries": 3, "dag_arcs": 5, "reached": 4}
    assert bench.algorithmic_bytes(st, 7, "batched", 4, 128, sigma_bytes=4) == 760
    # Plain form (width 1: no mask words), FP64 theta, 8-byte path counts:
    #   10 x (4 + 4) + 3 x 32 + 5 x (8 + 8) + 4 x (16 + 8) + 56 = 80 + 96 + 80 + 96 + 56
    assert bench.algorithmic_bytes(st, 7, "plain", 8, 1) == 408


def test_pair_model_worked_example():
    # 4 B per scanned arc, (2 + 8 + 2 + theta) per traversed (arc, source),
    # 40 B per (vertex, batch slot) and batch.
    st = {"scanned_arcs": 10, "traversed_arcs": 100}
    assert bench.pair_model_bytes(st, 7, 4, 128, 2) == 40 + 100 * 16 + 7 * 128 * 2 * 40


def _fake_tree(root):
    csrc = root / "paper_2401_02472_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for name, text in [("bc_batched.cuh", "batched kernel"), ("bc_batched_w4.cu", "width 4"),
                       ("api.cu", "launch and tuners"), ("common.cuh", "shared device code"),
                       ("internal.h", "declarations"), ("graph.cu", "validation, workspace"),
                       ("bc_plain_kernel.cuh", "plain form"), ("bc_small.cu", "small form"),
                       ("server.cu", "serving loop"), ("notes.txt", "not a source")]:
        (csrc / name).write_text(text)
    return csrc


def test_source_hash_follows_the_measured_path(tmp_path, monkeypatch):
    # The recorded traffic is the batched kernel's: its sources and the host
    # code that shapes its launch enter the hash, the other forms, the
    # serving loop and non-source files do not.
    csrc = _fake_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    for name in ("bc_plain_kernel.cuh", "bc_small.cu", "server.cu", "notes.txt"):
        (csrc / name).write_text("edited")
    assert bench.kernel_source_hash() == h0
    for name in ("bc_batched.cuh", "bc_batched_w4.cu", "api.cu", "common.cuh", "internal.h", "graph.cu"):
        saved = (csrc / name).read_text()
        (csrc / name).write_text(saved + " ")
        assert bench.kernel_source_hash() != h0, name
        (csrc / name).write_text(saved)
        assert bench.kernel_source_hash() == h0
    # a new batched-path file changes it too
    (csrc / "bc_batched_w16.cu").write_text("width 16")
    assert bench.kernel_source_hash() != h0
    os.remove(csrc / "bc_batched_w16.cu")
    shutil.copy(str(csrc / "notes.txt"), str(csrc / "notes2.txt"))
    assert bench.kernel_source_hash() == h0
