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
    for name, text in [("a.cu", "kernel a"), ("b.cuh", "kernel b"), ("c.h", "header"),
                       ("server.cu", "serving loop"), ("notes.txt", "not a source")]:
        (csrc / name).write_text(text)
    return csrc


def test_source_hash_follows_the_measured_path(tmp_path, monkeypatch):
    csrc = _fake_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    # the serving loop and non-source files do not enter the hash
    (csrc / "server.cu").write_text("serving loop, edited")
    (csrc / "notes.txt").write_text("edited")
    assert bench.kernel_source_hash() == h0
    # any kernel, header or launch source does
    for name in ("a.cu", "b.cuh", "c.h"):
        saved = (csrc / name).read_text()
        (csrc / name).write_text(saved + " ")
        assert bench.kernel_source_hash() != h0, name
        (csrc / name).write_text(saved)
        assert bench.kernel_source_hash() == h0
    # a renamed file changes it too
    shutil.move(str(csrc / "a.cu"), str(csrc / "a2.cu"))
    assert bench.kernel_source_hash() != h0
    assert os.path.exists(csrc / "a2.cu")
