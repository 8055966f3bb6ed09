"""Host-side checks of bench.py that need no GPU.

The roofline's `traffic` comes from an ncu capture recorded with the source
key of the captured kernel; the key must change with any edit of the
kernel's code (the file or a header it includes) and must not change with
an edit of its comments or blank lines.
"""
import os
import shutil

import bench


def _copy_sources(tmp_path):
    src = os.path.join(bench.ROOT, "paper_2609_28519_gb300", "csrc")
    dst = tmp_path / "paper_2609_28519_gb300" / "csrc"
    dst.mkdir(parents=True)
    for names in bench.KERNEL_SOURCES.values():
        for name in names:
            shutil.copy(os.path.join(src, name), dst / name)
    return dst


def test_source_key_tracks_code_not_comments(tmp_path, monkeypatch):
    dst = _copy_sources(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    key = bench.source_key("k_fused<16,16,FWD,tiled>")
    assert key == bench.source_key("k_fused<16,16,INV,tiled>")  # one key per kernel family

    kernel = dst / "fp32_fused.cu"
    text = kernel.read_text()
    kernel.write_text("// a new comment line\n\n" + text.replace("{\n", "{  // trailing comment\n", 1))
    assert bench.source_key("k_fused<16,16,FWD,tiled>") == key

    kernel.write_text(text.replace("{\n", "{ (void)0;\n", 1))
    assert bench.source_key("k_fused<16,16,FWD,tiled>") != key

    kernel.write_text(text)
    header = dst / "dct_cores.cuh"
    header.write_text(header.read_text() + "\nstatic const int kProbe = 1;\n")
    assert bench.source_key("k_fused<16,16,FWD,tiled>") != key
    # the tensor-core kernel does not include the 1D cores
    tc = bench.source_key("k_tc_split<16,tiled>")
    header.write_text(header.read_text().replace("\nstatic const int kProbe = 1;\n", "\nstatic const int kProbe = 2;\n"))
    assert bench.source_key("k_tc_split<16,tiled>") == tc

