"""Host logic of bench.py (no GPU): the kernel-source hash that ties the
committed ncu traffic figures to the code they were taken on."""
import os

import bench

HERE = os.path.dirname(os.path.abspath(__file__))


def test_comment_edits_keep_the_hash_and_code_edits_change_it():
    f = bench._code_without_comments
    src = ('int a = 1;  // Eq. 22\n/* block\n comment */ const char* s = "x//y /* z */";\n'
           "char q = '\\'';  asm volatile(\"mov.u32 %0, 1;\" : \"=r\"(a));\n")
    assert f(src) == f(src.replace("Eq. 22", "Eq. 23").replace("block", "other"))
    assert f(src) != f(src.replace("int a = 1", "int a = 2"))
    # literals survive whole, comments do not
    out = f(src)
    assert '"x//y /* z */"' in out and "'\\''" in out and "mov.u32" in out
    assert "Eq. 22" not in out and "block" not in out


def _fields(name):
    vals = {}
    with open(os.path.join(HERE, "..", "profiles", name)) as fh:
        for line in fh:
            if line.startswith("- ") and ":" in line:
                k, v = line[2:].split(":", 1)
                vals[k.strip()] = v.strip()
    return vals


def test_traffic_figure_is_reported_only_for_the_kernel_code_it_was_taken_on():
    # the sketch figure is what bench.py reports as roofline.traffic: the
    # committed one while its hash matches the current code, null otherwise
    sha = bench._kernel_source_sha("tc")
    f = _fields("tc_sketch_c4.md")
    got = bench._traffic_from_profiles("tc_sketch", "c4", sha)
    if f.get("kernel_source_sha") == sha:
        assert got == float(f["dram_bytes_per_launch"])
    else:
        assert got is None
    assert bench._traffic_from_profiles("tc_sketch", "c4", "0" * 16) is None
