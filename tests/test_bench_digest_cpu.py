"""The kernel-source digest that gates the committed DRAM counters: it follows
the code of csrc/ and ignores comments."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_comments_do_not_change_the_code():
    a = 'int f(int x) {  // twice x\n/* block\n comment */\n    return 2 * x;\n}\n'
    b = 'int f(int x) {\n\n    return 2 * x;   \n}\n'
    assert bench.code_only(a) == bench.code_only(b)


def test_code_and_strings_change_it():
    base = 'asm volatile("mov.u32 %0, 1; // not a comment" : "=r"(v));\nint y = 2;\n'
    assert "// not a comment" in bench.code_only(base)
    assert bench.code_only(base) != bench.code_only(base.replace("2;", "3;"))


def test_digest_of_a_tree(tmp_path):
    (tmp_path / "k.cu").write_text("__global__ void k() {}\n")
    d1 = bench.source_digest(str(tmp_path))
    (tmp_path / "k.cu").write_text("// a note\n__global__ void k() {}\n")
    assert bench.source_digest(str(tmp_path)) == d1
    (tmp_path / "k.cu").write_text("__global__ void k() { int z = 0; }\n")
    assert bench.source_digest(str(tmp_path)) != d1
