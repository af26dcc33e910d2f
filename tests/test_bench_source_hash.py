"""CPU checks of the source hash that decides whether bench.py reports the committed ncu
DRAM traffic of the fused CG kernel: comments and blank lines do not change it, code
does, and string or character literals that contain comment markers are kept."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_comments_and_blank_lines_are_dropped():
    src = 'int a = 1;  // trailing\n\n/* block\n   over lines */\nint b = 2;\n'
    assert bench._code_only(src) == "int a = 1;\nint b = 2;"


def test_literals_keep_comment_markers_and_escapes():
    src = 'const char* s = "x // y /* z */";\nchar q = \'"\';\nconst char* e = "a\\"b // c";  // gone\n'
    out = bench._code_only(src)
    assert '"x // y /* z */"' in out
    assert "'\"'" in out
    assert '"a\\"b // c"' in out
    assert "gone" not in out


def test_code_change_changes_the_stripped_text():
    a = "int f(int x) { return x + 1; }  // one\n"
    b = "int f(int x) { return x + 2; }  // one\n"
    c = "int f(int x) { return x + 1; }  /* another comment */\n"
    assert bench._code_only(a) != bench._code_only(b)
    assert bench._code_only(a) == bench._code_only(c)


def test_committed_profile_names_a_hash_of_the_right_form():
    txt = open(os.path.join(ROOT, "profiles", "k_cg_mixed_five_cylinders.md")).read()
    line = [ln for ln in txt.splitlines() if ln.startswith("kernel_source_hash:")][0]
    h = line.split(":", 1)[1].strip()
    assert len(h) == 16 and all(ch in "0123456789abcdef" for ch in h)
    assert len(bench.kernel_source_hash()) == 16
