"""Host-side pieces of bench.py that need no GPU: the kernel-source hash that
keys the stored DRAM-traffic record covers code only, so comment edits keep
the record and code edits drop it (the bench then reports traffic null)."""
import bench


def test_code_only_ignores_comments_and_blank_lines():
    a = "int f(int x) {\n  // one comment\n  return x + 1;  // trailing\n}\n\n/* block\n   comment */\n"
    b = "int f(int x) {\n  return x + 1;\n}\n"
    assert bench._code_only(a) == bench._code_only(b)


def test_code_only_sees_code_changes():
    a = "int f(int x) {\n  return x + 1;\n}\n"
    b = "int f(int x) {\n  return x + 2;\n}\n"
    assert bench._code_only(a) != bench._code_only(b)

