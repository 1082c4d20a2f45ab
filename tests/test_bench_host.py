"""Host logic of the benchmark (no GPU): the hash that ties the committed
DRAM-traffic record to the kernel sources leaves comments out."""
import bench


def test_strip_comments_keeps_code_and_strings():
    src = 'a = "x // y"; // note\n/* block\n comment */ b = \'/\';\nasm("ld // in a string");'
    out = bench._strip_comments(src)
    assert '"x // y"' in out and "'/'" in out and '"ld // in a string"' in out
    assert "note" not in out and "block" not in out


def test_source_hash_ignores_comments_but_not_code():
    base = {f: "int f() { return 1; }\n" for f in bench.KERNEL_SOURCES}
    commented = {f: "// about f\nint f() { return 1; }  /* one */\n" for f in bench.KERNEL_SOURCES}
    changed = {f: "int f() { return 2; }\n" for f in bench.KERNEL_SOURCES}
    assert bench._source_hash(base) == bench._source_hash(commented)
    assert bench._source_hash(base) != bench._source_hash(changed)
