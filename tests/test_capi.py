"""The C ABI library loads and exports every function include/cdl.h
declares (CPU only: nothing here launches a kernel)."""
import ctypes

import pytest

from paper_2501_13051_gb300 import build as B
from paper_2501_13051_gb300 import cdl


@pytest.fixture(scope="module")
def libcdl():
    B.build()
    return cdl.lib()


def test_header_declares_the_engine_and_step_calls():
    names = cdl.header_functions()
    for want in ("cdl_create", "cdl_destroy", "cdl_relation_create", "cdl_relation_load",
                 "cdl_rule_add", "cdl_run", "cdl_relation_size", "cdl_relation_export",
                 "cdl_last_error", "cdl_hash_build", "cdl_join_count", "cdl_exclusive_scan",
                 "cdl_join", "cdl_sort_unique", "cdl_diff_merge"):
        assert want in names


def test_every_declared_symbol_is_exported(libcdl):
    missing = [n for n in cdl.header_functions() if not hasattr(libcdl, n)]
    assert not missing, missing


def test_host_only_calls(libcdl):
    o = cdl.Options()
    libcdl.cdl_options_default(ctypes.byref(o))
    assert o.hash_load == 0.5 and o.radix_bits == 0 and o.max_iters == 0
    # 16-byte slots, power-of-two count, load factor respected
    for n, load in ((0, 0.5), (1, 0.5), (1000, 0.5), (1000, 0.8), (1 << 20, 0.5)):
        b = libcdl.cdl_hash_table_bytes(n, load)
        slots = b // 16
        assert b % 16 == 0 and slots & (slots - 1) == 0 and slots >= max(16, n / load)
    assert libcdl.cdl_last_error(None) == b"no engine"
    assert libcdl.cdl_create(None, None) == -1


def test_structs_match_header_sizes():
    # the ctypes mirrors must keep the header's field order and widths
    assert ctypes.sizeof(cdl.Term) == 8
    assert ctypes.sizeof(cdl.ColRef) == 8
    assert ctypes.sizeof(cdl.Atom) == 16
    assert ctypes.sizeof(cdl.Stats) == 8 * 17


def test_struct_sizes_equal_the_c_compilers(tmp_path):
    """sizeof of the ctypes mirrors equals sizeof in C for every struct of
    the boundary (a field added to the header but not to the binding, or in
    another order of widths, changes one of them)."""
    import os
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "sizes.c"
    src.write_text('#include <stdio.h>\n#include "cdl.h"\n'
                   "int main(void) { printf(\"%zu %zu %zu %zu %zu\\n\", sizeof(cdl_options), "
                   "sizeof(cdl_stats), sizeof(cdl_term), sizeof(cdl_atom), sizeof(cdl_rule)); "
                   "return 0; }\n")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    exe = tmp_path / "sizes"
    r = subprocess.run([cc, "-std=c99", "-I", inc, str(src), "-o", str(exe)], capture_output=True,
                       text=True)
    assert r.returncode == 0, r.stderr
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert got == [ctypes.sizeof(cdl.Options), ctypes.sizeof(cdl.Stats), ctypes.sizeof(cdl.Term),
                   ctypes.sizeof(cdl.Atom), ctypes.sizeof(cdl.RuleS)]


def test_field_offsets_equal_the_c_compilers(tmp_path):
    """Every field of the ctypes mirrors of cdl_options, cdl_stats and
    cdl_rule sits at the offset the C compiler gives the field of the same
    name in include/cdl.h (two fields of one width declared in swapped
    order keep the sizes equal but not the offsets)."""
    import os
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    mirrors = [("cdl_options", cdl.Options), ("cdl_stats", cdl.Stats), ("cdl_rule", cdl.RuleS),
               ("cdl_atom", cdl.Atom), ("cdl_term", cdl.Term)]
    lines = []
    want = []
    for cname, py in mirrors:
        for field in py._fields_:
            name = field[0]
            lines.append(f'  printf("%zu\\n", offsetof({cname}, {name}));')
            want.append((cname, name, getattr(py, name).offset))
    src = tmp_path / "offsets.c"
    src.write_text("#include <stddef.h>\n#include <stdio.h>\n#include \"cdl.h\"\n"
                   "int main(void) {\n" + "\n".join(lines) + "\n  return 0;\n}\n")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    exe = tmp_path / "offsets"
    r = subprocess.run([cc, "-std=c99", "-I", inc, str(src), "-o", str(exe)], capture_output=True,
                       text=True)
    assert r.returncode == 0, r.stderr
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert len(got) == len(want)
    for (cname, name, off), c_off in zip(want, got):
        assert off == c_off, (cname, name, off, c_off)


def test_header_is_plain_c(tmp_path):
    """include/cdl.h compiles as C99 (no C++ types in the boundary) and its
    declarations are usable from C."""
    import os
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_cdl.c"
    src.write_text(
        '#include "cdl.h"\n'
        "int main(void) {\n"
        "  cdl_options o;\n"
        "  cdl_options_default(&o);\n"
        "  cdl_engine* e = 0;\n"
        "  cdl_stats st = {0};\n"
        "  (void)st;\n"
        "  return cdl_create(&o, &e) == CDL_OK ? 0 : 1;\n"
        "}\n")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-fsyntax-only", "-I", inc, str(src)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_no_silent_fallback(monkeypatch, tmp_path):
    """The product path fails loudly: without the built library, and without
    a GPU (as in this container), nothing runs on the CPU instead."""
    monkeypatch.setattr(cdl, "_lib", None)
    monkeypatch.setattr(cdl, "LIB_PATH", str(tmp_path / "libcdl.so"))
    with pytest.raises(RuntimeError, match="missing"):
        cdl.lib()
    monkeypatch.undo()
    import torch
    if not torch.cuda.is_available():
        with pytest.raises(Exception):
            cdl.Engine()
