"""The C-ABI library builds for sm_103a, loads, and exports every function include/citron.h
declares; host-side argument checks answer without touching a GPU."""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent
HEADER = ROOT / "include" / "citron.h"


def declared_functions():
    text = HEADER.read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(citron_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def built():
    from paper_2112_10913_gb300 import build

    return build.build()


def test_header_lists_the_binding_exports():
    import paper_2112_10913_gb300 as cg

    assert declared_functions() == sorted(cg.EXPORTS)


def test_library_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(str(built))
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_status_strings_and_version(built):
    import paper_2112_10913_gb300 as cg

    L = cg.lib()
    for code in range(7):
        assert L.citron_status_str(code)
    assert L.citron_version() >= 100


def test_argument_checks_need_no_gpu(built):
    import paper_2112_10913_gb300 as cg

    L = cg.lib()
    out = ctypes.c_uint64(0)
    null = ctypes.c_void_p(0)
    # k = 0 is invalid; k above the compiled maximum is unsupported; missing output is invalid
    assert L.citron_count(10, ctypes.c_void_p(1), ctypes.c_void_p(1), 0, 0, ctypes.byref(out), null, null, 0, null) == 1
    assert L.citron_count(10, ctypes.c_void_p(1), ctypes.c_void_p(1), 13, 0, ctypes.byref(out), null, null, 0, null) == 6
    assert L.citron_count(10, ctypes.c_void_p(1), ctypes.c_void_p(1), 3, 0, null, null, null, 0, null) == 1
    # citron_count_ex: options are required; thresholds are range-checked
    o = cg.CountOpts(40, 0, 0, 0, 0, 0, None, 0)
    assert L.citron_count_ex(10, ctypes.c_void_p(1), ctypes.c_void_p(1), 3, 0, null, ctypes.byref(out), null, 0, null) == 1
    assert L.citron_count_ex(10, ctypes.c_void_p(1), ctypes.c_void_p(1), 3, 0, ctypes.byref(o), ctypes.byref(out), null, 0, null) == 1
    o = cg.CountOpts(0, 0, 0, 0, 100, 0, None, 0)  # compact_max must be 0, 1, 128 or 256
    assert L.citron_count_ex(10, ctypes.c_void_p(1), ctypes.c_void_p(1), 3, 0, ctypes.byref(o), ctypes.byref(out), null, 0, null) == 1
    assert L.citron_kernel_launches() == 0
    # no workspace
    assert L.citron_order(10, ctypes.c_void_p(1), ctypes.c_void_p(1), null, null, 0, null) == 2
    # odd arc count cannot be a symmetric CSR
    assert L.citron_build_dag(4, 3, ctypes.c_void_p(1), ctypes.c_void_p(1), null, ctypes.c_void_p(1),
                              ctypes.c_void_p(1), null, null, 0, null) == 1
    # n = 2^32 - 1 is reserved
    assert L.citron_validate(0xFFFFFFFF, 0, ctypes.c_void_p(1), null, null, null, 0, null) == 1
    # core ordering: odd arc count, missing rank, missing workspace
    one = ctypes.c_void_p(1)
    assert L.citron_core_order(4, 3, one, one, one, null, null, null, null, 0, null) == 1
    assert L.citron_core_order(4, 4, one, one, null, null, null, null, null, 0, null) == 1
    assert L.citron_core_order(4, 4, one, one, one, null, null, null, null, 0, null) == 2


def test_workspace_size_grows_with_graph(built):
    import paper_2112_10913_gb300 as cg

    a = cg.citron_workspace_bytes(1000, 20000, 100)
    b = cg.citron_workspace_bytes(100000, 2000000, 100)
    assert 0 < a < b
    # above the bitmap limit the sorted-list scratch is added
    assert cg.citron_workspace_bytes(1000, 20000, 5000) > a


def test_plain_c_caller_links_and_runs(built, tmp_path):
    """A plain C program (no C++, no torch) includes the header, links libcitron.so and gets
    answers that need no GPU: the version, status strings, workspace sizes, argument checks."""
    import shutil
    import subprocess

    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    src = tmp_path / "caller.c"
    src.write_text(r"""
#include <stdio.h>
#include <string.h>
#include "citron.h"
int main(void) {
    uint64_t count = 0;
    if (citron_version() < 100) return 1;
    if (strcmp(citron_status_str(CITRON_OK), "ok") != 0) return 2;
    if (citron_workspace_bytes(1000, 20000, 100) == 0) return 3;
    /* k = 0 is invalid before any device work */
    if (citron_count(10, (const uint64_t *)1, (const uint32_t *)1, 0, 0, &count, NULL, NULL, 0, NULL)
        != CITRON_E_INVALID) return 4;
    printf("ok %d\n", citron_version());
    return 0;
}
""")
    exe = tmp_path / "caller"
    lib_dir = Path(built).parent
    subprocess.run(["gcc", "-std=c99", "-Wall", f"-I{ROOT / 'include'}", str(src), "-o", str(exe),
                    f"-L{lib_dir}", "-lcitron", f"-Wl,-rpath,{lib_dir}"], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stderr
    assert out.stdout.startswith("ok ")


def test_python_mirrors_match_the_c_layout(tmp_path):
    """The binding's ctypes mirrors of citron_count_opts and citron_faults have the C header's
    field offsets and size (compiled with the host C compiler; no GPU)."""
    import shutil
    import subprocess

    import paper_2112_10913_gb300 as cg

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    structs = {"citron_count_opts": cg.CountOpts, "citron_faults": cg.Faults}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "citron.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", f"-I{ROOT / 'include'}", str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            parts = line.split()
            got[(parts[0], parts[1])] = int(parts[2])
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_debug_modes_k_range(built):
    import paper_2112_10913_gb300 as cg

    L = cg.lib()
    out = ctypes.c_uint64(0)
    null = ctypes.c_void_p(0)
    o = cg.CountOpts(0, 0, 0, 0, 0, 0, None, 0)
    o.d_per_arc = 1  # any non-NULL pointer: the check comes before any device access
    assert L.citron_count_ex(10, ctypes.c_void_p(1), ctypes.c_void_p(1), 2, 0, ctypes.byref(o),
                             ctypes.byref(out), null, 0, null) == 1
    # the instrumented kernel behind the debug modes is built for k <= 8
    assert L.citron_count_ex(10, ctypes.c_void_p(1), ctypes.c_void_p(1), 9, 0, ctypes.byref(o),
                             ctypes.byref(out), null, 0, null) == 6
    o.d_per_arc = None
    o.flags = cg.COUNT_WORK
    assert L.citron_count_ex(10, ctypes.c_void_p(1), ctypes.c_void_p(1), 12, 0, ctypes.byref(o),
                             ctypes.byref(out), null, 0, null) == 6
