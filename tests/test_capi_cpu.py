"""Host-side checks of the C-ABI library (no GPU needed): it builds, loads and
exports every entry point that include/xlbomd.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "xlbomd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(xlbomd_[A-Za-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1705_10845_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("xlbomd_init", "xlbomd_build_H", "xlbomd_density", "xlbomd_response",
              "xlbomd_kernel_update", "xlbomd_step", "xlbomd_get", "xlbomd_free"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing


def test_default_params_are_the_reference_workload(lib):
    from paper_1705_10845_gb300 import binding
    p = binding.default_params()
    assert p.n_sq == 10 and p.Te == 1000.0 and p.kmax == 5 and p.rank_m == 2
    assert list(p.c)[:6] == [-6.0, 14.0, -8.0, -3.0, 4.0, -1.0]
    assert p.kappa == 1.82 and p.alpha == 0.018
    assert p.kernel_c == pytest.approx(1.0 - 1.0 / p.mix_alpha)


def test_binding_struct_layout_matches_header(tmp_path):
    # compile a probe against the header with the host C compiler and compare
    # every field offset of the two structs with the ctypes mirror
    import shutil
    import subprocess
    from paper_1705_10845_gb300 import binding
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "xlbomd.h"', 'int main(void) {']
    for struct, cname in ((binding.Params, "xlbomd_params"), (binding.System, "xlbomd_system")):
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in struct._fields_:
            lines.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    for struct, cname in ((binding.Params, "xlbomd_params"), (binding.System, "xlbomd_system")):
        assert int(out[cname]) == ctypes.sizeof(struct)
        for f, _ in struct._fields_:
            assert int(out[f"{cname}.{f}"]) == getattr(struct, f).offset, f


def test_table_i_rows_of_the_library_match_the_printed_table(golden):
    # host-only call: the library's Table I (kappa, alpha, c_k) against the values printed in
    # the paper (tests/golden/table_i.txt)
    import paper_1705_10845_gb300 as X
    X.build.build()
    for kmax, (kappa, alpha, c) in golden.table_i().items():
        p = X.default_params(kmax=kmax)
        assert p.kmax == kmax and p.kappa == kappa and p.alpha == alpha
        assert [p.c[k] for k in range(kmax + 1)] == [float(x) for x in c]
        assert all(p.c[k] == 0.0 for k in range(kmax + 1, 8))
    with pytest.raises(X.XlbomdError):
        X.default_params(kmax=8)
