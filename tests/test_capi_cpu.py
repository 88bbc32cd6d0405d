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


def test_binding_precision_names_match_header_enum(tmp_path):
    # the binding's precision names carry the header's xlbomd_prec values
    import shutil
    import subprocess
    from paper_1705_10845_gb300 import binding
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    names = {"fp64": "XLBOMD_FP64", "fp16x3": "XLBOMD_FP16x3", "bf16x3": "XLBOMD_BF16x3", "tf32x3": "XLBOMD_TF32x3"}
    assert set(binding.PREC) == set(names)
    body = "".join(f'printf("{k} %d\\n", (int){v});' for k, v in names.items())
    src = tmp_path / "prec.c"
    src.write_text(f'#include <stdio.h>\n#include "xlbomd.h"\nint main(void) {{ {body} return 0; }}\n')
    exe = tmp_path / "prec"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    assert {k: int(v) for k, v in out.items()} == binding.PREC


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


BAD_PARAMS = [dict(mu_prec=2), dict(kernel_prec=-1), dict(graphs=2), dict(rank_m=9), dict(n_sq=0),
              dict(n_sq=41), dict(Te=0.0), dict(dt=0.0), dict(kernel_c=1.0), dict(mu_max_iter=0),
              dict(scf_mode=2), dict(kernel_mode=3), dict(kernel_every=-1), dict(rep_A=-1.0),
              dict(rep_rho=0.0), dict(prec=4), dict(prec=-1)]


@pytest.mark.parametrize("bad", BAD_PARAMS, ids=lambda d: "-".join(f"{k}={v}" for k, v in d.items()))
def test_init_rejects_bad_params_before_any_device_call(bad):
    # xlbomd_init validates every parameter on the host and returns ERR_ARG before it touches a
    # device, so these run without a GPU
    import numpy as np
    import paper_1705_10845_gb300 as X
    X.build.build()
    p = X.default_params(**bad)
    s = dict(natoms=2, L=12.0, R=np.array([[1.0, 1.0, 1.0], [2.4, 1.0, 1.0]]), V=np.zeros((2, 3)),
             Z=np.full(2, 4.0), mass=12.0)
    with pytest.raises(X.XlbomdError) as e:
        X.Context(p, [s])
    assert e.value.status == -1


@pytest.mark.parametrize("change", [dict(natoms=0), dict(L=4.0), dict(mass=0.0)],
                         ids=["natoms0", "box-inside-cutoff", "mass0"])
def test_init_rejects_bad_systems_before_any_device_call(change):
    import numpy as np
    import paper_1705_10845_gb300 as X
    X.build.build()
    s = dict(natoms=2, L=12.0, R=np.array([[1.0, 1.0, 1.0], [2.4, 1.0, 1.0]]), V=np.zeros((2, 3)),
             Z=np.full(2, 4.0), mass=12.0)
    s.update(change)
    with pytest.raises(X.XlbomdError) as e:
        X.Context(X.default_params(), [s])
    assert e.value.status == -1


C_CLIENT = r"""
#include <stdio.h>
#include "xlbomd.h"

int main(void) {
  xlbomd_params p;
  xlbomd_system s;
  xlbomd_ctx* ctx = (xlbomd_ctx*)&p;   /* must be overwritten with NULL on failure */
  const double R[6] = {1.0, 1.0, 1.0, 2.4, 1.0, 1.0}, V[6] = {0, 0, 0, 0, 0, 0}, Z[2] = {4.0, 4.0};
  xlbomd_default_params(&p);
  if (p.n_sq != 10 || p.kmax != 5 || p.rank_m != 2) return 1;
  if (xlbomd_table_i(&p, 6) != XLBOMD_OK || p.kmax != 6 || p.c[6] != 1.0 || p.kappa != 1.84) return 2;
  if (xlbomd_table_i(&p, 8) != XLBOMD_ERR_ARG) return 3;
  s.natoms = 2;
  s.box_L = 12.0;
  s.R = R;
  s.V = V;
  s.Z = Z;
  s.mass = 12.0;
  p.mu_prec = 2;                          /* out of range: refused on the host */
  if (xlbomd_init(&p, &s, 1, NULL, &ctx) != XLBOMD_ERR_ARG || ctx != NULL) return 4;
  if (xlbomd_init(NULL, &s, 1, NULL, &ctx) != XLBOMD_ERR_ARG) return 5;
  if (xlbomd_free(NULL) != XLBOMD_ERR_ARG) return 6;
  printf("ok %s\n", xlbomd_last_error(NULL));
  return 0;
}
"""


def test_c_client_links_and_calls_the_host_side_entry_points(tmp_path):
    # the boundary as a C user meets it: the header compiles as strict C99, the program links
    # against libxlbomd.so, and the calls that need no device behave as the header states
    import shutil
    import subprocess
    from paper_1705_10845_gb300 import build
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    libdir = os.path.dirname(build.build())
    src = tmp_path / "client.c"
    src.write_text(C_CLIENT)
    exe = tmp_path / "client"
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe), "-L", libdir, "-lxlbomd", f"-Wl,-rpath,{libdir}"], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, (out.returncode, out.stderr[-2000:])
    assert out.stdout.startswith("ok null context")
