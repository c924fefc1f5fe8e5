"""The C ABI library loads and exports every entry point include/*.h
declares; argument checks that need no GPU. No compute calls here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    inc = os.path.join(ROOT, "include")
    src = "\n".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*UST_API\s+(?:const\s+)?[a-z_0-9]+\s*\*?\s*(ust_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import paper_2006_13679_gb300 as pkg
    pkg.build()
    return pkg.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["ust_init", "ust_sample_aggregate", "ust_diag", "ust_free"]:
        assert required in names
    assert len(names) >= 14


def test_library_exports_every_declared_symbol(lib):
    from paper_2006_13679_gb300 import _binding
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in _binding.EXPORTS, name


def test_binding_structs_match_header_layout(lib):
    from paper_2006_13679_gb300 import _binding
    # ust_opts: 3 doubles, 9 int32 (+4 padding), pointer -> 3*8 + 9*4 + 4 + 8 = 72 bytes
    assert ctypes.sizeof(_binding.ust_opts) == 72
    assert ctypes.sizeof(_binding.ust_csr) == 32  # 2 int32, 2 pointers, int32 + padding
    o = _binding.default_opts()
    assert o.kappa == 0.3 and o.cg_tol == 1e-9 and o.skip_validation == 0


def test_init_rejects_bad_arguments_without_touching_the_gpu(lib):
    from paper_2006_13679_gb300 import _binding
    h = ctypes.c_void_p()
    g = _binding.ust_csr(n=1, nnz=0, row_ptr=None, col_idx=None, on_device=0)
    assert lib.ust_init(ctypes.byref(g), 0, None, ctypes.byref(h)) == _binding.UST_EINVAL
    assert h.value is None
    assert b"n >= 2" in lib.ust_last_error(None)
    assert lib.ust_strerror(-5) == b"UST_ETIMEOUT"
    lib.ust_free(None)
    assert lib.ust_tau(None, 0.3) == 0
    assert lib.ust_num_trees(None) == -1


def test_product_package_does_not_import_the_oracle():
    import subprocess
    import sys
    code = ("import sys, paper_2006_13679_gb300 as p; p.load(); "
            "assert 'oracle' not in sys.modules, 'product imported oracle'")
    subprocess.run([sys.executable, "-c", code], check=True, cwd=ROOT)
    # the CUDA sources never mention the oracle's C entry points
    csrc = os.path.join(ROOT, "paper_2006_13679_gb300", "csrc")
    for f in os.listdir(csrc):
        assert "orc_" not in open(os.path.join(csrc, f)).read(), f


def test_struct_layout_matches_a_c_compiler(tmp_path):
    """sizeof/offsetof of the ABI structs as gcc sees include/ust.h."""
    import shutil
    import subprocess
    from paper_2006_13679_gb300 import _binding
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stddef.h>\n#include <stdio.h>\n#include "ust.h"\n'
        'int main(void){printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(ust_csr), sizeof(ust_opts), sizeof(ust_info),'
        ' offsetof(ust_opts, stream), offsetof(ust_info, cg_relres), offsetof(ust_info, last_phase_cycles));'
        'return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(_binding.ust_csr), ctypes.sizeof(_binding.ust_opts), ctypes.sizeof(_binding.ust_info),
            _binding.ust_opts.stream.offset, _binding.ust_info.cg_relres.offset,
            _binding.ust_info.last_phase_cycles.offset]
    assert got == want
