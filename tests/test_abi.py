"""The C-ABI library builds and exports every entry point declared in include/sg.h (no GPU
needed: nothing is called)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "sg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sg_[a-z_]+)\s*\(", src)))


def test_header_declares_entry_points():
    names = declared()
    for n in ("sg_setup", "sg_step", "sg_solve_batch", "sg_get_field", "sg_get_state", "sg_set_state",
              "sg_destroy", "sg_strerror"):
        assert n in names


def test_library_exports_all_declared_symbols():
    from paper_2512_23027_gb300 import build as b
    import ctypes
    path = b.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing
    lib.sg_strerror.restype = ctypes.c_char_p
    assert lib.sg_strerror(-4) == b"PCG did not converge within max_iter"


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2512_23027_gb300 import binding
    saved = binding._LIB
    binding._LIB = None
    try:
        with pytest.raises(RuntimeError):
            binding.load_library(str(tmp_path / "missing.so"))
    finally:
        binding._LIB = saved


def test_noalloc_capacity_is_the_header_constant():
    """The static staging array of sg_get_moments_noalloc is sized by the header's
    SG_NOALLOC_MAX_FREE (2^20 free nodes), which the library source does not redefine."""
    hdr = open(os.path.join(ROOT, "include", "sg.h")).read()
    m = re.search(r"#define\s+SG_NOALLOC_MAX_FREE\s+\(1 << (\d+)\)", hdr)
    assert m and int(m.group(1)) == 20
    src = open(os.path.join(ROOT, "paper_2512_23027_gb300", "csrc", "sg_cuda.cu")).read()
    assert "g_noalloc_stage[2 * (size_t)SG_NOALLOC_MAX_FREE]" in src
    assert not re.search(r"(constexpr|#define)\s+\w*\s*SG_NOALLOC_MAX_FREE", src)


def test_header_is_plain_c(tmp_path):
    """include/sg.h is a C header (C99, pedantic, no warnings): the boundary carries no C++ or torch types."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    src = tmp_path / "h.c"
    src.write_text('#include "sg.h"\nint main(void) { sg_mesh m; sg_mesh_plan p; sg_plan q; sg_sizes z;\n'
                   '  (void)m; (void)p; (void)q; (void)z; return 0; }\n')
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                        "-c", str(src), "-o", str(tmp_path / "h.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
