"""The C ABI library builds, loads without a GPU and exports every entry
point that include/md.h declares; host-side validation paths that need no
device work."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "md.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(md_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1009_4330_gb300 import _build, _lib
    _build.build()
    return _lib.load(build_if_missing=False)


def test_header_declares_the_path_entry_points():
    names = declared_functions()
    for core in ("md_create", "md_build_neighbors", "md_compute_forces", "md_step", "md_energy_virial"):
        assert core in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1009_4330_gb300 import _lib
    names = declared_functions()
    assert sorted(_lib.EXPORTS) == names
    for name in names:
        assert hasattr(lib, name), name


def test_struct_layout_matches_header():
    # md_config: 16 fields, pointer-aligned; the ctypes mirror must have the C size
    from paper_1009_4330_gb300 import _lib
    assert ctypes.sizeof(_lib.MdConfig) == 128
    assert ctypes.sizeof(_lib.MdInfo) == 88


def test_null_arguments_are_rejected_without_device_work(lib):
    from paper_1009_4330_gb300 import _lib
    h = ctypes.c_void_p()
    assert lib.md_create(None, None, None, None, ctypes.byref(h)) == _lib.MD_ERR_INVALID
    assert b"null" in lib.md_last_error(None)
    assert lib.md_step(None, 1) == _lib.MD_ERR_INVALID
    assert lib.md_destroy(None) == _lib.MD_OK


def test_box_precondition_checked_on_host(lib):
    from paper_1009_4330_gb300 import _lib
    import numpy as np
    p = np.array([1.0, 1.0])
    m = np.array([1.0])
    cfg = _lib.MdConfig()
    cfg.n_atoms = 10
    cfg.n_types = 1
    for k in range(3):
        cfg.box[k] = 5.0  # < 2 * (2.5 + 0.3)
    cfg.pot = _lib.MD_POT_LJ
    cfg.params = p.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    cfg.n_params = 2
    cfg.cutoff, cfg.skin, cfg.dt = 2.5, 0.3, 0.005
    cfg.mass = m.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    cfg.ftm2v = 1.0
    cfg.prec = _lib.MD_PREC_MIXED
    cfg.list = _lib.MD_LIST_FULL
    cfg.tpa = 1
    dummy = ctypes.c_void_p(16)  # never dereferenced: the config is rejected first
    h = ctypes.c_void_p()
    assert lib.md_create(ctypes.byref(cfg), dummy, dummy, dummy, ctypes.byref(h)) == _lib.MD_ERR_BOX_TOO_SMALL
    for k in range(3):
        cfg.box[k] = 20.0
    cfg.tpa = 3
    assert lib.md_create(ctypes.byref(cfg), dummy, dummy, dummy, ctypes.byref(h)) == _lib.MD_ERR_INVALID
    cfg.tpa = 1
    cfg.n_params = 3
    assert lib.md_create(ctypes.byref(cfg), dummy, dummy, dummy, ctypes.byref(h)) == _lib.MD_ERR_INVALID


def test_product_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1009_4330_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "liboracle" not in text, f


def test_ctypes_mirrors_match_the_c_header(tmp_path):
    # compile a probe against include/md.h and compare sizes and field offsets
    import shutil
    import subprocess
    from paper_1009_4330_gb300 import _lib
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    fields = [f for f, _ in _lib.MdInfo._fields_]
    src = tmp_path / "probe.c"
    src.write_text("#include <stdio.h>\n#include <stddef.h>\n#include \"md.h\"\nint main(void) {\n"
                   "  printf(\"%zu %zu\\n\", sizeof(md_config), sizeof(md_info_t));\n"
                   + "".join(f"  printf(\"%zu\\n\", offsetof(md_info_t, {f}));\n" for f in fields)
                   + "  return 0;\n}\n")
    exe = tmp_path / "probe"
    subprocess.check_call([cc, "-I", inc, str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)], text=True).split()
    assert int(out[0]) == ctypes.sizeof(_lib.MdConfig)
    assert int(out[1]) == ctypes.sizeof(_lib.MdInfo)
    for f, off in zip(fields, out[2:]):
        assert int(off) == getattr(_lib.MdInfo, f).offset, f
    # the other structs of the header
    src2 = tmp_path / "probe2.c"
    src2.write_text("#include <stdio.h>\n#include <stddef.h>\n#include \"md.h\"\nint main(void) {\n"
                    "  printf(\"%zu %zu %zu\\n\", sizeof(md_tune_row), offsetof(md_tune_row, ms), sizeof(md_ceilings));\n"
                    "  return 0;\n}\n")
    exe2 = tmp_path / "probe2"
    subprocess.check_call([cc, "-I", inc, str(src2), "-o", str(exe2)])
    a, b, c = (int(t) for t in subprocess.check_output([str(exe2)], text=True).split())
    assert a == ctypes.sizeof(_lib.MdTuneRow) and b == _lib.MdTuneRow.ms.offset
    assert c == ctypes.sizeof(_lib.MdCeilings)


def test_every_entry_point_cites_its_passage():
    # each declaration's comment block names the paper passage that defines the
    # operation, or says that no passage does (plumbing, measurement, tests)
    src = open(HEADER).read()
    decls = [m for m in re.finditer(r"^(?:md_status|const char \*)\s*(md_[a-z_0-9]+)\s*\(", src, flags=re.M)]
    prev = 0
    for m in decls:
        block = src[prev:m.start()]
        assert "Cite:" in block, m.group(1)
        prev = m.end()


def test_empty_and_oversized_systems_rejected_on_host(lib):
    # no atoms, and more atoms than the 26-bit list entries can name: refused
    # before any device allocation
    from paper_1009_4330_gb300 import _lib
    import numpy as np
    p = np.array([1.0, 1.0])
    m = np.array([1.0])
    cfg = _lib.MdConfig()
    cfg.n_types = 1
    for k in range(3):
        cfg.box[k] = 1000.0
    cfg.pot = _lib.MD_POT_LJ
    cfg.params = p.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    cfg.n_params = 2
    cfg.cutoff, cfg.skin, cfg.dt = 2.5, 0.3, 0.005
    cfg.mass = m.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    cfg.ftm2v = 1.0
    cfg.prec = _lib.MD_PREC_MIXED
    cfg.list = _lib.MD_LIST_FULL
    cfg.tpa = 1
    dummy = ctypes.c_void_p(16)  # never dereferenced
    h = ctypes.c_void_p()
    cfg.n_atoms = 0
    assert lib.md_create(ctypes.byref(cfg), dummy, dummy, dummy, ctypes.byref(h)) == _lib.MD_ERR_INVALID
    cfg.n_atoms = (1 << 26) + 1
    assert lib.md_create(ctypes.byref(cfg), dummy, dummy, dummy, ctypes.byref(h)) == _lib.MD_ERR_UNSUPPORTED
    assert not h.value
