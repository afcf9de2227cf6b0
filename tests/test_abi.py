"""Host-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every entry point include/gm.h declares; the Python mirror of
gm_config has the C layout; argument errors are reported without touching
the GPU."""
import ctypes as ct
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gm.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2007_12273_gb300 import build, gm
    build.build()
    return gm.load()


def declared_functions():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^(?:int|size_t|const char\*)\s+(gm_\w+)\s*\(", txt, re.M)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert {"gm_compress", "gm_reconstruct", "gm_moments"} <= set(names)
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (gm_\w+)", out))
    for n in names:
        assert n in exported, n
        assert hasattr(lib, n)


def test_config_layout_matches_header(tmp_path):
    from paper_2007_12273_gb300.gm import GMConfig
    src = tmp_path / "lay.c"
    src.write_text(
        '#include <stddef.h>\n#include <stdio.h>\n#include "gm.h"\n'
        "int main(void){printf(\"%zu\", sizeof(gm_config));"
        + "".join(f'printf(" %zu", offsetof(gm_config, {f}));' for f, _ in GMConfig._fields_)
        + "return 0;}\n")
    exe = tmp_path / "lay"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = [int(t) for t in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert vals[0] == ct.sizeof(GMConfig)
    assert vals[1:] == [getattr(GMConfig, f).offset for f, _ in GMConfig._fields_]


def test_argument_errors_without_gpu(lib):
    from paper_2007_12273_gb300 import gm
    cfg = gm.config(dict(D=2, Kmax=4, shape_order=2, L=1.0))
    rc = lib.gm_compress(ct.byref(cfg), 1, 1, None, None, None, 0, None, None, None, None, None,
                         None, None, None, None, None)
    assert rc == -1 and b"D must be 1 or 3" in lib.gm_last_error()
    cfg = gm.config(dict(D=1, Kmax=40, shape_order=2, L=1.0))
    rc = lib.gm_reconstruct(ct.byref(cfg), 1, None, None, None, None, 0, None, None, None, None,
                            None, None, None)
    assert rc == -1 and b"Kmax" in lib.gm_last_error()
    cfg = gm.config(dict(D=1, Kmax=4, shape_order=3, L=1.0))
    assert lib.gm_moments(ct.byref(cfg), 1, 1, None, None, None, 0, None, None, None, None,
                          None, None, None) == -1
    # launch options are checked before any device call
    cfg = gm.config(dict(D=1, Kmax=4, shape_order=2, L=1.0), precision=2)
    ptr = ct.c_void_p(16)  # never dereferenced: the call fails on the option
    args = (1, 1, ptr, None, ptr, 0, ptr, ptr, ptr, ptr, None, ptr, ptr, ptr, ptr, None)
    assert lib.gm_compress(ct.byref(cfg), *args) == -1
    assert b"precision" in lib.gm_last_error()
    cfg = gm.config(dict(D=1, Kmax=4, shape_order=2, L=1.0), threads_per_cell=96)
    assert lib.gm_compress(ct.byref(cfg), *args) == -1
    assert b"threads_per_cell" in lib.gm_last_error()
    cfg = gm.config(dict(D=1, Kmax=4, shape_order=2, L=1.0), smem_particles=1 << 20)
    assert lib.gm_compress(ct.byref(cfg), *args) == -1
    assert b"smem_particles" in lib.gm_last_error()
    # a zero charge makes the mass matrix zero: refused by both reconstructions
    cfg = gm.config(dict(D=1, Kmax=4, shape_order=2, L=1.0, q=0.0))
    rargs = (1, ptr, ptr, ptr, ptr, 1, ptr, ptr, ptr, ptr, ptr, None, None)
    assert lib.gm_reconstruct(ct.byref(cfg), *rargs) == -1
    assert b"q must be nonzero" in lib.gm_last_error()
    assert lib.gm_reconstruct_noalloc(ct.byref(cfg), *rargs) == -1
    assert b"q must be nonzero" in lib.gm_last_error()
    # empty problems are valid no-ops
    cfg = gm.config(dict(D=1, Kmax=4, shape_order=2, L=1.0))
    assert lib.gm_mixture_moments(ct.byref(cfg), 0, None, None, None, None, None, None, None,
                                  None) == 0


def test_noalloc_scratch_holds_its_cell_limit(lib):
    """The static scratch of gm_reconstruct_noalloc (40 MiB) holds the
    workspace of its advertised 32768-cell limit for D = 1 and D = 3
    (host-side layout arithmetic, no device access)."""
    assert lib.gm_noalloc_limits_ok() == 1


def test_mlp_struct_layout_matches_header(tmp_path):
    from paper_2007_12273_gb300.gm import GMMlp
    src = tmp_path / "lay2.c"
    fields = [f for f, _ in GMMlp._fields_]
    src.write_text(
        '#include <stddef.h>\n#include <stdio.h>\n#include "gm.h"\n'
        "int main(void){printf(\"%zu\", sizeof(gm_mlp));"
        + "".join(f'printf(" %zu", offsetof(gm_mlp, {f}));' for f in fields)
        + "return 0;}\n")
    exe = tmp_path / "lay2"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = [int(t) for t in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert vals[0] == ct.sizeof(GMMlp)
    assert vals[1:] == [getattr(GMMlp, f).offset for f in fields]


def test_binding_argument_counts_match_header(lib):
    """Every entry point the Python binding declares to ctypes takes as
    many arguments as include/gm.h gives it."""
    txt = open(HEADER).read()
    decls = re.findall(r"^(?:int|size_t|const char\*)\s+(gm_\w+)\s*\((.*?)\);", txt, re.M | re.S)
    checked = 0
    for name, args in decls:
        at = getattr(lib, name).argtypes
        if at is None:
            continue
        n = 0 if args.strip() in ("", "void") else len(args.split(","))
        assert len(at) == n, (name, len(at), n)
        checked += 1
    assert checked >= 20


@pytest.mark.parametrize("py,c", [("GMMesh2d", "gm_mesh2d"), ("GMStdOpts", "gm_std_opts")])
def test_small_struct_layouts_match_header(tmp_path, py, c):
    from paper_2007_12273_gb300 import gm
    cls = getattr(gm, py)
    fields = [f for f, _ in cls._fields_]
    src = tmp_path / f"{c}.c"
    src.write_text(
        '#include <stddef.h>\n#include <stdio.h>\n#include "gm.h"\n'
        f"int main(void){{printf(\"%zu\", sizeof({c}));"
        + "".join(f'printf(" %zu", offsetof({c}, {f}));' for f in fields)
        + "return 0;}\n")
    exe = tmp_path / c
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = [int(t) for t in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert vals[0] == ct.sizeof(cls)
    assert vals[1:] == [getattr(cls, f).offset for f in fields]


def test_mesh2d_argument_errors_without_gpu(lib):
    from paper_2007_12273_gb300 import gm
    cfg = gm.config(dict(D=3, Kmax=4, shape_order=2, L=1.0))
    assert lib.gm_deposit_2d(ct.byref(cfg), None, None, None, None, None, None, None) == -1
    assert b"mesh" in lib.gm_last_error()
    mesh = gm.GMMesh2d(0, 4, 1.0, 1.0)
    assert lib.gm_deposit_2d(ct.byref(cfg), ct.byref(mesh), None, None, None, None, None, None) == -1
    mesh = gm.GMMesh2d(4, 4, 1.0, -1.0)
    assert lib.gm_deposit_2d(ct.byref(cfg), ct.byref(mesh), None, None, None, None, None, None) == -1
    mesh = gm.GMMesh2d(4, 4, 1.0, 1.0)
    cfg0 = gm.config(dict(D=3, Kmax=4, shape_order=2, L=1.0, q=0.0))
    assert lib.gm_reconstruct_2d(ct.byref(cfg0), ct.byref(mesh), None, None, None, None, 0, None,
                                 None, None, None, None, None, None, None) == -1
    assert b"q must be nonzero" in lib.gm_last_error()


def test_every_declaration_cites_the_paper_and_its_errors():
    """Each entry point of include/gm.h is documented (its own comment, or
    the comment of the group it is declared in) with the passage of the
    paper it implements or the statement that the paper has none, and with
    its error behaviour."""
    txt = open(HEADER).read()
    decl = list(re.finditer(r"^(?:int|size_t|const char\*)\s+(gm_\w+)\s*\(", txt, re.M))
    cite = re.compile(r"Sec\.|eqs?\.|not in the paper|no counterpart|not part of the paper",
                      re.I)
    errs = re.compile(r"GM_ERR|GM_OK|error|Returns", re.I)
    prev_end, prev_doc = 0, ""
    for m in decl:
        chunk = txt[prev_end:m.start()]
        doc = " ".join(re.findall(r"/\*.*?\*/", chunk, re.S)) or prev_doc
        doc = re.sub(r"\s+", " ", re.sub(r"\n\s*\*(?!/)", " ", doc))  # join wrapped lines
        assert cite.search(doc), m.group(1)
        assert errs.search(doc), m.group(1)
        prev_end = txt.index(";", m.end()) + 1
        prev_doc = doc


@pytest.mark.parametrize("lang,std,comp", [("c", "c99", "gcc"), ("c++", "c++17", "g++")])
def test_header_is_self_contained(tmp_path, lang, std, comp):
    """include/gm.h compiles on its own (first include, no other headers)
    as strict C99 and as C++17, warnings as errors."""
    src = tmp_path / ("h.c" if lang == "c" else "h.cpp")
    src.write_text('#include "gm.h"\nint main(void) { return 0; }\n')
    r = subprocess.run([comp, f"-std={std}", "-Wall", "-Wextra", "-pedantic", "-Werror",
                        "-fsyntax-only", "-I", os.path.join(ROOT, "include"), str(src)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
