"""The C ABI library builds for sm_103a, loads without a GPU, and exports every
function that include/fim.h declares.  No compute call is made here."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

from paper_2108_05038_gb300 import _build, fim

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    text = open(os.path.join(ROOT, "include", "fim.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fim_[a-z0-9_]+)\s*\(", text)))


def test_header_parsed():
    names = header_functions()
    assert "fim_mine" in names and "fim_build_vertical_db" in names and "fim_estimate_class_costs" in names


def test_library_builds_and_exports_header_symbols():
    path = _build.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    for name in header_functions():
        assert hasattr(lib, name), f"{name} declared in include/fim.h but not exported"
    assert sorted(fim.EXPORTED) == header_functions()


def test_status_strings_without_gpu():
    lib = fim.load()
    assert lib.fim_status_str(0) == b"FIM_OK"
    assert lib.fim_status_str(3) == b"FIM_ERR_OUTPUT_OVERFLOW"
    assert lib.fim_last_error() == b""


def test_launch_counter_starts_at_zero_without_gpu():
    """No kernel has been launched by a CPU-only process (failed calls launch nothing)."""
    lib = fim.load()
    lib.fim_build_vertical_db(None, None, 0, 1, 64, 0, None, None)
    assert fim.kernel_launches() == 0


def test_opts_struct_layout_matches_header():
    lib = fim.load()
    o = fim.MineOpts()
    lib.fim_mine_opts_init(ctypes.byref(o))
    assert o.struct_size == ctypes.sizeof(fim.MineOpts)
    assert o.donate == 0 and o.class_order == fim.FIM_ORDER_ESTIMATE and o.dfs_mode == fim.FIM_DFS_AUTO
    assert o.threads_per_cta == 0 and o.vec_per_lane == 0


@pytest.mark.parametrize("cname,pycls", [("fim_mine_stats", "MineStats"), ("fim_mine_opts", "MineOpts")])
def test_struct_offsets_match_header(cname, pycls, tmp_path):
    """Field offsets and sizes of the ctypes mirrors equal what a C compiler makes of include/fim.h."""
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    cls = getattr(fim, pycls)
    fields = [f for f, _ in cls._fields_]
    src = tmp_path / "layout.c"
    lines = ["#include <stdio.h>", "#include <stddef.h>", f'#include "{os.path.join(ROOT, "include", "fim.h")}"',
             "int main(void) {", f'  printf("size %zu\\n", sizeof({cname}));']
    lines += [f'  printf("{f} %zu\\n", offsetof({cname}, {f}));' for f in fields]
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-o", str(exe), str(src)])
    got = dict(line.split() for line in subprocess.check_output([str(exe)], text=True).splitlines())
    assert int(got["size"]) == ctypes.sizeof(cls)
    for f in fields:
        assert int(got[f]) == getattr(cls, f).offset, f


def test_invalid_arguments_rejected_without_gpu():
    lib = fim.load()
    h = ctypes.c_void_p()
    # NULL offsets, D == 0 and bad word size are rejected before any device call
    assert lib.fim_build_vertical_db(None, None, 0, 10, 64, 0, None, ctypes.byref(h)) == fim.FIM_ERR_INVALID
    assert b"D == 0" in lib.fim_last_error()
    off = (ctypes.c_uint32 * 2)(0, 0)
    assert lib.fim_build_vertical_db(off, None, 1, 10, 16, 0, None, ctypes.byref(h)) == fim.FIM_ERR_INVALID
    assert lib.fim_mine(None, 5, None, ctypes.byref(h)) == fim.FIM_ERR_INVALID
    assert lib.fim_estimate_class_costs(None, 0.01, 0.1, 1, None, None) == fim.FIM_ERR_INVALID


def test_no_oracle_import_in_product_path():
    """The GPU package never imports the oracle (parity would be void otherwise)."""
    pkg = os.path.join(ROOT, "paper_2108_05038_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".c", ".h")):
                text = open(os.path.join(dirpath, f), errors="replace").read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "fim_oracle" not in text, f


_SCALARS = {"uint8_t": ctypes.c_uint8, "uint32_t": ctypes.c_uint32, "uint64_t": ctypes.c_uint64,
            "int": ctypes.c_int, "fim_status": ctypes.c_int, "double": ctypes.c_double, "float": ctypes.c_float}
_STRUCTS = {"fim_mine_opts": "MineOpts", "fim_mine_stats": "MineStats"}


def header_prototypes():
    """(return type, name, [(base type, pointer depth)]) of every function declared in include/fim.h."""
    text = open(os.path.join(ROOT, "include", "fim.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = []
    for m in re.finditer(r"([A-Za-z_][\w\s\*]*?)\b(fim_[a-z0-9_]+)\s*\(([^)]*)\)\s*;", text):
        params = []
        for p in m.group(3).split(","):
            p = " ".join(p.replace("const", " ").split())
            if p in ("", "void"):
                continue
            depth = p.count("*")
            base = p.replace("*", " ").split()[0]
            params.append((base, depth))
        out.append((" ".join(m.group(1).split()), m.group(2), params))
    return out


def _matches(ct, base, depth):
    if depth == 0:
        return ct is _SCALARS[base]
    if ct in (ctypes.c_void_p, ctypes.c_char_p):
        return True  # an untyped pointer: buffers, opaque handles, the caller's stream
    target = getattr(ct, "_type_", None)
    if target is None:
        return False
    if depth >= 2:
        return target is ctypes.c_void_p  # out-pointer to a handle or a buffer address
    if base in _SCALARS:
        return target is _SCALARS[base]
    return base in _STRUCTS and target is getattr(fim, _STRUCTS[base])


def test_ctypes_signatures_match_header():
    """Every entry point's argument and return types in the binding agree with its prototype in
    include/fim.h: the same count, the same scalar widths, pointers where the header has pointers."""
    lib = fim.load()
    protos = header_prototypes()
    assert sorted(name for _, name, _ in protos) == header_functions()
    rets = {"fim_status": ctypes.c_int, "void": None, "const char*": ctypes.c_char_p, "uint64_t": ctypes.c_uint64}
    for ret, name, params in protos:
        f = getattr(lib, name)
        assert f.restype is rets[ret], name
        assert f.argtypes is not None and len(f.argtypes) == len(params), name
        for k, (ct, (base, depth)) in enumerate(zip(f.argtypes, params)):
            assert _matches(ct, base, depth), f"{name} argument {k}: {ct} for {base}{'*' * depth}"


def test_plain_c_program_links_and_calls_without_gpu(tmp_path):
    """The library is usable from plain C through include/fim.h alone: a C11 program links against it
    and makes the calls that need no device (option defaults, argument errors, status strings)."""
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    lib_path = _build.build()
    src = tmp_path / "use_abi.c"
    src.write_text(r'''
#include <stdio.h>
#include <string.h>
#include "fim.h"
int main(void) {
  fim_mine_opts o;
  fim_mine_opts_init(&o);
  if (o.struct_size != sizeof(fim_mine_opts) || o.class_order != FIM_ORDER_ESTIMATE) return 1;
  fim_db* db = (fim_db*)0;
  if (fim_build_vertical_db(NULL, NULL, 0, 10, 64, 0, NULL, &db) != FIM_ERR_INVALID || db) return 2;
  if (!strstr(fim_last_error(), "D == 0")) return 3;
  fim_result* r = (fim_result*)0;
  if (fim_mine(NULL, 5, &o, &r) != FIM_ERR_INVALID || r) return 4;
  if (strcmp(fim_status_str(FIM_ERR_TIMEOUT), "FIM_ERR_TIMEOUT") != 0) return 5;
  if (fim_kernel_launches() != 0) return 6;
  fim_db_free(NULL);
  fim_result_free(NULL);
  puts("ok");
  return 0;
}
''')
    exe = tmp_path / "use_abi"
    libdir = os.path.dirname(lib_path)
    subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                           "-o", str(exe), lib_path, f"-Wl,-rpath,{libdir}"])
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.returncode, r.stdout, r.stderr)


def test_stored_expected_values_come_from_the_oracle_only():
    """The script that writes tests/golden/digests.json imports the oracle, the input generator and the
    canonical-form helper, and nothing of the CUDA path (no expected value comes from the GPU)."""
    import ast

    for rel in ("tests/golden/make_digests.py", "tests/canon.py"):
        tree = ast.parse(open(os.path.join(ROOT, rel)).read())
        names = set()
        for node in ast.walk(tree):
            if isinstance(node, ast.Import):
                names |= {a.name for a in node.names}
            elif isinstance(node, ast.ImportFrom):
                names |= {f"{node.module}.{a.name}" for a in node.names}
        assert not any("fim" in n.split(".")[-1] or "torch" in n or "_build" in n for n in names), (rel, names)
