"""CPU checks of the C ABI boundary: the library builds, loads without a GPU and
exports every function include/mst.h declares; calls that need no device work
behave as documented."""
import ctypes

import pytest

from paper_2302_12199_gb300 import mst


@pytest.fixture(scope="module")
def lib():
    return mst.load()


def test_every_declared_symbol_is_exported(lib):
    names = mst.declared_symbols()
    assert "mst_solve" in names and "mst_solve_batched" in names and "mst_create" in names
    for name in names:
        assert hasattr(lib, name), name
    assert set(mst._SIGNATURES) >= set(names)


def test_default_config(lib):
    cfg = mst.MstConfig()
    lib.mst_config_default(ctypes.byref(cfg))
    assert cfg.variant == 0 and cfg.dedupe == 0
    assert cfg.pivot_sample == 1 << 16
    assert cfg.filter_max_avg_degree == 1.25
    assert cfg.tile_contract == 0 and cfg.tile_vertices == 1024
    assert cfg.base_case == 1 and cfg.graph_rounds == 1 and cfg.graph_jump_launches == 2
    assert cfg.jump_steps == 64 and cfg.tile_filter == 0
    assert cfg.filter_carry == 0
    assert cfg.spin_limit == 1 << 21 and cfg.block_threads == 0 and cfg.items_per_thread == 0
    assert cfg.filter_plan == 1 and cfg.relabel_block_threads == 0 and cfg.relabel_items_per_thread == 0
    assert cfg.pivot_quantile == 0.125


def test_bad_kernel_shapes_are_refused_without_device(lib):
    """Tile shapes outside 128/256/512 threads x 4/8/16 items are an invalid
    configuration (checked before any device is touched)."""
    for bt, it in ((384, 8), (256, 12), (1024, 8), (256, 2)):
        cfg = mst.MstConfig()
        lib.mst_config_default(ctypes.byref(cfg))
        cfg.block_threads, cfg.items_per_thread = bt, it
        h = ctypes.c_void_p()
        assert lib.mst_create(ctypes.byref(h), ctypes.byref(cfg)) == 1, (bt, it)
        lib.mst_config_default(ctypes.byref(cfg))
        cfg.relabel_block_threads, cfg.relabel_items_per_thread = bt, it  # the relabel compaction's own shape
        assert lib.mst_create(ctypes.byref(h), ctypes.byref(cfg)) == 1, ("relabel", bt, it)
    for flag in (-1, 2):
        lib.mst_config_default(ctypes.byref(cfg))
        cfg.filter_plan = flag
        assert lib.mst_create(ctypes.byref(h), ctypes.byref(cfg)) == 1, ("filter_plan", flag)
    for q in (0.0, 1.0 / 128, 0.51, 1.0, float("nan")):  # the pivot quantile is limited to [1/64, 1/2]
        lib.mst_config_default(ctypes.byref(cfg))
        cfg.pivot_quantile = q
        assert lib.mst_create(ctypes.byref(h), ctypes.byref(cfg)) == 1, ("pivot_quantile", q)


def test_status_strings(lib):
    for code in range(8):
        assert lib.mst_status_string(code)
    assert lib.mst_status_string(0) == b"ok"


def test_invalid_arguments_without_device(lib):
    h = ctypes.c_void_p()
    assert lib.mst_create(None, None) == 1
    assert lib.mst_solve(None, 1, 1, None, None, None, None, None, None, None) == 1
    assert lib.mst_get_error(None, None) == 1
    assert lib.mst_solve_host_many(None, 0, None, None) == 1
    assert lib.mst_profile_classes(None, 0) == 1
    assert lib.mst_profile_enable(None, 1) == 1
    lib.mst_destroy(None)
    del h


def test_workspace_bytes_grows_with_size(lib):
    cfg = mst.MstConfig()
    lib.mst_config_default(ctypes.byref(cfg))
    a = lib.mst_workspace_bytes(1000, 10000, ctypes.byref(cfg))
    b = lib.mst_workspace_bytes(1000, 20000, ctypes.byref(cfg))
    c = lib.mst_workspace_bytes(2000, 20000, ctypes.byref(cfg))
    assert 0 < a < b < c
    cfg.variant = 1
    assert lib.mst_workspace_bytes(1000, 20000, ctypes.byref(cfg)) > b


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of mst_config, mst_host_graph and mst_kernel_stats have
    the C compiler's size and field offsets (a mismatch would silently pass
    wrong values across the boundary)."""
    import os
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"mst_config": mst.MstConfig, "mst_host_graph": mst.HostGraph, "mst_kernel_stats": mst.KernelStats}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "mst.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'  printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-std=c11", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        cname, field, value = line.split()
        got[(cname, field)] = int(value)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for field, _ in py._fields_:
            assert got[(cname, field)] == getattr(py, field).offset, (cname, field)


def _header_prototypes():
    """{name: (return class, [parameter classes])} from include/mst.h, where a
    class is 'ptr' (any pointer or handle), 'u32', 'u64', 'int' (int and enums)
    or 'f32'."""
    import os
    import re
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "mst.h")
    text = re.sub(r"/\*.*?\*/", " ", open(path).read(), flags=re.S)
    text = re.sub(r"#[^\n]*", " ", text)
    out = {}
    for m in re.finditer(r"([A-Za-z_][\w\s\*]*?)\b(mst_[a-z_]+)\s*\(([^;{]*?)\)\s*;", text):
        ret, name, params = m.group(1), m.group(2), m.group(3)

        def cls(decl):
            decl = decl.strip()
            if "*" in decl or decl.startswith("mst_handle"):
                return "ptr"
            if decl.startswith("uint32_t"):
                return "u32"
            if decl.startswith("uint64_t"):
                return "u64"
            if decl.startswith("float"):
                return "f32"
            if decl.startswith("void"):
                return "void"
            return "int"  # int, mst_status
        plist = [] if params.strip() in ("", "void") else [cls(p) for p in params.split(",")]
        out[name] = (cls(ret.split()[-1] if "*" not in ret else "*"), plist)
    return out


def test_binding_signatures_match_the_header():
    """Every declared function's ctypes signature in the binding has the
    header's parameter count and the same class (pointer, 32-bit, 64-bit, int)
    for every parameter and for the result."""
    def cls(t):
        if t is None:
            return "void"
        if t in (ctypes.c_void_p, ctypes.c_char_p) or getattr(t, "_type_", None) is not None and \
                isinstance(t, type) and issubclass(t, ctypes._Pointer):
            return "ptr"
        return {ctypes.c_uint32: "u32", ctypes.c_uint64: "u64", ctypes.c_int: "int", ctypes.c_float: "f32"}[t]
    protos = _header_prototypes()
    assert set(protos) == set(mst.declared_symbols())
    for name, (ret, params) in protos.items():
        res, args = mst._SIGNATURES[name]
        assert [cls(a) for a in args] == params, name
        assert cls(res) == ret, name
