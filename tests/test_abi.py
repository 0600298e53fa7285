"""The C ABI: libcqk.so builds, loads without a GPU, and exports every function that
include/cqk.h declares.  No compute call is made here."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names.update(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(cqk_\w+)\s*\(", src, flags=re.M))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("cqk_solve", "cqk_project_simplex", "cqk_project_l1", "cqk_workspace_bytes", "cqk_status_string",
              "cqk_phi", "cqk_default_options"):
        assert f in names


def test_library_builds_loads_and_exports_every_symbol():
    from paper_2603_15910_b300 import build_lib
    path = build_lib.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_host_only_calls():
    from paper_2603_15910_b300 import api
    lib = api.library()
    assert lib.cqk_version() >= 200
    assert lib.cqk_status_string(0) == b"ok" and lib.cqk_status_string(5) == b"timeout"
    assert lib.cqk_workspace_bytes(10**8, 1, 0) > 0
    assert lib.cqk_workspace_bytes(-1, 1, 0) == 0
    assert lib.cqk_workspace_bytes(10, 1, 7) == 0
    o = api.make_options()
    assert o.max_iter == 100 and o.validate == 1 and o.spin_limit_us == 2_000_000 and o.final_step == 1
    assert ctypes.sizeof(api._Info) == 72
    assert ctypes.sizeof(api._Options) == 72 and api._Options.xbar.offset == 48


def test_bad_arguments_are_rejected_before_any_launch():
    from paper_2603_15910_b300 import api
    lib = api.library()
    null = ctypes.c_void_p(0)
    opt = api.make_options()
    # negative n, NULL arrays, bad dtype, bad r, missing workspace: CQK_BAD_ARG (7), nothing launched
    assert lib.cqk_solve(-1, 0, null, null, null, null, null, 1.0, null, null, ctypes.c_void_p(8),
                         ctypes.byref(opt), null, 0, null) == 7
    assert lib.cqk_solve(10, 0, null, null, null, null, null, 1.0, null, null, ctypes.c_void_p(8),
                         ctypes.byref(opt), null, 0, null) == 7
    assert lib.cqk_project_simplex(10, 9, ctypes.c_void_p(256), 1.0, ctypes.c_void_p(512), null,
                                   ctypes.c_void_p(8), ctypes.byref(opt), ctypes.c_void_p(1024), 1 << 20, null) == 7
    assert lib.cqk_project_simplex(10, 0, ctypes.c_void_p(256), -1.0, ctypes.c_void_p(512), null,
                                   ctypes.c_void_p(8), ctypes.byref(opt), ctypes.c_void_p(1024), 1 << 20, null) == 7
    assert lib.cqk_project_l1(10, 0, ctypes.c_void_p(256), 1.0, ctypes.c_void_p(512), null,
                              ctypes.c_void_p(8), ctypes.byref(opt), ctypes.c_void_p(1024), 16, null) == 7
