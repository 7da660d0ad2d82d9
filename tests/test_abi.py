"""The C-ABI library on the CPU: it builds for sm_103a, loads, exports every
entry point include/dawn.h declares, and rejects bad host-side arguments
before touching a device.  No compute call runs here."""
import ctypes
import subprocess

import numpy as np
import pytest

from paper_2208_04514_b300 import _build, dawn


def test_builds_for_sm103a_only():
    so = _build.build_dawn()
    assert so.exists()
    out = subprocess.run(["/usr/local/cuda/bin/cuobjdump", "--list-elf", str(so)],
                         capture_output=True, text=True)
    if out.returncode == 0:  # lists the embedded ELF names only (no disassembly)
        assert "sm_103a" in out.stdout
        assert "sm_90" not in out.stdout and "sm_100" not in out.stdout.replace("sm_103a", "")


def test_exports_every_header_entry_point(dawn):
    names = dawn.header_entry_points()
    assert len(names) >= 16
    lib = ctypes.CDLL(str(_build.DAWN_SO))
    for name in names:
        assert hasattr(lib, name), f"{name} declared in include/dawn.h but not exported"
    for name in names:
        assert name in dawn._SIGNATURES, f"{name} has no Python binding"


def test_version_and_last_error(dawn):
    assert dawn.dawn_version() >= 3
    assert isinstance(dawn.dawn_last_error(), str)


def test_host_side_argument_checks(dawn):
    lib = dawn.load()
    h = ctypes.c_void_p()
    rp = np.array([0, 1], dtype=np.int32)
    ci = np.array([0], dtype=np.int32)
    assert lib.dawn_graph_upload(rp.ctypes.data, ci.ctypes.data, 0, 1, 0, None, ctypes.byref(h)) == dawn.DAWN_E_INVALID
    assert "n = 0" in dawn.dawn_last_error()
    assert lib.dawn_graph_upload(rp.ctypes.data, ci.ctypes.data, 1, -1, 0, None, ctypes.byref(h)) == dawn.DAWN_E_INVALID
    assert lib.dawn_graph_upload(rp.ctypes.data, ci.ctypes.data, 1, 1 << 31, 0, None, ctypes.byref(h)) == dawn.DAWN_E_INVALID
    assert lib.dawn_graph_upload(rp.ctypes.data, ci.ctypes.data, 1, 1, 0x10, None, ctypes.byref(h)) == dawn.DAWN_E_INVALID
    assert lib.dawn_graph_upload(None, ci.ctypes.data, 1, 1, 0, None, ctypes.byref(h)) == dawn.DAWN_E_INVALID
    assert lib.dawn_graph_upload(rp.ctypes.data, ci.ctypes.data, 1, 1, 0, None, None) == dawn.DAWN_E_INVALID
    d = np.zeros(1, dtype=np.int32)
    assert lib.dawn_sssp(None, 0, d.ctypes.data, None) == dawn.DAWN_E_INVALID
    assert lib.dawn_graph_info(None, None, None, None) == dawn.DAWN_E_INVALID
    assert lib.dawn_graph_free(None) == dawn.DAWN_OK
    with pytest.raises(dawn.DawnError) as ei:
        dawn.dawn_sssp(None, 0, d)
    assert ei.value.code == dawn.DAWN_E_INVALID


def test_binding_rejects_noncontiguous(dawn):
    a = np.zeros((4, 4), dtype=np.int32)[:, 0]
    with pytest.raises(ValueError):
        dawn._ptr(a)


def test_struct_layouts_match_the_header(tmp_path):
    """Every struct the binding mirrors has the header's size and field
    offsets: a C program built against include/dawn.h prints them (gcc, no
    CUDA), and they are compared with the ctypes classes."""
    import shutil
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not found")
    structs = {name: cls for name, cls in vars(dawn).items()
               if isinstance(cls, type) and issubclass(cls, ctypes.Structure) and name.startswith("dawn_")}
    assert {"dawn_sssp_opts", "dawn_msbfs_opts", "dawn_tuning"} <= set(structs)
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "dawn.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'    printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'    printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c11", "-I", str(_build.INCLUDE), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        name, field, value = line.split()
        got[(name, field)] = int(value)
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)
