"""The C ABI used from plain C: tests/c_abi_host.c is compiled with the system C compiler against
include/mcsdp.h, linked to the built libmcsdp.so and run (host-only context, no GPU)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_plain_c_client(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_1310_6919_gb300 import build_library
    build_library()
    libdir = os.path.join(ROOT, "paper_1310_6919_gb300")
    exe = str(tmp_path / "c_abi_host")
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c_abi_host.c"), "-o", exe, "-L", libdir,
                    "-lmcsdp", "-Wl,-rpath," + libdir], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip().endswith("ok"), out.stdout + out.stderr
