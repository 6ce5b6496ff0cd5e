"""The C ABI from plain C (CPU): a C99 program includes include/cs_gb300.h, links against the
built library and calls the host-only entry points; its output is checked against the oracle's
draws."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import rng

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_client_compiles_links_and_runs(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_1509_03979_gb300 import build
    lib = build.build()
    libdir = os.path.dirname(lib)
    exe = tmp_path / "c_abi_check"
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c", "c_abi_check.c"), "-o", str(exe),
                    "-L", libdir, "-l:" + os.path.basename(lib), "-Wl,-rpath," + libdir],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    fields = dict(kv.split("=") for kv in out.split())
    om = rng.omega(4096, 1024, 0x0C5001)
    assert int(fields["omega[0]"]) == om[0] and int(fields["omega[M-1]"]) == om[-1]
    assert int(fields["d[0]"]) == int(rng.signs(4096, 0x0C5001)[0])
    assert int(fields["perm[0]"]) == int(rng.perm(4096, 7)[0])
