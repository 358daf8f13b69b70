"""The C ABI from C: tests/c/abi_step.c (a two-step Coulomb solve through the host-buffer entry
point, written against include/chasm.h alone) compiles as C11 with -Wall -Wextra -pedantic
-Werror, links against libchasm.so without Python or PyTorch and, on a machine without a GPU,
takes its error paths cleanly: EINVAL for a bad grid before any device work, then a CUDA status
with the runtime's message."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2205_02380_gb300")


def _build(tmp_path):
    import paper_2205_02380_gb300 as pkg
    pkg.chasm.lib()   # the library exists (built in-tree)
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path / "abi_step")
    r = subprocess.run([cc, "-std=c11", "-Wall", "-Wextra", "-pedantic", "-Werror", "-D_DEFAULT_SOURCE",
                        "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "c", "abi_step.c"),
                        "-L", PKG, "-lchasm", "-lm", "-Wl,-rpath," + PKG, "-o", exe],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_program_builds_and_takes_the_error_paths_without_a_gpu(tmp_path):
    exe = _build(tmp_path)
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the run is the gpu-marked test")
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 3, (r.returncode, r.stdout, r.stderr)
    assert "chasm_create" in r.stdout and len(r.stdout.strip()) > len("chasm_create: -3 ")
