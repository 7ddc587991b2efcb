"""Plain FP64 CPU oracle for the multipatch scalar-wave method (arXiv:2002.00088).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library in ``paper_2002_00088_gb300`` and neither side imports
the other.  ``pyoracle`` wraps the C oracle (``oracle.c``) with ctypes;
``build_oracle()`` compiles it with the system C compiler.  ``surrogate`` is
the numpy oracle of the learned surrogate (its layers, gradients, optimizer,
features, targets, update and residual check).
"""
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liboracle.so")


def build_oracle(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (OpenMP if the compiler has it)."""
    src = os.path.join(HERE, "oracle.c")
    hdr = os.path.join(HERE, "oracle.h")
    if (not force and os.path.exists(LIB_PATH)
            and os.path.getmtime(LIB_PATH) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return LIB_PATH
    cc = os.environ.get("CC") or shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("no C compiler found to build the oracle")
    # -ffp-contract=off: every FP64 operation rounds as written, identically
    # on x86-64 and AArch64 hosts.
    base = [cc, "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off", src, "-o", LIB_PATH + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(LIB_PATH + ".tmp", LIB_PATH)
    return LIB_PATH
