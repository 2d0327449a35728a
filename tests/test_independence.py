"""Structure: the FP64 oracle and the CUDA path share no code, and the
product path has no CPU fallback."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1503_03553_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _sources(top, exts):
    for dirpath, _, files in os.walk(top):
        if "__pycache__" in dirpath or "_build" in dirpath:
            continue
        for f in files:
            if f.endswith(exts):
                yield os.path.join(dirpath, f)


def test_oracle_does_not_use_the_cuda_path():
    for path in _sources(ORACLE, (".c", ".h", ".py")):
        src = open(path).read()
        assert "paper_1503_03553_gb300" not in src, path
        assert "csrc" not in src and "dem.h" not in src, path


def test_cuda_path_does_not_use_the_oracle():
    for path in _sources(PKG, (".py", ".cu", ".cuh", ".cpp", ".h")):
        src = open(path).read()
        assert not re.search(r"^\s*(import|from)\s+oracle\b", src, re.M), path
        assert "dem_oracle" not in src and "orc_" not in src, path


def test_product_path_needs_the_gpu():
    """Without a CUDA device the library refuses to run rather than fall
    back to the host."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1503_03553_gb300 as D
    from paper_1503_03553_gb300 import synth
    box = synth.w1_monodisperse(n=100, seed=1)
    with pytest.raises(RuntimeError):
        D.Context([box], precision="mixed")
