"""C ABI checks that need no GPU: the library builds, loads, exports every
entry point declared in include/dem.h, and its host-only restitution solver
agrees with the oracle's independent one."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dem_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1503_03553_gb300 import build
    build.build()
    import paper_1503_03553_gb300 as D
    return D.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "dem_create" in names and "dem_step" in names
    for n in names:
        assert hasattr(lib, n), n


def test_abi_version(lib):
    """The library reports the version the header defines."""
    import re
    import paper_1503_03553_gb300 as D
    hdr = open(os.path.join(ROOT, "include", "dem.h")).read()
    want = int(re.search(r"#define DEM_ABI_VERSION (\d+)", hdr).group(1))
    assert D.dem_abi_version() == want == D.ABI_VERSION


@pytest.mark.parametrize("eps", [0.3, 0.5, 0.9, 0.99])
def test_library_alpha_agrees_with_oracle(lib, eps):
    import oracle as O
    import paper_1503_03553_gb300 as D
    a = D.dem_alpha_of_restitution(eps)
    assert abs(a - O.alpha(eps)) < 1e-9
    assert abs(D.dem_restitution_of_alpha(a) - eps) < 1e-10


def test_alpha_rejects_bad_input(lib):
    import math
    import paper_1503_03553_gb300 as D
    assert math.isnan(D.dem_alpha_of_restitution(0.0))
    assert math.isnan(D.dem_alpha_of_restitution(1.5))
    assert D.dem_alpha_of_restitution(1.0) == 0.0


def test_create_rejects_bad_config_without_gpu(lib):
    """Argument checks run before any device call."""
    import paper_1503_03553_gb300 as D
    cfg = D.dem_config()
    with pytest.raises(D.DemError) as e:
        D.dem_create(cfg)
    assert e.value.status == D.DEM_ERR_ARG


@pytest.mark.parametrize("field, value, words", [
    ("l2_fetch", 7, "l2_fetch"), ("l2_fetch", 256, "l2_fetch"), ("block", 48, "block"),
    ("row_capacity", 2000, "row_capacity"), ("precision", 3, "precision")])
def test_create_rejects_bad_launch_settings_without_gpu(lib, field, value, words):
    """A config that is complete but for one bad setting is refused before
    any device call, with the setting named."""
    import ctypes as C
    import paper_1503_03553_gb300 as D
    mat = (D.dem_material * 1)()
    mat[0].E, mat[0].poisson, mat[0].density = 5e9, 0.3, 1000.0
    mat[0].restitution, mat[0].mu_d = 0.5, 0.5
    box = (D.dem_box * 1)()
    for a in range(3):
        box[0].L[a], box[0].periodic[a] = 1e-4, 1
    box[0].dt, box[0].max_particles, box[0].r_max = 1e-9, 16, 5e-6
    cfg = D.dem_config()
    cfg.nboxes, cfg.boxes = 1, C.cast(box, C.POINTER(D.dem_box))
    cfg.nmaterials, cfg.materials = 1, C.cast(mat, C.POINTER(D.dem_material))
    setattr(cfg, field, value)
    with pytest.raises(D.DemError) as e:
        D.dem_create(cfg)
    assert e.value.status == D.DEM_ERR_ARG
    assert words in str(e.value), str(e.value)


def test_header_compiles_as_c_and_matches_the_binding(tmp_path):
    """include/dem.h compiles as C99, and the sizes and member offsets of its
    structs are those of the ctypes structures of the binding."""
    import ctypes as C
    import subprocess
    import paper_1503_03553_gb300 as D
    structs = {"dem_material": D.dem_material, "dem_wall": D.dem_wall,
               "dem_box": D.dem_box, "dem_config": D.dem_config}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "dem.h"',
             'int main(void) {']
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{name} {fname} %zu\\n", offsetof({name}, {fname}));')
    lines += ['  return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    seen = {}
    for line in out.splitlines():
        name, field, value = line.split()
        seen[(name, field)] = int(value)
    for name, cls in structs.items():
        assert seen[(name, "size")] == C.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert seen[(name, fname)] == getattr(cls, fname).offset, (name, fname)


def test_host_arrays_of_the_wrong_size_are_refused_before_the_call(lib):
    """The binding checks the element count of every array a C call reads or
    writes (a short array would be read or written past its end)."""
    import numpy as np
    import paper_1503_03553_gb300 as D
    p, keep = D._ptr(np.zeros((4, 3)), D.DEM_HOST, elems=12, name="x")
    assert p.value == keep.ctypes.data
    with pytest.raises(ValueError, match="x must hold 12 elements, not 9"):
        D._ptr(np.zeros((3, 3)), D.DEM_HOST, elems=12, name="x")
    with pytest.raises(ValueError, match="radius must hold 4 elements, not 5"):
        D._ptr(np.zeros(5), D.DEM_HOST, elems=4, name="radius")
    assert D._ptr(None, D.DEM_HOST, elems=12) == (None, None)
    with pytest.raises(TypeError, match="CUDA tensors"):
        D._ptr(np.zeros((4, 3)), D.DEM_DEVICE, elems=12, name="x")
