"""CPU-side checks of the C ABI: the library loads, exports every symbol the
header declares, and its host-only logic (defaults, argument validation,
direction table) behaves as documented.  No call here touches a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1007_1388_gb300 import build

    build.build()
    import paper_1007_1388_gb300 as L

    return L


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b((?:lbm|unet)_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported(L):
    names = _declared_functions()
    assert len(names) >= 20
    lib = ctypes.CDLL(L.LIB_PATH)
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding declares a signature for each of them
    assert names == set(L.SIGNATURES), names ^ set(L.SIGNATURES)


def test_direction_table_matches_header_and_oracle(L, orc):
    e, w, opp = L.lbm_directions()
    hdr = open(os.path.join(ROOT, "include", "lbm.h")).read()
    rows = {}
    for axis in ("ex", "ey", "ez"):
        m = re.search(r"\*\s+%s :((?:\s+[+-]?\d)+)" % axis, hdr)
        rows[axis] = [int(v) for v in m.group(1).split()]
    assert e[:, 0].tolist() == rows["ex"]
    assert e[:, 1].tolist() == rows["ey"]
    assert e[:, 2].tolist() == rows["ez"]
    eo, wo, oo = orc.lattice()
    assert np.array_equal(e, eo) and np.array_equal(w, wo) and np.array_equal(opp, oo)


def test_default_params(L):
    p = L.lbm_default_params()
    assert p.collision == L.LBM_BGK and p.magic == 3 / 16 and p.rho0 == 1.0
    assert list(p.face_bc) == [L.LBM_NOSLIP] * 6 and list(p.periodic) == [0, 0, 0]
    assert p.storage == L.LBM_F32 and p.storage_scale == 1.0 and not p.stream
    assert list(p.tile) == [0, 0, 0] and p.graph_steps == 0


def test_struct_layouts_match_the_header(L, tmp_path):
    """ctypes mirrors of the ABI structs have the C compiler's offsets."""
    import subprocess

    structs = {"lbm_params": L.lbm_params, "lbm_info": L.lbm_info, "lbm_profile": L.lbm_profile}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lbm.h"', "int main(void){"]
    for name, cls in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (name, name))
        for fname, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, fname, name, fname))
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert int(got[f"{name}.{fname}"]) == getattr(cls, fname).offset, (name, fname)


@pytest.mark.parametrize("dims,bdims,tau", [
    ((32, 32, 32), (5, 32, 32), 0.6),    # not divisible
    ((32, 32, 32), (0, 32, 32), 0.6),    # zero block
    ((32, -1, 32), (32, 1, 32), 0.6),    # negative
    ((8, 8, 8), (8, 8, 8), 0.5),         # tau must exceed 1/2
    ((8, 8, 8), (8, 8, 8), float("nan")),
])
def test_create_rejects_bad_geometry_before_touching_the_gpu(L, dims, bdims, tau):
    p = L.lbm_default_params()
    p.stream = 1  # never used: validation fails first
    with pytest.raises(L.LBMError) as ei:
        L.lbm_create(dims, bdims, tau, None, p)
    assert ei.value.code == L.LBM_EINVAL
    assert L.lbm_last_error()


@pytest.mark.parametrize("field,value", [
    ("collision", 7), ("storage", 9), ("rho0", 0.0), ("storage_scale", 3.0),
    ("storage_scale", -2.0), ("streaming", 2), ("layout", 2),
])
def test_create_rejects_bad_params(L, field, value):
    p = L.lbm_default_params()
    p.stream = 1
    setattr(p, field, value)
    with pytest.raises(L.LBMError) as ei:
        L.lbm_create((8, 8, 8), (8, 8, 8), 0.7, None, p)
    assert ei.value.code == L.LBM_EINVAL


def test_bad_face_bc_and_batch_args(L):
    p = L.make_params(face_bc=(1, 1, 5, 1, 1, 1))
    p.stream = 1
    with pytest.raises(L.LBMError):
        L.lbm_create((8, 8, 8), (8, 8, 8), 0.7, None, p)
    with pytest.raises(L.LBMError) as ei:
        L.lbm_batch_create([(8, 8, 8), (4, 0, 4)], [0.7, 0.8], None, p)
    assert ei.value.code == L.LBM_EINVAL
    with pytest.raises(L.LBMError):
        L.lbm_batch_create([(8, 8, 8)], [0.4], None, p)


def test_in_place_streaming_rejects_batches_and_the_tma_sweep(L):
    p = L.make_params(streaming=L.LBM_STREAM_AA)
    p.stream = 1  # never used: the checks come first
    with pytest.raises(L.LBMError) as ei:
        L.lbm_batch_create([(8, 8, 8), (8, 8, 8)], [0.7, 0.8], None, p)
    assert ei.value.code == L.LBM_EINVAL and "in-place" in L.lbm_last_error()
    p = L.make_params(streaming=L.LBM_STREAM_AA, kernel=L.LBM_KERNEL_TMA)
    p.stream = 1
    with pytest.raises(L.LBMError) as ei:
        L.lbm_create((64, 8, 8), (64, 8, 8), 0.7, None, p)
    assert ei.value.code == L.LBM_EINVAL


def test_fluid_list_layout_rejects_batches_in_place_and_tma(L):
    for extra in (dict(streaming=L.LBM_STREAM_AA), dict(kernel=L.LBM_KERNEL_TMA)):
        p = L.make_params(layout=L.LBM_LAYOUT_SPARSE, **extra)
        p.stream = 1  # never used: the checks come first
        with pytest.raises(L.LBMError) as ei:
            L.lbm_create((64, 8, 8), (64, 8, 8), 0.7, None, p)
        assert ei.value.code == L.LBM_EINVAL and "fluid-cell list" in L.lbm_last_error()
    p = L.make_params(layout=L.LBM_LAYOUT_SPARSE)
    p.stream = 1
    with pytest.raises(L.LBMError) as ei:
        L.lbm_batch_create([(8, 8, 8), (8, 8, 8)], [0.7, 0.8], None, p)
    assert ei.value.code == L.LBM_EINVAL


def test_allocator_hooks_must_come_in_pairs(L):
    lib = L.lib()
    assert lib.lbm_set_allocator(L.ALLOC_FN(lambda n, s, u: None), L.FREE_FN(0), None) == L.LBM_EINVAL
    assert lib.lbm_set_allocator(L.ALLOC_FN(0), L.FREE_FN(0), None) == L.LBM_OK


def test_product_path_has_no_oracle_or_cpu_fallback():
    """The package never imports the oracle, and its sources name no CPU path."""
    pkg = os.path.join(ROOT, "paper_1007_1388_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in text and "from oracle" not in text, fn
                assert "lbm_oracle" not in text, fn


def test_noalloc_binding_checks_arguments_before_the_call(L):
    """lbm_invariants_noalloc's binding refuses a wrong dtype, size, layout or
    device with ValueError before any address reaches the library (checked
    here with CPU tensors: the device check comes last, so the earlier
    checks are reached)."""
    torch = pytest.importorskip("torch")
    n = 100
    f = torch.zeros(19 * n, dtype=torch.float32)
    out = torch.zeros(5, dtype=torch.float64)
    flags = torch.zeros(n, dtype=torch.uint8)
    cases = [
        (f.double(), flags, n, out, "float32"),
        (f[:-1], flags, n, out, "elements"),
        (f, flags, n + 1, out, "elements"),
        (f, flags, n, torch.zeros(4, dtype=torch.float64), "elements"),
        (f, flags, n, out.float(), "float64"),
        (f, flags[:-1], n, out, "elements"),
        (f, flags.to(torch.int32), n, out, "uint8"),
        (torch.zeros(2 * 19 * n, dtype=torch.float32)[::2], flags, n, out, "contiguous"),
        (f, flags, 0, out, "positive"),
        (f, flags, n, out, "CUDA"),
        (f.numpy(), flags, n, out, "torch tensor"),
    ]
    for ff, fl, nc, oo, what in cases:
        with pytest.raises(ValueError, match=what):
            L.lbm_invariants_noalloc(ff, fl, nc, 1.0, (0.0, 0.0, 0.0), oo)
