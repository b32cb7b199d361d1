"""The C-ABI library builds, loads and exports what include/lbm.h declares (no GPU needed)."""
import ctypes as C
import subprocess

import pytest

from paper_1002_3028_gb300 import build as B
from paper_1002_3028_gb300 import inputs as I
from paper_1002_3028_gb300 import lbm


def test_header_declares_the_boundary_calls():
    names = lbm.declared_symbols()
    for n in ("lbm_create", "lbm_set_inlet", "lbm_set_properties", "lbm_step", "lbm_get_fields",
              "lbm_destroy", "lbm_get_state", "lbm_set_state", "lbm_required_bytes",
              "lbm_last_error", "lbm_get_step", "lbm_set_launch", "lbm_get_launch", "lbm_check"):
        assert n in names


def test_library_exports_every_declared_symbol():
    path = B.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    missing = [n for n in lbm.declared_symbols() if n not in exported]
    assert not missing, missing
    L = lbm.lib()
    for n in lbm.declared_symbols():
        assert getattr(L, n) is not None


def test_desc_struct_matches_header_layout(tmp_path):
    """The ctypes mirror has the sizes and offsets the C compiler gives lbm_desc."""
    src = tmp_path / "layout.c"
    fields = [f[0] for f in lbm.Desc._fields_]
    body = "".join(f'printf("%zu ", offsetof(lbm_desc, {f}));' for f in fields)
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "lbm.h"\n'
                   'int main(void){' + body + 'printf("%zu", sizeof(lbm_desc)); return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", B.INCLUDE, str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                           check=True).stdout.split()]
    want = [getattr(lbm.Desc, f).offset for f in fields] + [C.sizeof(lbm.Desc)]
    assert got == want


def row_elems(nx, size):
    """Padded row: 32 leading elements, columns 0..nx rounded up to 64, 32 trailing elements,
    and for 4- and 8-byte values one 128-byte block more if the row would hold an even number
    of them."""
    row = 32 + (nx + 1 + 63) // 64 * 64 + 32
    return row + (128 // size if size >= 4 and (row * size // 128) % 2 == 0 else 0)


def test_required_bytes_counts_two_buffers():
    """Two buffers of 13 planes; each plane has ghost rows -1 and nr and padded rows."""
    cfg = I.LatticeConfig(nx=100, nr=40)
    assert [row_elems(100, sz) for sz in (8, 4, 2)] == [208, 224, 192]
    for st, sz in (("f64", 8), ("f32", 4), ("f16", 2), ("bf16", 2)):
        n = lbm.required_bytes(cfg, st)
        two = 2 * 13 * row_elems(100, sz) * (40 + 2) * sz
        assert two <= n < two + 200_000
    for st in ("f16s", "bf16s"):  # 13 two-byte planes and 3 FP32 moment planes per buffer
        n = lbm.required_bytes(cfg, st)
        two = 2 * (13 * 2 + 3 * 4) * row_elems(100, 2) * (40 + 2)
        assert two <= n < two + 200_000


def test_moment_split_storage_has_no_aa_pattern():
    d = lbm.make_desc(I.LatticeConfig(nx=40, nr=10), "f16s", pattern="aa")
    n = C.c_size_t(0)
    assert lbm.lib().lbm_required_bytes(C.byref(d), C.byref(n)) == -1
    assert "two-buffer" in lbm.lib().lbm_last_error().decode()


@pytest.mark.parametrize("bad", [
    dict(nx=0), dict(nr=0), dict(bc_in="periodic"), dict(r0=1.0), dict(nx=40000, nr=5000),
])
def test_invalid_descriptions_are_rejected(bad):
    cfg = I.LatticeConfig(nx=10, nr=10)
    d = lbm.make_desc(cfg, "f32")
    if "nx" in bad:
        d.nx = bad["nx"]
    if "nr" in bad:
        d.nr = bad["nr"]
    if "bc_in" in bad:
        d.bc_in = 1  # periodic on one end only
    if "r0" in bad:
        d.r0 = 1.0  # axis with an offset
    n = C.c_size_t(0)
    rc = lbm.lib().lbm_required_bytes(C.byref(d), C.byref(n))
    assert rc == -1
    assert lbm.lib().lbm_last_error().decode()
    h = C.c_void_p()
    assert lbm.lib().lbm_create(C.byref(d), None, 0, C.byref(h)) == -1
    assert h.value is None


def test_unknown_storage_rejected():
    d = lbm.make_desc(I.LatticeConfig(nx=4, nr=4), "f32")
    d.storage = 7
    n = C.c_size_t(0)
    assert lbm.lib().lbm_required_bytes(C.byref(d), C.byref(n)) == -1
