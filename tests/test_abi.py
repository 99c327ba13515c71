"""Host-side checks of the C ABI (no GPU needed): the library loads, exports every entry point
include/vdp.h declares, and rejects bad arguments before touching the device."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_1601_05448_gb300 as vdp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vdp.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(vdp_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1601_05448_gb300 import build
    build.build()
    return vdp.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for core in ("vdp_create", "vdp_set_density", "vdp_solve", "vdp_destroy"):
        assert core in names


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", vdp.LIB_PATH], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT\s+(vdp_[a-z0-9_]+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(lib, n)


def test_binding_covers_the_header():
    assert sorted(vdp.exported_symbols()) == declared_functions()


def declared_constants():
    """Every VDP_* enumerator with an explicit value and every integer #define of the header."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    consts = {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(VDP_[A-Z0-9_]+)\s*=\s*(\d+)", text)}
    consts.update({m.group(1): int(m.group(2))
                   for m in re.finditer(r"^#define\s+(VDP_[A-Z0-9_]+)\s+(\d+)\s*$", text, flags=re.M)})
    return consts


def test_binding_constants_match_the_header():
    consts = declared_constants()
    assert consts["VDP_SWEEP_KINDS"] == len(vdp.SWEEP_NAMES)
    checked = 0
    for name, value in consts.items():
        if hasattr(vdp, name):
            assert getattr(vdp, name) == value, name
            checked += 1
    assert checked >= 25


def test_host_only_entry_points(lib):
    assert vdp.vdp_version() >= 1
    assert vdp.vdp_strerror(vdp.VDP_EDENSITY).startswith("VDP_EDENSITY")
    assert vdp.vdp_strerror(999).startswith("VDP_?")
    o = vdp.vdp_default_options()
    assert o.precision == vdp.VDP_FP64 and o.max_iter > 0 and 0 < o.inner_tol < 1


@pytest.mark.parametrize("args", [(7, 8, 8, 1.0), (12, 8, 8, 1.0), (0, 8, 8, 1.0), (8, 0, 8, 1.0),
                                  (8, 8, 0, 1.0), (8, 8, 8, 0.0), (8, 8, 8, -1.0), (8, 8, 8, float("nan"))])
def test_create_rejects_bad_sizes(lib, args):
    h = ctypes.c_void_p()
    st = lib.vdp_create(*args, ctypes.byref(h))
    assert st == vdp.VDP_EINVAL and not h.value


def test_null_arguments(lib):
    assert lib.vdp_create(8, 8, 8, 1.0, None) == vdp.VDP_EINVAL
    assert lib.vdp_solve(None, None, None, 1e-8) == vdp.VDP_EINVAL
    assert lib.vdp_set_density(None, None) == vdp.VDP_EINVAL
    lib.vdp_destroy(None)  # NULL-safe


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    monkeypatch.setattr(vdp, "_lib", None)
    with pytest.raises(vdp.VdpUnavailable):
        vdp.load(str(tmp_path / "nope.so"))


def test_batch_tuning_keeps_to_batchable_layouts():
    from paper_1601_05448_gb300 import tune
    for n, prec in ((64, "mixed"), (96, "fp64"), (192, "mixed_bf16")):
        allc = tune.candidates(n, n, n, prec)
        bc = tune.candidates(n, n, n, prec, batchable=True)
        assert bc and all(c["stencil"] == 0 and "steps_per_sync" not in c for c in bc)
        assert any(c["stencil"] == 1 for c in allc)
        assert tune._key(n, n, n, prec) != tune._key(n, n, n, prec, batchable=True)


def test_multigrid_level_rule_matches_the_oracle(lib):
    from oracle import multigrid as MG
    for nx, ny, nz in ((256, 256, 256), (48, 48, 48), (40, 24, 16), (64, 48, 64), (8, 8, 1), (16, 8, 8),
                       (48, 36, 40), (24, 9, 16), (512, 512, 512), (80, 80, 80)):
        shapes = MG.level_shapes(nx, ny, nz)
        want = len(shapes) if shapes and len(shapes) > 1 else 0   # the library needs a coarser level
        assert vdp.vdp_mg_levels(nx, ny, nz) == want, (nx, ny, nz)
