"""CPU-only checks of the C ABI: the library builds, loads, exports every symbol declared in
include/lf2.h, and validates arguments on calls that touch no GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1508_05610_gb300 import build, lf2
    build.build()
    return lf2


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "lf2.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lf2_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("lf2_lattice_create", "lf2_field_alloc", "lf2_leapfrog", "lf2_energy", "lf2_field_update_halo",
                 "lf2_leapfrog_init", "lf2_field_upload", "lf2_field_download"):
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    so = ctypes.CDLL(lib.LIB_PATH)
    for name in declared_symbols():
        assert hasattr(so, name), name


def test_binding_covers_every_declared_symbol(lib):
    for name in declared_symbols():
        assert name in lib.SIGNATURES, name
        assert hasattr(lib, name), name


def test_status_strings_and_version(lib):
    assert lib.lf2_status_string(0) == "LF2_OK"
    assert lib.lf2_status_string(5) == "LF2_ERR_TIMEOUT"
    assert "sm_103a" in lib.lf2_version()


def test_lattice_argument_checks(lib):
    with pytest.raises(lib.LF2Error) as e:
        lib.lf2_lattice_create([8, 8], dim=2)
    assert e.value.status == lib.LF2_ERR_UNSUPPORTED
    with pytest.raises(lib.LF2Error) as e:
        lib.lf2_lattice_create([8, 8, 8, 8], dim=4)
    assert e.value.status == lib.LF2_ERR_UNSUPPORTED
    with pytest.raises(lib.LF2Error) as e:
        lib.lf2_lattice_create([8, 8, 8], dim=1)
    assert e.value.status == lib.LF2_ERR_INVALID
    with pytest.raises(lib.LF2Error) as e:
        lib.lf2_lattice_create([8, 0, 8])
    assert e.value.status == lib.LF2_ERR_INVALID
    with pytest.raises(lib.LF2Error) as e:
        lib.lf2_lattice_create([8, 8, 8], halo=0)
    assert e.value.status == lib.LF2_ERR_INVALID
    with pytest.raises(lib.LF2Error) as e:
        lib.lf2_lattice_create([1 << 14, 1 << 14, 1 << 14])
    assert e.value.status == lib.LF2_ERR_INVALID
    lat = lib.lf2_lattice_create([3, 4, 5])
    assert lib.lf2_lattice_sites(lat) == 60
    lib.lf2_lattice_destroy(lat)


def test_field_argument_checks_before_any_device_call(lib):
    lat = lib.lf2_lattice_create([4, 4, 4])
    try:
        with pytest.raises(lib.LF2Error) as e:
            lib.lf2_field_alloc(lat, 7, lib.LF2_F64)
        assert e.value.status == lib.LF2_ERR_UNSUPPORTED
        with pytest.raises(lib.LF2Error) as e:
            lib.lf2_field_alloc(lat, 0, lib.LF2_F64)
        assert e.value.status == lib.LF2_ERR_INVALID
        with pytest.raises(lib.LF2Error) as e:
            lib.lf2_field_alloc(lat, 1, 7)
        assert e.value.status == lib.LF2_ERR_INVALID
        with pytest.raises(lib.LF2Error) as e:
            lib.lf2_field_wrap(lat, 1, lib.LF2_F64, [0x1008])  # not 16-byte aligned
        assert e.value.status == lib.LF2_ERR_INVALID
        with pytest.raises(lib.LF2Error) as e:
            lib.lf2_field_wrap(lat, 1, lib.LF2_F64, [0x1000, 0x2000, 0x3000])  # comp needs F32_KAHAN
        assert e.value.status == lib.LF2_ERR_INVALID
        # wrap touches no device memory: a borrowed field can be created and freed on the host
        f = lib.lf2_field_wrap(lat, 2, lib.LF2_F32_KAHAN, [0x1000, 0x2000, 0x3000])
        with pytest.raises(lib.LF2Error) as e:
            lib.lf2_lattice_destroy(lat)
        assert e.value.status == lib.LF2_ERR_STATE
        assert lib.lf2_field_buffer(f, 0) == 0x1000 and lib.lf2_field_buffer(f, 2) == 0x3000
        lib.lf2_field_update_halo(f)
        g = lib.lf2_field_wrap(lat, 1, lib.LF2_F64, [0x1000])
        p = lib.params()
        with pytest.raises(lib.LF2Error) as e:
            lib.lf2_leapfrog(f, g, p, 1)  # mismatched ncomp / precision
        assert e.value.status == lib.LF2_ERR_INVALID
        with pytest.raises(lib.LF2Error) as e:
            lib.lf2_leapfrog(f, f, p, 1)
        assert e.value.status == lib.LF2_ERR_INVALID
        bad = lib.params(dx=0.0)
        h = lib.lf2_field_wrap(lat, 1, lib.LF2_F64, [0x4000])
        with pytest.raises(lib.LF2Error) as e:
            lib.lf2_leapfrog(g, h, bad, 1)
        assert e.value.status == lib.LF2_ERR_INVALID
        with pytest.raises(lib.LF2Error) as e:
            lib.lf2_leapfrog(g, h, p, -1)
        assert e.value.status == lib.LF2_ERR_INVALID
        # the fused step + energy and the error norms check their arguments first too
        for args in ((f, g, p, 1, 0x5000), (g, g, p, 1, 0x5000), (g, h, bad, 1, 0x5000), (g, h, p, -1, 0x5000),
                     (g, h, p, 2, None)):
            with pytest.raises(lib.LF2Error) as e:
                lib.lf2_leapfrog_energy(*args)
            assert e.value.status == lib.LF2_ERR_INVALID, args
        for which, ref, prec in ((0, None, lib.LF2_F64), (5, 0x5000, lib.LF2_F64), (0, 0x5000, 9)):
            with pytest.raises(lib.LF2Error) as e:
                lib.lf2_field_compare(g, ref, prec, which=which)
            assert e.value.status == lib.LF2_ERR_INVALID, (which, ref, prec)
        with pytest.raises(lib.LF2Error) as e:  # g was wrapped without a back buffer
            lib.lf2_field_compare(g, 0x5000, lib.LF2_F64, which=1)
        assert e.value.status == lib.LF2_ERR_STATE
        for x in (f, g, h):
            lib.lf2_field_free(x)
    finally:
        lib.lf2_lattice_destroy(lat)


def test_alloc_failure_is_reported_not_hidden(lib, monkeypatch):
    """Without a GPU (or with an injected failure) allocation reports an error status; there is
    no host fallback."""
    monkeypatch.setenv("LF2_FAULT", "alloc")
    lat = lib.lf2_lattice_create([4, 4, 4])
    try:
        with pytest.raises(lib.LF2Error) as e:
            lib.lf2_field_alloc(lat, 1, lib.LF2_F64)
        assert e.value.status == lib.LF2_ERR_NOMEM
    finally:
        lib.lf2_lattice_destroy(lat)


def test_injected_launch_failure_is_reported_before_any_device_call(lib, monkeypatch):
    """LF2_FAULT=launch: the stepping calls report LF2_ERR_CUDA without launching (checked here
    with borrowed, never-dereferenced pointers and no GPU); lf2_field_check on a field that has
    run nothing reports LF2_OK without a device call."""
    monkeypatch.setenv("LF2_FAULT", "launch")
    lat = lib.lf2_lattice_create([4, 4, 4])
    try:
        f = lib.lf2_field_wrap(lat, 1, lib.LF2_F64, [0x1000])
        g = lib.lf2_field_wrap(lat, 1, lib.LF2_F64, [0x2000])
        p = lib.params()
        try:
            for call in (lambda: lib.lf2_leapfrog(f, g, p, 3), lambda: lib.lf2_leapfrog_energy(f, g, p, 3, 0x3000)):
                with pytest.raises(lib.LF2Error) as e:
                    call()
                assert e.value.status == lib.LF2_ERR_CUDA and "LF2_FAULT=launch" in str(e.value)
            lib.lf2_field_check(f)
        finally:
            lib.lf2_field_free(f)
            lib.lf2_field_free(g)
    finally:
        lib.lf2_lattice_destroy(lat)


def test_release_library_has_no_index_checks(lib):
    """The index checks exist only in the debug build; the release library says so."""
    with pytest.raises(lib.LF2Error) as e:
        lib.lf2_debug_bounds()
    assert e.value.status == lib.LF2_ERR_UNSUPPORTED


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1508_05610_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, fn)).read()
                bad = re.search(r"(from\s+oracle|import\s+oracle|oracle\.|lf2_oracle|\bora_[a-z]+\()", text)
                assert bad is None, (os.path.join(dirpath, fn), bad and bad.group(0))


def test_ensemble_and_tune_argument_checks(lib):
    lat = lib.lf2_lattice_create([8, 8, 8])
    try:
        a = lib.lf2_field_wrap(lat, 1, lib.LF2_F32_KAHAN, [0x1000])
        b = lib.lf2_field_wrap(lat, 1, lib.LF2_F32_KAHAN, [0x2000])
        c = lib.lf2_field_wrap(lat, 1, lib.LF2_F64, [0x3000])
        p = lib.params()
        for phis, pis in (([a], [a]), ([a], [c]), ([a, a], [b, b]), ([], [])):
            with pytest.raises(lib.LF2Error) as e:
                lib.lf2_ensemble_create(phis, pis, [p] * len(phis))
            assert e.value.status == lib.LF2_ERR_INVALID
        with pytest.raises(lib.LF2Error) as e:
            lib.lf2_ensemble_create([a], [b], [lib.params(dx=-1.0)])
        assert e.value.status == lib.LF2_ERR_INVALID
        with pytest.raises(lib.LF2Error) as e:
            lib.lf2_tune_lookup((8, 8, 8), 1, lib.LF2_F32_KAHAN)
        assert e.value.status == lib.LF2_ERR_STATE
        for f in (a, b, c):
            lib.lf2_field_free(f)
    finally:
        lib.lf2_lattice_destroy(lat)
