"""C ABI checks that need no GPU: the library loads, exports every symbol that
include/etd.h declares, and rejects bad arguments before touching the device."""
import os
import re

import pytest

from paper_2601_06849_gb300 import etd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "etd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(etd_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    __graft_entry__.build()
    return etd.lib()


def test_header_and_binding_agree():
    assert declared_symbols() == sorted(etd.SYMBOLS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


@pytest.mark.parametrize("args,what", [
    ((5, 64, 0.1, 0.0, 1e-3, 2), "d"),
    ((2, 1, 0.1, 0.0, 1e-3, 2), "m"),
    ((3, 4096, 0.1, 0.0, 1e-3, 2), "m"),
    ((2, 64, -1.0, 0.0, 1e-3, 2), "kappa"),
    ((2, 64, 0.1, -0.5, 1e-3, 2), "q"),
    ((2, 64, 0.1, 0.0, 0.0, 2), "dt"),
    ((2, 64, 0.1, 0.0, 1e-3, 3), "pade"),
])
def test_plan_create_rejects_bad_arguments(lib, args, what):
    with pytest.raises(etd.EtdError) as ei:
        etd.etd_plan_create(*args)
    assert ei.value.status == etd.ETD_ERR_INVALID_ARG


def test_reaction_component_mismatch(lib):
    o = etd.etd_options_default()
    o.reaction = etd.REACTION["fhn"]
    o.n_comp = 1
    with pytest.raises(etd.EtdError) as ei:
        etd.etd_plan_create(2, 64, 0.1, 0.0, 1e-3, 2, o)
    assert ei.value.status == etd.ETD_ERR_INVALID_ARG


def test_null_plan_calls_fail_cleanly(lib):
    for call in (lambda: etd.etd_sync(0), lambda: etd.etd_plan_invalidate(0), lambda: etd.etd_set_time(0, 0.0)):
        with pytest.raises(etd.EtdError):
            call()
    etd.etd_plan_destroy(0)  # NULL-safe
    assert lib.etd_status_string(0) == b"ok"


def test_unknown_flags_rejected(lib):
    o = etd.etd_options_default()
    o.flags = 2  # not a defined ETD_FLAG_* bit
    with pytest.raises(etd.EtdError) as ei:
        etd.etd_plan_create(2, 64, 0.1, 0.0, 1e-3, 2, o)
    assert ei.value.status == etd.ETD_ERR_INVALID_ARG


def test_header_flag_and_binding_agree():
    src = open(os.path.join(ROOT, "include", "etd.h")).read()
    m = re.search(r"#define\s+ETD_FLAG_AUTOTUNE\s+(\d+)", src)
    assert m and int(m.group(1)) == etd.ETD_FLAG_AUTOTUNE


def test_plan_info_layout_matches_header():
    # the ctypes mirror must list the header's fields in order
    src = open(os.path.join(ROOT, "include", "etd.h")).read()
    body = re.search(r"typedef struct \{([^{}]*)\} etd_plan_info;", src).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        for part in decl.split(",") if "(" not in decl else [decl]:
            tok = re.findall(r"([A-Za-z_]\w*)\s*(?:\[\d+\])?\s*$", part.strip())
            names.append(tok[-1])
    assert names == [f[0] for f in etd.etd_plan_info._fields_]


def test_options_defaults_and_diag_validation(lib):
    """Defaults: FP64-split (the precision held to 1e-6, indeed 1e-10, of FP64 over
    every configuration's whole run), in-step check off; a negative check interval
    is rejected before any device work."""
    o = etd.etd_options_default()
    assert o.precision == etd.PRECISION["fp64split"]
    assert o.diag_every == 0 and o.diag_max_abs == 0.0
    o.diag_every = -1
    with pytest.raises(etd.EtdError) as ei:
        etd.etd_plan_create(2, 64, 0.1, 0.0, 1e-3, 2, o)
    assert ei.value.status == etd.ETD_ERR_INVALID_ARG



def test_fp64split_size_limit_rejected_before_device_work(lib):
    """FP64-split keeps its level sums exact in int32 up to K = 16384 values
    (128 groups of 128 products below 7 * 2^21 each), which is also the largest 2D
    grid a plan takes: a larger one is refused before anything touches the device."""
    o = etd.etd_options_default()
    o.precision = etd.PRECISION["fp64split"]
    with pytest.raises(etd.EtdError) as ei:
        etd.etd_plan_create(2, 16385, 0.1, 0.0, 1e-3, 2, o)
    assert ei.value.status in (etd.ETD_ERR_INVALID_ARG, etd.ETD_ERR_UNSUPPORTED)
    assert "16384" in str(ei.value)
