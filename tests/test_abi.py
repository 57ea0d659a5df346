"""The C-ABI library builds, loads, exports every declared symbol, and rejects
bad arguments before touching a GPU (CPU-only checks)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sbp.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2510_10070_gb300 import build as B
    from paper_2510_10070_gb300 import sbp

    B.build()
    return sbp.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sbp_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("sbp_plan_create", "sbp_solve", "sbp_solve_batched", "sbp_plan_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2510_10070_gb300 import sbp

    names = declared_functions()
    for name in names:
        assert hasattr(lib, name), name
    # the binding wraps exactly the declared set
    assert sorted(sbp.SIGNATURES) == names


def test_status_strings(lib):
    for s in range(9):
        assert lib.sbp_status_string(s)
    assert lib.sbp_status_string(0) == b"ok"
    assert lib.sbp_version().startswith(b"sbp")


def _create(lib, *args):
    h = ctypes.c_void_p()
    st = lib.sbp_plan_create(ctypes.byref(h), *args)
    return st, h


@pytest.mark.parametrize("dims,status", [
    ((3, 8, 8), 2), ((8, 2, 8), 2), ((8, 8, 1), 2), ((10, 8, 8), 2), ((8, 8, 5), 2), ((18, 8, 8), 2),
    ((4096, 8, 8), 2), ((8, 8, 9), 2),
])
def test_unsupported_sizes_rejected(lib, dims, status):
    st, h = _create(lib, *dims, 1.0, 1.0, 1.0, 1.5, 1.0, 1.0, 0)
    assert st == status and not h.value


@pytest.mark.parametrize("bad", [
    (0.0, 1.0, 1.0, 1.5, 1.0, 1.0), (1.0, -1.0, 1.0, 1.5, 1.0, 1.0), (1.0, 1.0, float("nan"), 1.5, 1.0, 1.0),
    (1.0, 1.0, 1.0, float("inf"), 1.0, 1.0), (1.0, 1.0, 1.0, 1.5, 0.0, 1.0), (1.0, 1.0, 1.0, 1.5, 1.0, -2.0),
])
def test_invalid_parameters_rejected(lib, bad):
    st, h = _create(lib, 8, 8, 8, *bad, 0)
    assert st == 1 and not h.value


def test_invalid_dtype_and_null_args(lib):
    assert _create(lib, 8, 8, 8, 1.0, 1.0, 1.0, 1.5, 1.0, 1.0, 2)[0] == 7
    assert _create(lib, 8, 8, 8, 1.0, 1.0, 1.0, 1.5, 1.0, 1.0, 3)[0] == 7
    assert _create(lib, 8, 8, 8, 1.0, 1.0, 1.0, 1.5, 1.0, 1.0, 9)[0] == 1
    assert lib.sbp_plan_create(None, 8, 8, 8, 1.0, 1.0, 1.0, 1.5, 1.0, 1.0, 0) == 1
    assert lib.sbp_solve(None, None, None, 0.0, None) == 1
    assert lib.sbp_run_stage(None, 0, None, None, 0.0, None) == 1
    assert lib.sbp_plan_info(None, None, None, None, None, None, None) == 1
    assert lib.sbp_plan_set_option(None, 0, 0.0) == 1
    lib.sbp_plan_destroy(None)  # NULL-safe
    assert lib.sbp_solve_batched(-1, None, None, None, None, None) == 1
    assert lib.sbp_solve_batched(0, None, None, None, None, None) == 0


def test_binding_checks_batch_lengths():
    # argument marshalling only: mismatched list lengths never reach the library
    from paper_2510_10070_gb300 import sbp

    with pytest.raises(ValueError):
        sbp.solve_batched([], [], [], [1.0])


def _header_enum(prefix):
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(" + prefix + r"[A-Z0-9_]*)\s*=\s*(\d+)", text)}


@pytest.mark.parametrize("enum_name,prefix,strip", [
    ("DType", "SBP_F", "SBP_"),
    ("Stage", "SBP_STAGE_", "SBP_STAGE_"),
    ("Option", "SBP_OPT_", "SBP_OPT_"),
])
def test_binding_enums_match_the_header(enum_name, prefix, strip):
    # the binding's enums carry exactly the header's names and values
    from paper_2510_10070_gb300 import sbp

    want = {k[len(strip):]: v for k, v in _header_enum(prefix).items()}
    got = {m.name: int(m.value) for m in getattr(sbp, enum_name)}
    assert got == want


def test_binding_status_codes_match_the_header():
    from paper_2510_10070_gb300 import sbp

    want = {k.replace("SBP_ERR_", "").replace("SBP_", ""): v for k, v in _header_enum("SBP_(?:ERR_|OK)").items()}
    got = {m.name: int(m.value) for m in sbp.Status}
    assert got == want
