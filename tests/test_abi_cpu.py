"""Host-side checks of the C ABI that need no GPU: the library loads and
exports every entry point include/orqa.h declares, and the argument checks
that run before any CUDA call."""
import ctypes
import os
import re

import pytest

from paper_2506_13241_gb300 import build, orqa

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "orqa.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return orqa.library()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^[A-Za-z_][\w \*]*?\b(orqa_\w+)\s*\(", text, re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    assert names == sorted(orqa.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_workspace_bytes_is_monotone_and_rejects_bad_sizes(lib):
    assert orqa.orqa_workspace_bytes(0, 10) == 0
    assert orqa.orqa_workspace_bytes(129, 10) == 0
    assert orqa.orqa_workspace_bytes(12, 0) == 0
    a = orqa.orqa_workspace_bytes(64, 1000)
    b = orqa.orqa_workspace_bytes(65, 1000)
    c = orqa.orqa_workspace_bytes(65, 100000)
    assert 0 < a < b < c
    assert a % 256 == 0 and b % 256 == 0


def test_create_validates_config_before_touching_cuda(lib):
    h = ctypes.c_void_p()
    assert lib.orqa_create(None, ctypes.byref(h)) == orqa.ORQA_EINVAL
    cfg = orqa.orqa_config(12, 0, 100, 0, 0, 0)       # null workspace
    assert lib.orqa_create(ctypes.byref(cfg), ctypes.byref(h)) == orqa.ORQA_EINVAL
    cfg = orqa.orqa_config(12, 0, 100, 256 + 3, 1 << 20, 0)  # misaligned
    assert lib.orqa_create(ctypes.byref(cfg), ctypes.byref(h)) == orqa.ORQA_EINVAL
    cfg = orqa.orqa_config(12, 0, 100, 4096, 10, 0)    # too small
    assert lib.orqa_create(ctypes.byref(cfg), ctypes.byref(h)) == orqa.ORQA_ENOMEM
    cfg = orqa.orqa_config(12, 8, 100, 4096, 1 << 30, 0)  # unknown flag bit
    assert lib.orqa_create(ctypes.byref(cfg), ctypes.byref(h)) == orqa.ORQA_EINVAL
    cfg = orqa.orqa_config(12, 0, 100, 4096, 1 << 30, 0, orqa.ORQA_MAX_PROBLEMS + 1, 0)  # too many problems
    assert lib.orqa_create(ctypes.byref(cfg), ctypes.byref(h)) == orqa.ORQA_EINVAL
    cfg = orqa.orqa_config(12, 0, 100, 4096, 1 << 30, 0, -1, 0)
    assert lib.orqa_create(ctypes.byref(cfg), ctypes.byref(h)) == orqa.ORQA_EINVAL
    cfg = orqa.orqa_config(12, orqa.ORQA_FLAG_RELATIVE, 100, 4096, 1 << 30, 0, 4, 0)  # relative + batched
    assert lib.orqa_create(ctypes.byref(cfg), ctypes.byref(h)) == orqa.ORQA_EINVAL
    cfg = orqa.orqa_config(12, 0, 100, 4096, 1 << 30, 0, 4, 1)  # reserved field set
    assert lib.orqa_create(ctypes.byref(cfg), ctypes.byref(h)) == orqa.ORQA_EINVAL


def test_batch_workspace_sizes(lib):
    one = orqa.orqa_workspace_bytes(127, 10000)
    assert orqa.orqa_workspace_bytes_batch(127, 10000, 1) == one
    assert orqa.orqa_workspace_bytes_batch(127, 10000, 0) == one
    b2, b96 = orqa.orqa_workspace_bytes_batch(127, 10000, 2), orqa.orqa_workspace_bytes_batch(127, 10000, 96)
    assert one < b2 < b96 and b96 % 256 == 0
    assert orqa.orqa_workspace_bytes_batch(127, 10000, orqa.ORQA_MAX_PROBLEMS + 1) == 0


def test_gate_array_marshalling():
    arr = orqa.gate_array([("rx", 3, None, 0.5), ("rzz", 1, 2, -1.5)])
    assert (arr[0].kind, arr[0].q0, arr[0].theta) == (orqa.ORQA_RX, 3, 0.5)
    assert (arr[1].kind, arr[1].q0, arr[1].q1) == (orqa.ORQA_RZZ, 1, 2)
    assert ctypes.sizeof(orqa.orqa_gate) == 24
    assert ctypes.sizeof(orqa.orqa_config) == 48
    assert ctypes.sizeof(orqa.orqa_stats_t) == 96
    assert ctypes.sizeof(orqa.orqa_kernel_profile) == 64
    assert ctypes.sizeof(orqa.orqa_layer_desc) == 24
    assert ctypes.sizeof(orqa.orqa_tuning) == 16


def test_label_encoding_matches_paper_codes():
    """x/z planes re-code the paper's two-bit index (z = high bit,
    x = high xor low)."""
    from paritylib import planes_to_codes
    x, z = orqa.strings_from_labels(["IXYZ" * 20], 80)
    codes = planes_to_codes(x, z, 80)
    assert list(codes[0][:4]) == [0, 1, 2, 3]


def test_bad_gates_and_programs_are_rejected():
    import numpy as np
    import pytest
    with pytest.raises(ValueError):
        orqa.gate_array([("ry", 0, None, 0.1)])
    xx = [("rx", q, None, 0.3) for q in range(4)]
    with pytest.raises(ValueError):
        orqa.Program([(xx, True, np.zeros((2, 3)))], n_problems=2)   # theta must be [P, n_gates]
    prog = orqa.Program([(xx, True, np.zeros((2, 4))), (xx, False, None)], n_problems=2)
    assert prog.n_expect_per_rep == 1 and prog.desc[0].n_gates == 4 and prog.desc[1].theta is None


def test_bad_labels_are_rejected():
    import pytest
    for bad in (["IXQZ"], ["x"], ["I" * 13]):
        with pytest.raises(ValueError):
            orqa.strings_from_labels(bad, 12)
    x, z = orqa.strings_from_labels(["", "I" * 12], 12)
    assert not x.any() and not z.any()


def test_null_context_is_rejected_before_any_cuda_call(lib):
    """Every entry point that takes a context returns ORQA_EINVAL for a null
    one, without touching CUDA."""
    E = orqa.ORQA_EINVAL
    n = ctypes.c_int64()
    d = ctypes.c_double()
    t = orqa.orqa_tuning()
    g = (orqa.orqa_gate * 1)()
    desc = (orqa.orqa_layer_desc * 1)()
    buf = (ctypes.c_uint64 * 4)()
    assert lib.orqa_set_operator(None, 0, None, None, None) == E
    assert lib.orqa_set_operator_batch(None, 0, None, None, None, None) == E
    assert lib.orqa_apply_layer(None, g, 1, 0.0, ctypes.byref(n)) == E
    assert lib.orqa_apply_layer_batch(None, g, 1, None, 0.0, ctypes.byref(n)) == E
    assert lib.orqa_apply_pauli_rotation(None, buf, buf, 0.1, 0.0, ctypes.byref(n)) == E
    assert lib.orqa_merge_truncate(None, 0.0, ctypes.byref(n)) == E
    assert lib.orqa_expect(None, ctypes.byref(d)) == E
    assert lib.orqa_expect_batch(None, ctypes.byref(d)) == E
    assert lib.orqa_problem_sizes(None, ctypes.byref(n)) == E
    assert lib.orqa_histogram(None, 4, -2.0, ctypes.byref(n), None) == E
    assert lib.orqa_run_program(None, desc, 1, 1, 0.0, None, 0) == E
    assert lib.orqa_get_tuning(None, ctypes.byref(t)) == E
    assert lib.orqa_set_tuning(None, ctypes.byref(t)) == E
    assert lib.orqa_autotune(None, desc, 1, 1, 0.0, 1, ctypes.byref(t), None) == E
    assert lib.orqa_stats(None, None) == E
    assert lib.orqa_profile(None, 0, None) == E
    assert lib.orqa_set_norm_tracking(None, 1) == E
    assert lib.orqa_debug_set(None, orqa.ORQA_DEBUG_PASS_LIMIT, 1) == E


def test_noalloc_rejects_bad_sizes_before_any_cuda_call(lib):
    d = ctypes.c_double()
    assert lib.orqa_expect_noalloc(0, 1, None, None, ctypes.byref(d), None) == orqa.ORQA_EINVAL
    assert lib.orqa_expect_noalloc(127, -1, None, None, ctypes.byref(d), None) == orqa.ORQA_EINVAL
    assert lib.orqa_expect_noalloc(127, orqa.ORQA_NOALLOC_MAX_STRINGS + 1, None, None, ctypes.byref(d),
                                   None) == orqa.ORQA_ECAPACITY
    assert lib.orqa_expect_noalloc(127, 5, None, None, ctypes.byref(d), None) == orqa.ORQA_EINVAL


def test_binding_constants_match_the_header():
    """Every ORQA_* constant the header defines (enum members with explicit
    values and #define'd numbers) has the same value in the binding, so the
    binding stays thin marshalling of the C declarations."""
    header = open(HEADER).read()
    header = re.sub(r"/\*.*?\*/", " ", header, flags=re.S)
    found = {}
    for name, value in re.findall(r"\b(ORQA_[A-Z0-9_]+)\s*=\s*(\d+)", header):
        found[name] = int(value)
    for name, value in re.findall(r"#define\s+(ORQA_[A-Z0-9_]+)\s+(\d+)(?:LL)?\b", header):
        found[name] = int(value)
    assert len(found) >= 20
    for name, value in sorted(found.items()):
        assert hasattr(orqa, name), name
        assert getattr(orqa, name) == value, (name, getattr(orqa, name), value)
