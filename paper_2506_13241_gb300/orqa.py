"""Thin Python binding of liborqa (include/orqa.h).

Each ``orqa_*`` function here has the name of the C entry point it calls and
only marshals arguments: numpy host arrays and torch device tensors become
pointers, workload gate tuples become ``orqa_gate`` records.  Every step of
the sparse Pauli dynamics runs in the CUDA library.  PyTorch supplies the
device workspace and the stream.  There is no CPU fallback: if the library
or a CUDA device is missing, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

ORQA_OK, ORQA_EINVAL, ORQA_ENOMEM, ORQA_ECAPACITY, ORQA_ECUDA, ORQA_ETIMEOUT, ORQA_ESTATE = range(7)
STATUS_NAMES = ["ORQA_OK", "ORQA_EINVAL", "ORQA_ENOMEM", "ORQA_ECAPACITY", "ORQA_ECUDA",
                "ORQA_ETIMEOUT", "ORQA_ESTATE"]
ORQA_RX, ORQA_RZZ = 1, 2
ORQA_FLAG_PROFILE = 1
ORQA_FLAG_RELATIVE = 2
ORQA_FLAG_FP32 = 4
EXPORTED = ["orqa_workspace_bytes", "orqa_create", "orqa_set_operator", "orqa_set_operator_device",
            "orqa_apply_layer", "orqa_merge_truncate", "orqa_expect", "orqa_export", "orqa_stats",
            "orqa_profile_count", "orqa_profile", "orqa_profile_reset",
            "orqa_last_error", "orqa_destroy", "orqa_expect_noalloc",
            "orqa_workspace_bytes_batch", "orqa_set_operator_batch", "orqa_apply_layer_batch",
            "orqa_expect_batch", "orqa_problem_sizes", "orqa_export_batch",
            "orqa_run_program", "orqa_get_tuning", "orqa_set_tuning", "orqa_autotune",
            "orqa_apply_pauli_rotation", "orqa_histogram", "orqa_set_norm_tracking", "orqa_debug_set",
            "orqa_shard_owner", "orqa_shard_split", "orqa_shard_append", "orqa_counters"]
ORQA_SHARD_MAX_RANKS = 512
ORQA_DEBUG_SPIN_LIMIT, ORQA_DEBUG_POISON_MERGE_TABLE, ORQA_DEBUG_MERGE_TABLE_SLOTS = 1, 2, 3
ORQA_DEBUG_PASS_LIMIT, ORQA_DEBUG_BUCKET_SHIFT, ORQA_DEBUG_NO_ZZ_FUSION = 4, 5, 6
ORQA_NOALLOC_MAX_STRINGS = 1 << 27
ORQA_MAX_PROBLEMS = 4096


class orqa_gate(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("q0", ctypes.c_int32), ("q1", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("theta", ctypes.c_double)]


class orqa_config(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_int32), ("flags", ctypes.c_int32), ("capacity", ctypes.c_int64),
                ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_uint64),
                ("stream", ctypes.c_void_p), ("n_problems", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class orqa_layer_desc(ctypes.Structure):
    _fields_ = [("gates", ctypes.POINTER(orqa_gate)), ("n_gates", ctypes.c_int32),
                ("expect_after", ctypes.c_int32), ("theta", ctypes.c_void_p)]


class orqa_tuning(ctypes.Structure):
    _fields_ = [("range_target", ctypes.c_int32), ("sub_max", ctypes.c_int32),
                ("bucket_density", ctypes.c_int32), ("grid_per_sm", ctypes.c_int32)]


class orqa_stats_t(ctypes.Structure):
    _fields_ = [("n_strings", ctypes.c_int64), ("last_layer_in", ctypes.c_int64),
                ("last_layer_peak", ctypes.c_int64), ("string_gate_updates", ctypes.c_int64),
                ("branch_events", ctypes.c_int64), ("dropped", ctypes.c_int64),
                ("pair_updates_one", ctypes.c_int64), ("pair_updates_two", ctypes.c_int64),
                ("chunk_passes", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("sum_sq", ctypes.c_double), ("max_abs", ctypes.c_double), ("dropped_sum_sq", ctypes.c_double)]


class orqa_kernel_profile(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("ms", ctypes.c_double),
                ("bytes", ctypes.c_double), ("floor_bytes", ctypes.c_double)]


class OrqaError(RuntimeError):
    def __init__(self, status, message):
        self.status = status
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < 7 else status, message))


_lib = None


def library(path: str | None = None) -> ctypes.CDLL:
    """Loads liborqa.so (built in-tree by ``build.build()``)."""
    global _lib
    if _lib is None:
        path = path or _build.LIB
        if not os.path.exists(path):
            raise OSError("liborqa.so not built: run paper_2506_13241_gb300.build.build() (%s)" % path)
        lib = ctypes.CDLL(path)
        vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        u64p = ctypes.POINTER(ctypes.c_uint64)
        dpp = ctypes.POINTER(ctypes.c_double)
        lib.orqa_workspace_bytes.restype = ctypes.c_uint64
        lib.orqa_workspace_bytes.argtypes = [i32, i64]
        lib.orqa_create.restype = i32
        lib.orqa_create.argtypes = [ctypes.POINTER(orqa_config), ctypes.POINTER(vp)]
        for name in ("orqa_set_operator", "orqa_set_operator_device"):
            f = getattr(lib, name)
            f.restype = i32
            f.argtypes = [vp, i64, vp, vp, vp]
        lib.orqa_apply_layer.restype = i32
        lib.orqa_apply_layer.argtypes = [vp, ctypes.POINTER(orqa_gate), i32, dp, ctypes.POINTER(i64)]
        lib.orqa_merge_truncate.restype = i32
        lib.orqa_merge_truncate.argtypes = [vp, dp, ctypes.POINTER(i64)]
        lib.orqa_expect.restype = i32
        lib.orqa_expect.argtypes = [vp, dpp]
        lib.orqa_export.restype = i32
        lib.orqa_export.argtypes = [vp, i64, u64p, u64p, dpp, ctypes.POINTER(i64)]
        lib.orqa_stats.restype = i32
        lib.orqa_stats.argtypes = [vp, ctypes.POINTER(orqa_stats_t)]
        lib.orqa_counters.restype = i32
        lib.orqa_counters.argtypes = [vp, ctypes.POINTER(orqa_stats_t)]
        lib.orqa_profile_count.restype = i32
        lib.orqa_profile_count.argtypes = []
        lib.orqa_profile.restype = i32
        lib.orqa_profile.argtypes = [vp, i32, ctypes.POINTER(orqa_kernel_profile)]
        lib.orqa_profile_reset.restype = i32
        lib.orqa_profile_reset.argtypes = [vp]
        lib.orqa_last_error.restype = ctypes.c_char_p
        lib.orqa_last_error.argtypes = [vp]
        lib.orqa_destroy.restype = None
        lib.orqa_destroy.argtypes = [vp]
        lib.orqa_expect_noalloc.restype = i32
        lib.orqa_expect_noalloc.argtypes = [i32, i64, vp, vp, dpp, vp]
        i32p = ctypes.POINTER(ctypes.c_int32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.orqa_workspace_bytes_batch.restype = ctypes.c_uint64
        lib.orqa_workspace_bytes_batch.argtypes = [i32, i64, i32]
        lib.orqa_set_operator_batch.restype = i32
        lib.orqa_set_operator_batch.argtypes = [vp, i64, vp, vp, vp, vp]
        lib.orqa_apply_layer_batch.restype = i32
        lib.orqa_apply_layer_batch.argtypes = [vp, ctypes.POINTER(orqa_gate), i32, vp, dp, i64p]
        lib.orqa_expect_batch.restype = i32
        lib.orqa_expect_batch.argtypes = [vp, dpp]
        lib.orqa_problem_sizes.restype = i32
        lib.orqa_problem_sizes.argtypes = [vp, i64p]
        lib.orqa_export_batch.restype = i32
        lib.orqa_export_batch.argtypes = [vp, i64, u64p, u64p, dpp, i32p, i64p]
        ldp = ctypes.POINTER(orqa_layer_desc)
        tp = ctypes.POINTER(orqa_tuning)
        lib.orqa_run_program.restype = i32
        lib.orqa_run_program.argtypes = [vp, ldp, i32, i32, dp, dpp, i64]
        lib.orqa_get_tuning.restype = i32
        lib.orqa_get_tuning.argtypes = [vp, tp]
        lib.orqa_set_tuning.restype = i32
        lib.orqa_set_tuning.argtypes = [vp, tp]
        lib.orqa_autotune.restype = i32
        lib.orqa_autotune.argtypes = [vp, ldp, i32, i32, dp, i32, tp, dpp]
        lib.orqa_apply_pauli_rotation.restype = i32
        lib.orqa_apply_pauli_rotation.argtypes = [vp, vp, vp, dp, dp, i64p]
        lib.orqa_histogram.restype = i32
        lib.orqa_histogram.argtypes = [vp, i32, dp, i64p, dpp]
        lib.orqa_set_norm_tracking.restype = i32
        lib.orqa_set_norm_tracking.argtypes = [vp, i32]
        lib.orqa_debug_set.restype = i32
        lib.orqa_debug_set.argtypes = [vp, i32, i64]
        lib.orqa_shard_owner.restype = i32
        lib.orqa_shard_owner.argtypes = [i32, i64, vp, i32, vp]
        lib.orqa_shard_split.restype = i32
        lib.orqa_shard_split.argtypes = [vp, i32, i32, i64, vp, i64p]
        lib.orqa_shard_append.restype = i32
        lib.orqa_shard_append.argtypes = [vp, i64, vp]
        _lib = lib
    return _lib


def words_per_plane(n_qubits: int) -> int:
    return 1 if n_qubits <= 64 else 2


def strings_from_labels(labels, n_qubits: int):
    """(x, z) uint64 planes [N, W] of Pauli labels (character q = qubit q)."""
    W = words_per_plane(n_qubits)
    x = np.zeros((len(labels), W), dtype=np.uint64)
    z = np.zeros((len(labels), W), dtype=np.uint64)
    for i, lab in enumerate(labels):
        if len(lab) > n_qubits or set(lab) - set("IXYZ"):
            raise ValueError("label %r: at most %d characters from I, X, Y, Z" % (lab, n_qubits))
        for q, ch in enumerate(lab):
            bit = np.uint64(1) << np.uint64(q % 64)
            if ch in "XY":
                x[i, q // 64] |= bit
            if ch in "ZY":
                z[i, q // 64] |= bit
    return x, z


def gate_array(gates):
    """orqa_gate[] from workload tuples (kind, q0, q1, theta)."""
    arr = (orqa_gate * len(gates))()
    kinds = {"rx": ORQA_RX, "rzz": ORQA_RZZ}
    for k, (kind, q0, q1, theta) in enumerate(gates):
        if kind not in kinds:
            raise ValueError("gate %d: kind %r is not one of %s" % (k, kind, sorted(kinds)))
        arr[k].kind = kinds[kind]
        arr[k].q0 = int(q0)
        arr[k].q1 = int(q1) if q1 is not None else 0
        arr[k].pad = 0
        arr[k].theta = float(theta)
    return arr


def _check(ctx, status):
    if status != ORQA_OK:
        msg = library().orqa_last_error(ctx).decode() if ctx else ""
        raise OrqaError(status, msg)


# --- the C entry points, same names -----------------------------------------

def orqa_workspace_bytes(n_qubits: int, capacity: int) -> int:
    return int(library().orqa_workspace_bytes(n_qubits, capacity))


def orqa_workspace_bytes_batch(n_qubits: int, capacity: int, n_problems: int) -> int:
    return int(library().orqa_workspace_bytes_batch(n_qubits, capacity, n_problems))


def orqa_create(n_qubits: int, capacity: int, workspace_ptr: int, workspace_bytes: int,
                stream_ptr: int = 0, flags: int = 0, n_problems: int = 0):
    cfg = orqa_config(n_qubits, flags, capacity, workspace_ptr, workspace_bytes, stream_ptr, n_problems, 0)
    h = ctypes.c_void_p()
    st = library().orqa_create(ctypes.byref(cfg), ctypes.byref(h))
    if st != ORQA_OK:
        raise OrqaError(st, "orqa_create")
    return h


def orqa_set_operator(ctx, x: np.ndarray, z: np.ndarray, c: np.ndarray):
    x = np.ascontiguousarray(x, dtype=np.uint64)
    z = np.ascontiguousarray(z, dtype=np.uint64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    _check(ctx, library().orqa_set_operator(ctx, len(c), x.ctypes.data, z.ctypes.data, c.ctypes.data))


def orqa_set_operator_device(ctx, x, z, c):
    """x, z: contiguous int64/uint64 torch tensors [N, W]; c: float64 [N]."""
    _check(ctx, library().orqa_set_operator_device(ctx, c.numel(), x.data_ptr(), z.data_ptr(),
                                                   c.data_ptr()))


def orqa_set_operator_batch(ctx, x: np.ndarray, z: np.ndarray, c: np.ndarray, problem: np.ndarray):
    x = np.ascontiguousarray(x, dtype=np.uint64)
    z = np.ascontiguousarray(z, dtype=np.uint64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    problem = np.ascontiguousarray(problem, dtype=np.int32)
    if len(problem) != len(c):
        raise ValueError("one problem index per string")
    _check(ctx, library().orqa_set_operator_batch(ctx, len(c), x.ctypes.data, z.ctypes.data, c.ctypes.data,
                                                  problem.ctypes.data))


def orqa_apply_layer_batch(ctx, gates, theta: np.ndarray, delta: float) -> int:
    """theta: [n_problems, n_gates] angles (row p: problem p)."""
    arr = gates if isinstance(gates, ctypes.Array) else gate_array(gates)
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    if theta.ndim != 2 or theta.shape[1] != len(arr):
        raise ValueError("theta must be [n_problems, n_gates]")
    n = ctypes.c_int64()
    _check(ctx, library().orqa_apply_layer_batch(ctx, arr, len(arr), theta.ctypes.data, float(delta),
                                                 ctypes.byref(n)))
    return n.value


def orqa_expect_batch(ctx, n_problems: int) -> np.ndarray:
    out = np.zeros(n_problems, dtype=np.float64)
    _check(ctx, library().orqa_expect_batch(ctx, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return out


def orqa_problem_sizes(ctx, n_problems: int) -> np.ndarray:
    out = np.zeros(n_problems, dtype=np.int64)
    _check(ctx, library().orqa_problem_sizes(ctx, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
    return out


def orqa_export_batch(ctx, n_qubits: int):
    W = words_per_plane(n_qubits)
    n = orqa_stats(ctx)["n_strings"]
    x = np.zeros((max(n, 1), W), dtype=np.uint64)
    z = np.zeros((max(n, 1), W), dtype=np.uint64)
    c = np.zeros(max(n, 1), dtype=np.float64)
    p = np.zeros(max(n, 1), dtype=np.int32)
    got = ctypes.c_int64()
    u64p = ctypes.POINTER(ctypes.c_uint64)
    _check(ctx, library().orqa_export_batch(ctx, n, x.ctypes.data_as(u64p), z.ctypes.data_as(u64p),
                                            c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                            p.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), ctypes.byref(got)))
    k = got.value
    return x[:k], z[:k], c[:k], p[:k]


class Program:
    """A layer sequence for orqa_run_program: items (gates, expect_after,
    theta) with theta an [n_problems, n_gates] array for batched X layers or
    None.  Keeps the ctypes arrays alive."""

    def __init__(self, layers, n_problems: int = 1):
        self.gates = [g if isinstance(g, ctypes.Array) else gate_array(g) for g, _, _ in layers]
        self.thetas = [None if t is None else np.ascontiguousarray(t, dtype=np.float64) for _, _, t in layers]
        self.desc = (orqa_layer_desc * len(layers))()
        self.n_expect_per_rep = 0
        for k, (_, e, _) in enumerate(layers):
            th = self.thetas[k]
            if th is not None and th.shape != (n_problems, len(self.gates[k])):
                raise ValueError("theta must be [n_problems, n_gates]")
            self.desc[k].gates = ctypes.cast(self.gates[k], ctypes.POINTER(orqa_gate))
            self.desc[k].n_gates = len(self.gates[k])
            self.desc[k].expect_after = 1 if e else 0
            self.desc[k].theta = th.ctypes.data if th is not None else None
            self.n_expect_per_rep += 1 if e else 0
        self.n_problems = n_problems


def orqa_run_program(ctx, program: Program, repeat: int, delta: float) -> np.ndarray:
    """Returns the expectation values as [repeat * n_expect_layers, n_problems]."""
    n = program.n_expect_per_rep * repeat * program.n_problems
    out = np.zeros(max(n, 1), dtype=np.float64)
    _check(ctx, library().orqa_run_program(ctx, program.desc, len(program.desc), repeat, float(delta),
                                           out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n))
    return out[:n].reshape(-1, program.n_problems)


def orqa_get_tuning(ctx) -> dict:
    t = orqa_tuning()
    _check(ctx, library().orqa_get_tuning(ctx, ctypes.byref(t)))
    return {name: getattr(t, name) for name, _ in orqa_tuning._fields_}


def orqa_set_tuning(ctx, **kw):
    t = orqa_tuning()
    _check(ctx, library().orqa_get_tuning(ctx, ctypes.byref(t)))
    for k, v in kw.items():
        setattr(t, k, int(v))
    _check(ctx, library().orqa_set_tuning(ctx, ctypes.byref(t)))


def orqa_autotune(ctx, program: Program, repeat: int, delta: float, trials: int = 2):
    t = orqa_tuning()
    ms = ctypes.c_double()
    _check(ctx, library().orqa_autotune(ctx, program.desc, len(program.desc), repeat, float(delta), trials,
                                        ctypes.byref(t), ctypes.byref(ms)))
    return {name: getattr(t, name) for name, _ in orqa_tuning._fields_}, ms.value


def orqa_apply_layer(ctx, gates, delta: float) -> int:
    arr = gates if isinstance(gates, ctypes.Array) else gate_array(gates)
    n = ctypes.c_int64()
    _check(ctx, library().orqa_apply_layer(ctx, arr, len(arr), float(delta), ctypes.byref(n)))
    return n.value


def orqa_apply_pauli_rotation(ctx, xj: np.ndarray, zj: np.ndarray, theta: float, delta: float) -> int:
    """One rotation exp(-i theta/2 sigma_J); xj, zj: the W plane words of J."""
    xj = np.ascontiguousarray(xj, dtype=np.uint64).reshape(-1)
    zj = np.ascontiguousarray(zj, dtype=np.uint64).reshape(-1)
    n = ctypes.c_int64()
    _check(ctx, library().orqa_apply_pauli_rotation(ctx, xj.ctypes.data, zj.ctypes.data, float(theta), float(delta),
                                                    ctypes.byref(n)))
    return n.value


def orqa_histogram(ctx, n_bins: int, log10_lo: float):
    """(counts [2, n_bins + 1] (row 0: c > 0, row 1: c < 0; column n_bins:
    below the lowest edge), max|c|)."""
    counts = np.zeros(2 * (n_bins + 1), dtype=np.int64)
    mx = ctypes.c_double()
    _check(ctx, library().orqa_histogram(ctx, n_bins, float(log10_lo),
                                         counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), ctypes.byref(mx)))
    return counts.reshape(2, n_bins + 1), mx.value


def orqa_merge_truncate(ctx, delta: float) -> int:
    n = ctypes.c_int64()
    _check(ctx, library().orqa_merge_truncate(ctx, float(delta), ctypes.byref(n)))
    return n.value


def orqa_expect(ctx) -> float:
    out = ctypes.c_double()
    _check(ctx, library().orqa_expect(ctx, ctypes.byref(out)))
    return out.value


def orqa_export(ctx, n_qubits: int):
    W = words_per_plane(n_qubits)
    n = orqa_stats(ctx)["n_strings"]
    x = np.zeros((max(n, 1), W), dtype=np.uint64)
    z = np.zeros((max(n, 1), W), dtype=np.uint64)
    c = np.zeros(max(n, 1), dtype=np.float64)
    got = ctypes.c_int64()
    lib = library()
    _check(ctx, lib.orqa_export(ctx, n, x.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                z.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(got)))
    return x[:got.value], z[:got.value], c[:got.value]


def orqa_stats(ctx) -> dict:
    s = orqa_stats_t()
    _check(ctx, library().orqa_stats(ctx, ctypes.byref(s)))
    return {name: getattr(s, name) for name, _ in orqa_stats_t._fields_ if name != "pad"}


def orqa_counters(ctx) -> dict:
    s = orqa_stats_t()
    _check(ctx, library().orqa_counters(ctx, ctypes.byref(s)))
    return {name: getattr(s, name) for name, _ in orqa_stats_t._fields_ if name != "pad"}


def orqa_set_norm_tracking(ctx, on: bool):
    _check(ctx, library().orqa_set_norm_tracking(ctx, 1 if on else 0))


def orqa_debug_set(ctx, knob: int, value: int):
    _check(ctx, library().orqa_debug_set(ctx, int(knob), int(value)))


def orqa_shard_owner(n_qubits: int, z: np.ndarray, n_ranks: int) -> np.ndarray:
    """Owner rank of each string's z plane (z: [N, W] uint64 host array)."""
    z = np.ascontiguousarray(z, dtype=np.uint64)
    out = np.zeros(max(len(z), 1), dtype=np.int32)
    st = library().orqa_shard_owner(n_qubits, len(z), z.ctypes.data, n_ranks, out.ctypes.data)
    if st != ORQA_OK:
        raise OrqaError(st, "orqa_shard_owner")
    return out[:len(z)]


def orqa_shard_split(ctx, n_ranks: int, rank: int, send_cap: int, send_ptr: int) -> np.ndarray:
    """Moves the strings other ranks own to the device buffer at send_ptr;
    returns the records per destination rank."""
    counts = np.zeros(n_ranks, dtype=np.int64)
    _check(ctx, library().orqa_shard_split(ctx, n_ranks, rank, send_cap, send_ptr,
                                           counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
    return counts


def orqa_shard_append(ctx, n: int, recv_ptr: int):
    _check(ctx, library().orqa_shard_append(ctx, n, recv_ptr))


def orqa_profile_count() -> int:
    return int(library().orqa_profile_count())


def orqa_profile(ctx, index: int) -> dict:
    p = orqa_kernel_profile()
    _check(ctx, library().orqa_profile(ctx, index, ctypes.byref(p)))
    return {"name": p.name.decode(), "launches": p.launches, "ms": p.ms, "bytes": p.bytes,
            "floor_bytes": p.floor_bytes}


def orqa_profile_reset(ctx):
    _check(ctx, library().orqa_profile_reset(ctx))


def orqa_last_error(ctx) -> str:
    return library().orqa_last_error(ctx).decode()


def orqa_destroy(ctx):
    library().orqa_destroy(ctx)


def orqa_expect_noalloc(n_qubits: int, n: int, x_ptr: int, c_ptr: int, stream_ptr: int = 0) -> float:
    """<0|O|0> of caller-owned device arrays (x: n*W words, c: n doubles),
    computed without a context and without any device allocation."""
    out = ctypes.c_double()
    st = library().orqa_expect_noalloc(n_qubits, n, x_ptr, c_ptr, ctypes.byref(out), stream_ptr)
    if st != ORQA_OK:
        raise OrqaError(st, "orqa_expect_noalloc (n=%d, limit %d)" % (n, ORQA_NOALLOC_MAX_STRINGS))
    return out.value


# --- convenience wrapper ------------------------------------------------------

class Context:
    """An operator on the current CUDA device.  The workspace is a torch
    uint8 tensor owned by this object; work runs on ``stream`` (a
    torch.cuda.Stream, default: the current stream)."""

    def __init__(self, n_qubits: int, capacity: int, stream=None, device=None, profile: bool = False,
                 relative: bool = False, fp32: bool = False, problems: int = 1):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("liborqa needs a CUDA device; none is available")
        library()
        self.n_qubits = n_qubits
        self.W = words_per_plane(n_qubits)
        self.capacity = capacity
        self.problems = problems
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            nbytes = orqa_workspace_bytes_batch(n_qubits, capacity, problems)
            if nbytes == 0:
                raise ValueError("bad n_qubits / capacity")
            self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
            base = self.workspace.data_ptr()
            aligned = (base + 255) // 256 * 256
            flags = ((ORQA_FLAG_PROFILE if profile else 0) | (ORQA_FLAG_RELATIVE if relative else 0) |
                     (ORQA_FLAG_FP32 if fp32 else 0))
            self.ctx = orqa_create(n_qubits, capacity, aligned, nbytes, self.stream.cuda_stream, flags,
                                   problems if problems > 1 else 0)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            orqa_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_operator(self, x, z, c):
        orqa_set_operator(self.ctx, x, z, c)

    def set_labels(self, terms):
        labels = [t[0] for t in terms]
        x, z = strings_from_labels(labels, self.n_qubits)
        self.set_operator(x, z, np.array([t[1] for t in terms], dtype=np.float64))

    def set_operator_device(self, x, z, c):
        orqa_set_operator_device(self.ctx, x, z, c)

    def set_operator_batch(self, x, z, c, problem):
        orqa_set_operator_batch(self.ctx, x, z, c, problem)

    def set_labels_batch(self, terms_per_problem):
        """terms_per_problem[p]: list of (label, coefficient) of problem p."""
        labels, coefs, pids = [], [], []
        for p, terms in enumerate(terms_per_problem):
            for lab, c in terms:
                labels.append(lab)
                coefs.append(c)
                pids.append(p)
        x, z = strings_from_labels(labels, self.n_qubits)
        self.set_operator_batch(x, z, np.array(coefs, dtype=np.float64), np.array(pids, dtype=np.int32))

    def apply_layer_batch(self, gates, theta, delta: float = 0.0) -> int:
        return orqa_apply_layer_batch(self.ctx, gates, theta, delta)

    def expect_batch(self) -> np.ndarray:
        return orqa_expect_batch(self.ctx, self.problems)

    def problem_sizes(self) -> np.ndarray:
        return orqa_problem_sizes(self.ctx, self.problems)

    def export_batch(self):
        return orqa_export_batch(self.ctx, self.n_qubits)

    def program(self, layers) -> Program:
        return Program(layers, self.problems)

    def run_program(self, program: Program, repeat: int, delta: float = 0.0) -> np.ndarray:
        return orqa_run_program(self.ctx, program, repeat, delta)

    def tuning(self) -> dict:
        return orqa_get_tuning(self.ctx)

    def set_tuning(self, **kw):
        orqa_set_tuning(self.ctx, **kw)

    def autotune(self, program: Program, repeat: int, delta: float = 0.0, trials: int = 2):
        return orqa_autotune(self.ctx, program, repeat, delta, trials)

    def apply_layer(self, gates, delta: float = 0.0) -> int:
        return orqa_apply_layer(self.ctx, gates, delta)

    def merge_truncate(self, delta: float = 0.0) -> int:
        return orqa_merge_truncate(self.ctx, delta)

    def histogram(self, n_bins: int, log10_lo: float):
        return orqa_histogram(self.ctx, n_bins, log10_lo)

    def apply_pauli_rotation(self, label: str, theta: float, delta: float = 0.0) -> int:
        """Rotation about the Pauli string `label` (character q = qubit q)."""
        x, z = strings_from_labels([label], self.n_qubits)
        return orqa_apply_pauli_rotation(self.ctx, x[0], z[0], theta, delta)

    def expect(self) -> float:
        return orqa_expect(self.ctx)

    def export(self):
        return orqa_export(self.ctx, self.n_qubits)

    def stats(self) -> dict:
        return orqa_stats(self.ctx)

    def counters(self) -> dict:
        return orqa_counters(self.ctx)

    def set_norm_tracking(self, on: bool = True):
        orqa_set_norm_tracking(self.ctx, on)

    def debug_set(self, knob: int, value: int):
        orqa_debug_set(self.ctx, knob, value)

    def profile(self) -> list:
        return [orqa_profile(self.ctx, k) for k in range(orqa_profile_count())]

    def profile_reset(self):
        orqa_profile_reset(self.ctx)

    def __len__(self):
        return self.stats()["n_strings"]
