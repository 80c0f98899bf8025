"""orqa_expect_noalloc: the expectation value for callers that cannot
allocate device memory (a host framework owning the memory pool, or a
latency-critical path).  Called through the C ABI on device arrays that the
test owns, and compared with the context-based orqa_expect on the same
operator, twice in a row (the shared scratch keeps the previous call's
contents).  This file is collected last on purpose."""
import math

import numpy as np
import pytest

from paper_2506_13241_gb300 import workloads as W

pytestmark = pytest.mark.gpu

M_TOL = 1e-10


def test_expect_noalloc_matches_context_expect():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2506_13241_gb300 import build, orqa
    build.build()
    n, edges = W.heavy_hex_eagle()
    layers = W.kicked_ising_layers(n, edges, math.pi / 4)
    ctx = orqa.Context(n, 1 << 21)
    ctx.set_labels([(W.z_label(n, [62]), 1.0)])
    stream = torch.cuda.current_stream().cuda_stream
    for step in range(5):
        for layer in layers:
            ctx.apply_layer(layer, 1e-4)
        ref = ctx.expect()
        x, z, c = ctx.export()
        x_d = torch.from_numpy(np.ascontiguousarray(x).view(np.int64)).cuda()
        c_d = torch.from_numpy(np.ascontiguousarray(c)).cuda()
        for _ in range(2):
            got = orqa.orqa_expect_noalloc(n, len(c), x_d.data_ptr(), c_d.data_ptr(), stream)
            assert abs(got - ref) < M_TOL, (step, got, ref)
    assert len(c) == 426052


def test_expect_noalloc_limits():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2506_13241_gb300 import orqa
    x_d = torch.zeros(2, dtype=torch.int64, device="cuda")
    c_d = torch.ones(1, dtype=torch.float64, device="cuda")
    assert orqa.orqa_expect_noalloc(12, 0, x_d.data_ptr(), c_d.data_ptr()) == 0.0
    assert orqa.orqa_expect_noalloc(12, 1, x_d.data_ptr(), c_d.data_ptr()) == 1.0
    with pytest.raises(orqa.OrqaError) as ei:
        orqa.orqa_expect_noalloc(12, orqa.ORQA_NOALLOC_MAX_STRINGS + 1, x_d.data_ptr(), c_d.data_ptr())
    assert ei.value.status == orqa.ORQA_ECAPACITY
    # host memory and misaligned addresses are refused before any launch
    x_h = np.zeros(2, dtype=np.uint64)
    c_h = np.ones(1, dtype=np.float64)
    for xp, cp in ((x_h.ctypes.data, c_d.data_ptr()), (x_d.data_ptr(), c_h.ctypes.data),
                   (x_d.data_ptr() + 4, c_d.data_ptr()), (x_d.data_ptr(), c_d.data_ptr() + 4)):
        with pytest.raises(orqa.OrqaError) as ei:
            orqa.orqa_expect_noalloc(12, 1, xp, cp)
        assert ei.value.status == orqa.ORQA_EINVAL
    # the refusals leave no CUDA error behind: a valid call still works
    assert orqa.orqa_expect_noalloc(12, 1, x_d.data_ptr(), c_d.data_ptr()) == 1.0
