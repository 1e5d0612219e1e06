"""The allocation-free left environment update against the regular one.

Some callers cannot allocate device memory while they run (a framework whose
allocator owns the device heap, a latency-critical loop); for them the
library offers tt_env_left_step_noalloc, which keeps its intermediates in a
fixed device array instead of allocating. This file is collected last so that
a failure here stops a `-x` run only after every other test has run.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2509_11890_gb300 as tg  # noqa: E402
from paper_2509_11890_gb300 import _lib, inputs  # noqa: E402

# (rw, rw2, R, R2, rv, rv2, m, n); the first two span several GEMM tiles with ragged tails
SHAPES = [(17, 9, 7, 3, 66, 5, 4, 4), (3, 70, 5, 33, 2, 65, 4, 4), (32, 32, 64, 64, 32, 32, 4, 4)]


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("shape", SHAPES)
def test_noalloc_matches_regular_entry_point_twice(shape):
    rw, rw2, R, R2, rv, rv2, m, n = shape
    dims = _lib.ContractDims(*shape)
    lib = tg.lib()
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        g = inputs.rng(100 + call, 7)
        phi, u = _t(g.standard_normal((rw, R, rv))), _t(g.standard_normal((rw, m, rw2)))
        op, v = _t(g.standard_normal((R, m, n, R2))), _t(g.standard_normal((rv, n, rv2)))
        ref = torch.empty(rw2 * R2 * rv2, dtype=torch.float64, device="cuda")
        got = torch.full_like(ref, float("nan"))
        st = lib.tt_env_left_step(ctypes.byref(dims), phi.data_ptr(), u.data_ptr(), op.data_ptr(), v.data_ptr(),
                                  ref.data_ptr(), 0, stream)
        assert st == 0
        st = lib.tt_env_left_step_noalloc(ctypes.byref(dims), phi.data_ptr(), u.data_ptr(), op.data_ptr(),
                                          v.data_ptr(), got.data_ptr(), stream)
        assert st == 0
        torch.cuda.synchronize()
        r, o = ref.cpu().numpy(), got.cpu().numpy()
        assert np.linalg.norm(o - r) <= 1e-11 * np.linalg.norm(r), (call, shape)


def test_noalloc_rejects_shapes_beyond_its_scratch():
    # intermediates of 2 * 64*200*4*64 doubles (6.6M) exceed the 2^22-double array;
    # the buffers have their full sizes, so the call touches nothing out of bounds
    # whatever it returns
    rw, rw2, R, R2, rv, rv2, m, n = 64, 64, 200, 200, 64, 64, 4, 4
    assert rw * R * n * rv2 + rw * m * R2 * rv2 > (1 << 22)
    dims = _lib.ContractDims(rw, rw2, R, R2, rv, rv2, m, n)
    z = lambda k: torch.zeros(k, dtype=torch.float64, device="cuda")
    phi, u, op, v, out = z(rw * R * rv), z(rw * m * rw2), z(R * m * n * R2), z(rv * n * rv2), z(rw2 * R2 * rv2)
    st = tg.lib().tt_env_left_step_noalloc(ctypes.byref(dims), phi.data_ptr(), u.data_ptr(), op.data_ptr(),
                                           v.data_ptr(), out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert st == 3  # TT_E_NOMEM
