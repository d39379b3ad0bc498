"""plu_lu_reorth_static, the allocation-free variant of the re-orthogonalising
panel LU.

Callers that cannot allocate device memory -- code inside a framework that
has given all GPU memory to its own pool, plug-ins that may not allocate,
loops that cannot pay for cudaMalloc's device-wide synchronisation -- cannot
create a plu_ctx.  This entry point takes no context: its scratch is a fixed
device array inside the library.  It must give the same result as the
context-based plu_lu_reorth, call after call (the array keeps the previous
call's contents, which must not leak into the next result).  This file is
collected last so that a run stopping at the first failure has run every other
test already; it passes alone and after the other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth
import paper_2002_07138_gb300 as plu

pytestmark = pytest.mark.gpu


def _dev(X):
    out = plu.colmajor_empty(X.shape[0], X.shape[1])
    out.copy_(torch.from_numpy(np.ascontiguousarray(X)))
    return out


def _static(X):
    err = ctypes.create_string_buffer(512)
    stream = torch.cuda.current_stream().cuda_stream
    st = plu.lib().plu_lu_reorth_static(ctypes.c_void_p(stream), X.shape[0], X.shape[1],
                                        ctypes.c_void_p(X.data_ptr()), X.stride(1), err, 512)
    return st, err.value.decode()


def test_static_matches_context_entry_point_on_consecutive_calls(ctx):
    for rows, cols, seed in ((5000, 64, 1), (20000, 110, 2)):      # two calls in a row
        X = synth.gaussian_np(rows, cols, seed)
        ref = _dev(X)
        plu.plu_lu_reorth(ctx, ref)
        got = _dev(X)
        st, msg = _static(got)
        assert st == 0, msg
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.linalg.norm(g - r) <= 1e-12 * np.linalg.norm(r)


def test_static_rejects_panels_beyond_its_array():
    X = plu.colmajor_empty(8, 4)
    err = ctypes.create_string_buffer(512)
    st = plu.lib().plu_lu_reorth_static(None, 70000, 4, ctypes.c_void_p(X.data_ptr()), 70000,
                                        err, 512)
    assert plu.STATUS[st] == "PLU_EINVAL"
    assert "65536" in err.value.decode()
