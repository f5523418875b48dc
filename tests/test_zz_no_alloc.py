"""The allocation-free solve entry point (lsp_hj_solve_noalloc), for callers
that cannot allocate device memory (real-time loops that must not call
cudaMalloc, hosts whose device memory belongs to another allocator).

It is called through the C ABI and must give the same field as the
workspace entry point lsp_hj_solve on the same input, on two calls in a row
(the second on different data, so the built-in scratch holds the first
call's values when it starts), and must reject grids whose scratch need
exceeds its fixed size with a clear error.  This file is collected last and
runs alone or after the other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2411_03501_gb300 import binding as B
from paper_2411_03501_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def test_noalloc_solve_matches_workspace_solve_twice():
    spec, phi0, g = W.air3d(n=41, t_final=0.5)
    P = B.Problem(spec)
    lib = B.load()
    gt = _dev(g)
    inputs = [phi0, phi0 + 0.3 * W.smooth_field(spec, seed=17)]
    for call, p0 in enumerate(inputs):
        ref = _dev(p0)
        st_ref = P.solve(ref, gt, 0.0, 0.5)
        out = _dev(p0)
        st = B.lsp_solve_stats()
        rc = lib.lsp_hj_solve_noalloc(P.grid.handle, ctypes.byref(P.opts),
                                      ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_void_p(gt.data_ptr()), 0.0, 0.5, ctypes.byref(st),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == B.LSP_OK, lib.lsp_last_error()
        torch.cuda.synchronize()
        assert st.steps == st_ref["steps"] and st.stages == st_ref["stages"]
        # same kernels, same sequence: equal to the FP32 step tolerance of the
        # parity tests (8 u max|phi|), in practice bit for bit
        tol = 8 * 2.0 ** -24 * float(ref.abs().max())
        err = float((out - ref).abs().max())
        assert err <= tol, (call, err, tol)


def test_noalloc_rejects_grids_beyond_its_scratch():
    spec, phi0, g = W.air3d(n=201, t_final=0.01)  # 2 x 32.5 MB of stage fields > 32 MiB
    P = B.Problem(spec)
    x = _dev(phi0)
    with pytest.raises(B.LspError) as e:
        B.lsp_hj_solve_noalloc(P.grid, P.opts, x, _dev(g), 0.0, 0.01)
    assert e.value.status == B.LSP_ENOMEM
    assert "bytes" in str(e.value)
    # and a graph request is refused rather than allocating
    o = B.make_opts(rk_order=3, scheme="weno5", dtype="f32", tube=True, cfl=0.75, use_graph=True)
    small = W.air3d(n=21, t_final=0.01)
    P2 = B.Problem(small[0])
    with pytest.raises(B.LspError) as e:
        B.lsp_hj_solve_noalloc(P2.grid, o, _dev(small[1]), _dev(small[2]), 0.0, 0.01)
    assert e.value.status == B.LSP_EINVAL
