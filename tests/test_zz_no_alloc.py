"""The allocation-free Frank-Wolfe entry point (lds_fw_exact_noalloc).

It is for callers that cannot allocate device memory themselves (a framework
that owns the device heap, a loop that cannot take cudaMalloc's implicit
synchronisation, a fixed memory budget); its only scratch is a fixed device
array inside the library.  This test calls it through the C-ABI twice in a row,
on one graph with two iteration counts, and checks its loads and weights bit
for bit against lds_fw's exact path (the tolerance of the other FW tests).  The
file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_2504_10937_gb300 import synth

pytestmark = pytest.mark.gpu


def test_noalloc_matches_lds_fw_on_two_calls():
    import torch
    from paper_2504_10937_gb300 import lds
    lib = lds.load()
    fn = lib.lds_fw_exact_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    n, u, v, _ = synth.chung_lu(5000, 20000, 2.1, seed=12, n_blocks=3, block_size_range=(20, 50))
    m = len(u)
    du = torch.from_numpy(u.astype(np.int32)).cuda()
    dv = torch.from_numpy(v.astype(np.int32)).cuda()
    R = torch.empty(n, dtype=torch.int64, device="cuda")
    W = torch.empty(m, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    with lds.Graph(n, u, v) as g:
        for iters in (57, 23):
            ref = g.fw(iters, precision="exact", want=("R", "W"))
            st = fn(n, m, du.data_ptr(), dv.data_ptr(), iters, R.data_ptr(), W.data_ptr(), stream)
            assert st == lds.OK, lib.lds_last_error()
            torch.cuda.synchronize()
            assert np.array_equal(R.cpu().numpy(), ref["R"])
            assert np.array_equal(W.cpu().numpy(), ref["W"])
    # a repeated edge and an unsorted list are refused (both would silently
    # differ from lds_fw on the same graph)
    for perm in (np.r_[0, np.arange(m - 1)], np.r_[1, 0, np.arange(2, m)]):
        pu = torch.from_numpy(u[perm].astype(np.int32)).cuda()
        pv = torch.from_numpy(v[perm].astype(np.int32)).cuda()
        st = fn(n, m, pu.data_ptr(), pv.data_ptr(), 3, R.data_ptr(), W.data_ptr(), stream)
        assert st == lds.EINVAL
        assert b"sorted" in lib.lds_last_error()
    # sizes beyond the fixed scratch are refused, and nothing is launched for them
    big = (1 << 20) + 1
    st = fn(big, 0, None, None, 1, R.data_ptr(), None, stream)
    assert st == lds.EINVAL
    assert b"scratch limit" in lib.lds_last_error()
