"""sld_restrict_noalloc: Z^T v computed without allocating device memory, for
callers whose device memory belongs to another allocator or who must not
call cudaMalloc / cudaFree.  Checked against sld_restrict (the allocating
entry point) on two calls in a row, through the C ABI.  Kept in a file that
pytest collects last."""
import ctypes as C

import numpy as np
import pytest

from paper_1510_02148_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1510_02148_gb300 import _build, sld
    _build.build()
    lib = sld.load()
    lib.sld_restrict_noalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    lib.sld_restrict_noalloc.restype = C.c_int
    return torch, sld, lib


def test_restrict_noalloc_matches_restrict_twice(env):
    torch, sld, lib = env
    P = W.lognormal_point_source(96, 80, 48, 6, (4, 4, 3), seed=11)
    s = sld.from_problem(P, stream=torch.cuda.current_stream().cuda_stream)
    out = torch.empty(P.d, dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(0)
    for call in range(2):
        v = rng.standard_normal(P.n) * (1.0 + call)
        vd = torch.from_numpy(v).cuda()
        st = lib.sld_restrict_noalloc(s._h, vd.data_ptr(), out.data_ptr())
        assert st == sld.OK, lib.sld_last_error().decode()
        torch.cuda.synchronize()
        ref = s.restrict(v)  # the allocating entry point
        assert np.max(np.abs(out.cpu().numpy() - ref)) <= 1e-13 * np.abs(v).sum(), call
    s.close()


def test_restrict_noalloc_rejects(env):
    torch, sld, lib = env
    P = W.lognormal_point_source(32, 32, 16, 4, (2, 2, 2), seed=3)
    s = sld.from_problem(P)
    vh = np.zeros(P.n)
    out = torch.empty(P.d, dtype=torch.float64, device="cuda")
    st = lib.sld_restrict_noalloc(s._h, vh.ctypes.data, out.data_ptr())  # host input
    assert st == sld.ERR_INVALID_ARG and b"device memory" in lib.sld_last_error()
    s.close()
    big = W.lognormal_point_source(64, 64, 32, 4, (16, 16, 4), seed=3)  # d = 2048 > 1024
    s = sld.from_problem(big)
    vd = torch.zeros(big.n, dtype=torch.float64, device="cuda")
    outb = torch.empty(big.d, dtype=torch.float64, device="cuda")
    st = lib.sld_restrict_noalloc(s._h, vd.data_ptr(), outb.data_ptr())
    assert st == sld.ERR_INVALID_ARG and b"d <= 1024" in lib.sld_last_error()
    s.close()
