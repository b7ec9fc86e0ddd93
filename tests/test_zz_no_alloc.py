"""shg_eval_2c_noalloc: the entry point for callers that cannot allocate device
memory during a call (their memory comes only from their own pool, or they
must avoid allocation latency and its implicit synchronisation).  Its plan
lives in a fixed array inside the library instead of cudaMallocAsync memory.

Checked through the C ABI against shg_eval_2c on calls in a row (each call
reuses the array the previous one left behind): the results must be bitwise
equal, since both run the same kernel on the same bucketing.  After the
first call on the device, which sets up the array's address, the calls must
not draw on the device's stream-ordered memory pool (the pool shg_eval_2c
allocates its plan from) nor change the free device memory.
This file is collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_1701_06588_gb300 import _lib as L
from paper_1701_06588_gb300 import workloads as W

pytestmark = pytest.mark.gpu

_USED_MEM_CURRENT, _USED_MEM_HIGH = 7, 8          # CUmemPool_attribute


class _DefaultPool:
    """Usage counters of the current device's default memory pool (driver API)."""

    def __init__(self, device):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int()
        assert self.cu.cuDeviceGet(ctypes.byref(dev), device) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def get(self, attr):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        v = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, _USED_MEM_HIGH, ctypes.byref(v)) == 0


def test_noalloc_matches_eval_2c_on_two_calls_in_a_row():
    import torch
    from paper_1701_06588_gb300 import api, build
    build.build()
    stream = torch.cuda.current_stream().cuda_stream
    pool = _DefaultPool(torch.cuda.current_device())
    cases = [("c2_200k_l4_k8", 6000, "coulomb", 0.0), ("c3_2m_l6_k20", 3000, "erfc", 0.11)]
    for name, n, opname, omega in cases:
        shells, pa, pb = W.make(name, n=n)
        basis = api.Basis(shells)
        off, total = basis.pair_offsets(pa, pb)
        d_pa = torch.from_numpy(pa).cuda()
        d_pb = torch.from_numpy(pb).cuda()
        d_off = torch.from_numpy(off).cuda()
        op = L.OPERATORS[opname]
        ref = torch.full((total,), float("nan"), dtype=torch.float64, device="cuda")
        L.shg_eval_2c(basis.handle, len(pa), d_pa, d_pb, op, omega, 0.0, L.SHG_PREC_FP64, d_off, ref, stream)
        torch.cuda.synchronize()
        ref_h = ref.cpu().numpy()
        outs = [torch.full((total,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(3)]
        # the first call on a device looks up the array's address, which may load
        # the library's module holding it (the array's memory is committed then)
        L.shg_eval_2c_noalloc(basis.handle, len(pa), d_pa, d_pb, op, omega, L.SHG_PREC_FP64, d_off, outs[0], stream)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        used_before = pool.get(_USED_MEM_CURRENT)
        pool.reset_high()
        for call in (1, 2):
            L.shg_eval_2c_noalloc(basis.handle, len(pa), d_pa, d_pb, op, omega, L.SHG_PREC_FP64, d_off, outs[call],
                                  stream)
            torch.cuda.synchronize()
        assert pool.get(_USED_MEM_HIGH) <= used_before, (name, "drew on the stream-ordered pool")
        assert torch.cuda.mem_get_info()[0] == free_before, (name, "free device memory changed")
        assert L.shg_last_error() == ""
        for call in range(3):
            got = outs[call].cpu().numpy()
            assert np.array_equal(got, ref_h), (name, call, np.nanmax(np.abs(got - ref_h)))
        basis.close()


def test_noalloc_rejects_lists_beyond_its_maximum_and_other_precisions():
    import torch
    from paper_1701_06588_gb300 import api
    shells, pa, pb = W.make("c1_2k_l3_k4", n=4)
    basis = api.Basis(shells)
    st = torch.cuda.current_stream().cuda_stream
    with pytest.raises(L.ShgError) as e:
        L.shg_eval_2c_noalloc(basis.handle, (1 << 20) + 1, 1, 1, L.SHG_OP_OVERLAP, 0.0, L.SHG_PREC_FP64, 1, 1, st)
    assert e.value.code == L.SHG_ERANGE
    assert "maximum" in str(e.value)
    off, total = basis.pair_offsets(pa, pb)
    d_pa, d_pb, d_off = (torch.from_numpy(x).cuda() for x in (pa, pb, off))
    out = torch.zeros(total, dtype=torch.float64, device="cuda")
    with pytest.raises(L.ShgError) as e:
        L.shg_eval_2c_noalloc(basis.handle, len(pa), d_pa, d_pb, L.SHG_OP_COULOMB, 0.0, L.SHG_PREC_MIXED, d_off, out,
                              st)
    assert e.value.code == L.SHG_EINVAL and "FP64" in str(e.value)
    # a valid call after the failures leaves no error message behind
    L.shg_eval_2c_noalloc(basis.handle, len(pa), d_pa, d_pb, L.SHG_OP_COULOMB, 0.0, L.SHG_PREC_FP64, d_off, out, st)
    torch.cuda.synchronize()
    assert L.shg_last_error() == ""
    assert np.all(np.isfinite(out.cpu().numpy()))
    basis.close()
