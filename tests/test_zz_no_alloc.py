"""shg_eval_2c_noalloc: the entry point for callers that cannot allocate device
memory during a call (their memory comes only from their own pool, or they
must avoid allocation latency and its implicit synchronisation).  Its plan
lives in a fixed array inside the library instead of cudaMallocAsync memory.

Checked through the C ABI against shg_eval_2c on two calls in a row (the
second call reuses the array the first one left behind), with the same parity
bar as the other two-center tests.  This file is collected last.
"""
import numpy as np
import pytest

from paper_1701_06588_gb300 import _lib as L
from paper_1701_06588_gb300 import workloads as W
from tests.parity import TOL_FP64, excess

pytestmark = pytest.mark.gpu


def test_noalloc_matches_eval_2c_on_two_calls_in_a_row():
    import torch
    from paper_1701_06588_gb300 import api, build
    build.build()
    stream = torch.cuda.current_stream().cuda_stream
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
        for call in range(2):
            out = torch.full((total,), float("nan"), dtype=torch.float64, device="cuda")
            L.shg_eval_2c_noalloc(basis.handle, len(pa), d_pa, d_pb, op, omega, L.SHG_PREC_FP64, d_off, out, stream)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert np.all(np.isfinite(got)), (name, call)
            e = excess(got, ref_h, TOL_FP64[:2])
            assert e <= 1.0, (name, call, e)
        basis.close()


def test_noalloc_rejects_lists_beyond_its_maximum():
    import torch
    from paper_1701_06588_gb300 import api
    shells, pa, pb = W.make("c1_2k_l3_k4", n=4)
    basis = api.Basis(shells)
    with pytest.raises(L.ShgError) as e:
        L.shg_eval_2c_noalloc(basis.handle, (1 << 20) + 1, 1, 1, L.SHG_OP_OVERLAP, 0.0, L.SHG_PREC_FP64, 1, 1,
                              torch.cuda.current_stream().cuda_stream)
    assert e.value.code == L.SHG_ERANGE
    assert "maximum" in str(e.value)
    basis.close()
