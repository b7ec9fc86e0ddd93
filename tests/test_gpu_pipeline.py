"""api.HostPipeline2c: host pair lists in, host blocks out, the pair list
planned in contiguous chunks whose read-back overlaps the next chunk's
fused pass.  Every pair is computed by the same kernel code whatever chunk
or tile it lands in, so the blocks must equal those of one fused pass over
the whole list bit for bit; and the planner's chunked scan must give the
same tiles for any chunk boundary (ragged chunks, a chunk of one pair)."""
import numpy as np
import pytest

from paper_1701_06588_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def shg():
    import torch
    from paper_1701_06588_gb300 import api, build
    build.build()
    torch.cuda.init()
    return api


@pytest.mark.parametrize("name,n,ops", [
    ("c2_200k_l4_k8", 5001, [("overlap", 0.0), ("coulomb", 0.0), ("erfc", 0.11), ("erf", 0.11), ("gauss", 1.0)]),
    ("c3_2m_l6_k20", 3001, [("coulomb", 0.0), ("erfc", 0.11)])])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_pipeline_equals_one_fused_pass(shg, name, n, ops, precision):
    import torch
    sh, pa, pb = W.make(name, n=n)
    b = shg.Basis(sh)
    off, total = b.pair_offsets(pa, pb)
    names, oms = [o[0] for o in ops], [o[1] for o in ops]
    d_off = torch.from_numpy(off).cuda()
    outs = [torch.full((total,), float("nan"), dtype=torch.float64, device="cuda") for _ in ops]
    plan = shg.Plan2c(b, pa, pb)
    plan.exec_fused(names, d_off, outs, omegas=oms, precision=precision)
    torch.cuda.synchronize()
    ref = [o.cpu().numpy() for o in outs]
    plan.close()
    pa_h = torch.from_numpy(pa).pin_memory()
    pb_h = torch.from_numpy(pb).pin_memory()
    off_h = torch.from_numpy(off).pin_memory()
    for chunks in (1, 3, 7, n):
        pipe = shg.HostPipeline2c(b, n_chunks=chunks)
        outs_h = [torch.full((total,), float("nan"), dtype=torch.float64).pin_memory() for _ in ops]
        pipe.run(pa_h, pb_h, off_h, names, outs_h, omegas=oms, precision=precision,
                 centers=np.asarray(sh["centers"]))
        torch.cuda.synchronize()
        for r, o in zip(ref, outs_h):
            assert np.array_equal(o.numpy(), r), (chunks, precision)
    b.close()
