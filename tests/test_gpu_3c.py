"""GPU parity of the three-index overlap (a b a~) path (C ABI) against the oracle."""
import numpy as np
import pytest

from paper_1701_06588_gb300 import workloads as W
from tests.parity import TOL_FP64, TOL_MIXED, assert_parity, reference_3c

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def shg():
    import torch
    from paper_1701_06588_gb300 import api, build
    build.build()
    torch.cuda.init()
    return api


def _run(api, shells, ta, tt, tb, precision="fp64"):
    import torch
    b = api.Basis(shells)
    out, off = api.eval_3c_aab(b, b, ta, tt, tb, precision=precision)
    torch.cuda.synchronize()
    res = out.cpu().numpy()
    b.close()
    return res


@pytest.mark.parametrize("layout", ["orbital_pairs_on_A", "aux_on_A"])
def test_aab_subset(shg, layout):
    """Atom-pair blocks of the 32-atom-cluster recipe (seed 3): orbital pairs
    on A with auxiliary b on B, and the paper's layout (orbital a and
    auxiliary a~ on A, orbital b on B, la + la~ up to 10)."""
    sh, ta, tt, tb, per = W.aab_workload(12, seed=3, layout=layout)
    got = _run(shg, sh, ta, tt, tb)
    ref, scale = reference_3c(sh, ta, tt, tb)
    assert_parity(got, ref, TOL_FP64, "aab " + layout, scale)


def test_aab_full_size_sampled(shg):
    """The 20,000 atom-pair workload (3,000,000 triples) in one call; 300
    sampled triples checked element by element against the oracle."""
    import torch
    sh, ta, tt, tb, per = W.make("c4_aab_20k")
    b = shg.Basis(sh)
    out, off = shg.eval_3c_aab(b, b, ta, tt, tb)
    torch.cuda.synchronize()
    l = sh["l"].astype(np.int64)
    sizes = (2 * l[ta] + 1) * (2 * l[tt] + 1) * (2 * l[tb] + 1)
    rng = np.random.default_rng(77)
    idx = np.sort(rng.choice(len(ta), 300, replace=False))
    res = torch.cat([out[int(off[i]):int(off[i] + sizes[i])] for i in idx]).cpu().numpy()
    ref, scale = reference_3c(sh, ta[idx], tt[idx], tb[idx])
    assert_parity(res, ref, TOL_FP64, "aab full-size sampled", scale)
    b.close()


def test_aab_one_center_and_errors(shg):
    import torch
    from paper_1701_06588_gb300 import _lib as L
    sh, ta, tt, tb, per = W.aab_workload(2, seed=5)
    sh1 = dict(sh, centers=np.zeros_like(sh["centers"]))
    got = _run(shg, sh1, ta, tt, tb)
    ref, scale = reference_3c(sh1, ta, tt, tb)
    assert_parity(got, ref, TOL_FP64, "aab R=0", scale)
    # a and a~ on different centers is rejected
    b = shg.Basis(sh)
    other = np.where(sh["center_of"] != sh["center_of"][ta[0]])[0][0]
    with pytest.raises(L.ShgError) as e:
        shg.eval_3c_aab(b, b, ta[:1], np.array([other], np.int32), tb[:1])
    assert e.value.code == L.SHG_EINVAL and "same center" in str(e.value)
    b.close()


@pytest.mark.parametrize("layout", ["orbital_pairs_on_A", "aux_on_A"])
def test_aab_mixed_subset(shg, layout):
    """Mixed form (radial sums FP64, angular part and Gaunt sum in
    double-float) against the oracle with the mixed bar, both layouts."""
    sh, ta, tt, tb, per = W.aab_workload(12, seed=3, layout=layout)
    got = _run(shg, sh, ta, tt, tb, precision="mixed")
    ref, scale = reference_3c(sh, ta, tt, tb)
    assert_parity(got, ref, TOL_MIXED, "aab mixed " + layout, scale)


def test_aab_mixed_full_size_sampled_and_one_center(shg):
    import torch
    from paper_1701_06588_gb300 import _lib as L
    sh, ta, tt, tb, per = W.make("c4_aab_20k")
    b = shg.Basis(sh)
    out, off = shg.eval_3c_aab(b, b, ta, tt, tb, precision="mixed")
    torch.cuda.synchronize()
    l = sh["l"].astype(np.int64)
    sizes = (2 * l[ta] + 1) * (2 * l[tt] + 1) * (2 * l[tb] + 1)
    idx = np.sort(np.random.default_rng(78).choice(len(ta), 300, replace=False))
    res = torch.cat([out[int(off[i]):int(off[i] + sizes[i])] for i in idx]).cpu().numpy()
    ref, scale = reference_3c(sh, ta[idx], tt[idx], tb[idx])
    assert_parity(res, ref, TOL_MIXED, "aab mixed full-size sampled", scale)
    w = torch.ones(int(sizes.sum()), dtype=torch.float64, device="cuda")
    with pytest.raises(L.ShgError) as e:          # the (aab) gradient is FP64 only
        shg.eval_3c_aab_grad(b, b, ta[:5], tt[:5], tb[:5], w[:int(sizes[:5].sum())], precision="mixed")
    assert e.value.code == L.SHG_EINVAL
    b.close()
    sh2, ta2, tt2, tb2, _ = W.aab_workload(2, seed=5)
    sh1 = dict(sh2, centers=np.zeros_like(sh2["centers"]))
    got = _run(shg, sh1, ta2, tt2, tb2, precision="mixed")
    ref, scale = reference_3c(sh1, ta2, tt2, tb2)
    assert_parity(got, ref, TOL_MIXED, "aab mixed R=0", scale)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_aab_screening_bound(shg, precision):
    """screen_thresh > 0 writes zeros only for triples whose bound is below
    it: every element stays within the threshold of the unscreened result,
    some blocks are screened at 1e-6, and the others are unchanged."""
    import torch
    sh, ta, tt, tb, per = W.aab_workload(60, seed=3)
    b = shg.Basis(sh)
    exact, off = shg.eval_3c_aab(b, b, ta, tt, tb, precision=precision)
    e = exact.cpu().numpy()
    l = sh["l"].astype(np.int64)
    sizes = (2 * l[ta] + 1) * (2 * l[tt] + 1) * (2 * l[tb] + 1)
    for thr in (1e-10, 1e-6):
        scr, _ = shg.eval_3c_aab(b, b, ta, tt, tb, precision=precision, screen_thresh=thr)
        torch.cuda.synchronize()
        s_ = scr.cpu().numpy()
        assert np.all(np.isfinite(s_))
        assert np.max(np.abs(s_ - e)) <= thr, (precision, thr)
        zero = np.array([not np.any(s_[o:o + z]) and np.any(e[o:o + z]) for o, z in zip(off, sizes)])
        kept = ~np.array([not np.any(s_[o:o + z]) for o, z in zip(off, sizes)])
        for o, z, k in zip(off, sizes, kept):
            if k:
                assert np.array_equal(s_[o:o + z], e[o:o + z])
        if thr == 1e-6:
            assert zero.mean() > 0.01, zero.mean()
    with pytest.raises(Exception):
        shg.eval_3c_aab(b, b, ta, tt, tb, precision=precision, screen_thresh=-1.0)
    b.close()
