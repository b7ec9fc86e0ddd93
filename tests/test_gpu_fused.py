"""GPU parity of the fused multi-operator pass (shg_plan_2c_exec_fused: the
geometry-only factor Q_j of Sec. II B built once per shell pair and
contracted with the radial orders of every requested operator of Table S1),
FP64 and double-float, against the CPU oracle, and its agreement with the
single-operator pass of the same precision."""
import numpy as np
import pytest

from paper_1701_06588_gb300 import workloads as W
from tests.parity import _bar, TOL_FP64, TOL_MIXED, assert_parity, reference_2c

pytestmark = pytest.mark.gpu

C2_OPS = [("overlap", 0, 0.0), ("coulomb", 1, 0.0), ("erfc", 2, 0.11), ("erf", 3, 0.11), ("gauss", 4, 1.0)]
_REF = {}


@pytest.fixture(scope="module")
def shg():
    import torch
    from paper_1701_06588_gb300 import api, build
    build.build()
    torch.cuda.init()
    return api


def _ref(name, n, op, omega):
    key = (name, n, op, omega)
    if key not in _REF:
        sh, pa, pb = W.make(name, n=n)
        _REF[key] = reference_2c(sh, pa, pb, op, omega)
    return _REF[key]


def _tol(precision):
    return TOL_FP64 if precision == "fp64" else TOL_MIXED


def _fused(api, shells, pa, pb, ops, schedule="persistent", graph=False, precision="fp64"):
    """Fused pass over (name, op id, omega) triples; returns {name: blocks} and
    the single-operator results of the same plan."""
    import torch
    b = api.Basis(shells)
    off, total = b.pair_offsets(pa, pb)
    d_off = torch.from_numpy(off).cuda()
    plan = api.Plan2c(b, pa, pb, schedule=schedule)
    outs = [torch.full((max(total, 1),), float("nan"), dtype=torch.float64, device="cuda") for _ in ops]
    names = [o[0] for o in ops]
    omegas = [o[2] for o in ops]
    if graph:
        g = api.Graph2c(plan, names, omegas, d_off, outs, precision=precision, fused=True)
        g.launch()
        torch.cuda.synchronize()
        g.close()
    else:
        plan.exec_fused(names, d_off, outs, omegas=omegas, precision=precision)
    single = {}
    for name, _, om in ops:
        o = torch.full((max(total, 1),), float("nan"), dtype=torch.float64, device="cuda")
        plan.exec(name, d_off, o, omega=om, precision=precision)
        single[name] = o[:total].cpu().numpy()
    torch.cuda.synchronize()
    fused = {n: o[:total].cpu().numpy() for n, o in zip(names, outs)}
    plan.close()
    b.close()
    return fused, single


def _check(fused, single, ops, refs, what, precision="fp64"):
    worst = 0.0
    for name, op, om in ops:
        ref, scale = refs[(op, om)]
        worst = max(worst, assert_parity(fused[name], ref, _tol(precision), "%s fused %s %s" % (what, precision, name),
                                         scale))
        # same formula, sums in another order (the fused 1/r sum takes its far field,
        # T >= 120, as a product of per-primitive weights): agreement inside twice the
        # element-wise parity bar of the precision
        d = np.abs(fused[name] - single[name])
        bar = 2.0 * _bar(ref, _tol(precision), scale)
        assert np.all(d <= bar), (name, float(np.max(d / bar)))
    return worst


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("schedule,graph", [("persistent", False), ("per_class", False), ("persistent", True)])
def test_fused_c2_subset_all_five(shg, schedule, graph, precision):
    """First 3,000 pairs of the 200k recipe (every class up to l = 4, many
    tiles, ragged tails): the five headline operators in one pass."""
    sh, pa, pb = W.make("c2_200k_l4_k8", n=3000)
    fused, single = _fused(shg, sh, pa, pb, C2_OPS, schedule, graph, precision)
    refs = {(op, om): _ref("c2_200k_l4_k8", 3000, op, om) for _, op, om in C2_OPS}
    worst = _check(fused, single, C2_OPS, refs, "c2 %s graph=%s" % (schedule, graph), precision)
    print("fused %s %s graph=%s: largest parity excess %.3g" % (precision, schedule, graph, worst))


@pytest.mark.parametrize("ops", [
    [("erfc", 2, 0.11)],                                     # erfc alone: its own attenuated sum
    [("erf", 3, 0.3), ("erfc", 2, 0.11)],                    # different omegas: two attenuated sums
    [("gauss", 4, 1.0), ("overlap", 0, 0.0)],                # no Boys sums, order of the list reversed
    [("coulomb", 1, 0.0)],
    [("erf", 3, 0.11), ("coulomb", 1, 0.0)],
])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fused_operator_subsets(shg, ops, precision):
    sh, pa, pb = W.make("c2_200k_l4_k8", n=1200)
    fused, single = _fused(shg, sh, pa, pb, ops, precision=precision)
    refs = {(op, om): _ref("c2_200k_l4_k8", 1200, op, om) for _, op, om in ops}
    _check(fused, single, ops, refs, "c2 subset %s" % [o[0] for o in ops], precision)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fused_c3_high_l(shg, precision):
    """l up to 6 (J up to 7), K up to 20, exponents to 5000."""
    ops = [("coulomb", 1, 0.0), ("erfc", 2, 0.11), ("overlap", 0, 0.0)]
    sh, pa, pb = W.make("c3_2m_l6_k20", n=1500)
    fused, single = _fused(shg, sh, pa, pb, ops, precision=precision)
    refs = {(op, om): _ref("c3_2m_l6_k20", 1500, op, om) for _, op, om in ops}
    worst = _check(fused, single, ops, refs, "c3", precision)
    print("fused %s c3: largest parity excess %.3g" % (precision, worst))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fused_full_size_c2_sampled(shg, precision):
    """The full 200k-pair workload in the benchmark's form (autotuned plan
    launch shape aside, one fused graph replay); 400 sampled pairs of every
    operator checked element by element against the oracle."""
    import torch
    sh, pa, pb = W.make("c2_200k_l4_k8")
    b = shg.Basis(sh)
    off, total = b.pair_offsets(pa, pb)
    plan = shg.Plan2c(b, pa, pb, schedule="persistent")
    d_off = torch.from_numpy(off).cuda()
    outs = [torch.full((total,), float("nan"), dtype=torch.float64, device="cuda") for _ in C2_OPS]
    g = shg.Graph2c(plan, [o[0] for o in C2_OPS], [o[2] for o in C2_OPS], d_off, outs, precision=precision, fused=True)
    g.launch()
    torch.cuda.synchronize()
    idx = np.sort(np.random.default_rng(124).choice(len(pa), 400, replace=False))
    sub, spa, spb = W.subset_pairs(sh, pa, pb, idx)
    l = sh["l"]
    for (opname, op, omega), out in zip(C2_OPS, outs):
        res = out.cpu().numpy()
        assert np.all(np.isfinite(res)), opname
        got = np.concatenate([res[off[p]:off[p] + (2 * l[pa[p]] + 1) * (2 * l[pb[p]] + 1)] for p in idx])
        ref, scale = reference_2c(sub, spa, spb, op, omega)
        assert_parity(got, ref, _tol(precision), "c2 full-size fused sampled %s %s" % (precision, opname), scale)
    g.close()
    plan.close()
    b.close()


def test_fused_edge_cases_and_errors(shg):
    import torch
    from paper_1701_06588_gb300 import _lib as L
    sh, pa, pb = W.make("c1_2k_l3_k4", n=40)
    b = shg.Basis(sh)
    # empty pair list: nothing to do, no error
    plan0 = shg.Plan2c(b, pa[:0], pb[:0])
    z = torch.zeros(1, dtype=torch.float64, device="cuda")
    plan0.exec_fused(["coulomb", "overlap"], torch.zeros(1, dtype=torch.int64, device="cuda"), [z, z.clone()])
    plan0.close()
    off, total = b.pair_offsets(pa, pb)
    d_off = torch.from_numpy(off).cuda()
    plan = shg.Plan2c(b, pa, pb)
    outs = [torch.zeros(total, dtype=torch.float64, device="cuda") for _ in range(6)]
    bad = [
        (["ra2n"], [1.0]),                         # not a fused operator
        (["gauss_coulomb"], [0.3]),
        (["coulomb", "coulomb"], [0.0, 0.0]),      # repeated
        (["erf"], [0.0]),                          # omega must be > 0
        (["gauss"], [float("nan")]),
        ([], []),
        (["overlap", "coulomb", "erfc", "erf", "gauss", "overlap"], [0, 0, 0.1, 0.1, 1, 0]),
    ]
    for ops, om in bad:
        with pytest.raises(L.ShgError) as e:
            plan.exec_fused(ops, d_off, outs[:len(ops)], omegas=om)
        assert e.value.code == L.SHG_EINVAL, ops
        with pytest.raises(L.ShgError):
            shg.Graph2c(plan, ops, om, d_off, outs[:len(ops)], fused=True)
    for prec in (2, -1):                           # not a precision
        with pytest.raises(L.ShgError) as e:
            L.shg_plan_2c_exec_fused(plan.handle, [1], [0.0], prec, d_off, outs[:1], None)
        assert e.value.code == L.SHG_EINVAL
    # the gauss_coulomb and ra2n operators are not part of the fused pass in either precision
    with pytest.raises(L.ShgError):
        plan.exec_fused(["gauss_coulomb"], d_off, outs[:1], omegas=[0.3], precision="mixed")
    # a valid call after the errors still works and matches the single-operator pass
    plan.exec_fused(["erfc", "gauss"], d_off, outs[:2], omegas=[0.2, 0.5])
    ref = torch.zeros(total, dtype=torch.float64, device="cuda")
    plan.exec("gauss", d_off, ref, omega=0.5)
    torch.cuda.synchronize()
    r = ref.cpu().numpy()
    assert np.all(np.abs(outs[1].cpu().numpy() - r) <= 1e-13 * (np.abs(r) + np.abs(r).max()))
    plan.close()
    b.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fused_kernel_variants_are_bitwise_equal(shg, precision):
    """The compiled variants of the persistent fused kernels differ only in
    their register caps: the same operations in the same order, so every
    block must be bitwise equal; a variant outside 0..2 is rejected."""
    import torch
    from paper_1701_06588_gb300 import _lib as L
    sh, pa, pb = W.make("c3_2m_l6_k20", n=4000)
    b = shg.Basis(sh)
    off, total = b.pair_offsets(pa, pb)
    d_off = torch.from_numpy(off).cuda()
    names, oms = ["coulomb", "erfc"], [0.0, 0.11]
    plan = shg.Plan2c(b, pa, pb)
    res = []
    for variant in (0, 1, 2):
        shg.set_launch(plan, 128, 0, variant)
        outs = [torch.full((total,), float("nan"), dtype=torch.float64, device="cuda") for _ in names]
        plan.exec_fused(names, d_off, outs, omegas=oms, precision=precision)
        torch.cuda.synchronize()
        res.append([o.cpu().numpy() for o in outs])
    for v in (1, 2):
        for a, r in zip(res[v], res[0]):
            assert np.array_equal(a, r), (precision, v)
    with pytest.raises(L.ShgError):
        L.shg_plan_2c_set_variant(plan.handle, 3)
    plan.close()
    b.close()
