"""GPU parity of the two-center SHG path (C ABI) against the CPU oracle."""
import numpy as np
import pytest

import oracle
from paper_1701_06588_gb300 import workloads as W
from tests.parity import TOL_FP64, assert_parity, reference_2c

pytestmark = pytest.mark.gpu

OPS = [("overlap", 0, 0.0), ("coulomb", 1, 0.0), ("erfc", 2, 0.11), ("erf", 3, 0.11), ("gauss", 4, 1.0),
       ("gauss_coulomb", 5, 0.3)]
_REF = {}


def _oracle(name, n, op, omega):
    """Oracle blocks of a named workload, computed once per module."""
    key = (name, n, op, omega)
    if key not in _REF:
        sh, pa, pb = W.make(name, n=n)
        _REF[key] = reference_2c(sh, pa, pb, op, omega)
    return _REF[key]


@pytest.fixture(scope="module")
def shg():
    import torch
    from paper_1701_06588_gb300 import api, build
    build.build()
    torch.cuda.init()
    return api


def _run(api, shells, pa, pb, opname, omega, schedule="persistent", precision="fp64"):
    import torch
    b = api.Basis(shells)
    off, total = b.pair_offsets(pa, pb)
    plan = api.Plan2c(b, pa, pb, schedule=schedule)
    out = torch.full((max(total, 1),), float("nan"), dtype=torch.float64, device="cuda")
    plan.exec(opname, torch.from_numpy(off).cuda(), out, omega=omega, precision=precision)
    torch.cuda.synchronize()
    res = out[:total].cpu().numpy()
    plan.close()
    b.close()
    return res


@pytest.mark.parametrize("opname,op,omega", OPS)
@pytest.mark.parametrize("schedule", ["per_class", "persistent"])
def test_c1_full(shg, opname, op, omega, schedule):
    """2,000 pairs, l <= 3, K = 4 (the small configuration), every element."""
    sh, pa, pb = W.make("c1_2k_l3_k4")
    got = _run(shg, sh, pa, pb, opname, omega, schedule)
    ref, scale = _oracle("c1_2k_l3_k4", None, op, omega)
    assert_parity(got, ref, TOL_FP64, "c1 %s %s" % (opname, schedule), scale)


@pytest.mark.parametrize("opname,op,omega", OPS)
def test_c2_subset(shg, opname, op, omega):
    """First 3,000 pairs of the 200k workload recipe (l <= 4, K 1..8): spans
    every class, many tiles and ragged tile tails."""
    sh, pa, pb = W.make("c2_200k_l4_k8", n=3000)
    got = _run(shg, sh, pa, pb, opname, omega)
    ref, scale = reference_2c(sh, pa, pb, op, omega)
    assert_parity(got, ref, TOL_FP64, "c2 %s" % opname, scale)


@pytest.mark.parametrize("opname,op,omega", [("coulomb", 1, 0.0), ("erfc", 2, 0.11), ("gauss_coulomb", 5, 0.3)])
def test_c3_subset_high_l_long_contractions(shg, opname, op, omega):
    """l up to 6, K up to 20, exponents to 5000."""
    sh, pa, pb = W.make("c3_2m_l6_k20", n=1500)
    got = _run(shg, sh, pa, pb, opname, omega)
    ref, scale = reference_2c(sh, pa, pb, op, omega)
    assert_parity(got, ref, TOL_FP64, "c3 %s" % opname, scale)


def test_full_size_c2_sampled(shg):
    """The full 200k-pair workload in the benchmark's launch configuration;
    400 sampled pairs checked element by element against the oracle."""
    import torch
    sh, pa, pb = W.make("c2_200k_l4_k8")
    b = shg.Basis(sh)
    off, total = b.pair_offsets(pa, pb)
    plan = shg.Plan2c(b, pa, pb, schedule="persistent")
    d_off = torch.from_numpy(off).cuda()
    rng = np.random.default_rng(123)
    idx = np.sort(rng.choice(len(pa), 400, replace=False))
    sub, spa, spb = W.subset_pairs(sh, pa, pb, idx)
    for opname, op, omega in OPS:
        out = torch.full((total,), float("nan"), dtype=torch.float64, device="cuda")
        plan.exec(opname, d_off, out, omega=omega)
        torch.cuda.synchronize()
        res = out.cpu().numpy()
        assert np.all(np.isfinite(res)), opname
        got = np.concatenate([res[off[p]:off[p] + (2 * sh["l"][pa[p]] + 1) * (2 * sh["l"][pb[p]] + 1)] for p in idx])
        ref, scale = reference_2c(sub, spa, spb, op, omega)
        assert_parity(got, ref, TOL_FP64, "c2 full-size sampled %s" % opname, scale)
    plan.close()
    b.close()


def test_edge_cases(shg):
    import torch
    # empty pair list
    sh, pa, pb = W.make("c1_2k_l3_k4", n=5)
    b = shg.Basis(sh)
    out, off = shg.eval_2c(b, pa[:0], pb[:0], "coulomb")
    assert out.numel() == 0
    # one pair, both shells on one center (R = 0), every l combination up to 6, K = 1 and K = 20
    rng = np.random.default_rng(5)
    ls, ks = [], []
    for la in range(7):
        for lb in range(7):
            ls += [la, lb]
    n = len(ls) // 2
    for K in (1, 20):
        nprim = np.full(2 * n, K, np.int32)
        shells = dict(l=np.array(ls, np.int32), nprim=nprim, exps=np.exp(rng.uniform(np.log(0.05), np.log(500), 2 * n * K)),
                      coefs=rng.uniform(-1, 1, 2 * n * K), centers=np.zeros((1, 3)),
                      center_of=np.zeros(2 * n, np.int32))
        pa = np.arange(0, 2 * n, 2, dtype=np.int32)
        pb = pa + 1
        for opname, op, omega in OPS:
            got = _run(shg, shells, pa, pb, opname, omega)
            ref, scale = reference_2c(shells, pa, pb, op, omega)
            assert_parity(got, ref, TOL_FP64, "R=0 K=%d %s" % (K, opname), scale)
    # a pair of one shell with itself, and a pair list with repeated pairs
    sh, pa, pb = W.make("c2_200k_l4_k8", n=40)
    pa2 = np.r_[pa, pa[:7], pb[:3]].astype(np.int32)
    pb2 = np.r_[pb, pb[:7], pb[:3]].astype(np.int32)
    got = _run(shg, sh, pa2, pb2, "overlap", 0.0)
    ref, scale = reference_2c(sh, pa2, pb2, 0, 0.0)
    assert_parity(got, ref, TOL_FP64, "repeated pairs", scale)
    b.close()


def test_errors_are_reported(shg):
    import torch
    from paper_1701_06588_gb300 import _lib as L
    sh, pa, pb = W.make("c1_2k_l3_k4", n=4)
    b = shg.Basis(sh)
    bad = torch.tensor([0, 1, 2, 10_000], dtype=torch.int32, device="cuda")
    good = torch.tensor([0, 1, 2, 3], dtype=torch.int32, device="cuda")
    with pytest.raises(L.ShgError) as e:
        shg.Plan2c(b, bad, good)
    assert e.value.code == L.SHG_EINVAL
    plan = shg.Plan2c(b, good, good)
    out = torch.zeros(100, dtype=torch.float64, device="cuda")
    off = torch.zeros(4, dtype=torch.int64, device="cuda")
    for op, om in [("erf", 0.0), ("gauss", -1.0), ("gauss_coulomb", 0.0), (7, 1.0)]:
        with pytest.raises(L.ShgError):
            plan.exec(op, off, out, omega=om)
    plan.close()
    b.close()


def test_set_centers_rejects_non_finite_and_keeps_previous(shg):
    """shg_basis_set_centers packs and checks the coordinates on the device:
    a non-finite coordinate is reported with the first bad center and the
    basis keeps its previous centers; a valid update is seen by a new plan."""
    import torch
    from paper_1701_06588_gb300 import _lib as L
    sh, pa, pb = W.make("c1_2k_l3_k4", n=200)
    b = shg.Basis(sh)

    def run():
        off, total = b.pair_offsets(pa, pb)
        plan = shg.Plan2c(b, pa, pb)
        out = torch.zeros(total, dtype=torch.float64, device="cuda")
        plan.exec("coulomb", torch.from_numpy(off).cuda(), out)
        torch.cuda.synchronize()
        plan.close()
        return out.cpu().numpy()

    before = run()
    c = sh["centers"].copy()
    for bad_center, val in ((7, np.nan), (3, np.inf), (len(c) - 1, -np.inf)):
        cb = c.copy()
        cb[bad_center, 1] = val
        cb[bad_center + 1:, 0] = np.nan      # later bad centers: the first one is named
        with pytest.raises(L.ShgError) as e:
            b.set_centers(cb)
        assert e.value.code == L.SHG_EINVAL
        assert "center %d " % bad_center in str(e.value), str(e.value)
        assert np.array_equal(run(), before)
    moved = c + np.array([0.25, -0.5, 1.0])
    b.set_centers(moved)
    assert np.allclose(run(), before, rtol=1e-12, atol=1e-14)   # a rigid translation
    c2 = c.copy()
    c2[::2] *= 1.1
    b.set_centers(c2)
    sh2 = dict(sh, centers=c2)
    ref, scale = reference_2c(sh2, pa, pb, 1, 0.0)
    assert_parity(run(), ref, TOL_FP64, "c1 coulomb after set_centers", scale)
    b.close()


def test_device_boys_against_oracle(shg):
    import torch
    from paper_1701_06588_gb300 import _lib as L
    T = np.concatenate([[0.0, 1e-12, 1e-3], np.linspace(0, 40, 3001), np.exp(np.linspace(np.log(30), np.log(800), 300)),
                        np.array([35.999999, 36.0, 36.000001])])
    dT = torch.from_numpy(T).cuda()
    nmax = 15
    dF = torch.empty(len(T) * (nmax + 1), dtype=torch.float64, device="cuda")
    L.shg_debug_boys(len(T), dT, nmax, dF, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    F = dF.cpu().numpy().reshape(len(T), nmax + 1)
    ref = np.stack([oracle.boys(nmax, t) for t in T])
    rel = np.abs(F - ref) / ref
    # 15 downward recursion steps from F_15: about 20 ulp at F_0
    assert rel.max() < 1e-14, rel.max()


def test_graph_replay_and_launch_shapes(shg):
    """A captured CUDA graph of several operators reproduces the direct plan
    execution, sees later shg_basis_set_centers updates, and every launch
    shape the autotuner may pick gives the same blocks."""
    import torch
    from paper_1701_06588_gb300 import autotune
    sh, pa, pb = W.make("c2_200k_l4_k8", n=4000)
    b = shg.Basis(sh)
    off, total = b.pair_offsets(pa, pb)
    d_off = torch.from_numpy(off).cuda()
    names = ["overlap", "coulomb", "erfc"]
    omegas = [0.0, 0.0, 0.11]
    for prec in ("fp64", "mixed"):
        plan = shg.Plan2c(b, pa, pb)
        ref = []
        for n, w in zip(names, omegas):
            o = torch.empty(total, dtype=torch.float64, device="cuda")
            plan.exec(n, d_off, o, omega=w, precision=prec)
            ref.append(o)
        outs = [torch.full((total,), float("nan"), dtype=torch.float64, device="cuda") for _ in names]
        g = shg.Graph2c(plan, names, omegas, d_off, outs, precision=prec)
        g.launch()
        torch.cuda.synchronize()
        for o, r in zip(outs, ref):
            assert torch.equal(o, r)
        # new geometry: graph replay follows the basis
        c2 = sh["centers"] + 0.01
        b.set_centers(c2)
        g.launch()
        torch.cuda.synchronize()
        ref2, _ = shg.eval_2c(b, pa, pb, "coulomb", precision=prec)
        assert torch.equal(outs[1], ref2)
        b.set_centers(sh["centers"])
        g.close()
        for sched, threads, ctas in autotune.CANDIDATES:
            p2 = autotune.tuned_plan(b, pa, pb, {"schedule": sched, "threads_per_cta": threads, "ctas_per_sm": ctas})
            o = torch.full((total,), float("nan"), dtype=torch.float64, device="cuda")
            p2.exec("erfc", d_off, o, omega=0.11, precision=prec)
            torch.cuda.synchronize()
            assert torch.equal(o, ref[2]), (prec, sched, threads, ctas)
            p2.close()
        plan.close()
    b.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_screening_bound(shg, precision):
    """With screen_thresh > 0, overlap and Gaussian-operator pairs whose bound
    is below it write zeros: every element stays within thr of the exact
    block, and on the 0..10 bohr workload a share of the pairs is screened.
    Coulomb-type operators are never screened."""
    import torch
    sh, pa, pb = W.make("c2_200k_l4_k8", n=4000)
    b = shg.Basis(sh)
    off, total = b.pair_offsets(pa, pb)
    d_off = torch.from_numpy(off).cuda()
    plan = shg.Plan2c(b, pa, pb)
    sizes = np.diff(np.r_[off, total])
    for opname, omega in [("overlap", 0.0), ("gauss", 1.0), ("coulomb", 0.0)]:
        exact = torch.empty(total, dtype=torch.float64, device="cuda")
        plan.exec(opname, d_off, exact, omega=omega, precision=precision)
        for thr in (1e-10, 1e-6):
            scr = torch.full((total,), float("nan"), dtype=torch.float64, device="cuda")
            plan.exec(opname, d_off, scr, omega=omega, precision=precision, screen_thresh=thr)
            torch.cuda.synchronize()
            e, s = exact.cpu().numpy(), scr.cpu().numpy()
            assert np.all(np.isfinite(s))
            assert np.max(np.abs(s - e)) <= thr, (opname, thr)
            zero_blocks = np.array([not np.any(s[o:o + z]) and np.any(e[o:o + z]) for o, z in zip(off, sizes)])
            if opname == "coulomb":
                np.testing.assert_array_equal(s, e)
            elif thr == 1e-6:
                assert zero_blocks.mean() > 0.01, (opname, zero_blocks.mean())
    plan.close()
    b.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_full_size_c3_sampled(shg, precision):
    """The full 2,000,000-pair workload (l up to 6, K up to 20) in one
    persistent launch per operator; 300 sampled pairs against the oracle."""
    import torch
    from tests.parity import TOL_MIXED
    sh, pa, pb = W.make("c3_2m_l6_k20")
    b = shg.Basis(sh)
    off, total = b.pair_offsets(pa, pb)
    plan = shg.Plan2c(b, pa, pb, schedule="persistent")
    d_off = torch.from_numpy(off).cuda()
    idx = np.sort(np.random.default_rng(321).choice(len(pa), 300, replace=False))
    sub, spa, spb = W.subset_pairs(sh, pa, pb, idx)
    l = sh["l"]
    for opname, op, omega in [("coulomb", 1, 0.0), ("erfc", 2, 0.11)]:
        out = torch.full((total,), float("nan"), dtype=torch.float64, device="cuda")
        plan.exec(opname, d_off, out, omega=omega, precision=precision)
        torch.cuda.synchronize()
        got = torch.cat([out[int(off[p]):int(off[p]) + (2 * int(l[pa[p]]) + 1) * (2 * int(l[pb[p]]) + 1)]
                         for p in idx]).cpu().numpy()
        ref, scale = reference_2c(sub, spa, spb, op, omega)
        assert_parity(got, ref, TOL_FP64 if precision == "fp64" else TOL_MIXED,
                      "c3 full-size sampled %s %s" % (precision, opname), scale)
        del out
    plan.close()
    b.close()


def test_alu_peak_probes_report_positive_rates():
    """The three throughput probes (FP64 FMA, FP32 FMA, FP64 tensor-core MMA)
    run and report finite positive rates; a bad kind is rejected."""
    import torch
    from paper_1701_06588_gb300 import _lib as L, build
    build.build()
    st = torch.cuda.current_stream().cuda_stream
    rates = [L.shg_measure_alu_peak(k, 256, st) for k in (0, 1, 2)]
    assert all(np.isfinite(r) and r > 1e9 for r in rates), rates
    assert rates[1] > rates[0]
    with pytest.raises(L.ShgError):
        L.shg_measure_alu_peak(3, 256, st)
