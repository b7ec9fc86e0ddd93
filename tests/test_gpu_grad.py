"""GPU parity of the two-center gradient kernel (vector-Jacobian product with
respect to both centers) against the oracle's analytic gradients, central
finite differences and translation invariance; and the autograd wrapper."""
import numpy as np
import pytest

import oracle
from paper_1701_06588_gb300 import workloads as W
from tests.parity import normalised, vjp_reference

pytestmark = pytest.mark.gpu

GRAD_OPS = [("coulomb", 1, 0.0), ("erfc", 2, 0.11), ("overlap", 0, 0.0), ("erf", 3, 0.11), ("gauss", 4, 1.0),
            ("gauss_coulomb", 5, 0.3)]


@pytest.fixture(scope="module")
def shg():
    import torch
    from paper_1701_06588_gb300 import api, build
    build.build()
    torch.cuda.init()
    return api


def _oracle_vjp(shells, pa, pb, op, omega, w):
    """sum_e W_e dI_e/dR_a from the oracle Jacobian, and the element-wise bar
    scale sum_e |W_e| |dI_e/dR_a| with the |N c| Jacobian (conditioning of the
    dot product and of the contractions in it)."""
    shn, sha = normalised(shells)
    J, off, sz = oracle.eval_2c_grad(shn, pa, pb, op, omega, center="A", normalize=False)
    if op == oracle.OP_ERFC:
        J1, _, _ = oracle.eval_2c_grad(sha, pa, pb, oracle.OP_COULOMB, 0.0, center="A", normalize=False)
        J2, _, _ = oracle.eval_2c_grad(sha, pa, pb, oracle.OP_ERF, omega, center="A", normalize=False)
        Ja = np.abs(J1) + np.abs(J2)
    else:
        Ja, _, _ = oracle.eval_2c_grad(sha, pa, pb, op, omega, center="A", normalize=False)
    return vjp_reference(J, Ja, off, sz, w)


@pytest.mark.parametrize("name,n", [("c5_grad_500k_l5_k12", 1200), ("c2_200k_l4_k8", 800)])
@pytest.mark.parametrize("opname,op,omega", GRAD_OPS)
def test_grad_against_oracle(shg, name, n, opname, op, omega):
    import torch
    sh, pa, pb = W.make(name, n=n)
    b = shg.Basis(sh)
    off, total = b.pair_offsets(pa, pb)
    rng = np.random.default_rng(4)
    w = rng.uniform(-1, 1, total)
    ga, gb = shg.eval_2c_grad(b, pa, pb, opname, torch.from_numpy(w).cuda(), offsets=off, omega=omega)
    torch.cuda.synchronize()
    ga, gb = ga.cpu().numpy(), gb.cpu().numpy()
    np.testing.assert_array_equal(gb, -ga)
    ref, scale = _oracle_vjp(sh, pa, pb, op, omega, w)
    bar = 1e-10 * np.abs(ref) + 1e-12 + 1e-15 * scale
    ex = np.abs(ga - ref) / bar
    assert ex.max() <= 1.0, (opname, ex.max(), np.unravel_index(ex.argmax(), ex.shape))
    b.close()


@pytest.mark.parametrize("opname,op,omega", [("coulomb", 1, 0.0), ("erfc", 2, 0.11)])
def test_grad_against_finite_differences_of_gpu_forward(shg, opname, op, omega):
    """Central differences (h = 1e-5 bohr) of the GPU integrals themselves."""
    import torch
    sh, pa, pb = W.make("c5_grad_500k_l5_k12", n=300)
    b = shg.Basis(sh)
    off, total = b.pair_offsets(pa, pb)
    w = np.random.default_rng(8).uniform(-1, 1, total)
    ga, _ = shg.eval_2c_grad(b, pa, pb, opname, torch.from_numpy(w).cuda(), offsets=off, omega=omega)
    ga = ga.cpu().numpy()
    h = 1e-5
    fd = np.zeros_like(ga)
    ca = sh["center_of"][pa]
    for d in range(3):
        c = sh["centers"].copy()
        c[ca, d] += h
        b.set_centers(c)
        vp, _ = shg.eval_2c(b, pa, pb, opname, omega=omega)
        c[ca, d] -= 2 * h
        b.set_centers(c)
        vm, _ = shg.eval_2c(b, pa, pb, opname, omega=omega)
        diff = ((vp - vm) / (2 * h)).cpu().numpy() * w
        fd[:, d] = np.add.reduceat(diff, off)
    err = np.abs(ga - fd)
    assert np.all(err <= 1e-7 * np.maximum(1.0, np.abs(fd))), err.max()
    b.close()


def test_autograd_function_matches_finite_differences(shg):
    import torch
    sh, pa, pb = W.make("c2_200k_l4_k8", n=40)
    b = shg.Basis(sh)
    centers = torch.tensor(sh["centers"], dtype=torch.float64, requires_grad=True)
    out = shg.TwoCenterIntegrals.apply(centers, b, pa, pb, "coulomb", 0.0)
    wt = torch.from_numpy(np.random.default_rng(2).uniform(-1, 1, out.numel())).cuda()
    loss = (out * wt).sum()
    loss.backward()
    g = centers.grad.numpy()
    h = 1e-5
    for c_idx in [0, 1, 7, 30]:
        for d in range(3):
            cp = sh["centers"].copy(); cp[c_idx, d] += h
            cm = sh["centers"].copy(); cm[c_idx, d] -= h
            b.set_centers(cp)
            lp = float((shg.eval_2c(b, pa, pb, "coulomb")[0] * wt).sum())
            b.set_centers(cm)
            lm = float((shg.eval_2c(b, pa, pb, "coulomb")[0] * wt).sum())
            fd = (lp - lm) / (2 * h)
            assert abs(g[c_idx, d] - fd) <= 1e-7 * max(1.0, abs(fd)), (c_idx, d, g[c_idx, d], fd)
    b.close()


def _oracle_vjp_3c(shells, ta, tt, tb, w):
    shn, sha = normalised(shells)
    J, off, sz = oracle.eval_3c_aab_grad(shn, ta, tt, tb, center="A", normalize=False)
    Ja, _, _ = oracle.eval_3c_aab_grad(sha, ta, tt, tb, center="A", normalize=False)
    return vjp_reference(J, Ja, off, sz, w)


@pytest.mark.parametrize("layout", ["orbital_pairs_on_A", "aux_on_A"])
def test_aab_grad_against_oracle_and_translation(shg, layout):
    import torch
    sh, ta, tt, tb, per = W.aab_workload(6, seed=4, layout=layout)
    b = shg.Basis(sh)
    off, total = b.triple_offsets(b, ta, tt, tb)
    w = np.random.default_rng(14).uniform(-1, 1, total)
    ga, gb = shg.eval_3c_aab_grad(b, b, ta, tt, tb, torch.from_numpy(w).cuda(), offsets=off)
    torch.cuda.synchronize()
    ga, gb = ga.cpu().numpy(), gb.cpu().numpy()
    np.testing.assert_array_equal(gb, -ga)
    ref, scale = _oracle_vjp_3c(sh, ta, tt, tb, w)
    ex = np.abs(ga - ref) / (1e-10 * np.abs(ref) + 1e-12 + 1e-15 * scale)
    assert ex.max() <= 1.0, (layout, ex.max())
    b.close()


def test_aab_grad_against_finite_differences_of_gpu_forward(shg):
    import torch
    sh, ta, tt, tb, per = W.aab_workload(3, seed=6)
    b = shg.Basis(sh)
    off, total = b.triple_offsets(b, ta, tt, tb)
    w = np.random.default_rng(15).uniform(-1, 1, total)
    ga, _ = shg.eval_3c_aab_grad(b, b, ta, tt, tb, torch.from_numpy(w).cuda(), offsets=off)
    ga = ga.cpu().numpy()
    h = 1e-5
    cb = sh["center_of"][tb]
    fd = np.zeros_like(ga)
    for d in range(3):
        c = sh["centers"].copy()
        c[cb, d] += h
        b.set_centers(c)
        vp, _ = shg.eval_3c_aab(b, b, ta, tt, tb)
        c[cb, d] -= 2 * h
        b.set_centers(c)
        vm, _ = shg.eval_3c_aab(b, b, ta, tt, tb)
        diff = ((vp - vm) / (2 * h)).cpu().numpy() * w
        fd[:, d] = -np.add.reduceat(diff, off)      # d/dR_a = -d/dR_b
    # every B center moved; keep the triples whose A center did not move with them
    moved = set(cb.tolist())
    ok = np.array([c not in moved for c in sh["center_of"][ta]])
    assert ok.sum() > 50
    err = np.abs(ga - fd)[ok]
    assert np.all(err <= 1e-7 * np.maximum(1.0, np.abs(fd[ok]))), err.max()
    b.close()


def test_aab_autograd_function_matches_finite_differences(shg):
    """ThreeIndexOverlap through torch.autograd: d(sum W (a b a~))/dR of every
    center against central differences of the GPU forward pass."""
    import torch
    sh, ta, tt, tb, per = W.aab_workload(4, seed=21)
    b = shg.Basis(sh)
    centers = torch.tensor(sh["centers"], dtype=torch.float64, requires_grad=True)
    out = shg.ThreeIndexOverlap.apply(centers, b, b, ta, tt, tb)
    wt = torch.from_numpy(np.random.default_rng(5).uniform(-1, 1, out.numel())).cuda()
    (out * wt).sum().backward()
    g = centers.grad.numpy()
    used = sorted(set(sh["center_of"][ta].tolist()) | set(sh["center_of"][tb].tolist()))
    h = 1e-5
    for c_idx in used[:6]:
        for d in range(3):
            cp = sh["centers"].copy(); cp[c_idx, d] += h
            cm = sh["centers"].copy(); cm[c_idx, d] -= h
            b.set_centers(cp)
            lp = float((shg.eval_3c_aab(b, b, ta, tt, tb)[0] * wt).sum())
            b.set_centers(cm)
            lm = float((shg.eval_3c_aab(b, b, ta, tt, tb)[0] * wt).sum())
            fd = (lp - lm) / (2 * h)
            assert abs(g[c_idx, d] - fd) <= 1e-7 * max(1.0, abs(fd)), (c_idx, d, g[c_idx, d], fd)
    b.close()


@pytest.mark.parametrize("opname,op,omega", [("coulomb", 1, 0.0), ("erfc", 2, 0.11)])
def test_grad_full_size_c5_sampled(shg, opname, op, omega):
    """The full 500,000-pair gradient workload (l up to 5, K up to 12) in one
    call; 200 sampled pair gradients against the oracle's vector-Jacobian
    products with the gradient bar."""
    import torch
    sh, pa, pb = W.make("c5_grad_500k_l5_k12")
    b = shg.Basis(sh)
    off, total = b.pair_offsets(pa, pb)
    w = np.random.default_rng(44).uniform(-1, 1, total)
    ga, gb = shg.eval_2c_grad(b, pa, pb, opname, torch.from_numpy(w).cuda(), offsets=off, omega=omega)
    torch.cuda.synchronize()
    ga = ga.cpu().numpy()
    idx = np.sort(np.random.default_rng(45).choice(len(pa), 200, replace=False))
    sub, spa, spb = W.subset_pairs(sh, pa, pb, idx)
    l = sh["l"].astype(np.int64)
    sizes = (2 * l[pa] + 1) * (2 * l[pb] + 1)
    ws = np.concatenate([w[off[p]:off[p] + sizes[p]] for p in idx])
    ref, scale = _oracle_vjp(sub, spa, spb, op, omega, ws)
    bar = 1e-10 * np.abs(ref) + 1e-12 + 1e-15 * scale
    ex = np.abs(ga[idx] - ref) / bar
    assert ex.max() <= 1.0, (opname, ex.max())
    b.close()


@pytest.mark.parametrize("name,n", [("c5_grad_500k_l5_k12", 1200), ("c2_200k_l4_k8", 800)])
@pytest.mark.parametrize("opname,op,omega", GRAD_OPS)
def test_grad_mixed_against_oracle(shg, name, n, opname, op, omega):
    """Mixed precision: double-float radial orders, FP64 angular part; the
    oracle's vector-Jacobian products with the mixed gradient bar."""
    import torch
    from tests.parity import TOL_GRAD_MIXED
    sh, pa, pb = W.make(name, n=n)
    b = shg.Basis(sh)
    off, total = b.pair_offsets(pa, pb)
    w = np.random.default_rng(4).uniform(-1, 1, total)
    ga, gb = shg.eval_2c_grad(b, pa, pb, opname, torch.from_numpy(w).cuda(), offsets=off, omega=omega,
                              precision="mixed")
    torch.cuda.synchronize()
    ga, gb = ga.cpu().numpy(), gb.cpu().numpy()
    np.testing.assert_array_equal(gb, -ga)
    ref, scale = _oracle_vjp(sh, pa, pb, op, omega, w)
    rtol, atol, gamma = TOL_GRAD_MIXED
    ex = np.abs(ga - ref) / (rtol * np.abs(ref) + atol + gamma * scale)
    assert ex.max() <= 1.0, (opname, ex.max(), np.unravel_index(ex.argmax(), ex.shape))
    b.close()


def test_grad_mixed_runs_high_l_classes_in_fp64(shg):
    """Pairs with both l >= 4 take the FP64 gradient kernel under mixed
    precision (bitwise equal to FP64); the others the double-float radial
    orders (not bitwise equal)."""
    import torch
    sh, pa, pb = W.make("c5_grad_500k_l5_k12", n=3000)
    b = shg.Basis(sh)
    off, total = b.pair_offsets(pa, pb)
    w = torch.from_numpy(np.random.default_rng(9).uniform(-1, 1, total)).cuda()
    g64, _ = shg.eval_2c_grad(b, pa, pb, "coulomb", w, offsets=off, precision="fp64")
    gmx, _ = shg.eval_2c_grad(b, pa, pb, "coulomb", w, offsets=off, precision="mixed")
    torch.cuda.synchronize()
    g64, gmx = g64.cpu().numpy(), gmx.cpu().numpy()
    hi = (sh["l"][pa] >= 4) & (sh["l"][pb] >= 4)
    assert hi.sum() > 20
    np.testing.assert_array_equal(g64[hi], gmx[hi])
    assert not np.array_equal(g64[~hi], gmx[~hi])
    with pytest.raises(Exception):
        shg.eval_2c_grad(b, pa, pb, "ra2n", w, offsets=off, omega=1.0, precision="mixed")
    b.close()


def test_grad_mixed_single_kind_lists(shg):
    """Mixed-precision gradients of a list with no class run in FP64 (l <= 3:
    one double-float launch, no side streams) and of a list with only such
    classes (both l >= 4: the FP64 kernel alone, bitwise equal to FP64)."""
    import torch
    from tests.parity import TOL_GRAD_MIXED
    sh, pa, pb = W.make("c1_2k_l3_k4", n=300)
    b = shg.Basis(sh)
    off, total = b.pair_offsets(pa, pb)
    w = np.random.default_rng(21).uniform(-1, 1, total)
    ga, _ = shg.eval_2c_grad(b, pa, pb, "erfc", torch.from_numpy(w).cuda(), offsets=off, omega=0.11,
                             precision="mixed")
    torch.cuda.synchronize()
    ref, scale = _oracle_vjp(sh, pa, pb, oracle.OP_ERFC, 0.11, w)
    rtol, atol, gamma = TOL_GRAD_MIXED
    ex = np.abs(ga.cpu().numpy() - ref) / (rtol * np.abs(ref) + atol + gamma * scale)
    assert ex.max() <= 1.0, ex.max()
    b.close()

    sh, pa, pb = W.make("c5_grad_500k_l5_k12", n=20000)
    l = np.asarray(sh["l"])
    keep = np.where((l[pa] >= 4) & (l[pb] >= 4))[0][:300]
    sh, pa, pb = W.subset_pairs(sh, pa, pb, keep)
    b = shg.Basis(sh)
    off, total = b.pair_offsets(pa, pb)
    w = torch.from_numpy(np.random.default_rng(22).uniform(-1, 1, total)).cuda()
    g64, _ = shg.eval_2c_grad(b, pa, pb, "coulomb", w, offsets=off, precision="fp64")
    gmx, _ = shg.eval_2c_grad(b, pa, pb, "coulomb", w, offsets=off, precision="mixed")
    torch.cuda.synchronize()
    np.testing.assert_array_equal(g64.cpu().numpy(), gmx.cpu().numpy())
    b.close()
