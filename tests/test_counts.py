"""Count model against the paper's printed Table II, and sanity of the flop model."""
import json
import os

import numpy as np

from paper_1701_06588_gb300 import counts

HERE = os.path.dirname(os.path.abspath(__file__))


def test_table2_contracted_element_counts():
    g = json.load(open(os.path.join(HERE, "golden", "table2_contracted_elements.json")))
    for name, spec in g["bases"].items():
        for col, grad in (("Int.", False), ("Int.+Dev.", True)):
            shg = counts.shg_contracted_elements(spec["l"], spec["l"], spec["K"], spec["K"], grad)
            os_ = counts.os_contracted_elements(spec["l"], spec["l"], spec["K"], spec["K"], grad)
            assert shg == g["values"]["SHG"][name][col], (name, col, shg)
            assert os_ == g["values"]["OS"][name][col], (name, col, os_)


def test_flop_model_monotone_and_positive():
    for op in range(7):
        f = counts.pair_flops(np.array([0, 1, 2, 4, 6]), np.array([0, 1, 2, 4, 6]), np.ones(5), np.ones(5), op)
        assert np.all(f > 0) and np.all(np.diff(f) > 0)
        g = counts.pair_flops(np.full(4, 2), np.full(4, 3), np.array([1, 2, 4, 8]), np.array([1, 2, 4, 8]), op)
        assert np.all(np.diff(g) > 0)
    # erfc costs the Coulomb and the erf radial parts together
    a = counts.pair_flops(3, 2, 5, 5, counts.OP_ERFC)
    assert a > counts.pair_flops(3, 2, 5, 5, counts.OP_COULOMB)
    assert a > counts.pair_flops(3, 2, 5, 5, counts.OP_ERF)


def test_triple_and_gradient_flop_models():
    # more primitives or higher l cost more; the gradient costs more than the forward pass
    f = counts.triple_flops(np.array([0, 1, 2, 3]), np.array([0, 1, 2, 3]), np.array([1, 2, 3, 4]), 2, 2, 2)
    assert np.all(f > 0) and np.all(np.diff(f) > 0)
    g = counts.triple_flops(2, 2, 2, np.array([1, 2, 4]), 3, 2)
    assert np.all(np.diff(g) > 0)
    for op in range(7):
        assert counts.grad_pair_flops(3, 2, 4, 4, op) > counts.pair_flops(3, 2, 4, 4, op)


def test_fused_flop_model():
    five = [(counts.OP_OVERLAP, 0.0), (counts.OP_COULOMB, 0.0), (counts.OP_ERFC, 0.11), (counts.OP_ERF, 0.11),
            (counts.OP_GAUSS, 1.0)]
    la, lb = np.array([0, 1, 2, 4, 4]), np.array([0, 2, 2, 3, 4])
    k = np.array([1, 3, 5, 8, 8])
    fused = counts.fused_pair_flops(la, lb, k, k, five)
    separate = sum(counts.pair_flops(la, lb, k, k, op) for op, _ in five)
    assert np.all(fused > 0) and np.all(fused < separate)
    # erf and erfc with the same omega share one attenuated sum; different omegas need two
    same = counts.fused_pair_flops(3, 3, 6, 6, [(counts.OP_ERF, 0.2), (counts.OP_ERFC, 0.2)])
    diff = counts.fused_pair_flops(3, 3, 6, 6, [(counts.OP_ERF, 0.2), (counts.OP_ERFC, 0.3)])
    assert diff > same
    # erfc costs one Boys sum more than erf alone (the 1/r part)
    assert (counts.fused_pair_flops(3, 3, 6, 6, [(counts.OP_ERFC, 0.2)]) >
            counts.fused_pair_flops(3, 3, 6, 6, [(counts.OP_ERF, 0.2)]))
    # adding an operator to the pass adds less than the operator costs on its own
    for op, w in five:
        rest = [o for o in five if o[0] != op]
        extra = counts.fused_pair_flops(4, 4, 8, 8, five) - counts.fused_pair_flops(4, 4, 8, 8, rest)
        assert 0 < extra < counts.pair_flops(4, 4, 8, 8, op)


def test_far_primitive_pairs_against_brute_force():
    from paper_1701_06588_gb300 import workloads as W
    sh, pa, pb = W.make("c3_2m_l6_k20", n=400)
    nf = counts.far_primitive_pairs(sh, pa, pb)
    off = np.concatenate([[0], np.cumsum(sh["nprim"])])
    c, co = sh["centers"], sh["center_of"]
    for p in range(len(pa)):
        A = sh["exps"][off[pa[p]]:off[pa[p] + 1]]
        B = sh["exps"][off[pb[p]]:off[pb[p] + 1]]
        R2 = float(((c[co[pa[p]]] - c[co[pb[p]]]) ** 2).sum())
        assert nf[p] == sum(1 for a in A for b in B if a * b / (a + b) * R2 >= counts.KBOYS_TMAX)
    assert 0 < nf.sum() < (sh["nprim"][pa] * sh["nprim"][pb]).sum()


def test_fused_flops_count_far_pairs_as_one_multiply_add():
    ops = [(counts.OP_COULOMB, 0.0), (counts.OP_ERFC, 0.11)]
    la, lb, ka, kb = np.array([0, 2]), np.array([3, 2]), np.array([5, 4]), np.array([6, 3])
    near = counts.fused_pair_flops(la, lb, ka, kb, ops)
    half = counts.fused_pair_flops(la, lb, ka, kb, ops, n_far=(ka * kb) // 2)
    allfar = counts.fused_pair_flops(la, lb, ka, kb, ops, n_far=ka * kb)
    assert np.all(allfar < half) and np.all(half < near)
    # per far primitive pair the 1/r part costs 2 flops instead of the Boys head,
    # (-rho)^kmin and J orders; the attenuated erfc part is unchanged
    J = np.minimum(la, lb) + 1
    kmin = np.maximum(la, lb)
    for i in range(2):
        d = counts._fused_radial_flops(ops, J[i], kmin[i]) - counts._fused_radial_flops(ops, J[i], kmin[i], far=True)
        assert d == (2 * int(np.ceil(np.log2(kmin[i] + 1))) + counts._boys(J[i]) + 3 * (J[i] - 1) + 3 * J[i] - 2)
