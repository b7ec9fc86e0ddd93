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
