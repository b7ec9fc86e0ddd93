"""The plain accuracy bars, with no conditioning term, on well-conditioned
inputs:

  FP64 integrals   |x - ref| <= 1e-12 |ref| + 1e-14
  mixed precision  |x - ref| <= 1e-10 |ref| + 1e-14
  gradients        |g - ref| <= 1e-10 |ref| + 1e-12   (FP64 and mixed)

Inputs: the synthetic recipes with every contraction coefficient replaced by
its magnitude, so that no contraction over primitives cancels (Eq.
O_rab2_deriv: all primitive terms of one derivative order then share a
sign).  The angular part can still cancel where an element passes through a
node as a function of the separation; those elements are the ones with a
large G_e (tests/parity.py), and the check runs over the elements with
S_e + G_e <= 1e3 |ref_e|, which must be at least 90% of the total (the rest
are held to the conditioned bar by the other parity tests).
"""
import numpy as np
import pytest

import oracle
from paper_1701_06588_gb300 import workloads as W
from tests.accuracy import KAPPA_WC, c3_stratified, element_stats, references, run_forms, same_sign
from tests.parity import PLAIN_FP64, PLAIN_GRAD, PLAIN_MIXED, normalised, vjp_reference

pytestmark = pytest.mark.gpu

C2_OPS = [("overlap", 0, 0.0), ("coulomb", 1, 0.0), ("erfc", 2, 0.11), ("erf", 3, 0.11), ("gauss", 4, 1.0)]
C3_OPS = [("coulomb", 1, 0.0), ("erfc", 2, 0.11)]


@pytest.fixture(scope="module")
def shg():
    import torch
    from paper_1701_06588_gb300 import api, build
    build.build()
    torch.cuda.init()
    return api


def _workload(name):
    if name == "c2":
        sh, pa, pb = W.make("c2_200k_l4_k8", n=3000)
        ops = C2_OPS + [("gauss_coulomb", 5, 0.3)]
    else:
        sh, pa, pb = c3_stratified()
        ops = C3_OPS
    return same_sign(sh), pa, pb, ops


@pytest.mark.parametrize("name", ["c2", "c3"])
def test_plain_bars_same_sign_coefficients(shg, name):
    sh, pa, pb, ops = _workload(name)
    fused_ops = [o for o in ops if o[1] <= 4]
    refs = references(sh, pa, pb, ops)
    res = run_forms(shg, sh, pa, pb, ops, ["fp64", "mixed"])
    res.update(run_forms(shg, sh, pa, pb, fused_ops, ["fp64_fused", "mixed_fused"]))
    report = []
    for form, blocks in res.items():
        tol = PLAIN_FP64 if form.startswith("fp64") else PLAIN_MIXED
        for opname, got in blocks.items():
            st = element_stats(got, refs[opname], tol)
            report.append((form, opname, st["max_plain_wc"], st["wc_fraction"], st["max_rel_wc"]))
            assert st["wc_fraction"] >= 0.9, (name, form, opname, st)
            assert st["max_plain_wc"] <= 1.0, (name, form, opname, st)
    for r in report:
        print("%s %-12s %-14s plain excess %.3g  well-conditioned %.4f  max rel %s" % ((name,) + r))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("opname,op,omega", [("coulomb", 1, 0.0), ("erfc", 2, 0.11)])
def test_plain_gradient_bar_same_sign_coefficients(shg, opname, op, omega, precision):
    """Vector-Jacobian products with upstream weights uniform in [0, 1] on
    1,000 pairs of the gradient recipe (l up to 5, K up to 12), same-sign
    coefficients; components whose magnitude sum sum_e |W_e| |dI_e/dR| is
    within 1e3 of |ref|."""
    import torch
    sh, pa, pb = W.make("c5_grad_500k_l5_k12", n=1000)
    sh = same_sign(sh)
    b = shg.Basis(sh)
    off, total = b.pair_offsets(pa, pb)
    w = np.random.default_rng(17).uniform(0.0, 1.0, total)
    ga, _ = shg.eval_2c_grad(b, pa, pb, opname, torch.from_numpy(w).cuda(), offsets=off, omega=omega,
                             precision=precision)
    torch.cuda.synchronize()
    ga = ga.cpu().numpy()
    b.close()
    shn, _ = normalised(sh)
    J, o, z = oracle.eval_2c_grad(shn, pa, pb, op, omega, center="A", normalize=False)
    ref, scale = vjp_reference(J, J, o, z, w)
    wc = scale <= KAPPA_WC * np.abs(ref)
    assert wc.mean() >= 0.9, wc.mean()
    ex = np.abs(ga - ref)[wc] / (PLAIN_GRAD[0] * np.abs(ref[wc]) + PLAIN_GRAD[1])
    print("plain gradient bar %s %s: excess %.3g over %.4f of the components" % (precision, opname, ex.max(),
                                                                                  wc.mean()))
    assert ex.max() <= 1.0, ex.max()
