"""GPU parity of the (a|r_a^{2n}|b) integrals (Sec. II C, Eqs. ara2nb and
T_rab2_deriv; operator SHG_OP_RA2N with n in omega) and of their gradients
against the oracle, whose route is the multinomial expansion of r_A^{2n}
over closed-form 1-D Gaussian overlaps."""
import numpy as np
import pytest

import oracle
from paper_1701_06588_gb300 import workloads as W
from tests.parity import TOL_FP64, assert_parity, normalised, reference_ra2n, vjp_reference

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def shg():
    import torch
    from paper_1701_06588_gb300 import api, build
    build.build()
    torch.cuda.init()
    return api


def _run(api, shells, pa, pb, n, schedule="persistent"):
    import torch
    b = api.Basis(shells)
    off, total = b.pair_offsets(pa, pb)
    plan = api.Plan2c(b, pa, pb, schedule=schedule)
    out = torch.full((max(total, 1),), float("nan"), dtype=torch.float64, device="cuda")
    plan.exec("ra2n", torch.from_numpy(off).cuda(), out, omega=float(n))
    torch.cuda.synchronize()
    res = out[:total].cpu().numpy()
    plan.close()
    b.close()
    return res


@pytest.mark.parametrize("n", [0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("schedule", ["per_class", "persistent"])
def test_ra2n_c1(shg, n, schedule):
    sh, pa, pb = W.make("c1_2k_l3_k4", n=600)
    got = _run(shg, sh, pa, pb, n, schedule)
    ref, scale = reference_ra2n(sh, pa, pb, n)
    assert_parity(got, ref, TOL_FP64, "ra2n c1 n=%d %s" % (n, schedule), scale)


@pytest.mark.parametrize("n", [1, 5])
def test_ra2n_c2_subset(shg, n):
    sh, pa, pb = W.make("c2_200k_l4_k8", n=1000)
    got = _run(shg, sh, pa, pb, n)
    ref, scale = reference_ra2n(sh, pa, pb, n)
    assert_parity(got, ref, TOL_FP64, "ra2n c2 n=%d" % n, scale)


@pytest.mark.parametrize("n", [2, 5])
def test_ra2n_high_l_and_one_center(shg, n):
    """l up to 6 and K up to 20 (C3 recipe), and every (la, lb) up to 6 at R = 0."""
    sh, pa, pb = W.make("c3_2m_l6_k20", n=400)
    got = _run(shg, sh, pa, pb, n)
    ref, scale = reference_ra2n(sh, pa, pb, n)
    assert_parity(got, ref, TOL_FP64, "ra2n c3 n=%d" % n, scale)
    rng = np.random.default_rng(17)
    ls = [l for la in range(7) for lb in range(7) for l in (la, lb)]
    m = len(ls) // 2
    K = 3
    shells = dict(l=np.array(ls, np.int32), nprim=np.full(2 * m, K, np.int32),
                  exps=np.exp(rng.uniform(np.log(0.05), np.log(200), 2 * m * K)),
                  coefs=rng.uniform(-1, 1, 2 * m * K), centers=np.zeros((1, 3)), center_of=np.zeros(2 * m, np.int32))
    pa1 = np.arange(0, 2 * m, 2, dtype=np.int32)
    got = _run(shg, shells, pa1, pa1 + 1, n)
    ref, scale = reference_ra2n(shells, pa1, pa1 + 1, n)
    assert_parity(got, ref, TOL_FP64, "ra2n R=0 n=%d" % n, scale)


@pytest.mark.parametrize("n", [1, 4])
def test_ra2n_gradient_against_oracle(shg, n):
    import torch
    sh, pa, pb = W.make("c2_200k_l4_k8", n=500)
    b = shg.Basis(sh)
    off, total = b.pair_offsets(pa, pb)
    w = np.random.default_rng(8).uniform(-1, 1, total)
    ga, gb = shg.eval_2c_grad(b, pa, pb, "ra2n", torch.from_numpy(w).cuda(), offsets=off, omega=float(n))
    torch.cuda.synchronize()
    ga, gb = ga.cpu().numpy(), gb.cpu().numpy()
    np.testing.assert_array_equal(gb, -ga)
    shn, sha = normalised(sh)
    J, o, z = oracle.eval_2c_ra2n_grad(shn, pa, pb, n, center="A", normalize=False)
    Ja, _, _ = oracle.eval_2c_ra2n_grad(sha, pa, pb, n, center="A", normalize=False)
    ref, scale = vjp_reference(J, Ja, o, z, w)
    bar = 1e-10 * np.abs(ref) + 1e-12 + 1e-15 * scale
    ex = np.abs(ga - ref) / bar
    assert ex.max() <= 1.0, (n, ex.max(), np.unravel_index(ex.argmax(), ex.shape))
    b.close()


def test_ra2n_argument_errors(shg):
    import torch
    from paper_1701_06588_gb300 import _lib as L
    sh, pa, pb = W.make("c1_2k_l3_k4", n=4)
    b = shg.Basis(sh)
    plan = shg.Plan2c(b, pa, pb)
    off, total = b.pair_offsets(pa, pb)
    out = torch.zeros(total, dtype=torch.float64, device="cuda")
    d_off = torch.from_numpy(off).cuda()
    for om, prec in [(6.0, "fp64"), (1.5, "fp64"), (-1.0, "fp64"), (2.0, "mixed")]:
        with pytest.raises(L.ShgError) as e:
            plan.exec("ra2n", d_off, out, omega=om, precision=prec)
        assert e.value.code == L.SHG_EINVAL
    plan.close()
    b.close()
