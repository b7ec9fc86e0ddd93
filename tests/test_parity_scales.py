"""CPU checks of the parity bar's element-wise conditioning scales
(tests/parity.py): the separation term G_e against central differences of the
oracle, the contraction term S_e against a direct sum over primitives, and
the vector-Jacobian helper."""
import numpy as np

import oracle
from paper_1701_06588_gb300 import workloads as W
from tests.accuracy import element_stats, same_sign
from tests.parity import geometric_scale, normalised, reference_2c_parts, separations, vjp_reference


def test_geometric_scale_matches_central_differences():
    sh, pa, pb = W.make("c2_200k_l4_k8", n=40)
    shn, _ = normalised(sh)
    r = reference_2c_parts(sh, pa, pb, oracle.OP_COULOMB, 0.0)
    v = separations(sh, pa, pb)
    h = 1e-6
    fd = []
    for i in range(3):
        cp = sh["centers"].copy()
        cm = sh["centers"].copy()
        cp[sh["center_of"][pa], i] += h
        cm[sh["center_of"][pa], i] -= h
        vp, _, _ = oracle.eval_2c(dict(shn, centers=cp), pa, pb, 1, 0.0, normalize=False)
        vm, _, _ = oracle.eval_2c(dict(shn, centers=cm), pa, pb, 1, 0.0, normalize=False)
        fd.append((vp - vm) / (2 * h))
    ent = np.repeat(np.arange(len(pa)), r["sz"])
    g_fd = sum(np.abs(fd[i]) * np.abs(v[ent, i]) for i in range(3))
    np.testing.assert_allclose(r["G"], g_fd, rtol=1e-5, atol=1e-12)
    # one element by hand: entry p, element e
    p, e = 7, 2
    jac, off, sz = oracle.eval_2c_grad(shn, pa, pb, 1, 0.0, center="A", normalize=False)
    o = 3 * off[p]
    want = sum(abs(jac[o + i * sz[p] + e]) * abs(v[p, i]) for i in range(3))
    assert abs(geometric_scale(jac, off, sz, v)[off[p] + e] - want) <= 1e-15 * want


def test_contraction_scale_is_the_sum_of_primitive_magnitudes():
    """S_e equals sum over primitive pairs of |N c_a N c_b| |primitive element|
    whenever every primitive element of one entry has one sign (an s-s pair)."""
    rng = np.random.default_rng(3)
    K = 4
    sh = dict(l=np.array([0, 0], np.int32), nprim=np.array([K, K], np.int32),
              exps=np.exp(rng.uniform(np.log(0.1), np.log(50), 2 * K)), coefs=rng.uniform(-1, 1, 2 * K),
              centers=np.array([[0.0, 0.0, 0.0], [0.3, -0.4, 1.1]]), center_of=np.array([0, 1], np.int32))
    pa, pb = np.array([0], np.int32), np.array([1], np.int32)
    r = reference_2c_parts(sh, pa, pb, oracle.OP_OVERLAP, 0.0)
    shn, _ = normalised(sh)
    tot = 0.0
    for i in range(K):
        for j in range(K):
            one = dict(shn, nprim=np.array([1, 1], np.int32), exps=shn["exps"][[i, K + j]],
                       coefs=shn["coefs"][[i, K + j]])
            val, _, _ = oracle.eval_2c(one, pa, pb, 0, 0.0, normalize=False)
            tot += abs(val[0])
    np.testing.assert_allclose(r["S"][0], tot, rtol=1e-13)
    assert r["S"][0] >= abs(r["ref"][0])


def test_same_sign_shells_have_contraction_scale_equal_to_value():
    sh, pa, pb = W.make("c2_200k_l4_k8", n=30)
    r = reference_2c_parts(same_sign(sh), pa, pb, oracle.OP_COULOMB, 0.0)
    np.testing.assert_allclose(r["S"], np.abs(r["ref"]), rtol=1e-14, atol=1e-300)


def test_vjp_reference_and_element_stats():
    rng = np.random.default_rng(5)
    sz = np.array([3, 1, 5])
    off = np.concatenate([[0], np.cumsum(sz)[:-1]])
    jac = rng.standard_normal(3 * sz.sum())
    w = rng.uniform(-1, 1, sz.sum())
    g, s = vjp_reference(jac, jac, off, sz, w)
    for p in range(3):
        blk = jac[3 * off[p]: 3 * (off[p] + sz[p])].reshape(3, sz[p])
        np.testing.assert_allclose(g[p], blk @ w[off[p]: off[p] + sz[p]], rtol=1e-15)
        np.testing.assert_allclose(s[p], np.abs(blk) @ np.abs(w[off[p]: off[p] + sz[p]]), rtol=1e-15)
    ref = np.array([1.0, -2.0, 1e-20, 3.0])  # element 2 is below atol
    parts = dict(ref=ref, S=np.abs(ref), G=np.array([0.0, 1.0, 1.0, 1e4]))
    got = ref + np.array([1e-13, 0.0, 0.0, 2e-12])
    st = element_stats(got, parts, (1e-12, 1e-14, 1e-15))
    assert st["wc_fraction"] == 0.5               # elements 2 (G >> |ref|) and 3 (G > 1e3 |ref|) are not
    d0 = (1.0 + 1e-13) - 1.0                      # the error of element 0 as stored
    assert st["max_rel_wc"] == d0
    assert abs(st["max_plain_wc"] - d0 / (1e-12 + 1e-14)) < 1e-12
    d3 = (3.0 + 2e-12) - 3.0
    assert abs(st["max_excess"] - d3 / (3e-12 + 1e-14 + 1e-15 * (3 + 1e4))) < 1e-12
