"""GPU parity of the family path (radial terms once per primitive pair of a
family pair, contracted per shell pair; shg_family_plan_*) against the
oracle and against the regular per-pair path, including pairs the plan routes
to the regular path (K_a K_b > 100)."""
import numpy as np
import pytest

from paper_1701_06588_gb300 import workloads as W
from tests.parity import TOL_FP64, assert_parity, reference_2c

pytestmark = pytest.mark.gpu

OPS = [("overlap", 0, 0.0), ("coulomb", 1, 0.0), ("erfc", 2, 0.11), ("erf", 3, 0.11), ("gauss", 4, 1.0),
       ("gauss_coulomb", 5, 0.3)]


@pytest.fixture(scope="module")
def shg():
    import torch
    from paper_1701_06588_gb300 import api, build
    build.build()
    torch.cuda.init()
    return api


def _both(api, shells, pa, pb, opname, omega):
    import torch
    b = api.Basis(shells)
    off, total = b.pair_offsets(pa, pb)
    d_off = torch.from_numpy(off).cuda()
    fam = torch.full((total,), float("nan"), dtype=torch.float64, device="cuda")
    reg = torch.full((total,), float("nan"), dtype=torch.float64, device="cuda")
    fp = api.FamilyPlan(b, pa, pb)
    fp.exec(opname, d_off, fam, omega=omega)
    plan = api.Plan2c(b, pa, pb)
    plan.exec(opname, d_off, reg, omega=omega)
    torch.cuda.synchronize()
    counts = (fp.n_family_pairs, fp.n_groups)
    fp.close()
    plan.close()
    b.close()
    return fam.cpu().numpy(), reg.cpu().numpy(), counts


def _molecule_pairs(n_atoms, seed):
    from paper_1701_06588_gb300 import molecule
    coords, el, bs = W.molecule_workload(n_atoms, seed=seed)
    shells, _, _ = molecule.molecule_shells(coords, el, bs)
    pa, pb = molecule.shell_pairs(len(shells["l"]), True)
    return shells, pa, pb


@pytest.mark.parametrize("opname,op,omega", OPS)
def test_family_molecule_against_oracle_and_regular_path(shg, opname, op, omega):
    shells, pa, pb = _molecule_pairs(12, 41)
    fam, reg, (nf, ng) = _both(shg, shells, pa, pb, opname, omega)
    assert nf == len(pa)                                   # every pair has K_a K_b = 49
    atoms = shells["center_of"]
    assert ng == len(set(zip(atoms[pa].tolist(), atoms[pb].tolist())))   # one family per atom
    ref, scale = reference_2c(shells, pa, pb, op, omega)
    assert_parity(fam, ref, TOL_FP64, "family " + opname, scale)
    assert np.all(np.abs(fam - reg) <= 1e-14 * scale + 1e-13 * np.abs(reg)), opname


@pytest.mark.parametrize("opname,op,omega", [("coulomb", 1, 0.0), ("erfc", 2, 0.11)])
def test_family_mixed_with_regular_pairs(shg, opname, op, omega):
    """C3 recipe (K up to 20): pairs with K_a K_b <= 100 take the family path
    as single-pair groups, the others the regular path inside the plan."""
    sh, pa, pb = W.make("c3_2m_l6_k20", n=1200)
    fam, reg, (nf, ng) = _both(shg, sh, pa, pb, opname, omega)
    k = sh["nprim"]
    assert nf == int(np.sum(k[pa] * k[pb] <= 100)) and 0 < nf < len(pa)
    ref, scale = reference_2c(sh, pa, pb, op, omega)
    assert_parity(fam, ref, TOL_FP64, "family c3 " + opname, scale)


@pytest.mark.parametrize("opname,op,omega", [("coulomb", 1, 0.0), ("gauss", 4, 1.0)])
def test_family_groups_of_more_than_32_pairs(shg, opname, op, omega):
    """Ten shells (l up to 3) on one family per atom: 100 shell pairs per atom
    pair and 55 on the diagonal, so a group's contraction runs over several
    chunks of 32 shell pairs with up to 4 orders each."""
    from paper_1701_06588_gb300 import molecule
    rng = np.random.default_rng(43)
    ls = (0, 0, 1, 1, 2, 2, 3, 3, 1, 0)
    e = np.sort(np.exp(rng.uniform(np.log(0.08), np.log(40.0), 6)))[::-1].copy()
    bs = {"Z": [(l, e, rng.uniform(-1.0, 1.0, 6)) for l in ls]}
    coords = np.array([[0.0, 0.0, 0.0], [2.1, 0.3, -0.4], [-0.5, 2.6, 1.2]])
    shells, _, _ = molecule.molecule_shells(coords, ["Z"] * 3, bs)
    pa, pb = molecule.shell_pairs(len(shells["l"]), True)
    fam, reg, (nf, ng) = _both(shg, shells, pa, pb, opname, omega)
    assert nf == len(pa) == 465 and ng == 6
    ref, scale = reference_2c(shells, pa, pb, op, omega)
    assert_parity(fam, ref, TOL_FP64, "family big groups " + opname, scale)
    assert np.all(np.abs(fam - reg) <= 1e-14 * scale + 1e-13 * np.abs(reg)), opname


def test_family_errors(shg):
    import torch
    from paper_1701_06588_gb300 import _lib as L
    shells, pa, pb = _molecule_pairs(4, 42)
    b = shg.Basis(shells)
    off, total = b.pair_offsets(pa, pb)
    fp = shg.FamilyPlan(b, pa, pb)
    out = torch.zeros(total, dtype=torch.float64, device="cuda")
    for op, om in [("ra2n", 1.0), ("erf", 0.0), (9, 1.0)]:
        with pytest.raises(L.ShgError) as e:
            fp.exec(op, torch.from_numpy(off).cuda(), out, omega=om)
        assert e.value.code == L.SHG_EINVAL
    fp.close()
    with pytest.raises(L.ShgError):
        shg.FamilyPlan(b, pa, np.full_like(pb, 10_000))
    b.close()
