"""Molecular assembly through the library: dense AO matrices scattered from
the blocks, forces from gathered weights, the gradient kernel and the
per-center reduction, against the oracle's blocks and Jacobians assembled
on the host, finite differences of the GPU energy and the adjoint identity
of scatter and gather."""
import numpy as np
import pytest

import oracle
from paper_1701_06588_gb300 import workloads as W
from tests.parity import TOL_FP64, assert_parity, normalised, reference_2c, reference_ra2n

pytestmark = pytest.mark.gpu

OPS = [("overlap", 0, 0.0), ("coulomb", 1, 0.0), ("erfc", 2, 0.11), ("gauss_coulomb", 5, 0.3)]


@pytest.fixture(scope="module")
def mol_mod():
    import torch
    from paper_1701_06588_gb300 import build, molecule
    build.build()
    torch.cuda.init()
    return molecule


def _dense(vals, shells, ao_off, nao, pa, pb, sym):
    l = shells["l"].astype(np.int64)
    sz = (2 * l[pa] + 1) * (2 * l[pb] + 1)
    off = np.concatenate([[0], np.cumsum(sz)[:-1]])
    M = np.zeros((nao, nao))
    for p in range(len(pa)):
        a, b = pa[p], pb[p]
        na, nb = 2 * l[a] + 1, 2 * l[b] + 1
        blk = vals[off[p]:off[p] + sz[p]].reshape(na, nb)
        M[ao_off[a]:ao_off[a] + na, ao_off[b]:ao_off[b] + nb] = blk
        if sym and a != b:
            M[ao_off[b]:ao_off[b] + nb, ao_off[a]:ao_off[a] + na] = blk.T
    return M


@pytest.mark.parametrize("opname,op,omega", OPS)
def test_matrix_against_oracle(mol_mod, opname, op, omega):
    coords, el, bs = W.molecule_workload(10, seed=31)
    mol = mol_mod.Molecule(coords, el, bs)
    M = mol.matrix(opname, omega=omega).cpu().numpy()
    pa, pb = mol.shell_pairs(True)
    ref, scale = reference_2c(mol.shells, pa, pb, op, omega)
    Mref = _dense(ref, mol.shells, mol.ao_off, mol.nao, pa, pb, True)
    Sref = _dense(scale, mol.shells, mol.ao_off, mol.nao, pa, pb, True)
    assert_parity(M.ravel(), Mref.ravel(), TOL_FP64, "molecule " + opname, Sref.ravel())
    assert np.array_equal(M, M.T)
    Mf = mol.matrix(opname, omega=omega, path="family").cpu().numpy()
    assert_parity(Mf.ravel(), Mref.ravel(), TOL_FP64, "molecule family " + opname, Sref.ravel())
    if opname == "overlap":                      # normalised functions
        np.testing.assert_allclose(np.diag(M), 1.0, rtol=0, atol=1e-12)
    mol.close()


def test_ra2n_matrix_is_not_symmetric(mol_mod):
    coords, el, bs = W.molecule_workload(6, seed=32)
    mol = mol_mod.Molecule(coords, el, bs)
    M = mol.matrix("ra2n", omega=1.0).cpu().numpy()
    pa, pb = mol.shell_pairs(False)
    ref, scale = reference_ra2n(mol.shells, pa, pb, 1)
    Mref = _dense(ref, mol.shells, mol.ao_off, mol.nao, pa, pb, False)
    Sref = _dense(scale, mol.shells, mol.ao_off, mol.nao, pa, pb, False)
    assert_parity(M.ravel(), Mref.ravel(), TOL_FP64, "molecule ra2n", Sref.ravel())
    assert not np.allclose(M, M.T)
    mol.close()


@pytest.mark.parametrize("opname,op,omega", [("coulomb", 1, 0.0), ("overlap", 0, 0.0)])
def test_forces_against_oracle_and_finite_differences(mol_mod, opname, op, omega):
    import torch
    coords, el, bs = W.molecule_workload(8, seed=33)
    mol = mol_mod.Molecule(coords, el, bs)
    rng = np.random.default_rng(9)
    Wm = rng.uniform(-1, 1, (mol.nao, mol.nao))
    Wm = 0.5 * (Wm + Wm.T)
    F = mol.forces(opname, torch.from_numpy(Wm), omega=omega).cpu().numpy()
    # oracle: Jacobians of every block (a <= b) with respect to both centers
    pa, pb = mol.shell_pairs(True)
    shn, _ = normalised(mol.shells)
    JA, off, sz = oracle.eval_2c_grad(shn, pa, pb, op, omega, center="A", normalize=False)
    JB, _, _ = oracle.eval_2c_grad(shn, pa, pb, op, omega, center="B", normalize=False)
    l = mol.shells["l"]
    Fref = np.zeros((mol.n_atoms, 3))
    for p in range(len(pa)):
        a, b = pa[p], pb[p]
        na, nb = 2 * l[a] + 1, 2 * l[b] + 1
        u = Wm[mol.ao_off[a]:mol.ao_off[a] + na, mol.ao_off[b]:mol.ao_off[b] + nb].copy()
        if a != b:
            u += Wm[mol.ao_off[b]:mol.ao_off[b] + nb, mol.ao_off[a]:mol.ao_off[a] + na].T
        u = u.ravel()
        Fref[mol.shells["center_of"][a]] += JA[3 * off[p]:3 * (off[p] + sz[p])].reshape(3, sz[p]) @ u
        Fref[mol.shells["center_of"][b]] += JB[3 * off[p]:3 * (off[p] + sz[p])].reshape(3, sz[p]) @ u
    np.testing.assert_allclose(F, Fref, rtol=1e-9, atol=1e-11 * np.abs(Fref).max())
    # finite differences of E = sum W M with the GPU matrix
    h = 1e-5
    Wt = torch.from_numpy(Wm).cuda()
    for atom in (0, 3):
        for d in range(3):
            cp, cm = coords.copy(), coords.copy()
            cp[atom, d] += h
            cm[atom, d] -= h
            mol.set_coords(cp)
            ep = float((mol.matrix(opname, omega=omega) * Wt).sum())
            mol.set_coords(cm)
            em = float((mol.matrix(opname, omega=omega) * Wt).sum())
            fd = (ep - em) / (2 * h)
            assert abs(F[atom, d] - fd) <= 1e-7 * max(1.0, abs(fd)), (atom, d, F[atom, d], fd)
    mol.set_coords(coords)
    mol.close()


@pytest.mark.parametrize("sym", [True, False])
def test_scatter_gather_adjoint_and_errors(mol_mod, sym):
    """<gather(W), b> = <W, scatter(b)> for random blocks b and matrix W."""
    import torch
    from paper_1701_06588_gb300 import _lib as L
    coords, el, bs = W.molecule_workload(7, seed=34)
    mol = mol_mod.Molecule(coords, el, bs)
    pa, pb = mol.shell_pairs(sym)
    off, total = mol.basis.pair_offsets(pa, pb)
    d_pa, d_pb, d_off = (torch.from_numpy(x).cuda() for x in (pa, pb, off))
    rng = np.random.default_rng(3)
    blocks = torch.from_numpy(rng.uniform(-1, 1, total)).cuda()
    Wm = torch.from_numpy(rng.uniform(-1, 1, (mol.nao, mol.nao))).cuda()
    M = torch.zeros((mol.nao, mol.nao), dtype=torch.float64, device="cuda")
    g = torch.empty(total, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    L.shg_scatter_2c(mol.basis.handle, len(pa), d_pa, d_pb, d_off, blocks, mol.d_ao_off, mol.nao, sym, M, st)
    L.shg_gather_2c(mol.basis.handle, len(pa), d_pa, d_pb, d_off, Wm, mol.d_ao_off, mol.nao, sym, g, st)
    lhs = float((g * blocks).sum())
    rhs = float((Wm * M).sum())
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(rhs)), (lhs, rhs)
    with pytest.raises(L.ShgError) as e:
        L.shg_scatter_2c(mol.basis.handle, len(pa), d_pa, d_pb, d_off, blocks, mol.d_ao_off, 0, sym, M, st)
    assert e.value.code == L.SHG_EINVAL
    mol.close()
