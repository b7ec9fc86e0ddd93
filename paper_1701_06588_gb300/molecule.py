"""Molecular assembly on top of the integral library.

A molecule's shells come from per-element basis sets; the symmetric shell-pair
list (a <= b) covers each unordered pair once; the blocks of one evaluation
are scattered into a dense AO matrix by the library's scatter kernel, and
forces sum_{mu,nu} W_{mu nu} dM_{mu nu}/dR_atom come from the gather kernel
(upstream weights), the gradient kernel and the per-center reduction.  The
sharded forms split the pair list across ranks (cost-balanced, no exchange
of integrals) and sum the partial matrices or forces with one all-reduce.
Every step runs in the CUDA library; there is no host fallback.
"""
import numpy as np
import torch

from . import _lib as L
from . import api, shard

# operators whose matrix is symmetric (M_ba = M_ab^T); (a|r_a^{2n}|b) is not
_SYMMETRIC = {"overlap", "coulomb", "erfc", "erf", "gauss", "gauss_coulomb"}


def _is_symmetric(op):
    name = op if isinstance(op, str) else {v: k for k, v in L.OPERATORS.items()}[int(op)]
    return name in _SYMMETRIC


def molecule_shells(coords, elements, basis_sets):
    """Shell list of a molecule (layout of api.Basis; centers = atoms), the AO
    offset of every shell and the number of AOs (host only)."""
    coords = np.ascontiguousarray(coords, dtype=np.float64).reshape(-1, 3)
    l, nprim, exps, coefs, center_of = [], [], [], [], []
    for i, el in enumerate(elements):
        for (ls, e, c) in basis_sets[el]:
            e = np.asarray(e, dtype=np.float64)
            c = np.asarray(c, dtype=np.float64)
            if e.shape != c.shape:
                raise ValueError("exponents and coefficients of a shell differ in length")
            l.append(int(ls))
            nprim.append(len(e))
            exps.append(e)
            coefs.append(c)
            center_of.append(i)
    shells = dict(l=np.array(l, np.int32), nprim=np.array(nprim, np.int32), exps=np.concatenate(exps),
                  coefs=np.concatenate(coefs), centers=coords, center_of=np.array(center_of, np.int32))
    size = 2 * shells["l"].astype(np.int64) + 1
    ao_off = np.concatenate([[0], np.cumsum(size)[:-1]]).astype(np.int64)
    return shells, ao_off, int(size.sum())


def shell_pairs(n_shells, symmetric=True):
    """(pair_a, pair_b): a <= b when symmetric, else every ordered pair."""
    if symmetric:
        a, b = np.triu_indices(n_shells)
    else:
        a, b = np.indices((n_shells, n_shells)).reshape(2, -1)
    return a.astype(np.int32), b.astype(np.int32)


class Molecule:
    """Atoms with coordinates (bohr) and element keys into `basis_sets`,
    {element: [(l, exponents, coefficients), ...]}.  Shell s of atom i
    starts at AO row ao_off[s]; functions of a shell are consecutive in
    m = -l..l.  The centers of the underlying basis are the atoms."""

    def __init__(self, coords, elements, basis_sets, normalize=True):
        self.shells, self.ao_off, self.nao = molecule_shells(coords, elements, basis_sets)
        self.n_atoms = len(self.shells["centers"])
        self.basis = api.Basis(self.shells, normalize=normalize)
        self.d_ao_off = torch.from_numpy(self.ao_off).cuda()

    def set_coords(self, coords):
        coords = np.ascontiguousarray(coords, dtype=np.float64).reshape(-1, 3)
        self.shells["centers"] = coords
        self.basis.set_centers(coords)

    def shell_pairs(self, symmetric=True):
        return shell_pairs(len(self.shells["l"]), symmetric)

    def _pairs(self, op, pairs):
        return self.shell_pairs(_is_symmetric(op)) if pairs is None else pairs

    def matrix(self, op, omega=0.0, precision="fp64", pairs=None, out=None, stream=None, path="pairs"):
        """Dense (nao, nao) float64 CUDA matrix of the operator; with a pair
        subset only the entries of those pairs are written (out defaults to
        zeros).  path="family" evaluates the blocks on the family path
        (FP64; radial terms shared by the shell pairs of each atom pair)."""
        pa, pb = self._pairs(op, pairs)
        if out is None:
            out = torch.zeros((self.nao, self.nao), dtype=torch.float64, device="cuda")
        if len(pa) == 0:
            return out
        off, total = self.basis.pair_offsets(pa, pb)
        d_pa, d_pb = torch.from_numpy(pa).cuda(), torch.from_numpy(pb).cuda()
        d_off = torch.from_numpy(off).cuda()
        blocks = torch.empty(total, dtype=torch.float64, device="cuda")
        if path == "family":
            if precision != "fp64":
                raise ValueError("the family path is FP64")
            plan = api.FamilyPlan(self.basis, d_pa, d_pb, stream=stream)
            plan.exec(op, d_off, blocks, omega=omega, stream=stream)
        else:
            plan = api.Plan2c(self.basis, d_pa, d_pb, stream=stream)
            plan.exec(op, d_off, blocks, omega=omega, precision=precision, stream=stream)
        L.shg_scatter_2c(self.basis.handle, len(pa), d_pa, d_pb, d_off, blocks, self.d_ao_off, self.nao,
                         _is_symmetric(op), out, api._stream(stream))
        plan.close()
        return out

    def forces(self, op, weights, omega=0.0, pairs=None, out=None, stream=None):
        """(n_atoms, 3) CUDA tensor d/dR_atom of sum_{mu,nu} W_{mu nu} M_{mu nu}
        (added into `out` when given), for a (nao, nao) weight matrix W; for a
        symmetric operator and a pair list with a <= b, W may be any matrix
        (its symmetric part counts)."""
        pa, pb = self._pairs(op, pairs)
        if out is None:
            out = torch.zeros((self.n_atoms, 3), dtype=torch.float64, device="cuda")
        if len(pa) == 0:
            return out
        off, total = self.basis.pair_offsets(pa, pb)
        d_pa, d_pb = torch.from_numpy(pa).cuda(), torch.from_numpy(pb).cuda()
        d_off = torch.from_numpy(off).cuda()
        up = torch.empty(total, dtype=torch.float64, device="cuda")
        st = api._stream(stream)
        W = weights.to("cuda", torch.float64).contiguous()
        L.shg_gather_2c(self.basis.handle, len(pa), d_pa, d_pb, d_off, W, self.d_ao_off, W.shape[1],
                        _is_symmetric(op), up, st)
        ga, gb = api.eval_2c_grad(self.basis, d_pa, d_pb, op, up, offsets=off, omega=omega, stream=stream)
        L.shg_reduce_centers(self.basis.handle, len(pa), d_pa, d_pb, ga, gb, out, st)
        return out

    def close(self):
        self.basis.close()


def local_pairs(shells, rank, world, op="coulomb"):
    """This rank's cost-balanced contiguous slice of a molecule's pair list."""
    pa, pb = shell_pairs(len(shells["l"]), _is_symmetric(op))
    opn = L.OPERATORS[op] if isinstance(op, str) else int(op)
    a, b, _ = shard.shard_pairs(shells["l"], shells["nprim"], pa, pb, rank, world, op=opn)
    return a, b


def allreduce_sum(t, group=None):
    """Sum of a tensor over the ranks of the default (or given) process group."""
    import torch.distributed as dist
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def matrix_sharded(mol, op, rank, world, omega=0.0, precision="fp64", group=None):
    """Full matrix on every rank: each evaluates its slice, one all-reduce."""
    m = mol.matrix(op, omega=omega, precision=precision, pairs=local_pairs(mol.shells, rank, world, op))
    return allreduce_sum(m, group)


def forces_sharded(mol, op, weights, rank, world, omega=0.0, group=None):
    """Forces on every rank: each differentiates its slice, one all-reduce of 3 n_atoms values."""
    f = mol.forces(op, weights, omega=omega, pairs=local_pairs(mol.shells, rank, world, op))
    return allreduce_sum(f, group)
