"""Seeded synthetic inputs (shell lists, pair and triple lists).

This module holds only random-number draws and bookkeeping: no integral
arithmetic, no normalisation, no table.  Both the CUDA path and the CPU oracle
are fed from it.  Contraction coefficients are returned raw (uniform in
[-1, 1]); each side normalises them on its own.

A shell set is a dict of numpy arrays:
    l[n_shells] int32, nprim[n_shells] int32,
    exps[sum nprim] float64, coefs[sum nprim] float64  (concatenated per shell),
    centers[n_centers, 3] float64, center_of[n_shells] int32.
"""
import numpy as np

__all__ = ["two_center_workload", "aab_workload", "WORKLOADS", "make", "subset_pairs"]


def _log_uniform(rng, lo, hi, n):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=n))


def _unit_vectors(rng, n):
    v = rng.standard_normal((n, 3))
    nrm = np.linalg.norm(v, axis=1, keepdims=True)
    nrm[nrm == 0] = 1.0
    return v / nrm


def two_center_workload(n_pairs, l_values, l_probs, k_sampler, exp_range, d_range, seed):
    """One independent geometry per pair: shell 2p on center 2p (uniform in
    [-10,10]^3), shell 2p+1 on center 2p+1 = center 2p + d * u, d uniform in
    d_range, u a normalised 3-D standard normal."""
    rng = np.random.default_rng(seed)
    n_sh = 2 * n_pairs
    l = rng.choice(np.asarray(l_values), size=n_sh, p=np.asarray(l_probs, dtype=np.float64)).astype(np.int32)
    nprim = k_sampler(rng, n_sh).astype(np.int32)
    nprim_total = int(nprim.sum())
    exps = _log_uniform(rng, exp_range[0], exp_range[1], nprim_total)
    coefs = rng.uniform(-1.0, 1.0, size=nprim_total)
    A = rng.uniform(-10.0, 10.0, size=(n_pairs, 3))
    d = rng.uniform(d_range[0], d_range[1], size=n_pairs)
    u = _unit_vectors(rng, n_pairs)
    B = A + d[:, None] * u
    centers = np.empty((n_sh, 3))
    centers[0::2] = A
    centers[1::2] = B
    shells = dict(l=l, nprim=nprim, exps=exps, coefs=coefs, centers=centers,
                  center_of=np.arange(n_sh, dtype=np.int32))
    pair_a = np.arange(0, n_sh, 2, dtype=np.int32)
    pair_b = np.arange(1, n_sh, 2, dtype=np.int32)
    return shells, pair_a, pair_b


def _k_uniform(lo, hi):
    return lambda rng, n: rng.integers(lo, hi + 1, size=n)


def _k_c3(rng, n):
    heavy = rng.uniform(size=n) < 0.30
    k = rng.integers(1, 12, size=n)
    k[heavy] = rng.integers(12, 21, size=int(heavy.sum()))
    return k


def _uniform_l(lmax):
    return list(range(lmax + 1)), [1.0 / (lmax + 1)] * (lmax + 1)


def _geometric_l(lmax):
    w = np.array([2.0 ** -l for l in range(lmax + 1)])
    return list(range(lmax + 1)), list(w / w.sum())


def _cluster(rng, n_atoms, box, dmin):
    """Uniform positions in a cube of side `box`, rejecting any atom closer
    than dmin to one already placed."""
    pos = []
    tries = 0
    while len(pos) < n_atoms:
        tries += 1
        if tries > 1_000_000:
            raise RuntimeError("cluster rejection sampling did not converge")
        p = rng.uniform(0.0, box, size=3)
        if all(np.linalg.norm(p - q) >= dmin for q in pos):
            pos.append(p)
    return np.array(pos)


def aab_workload(n_atom_pairs, seed, n_clusters=21, n_atoms=32, box=12.0, dmin=1.8,
                 n_orb=5, orb_l=(0, 4), orb_k=(1, 10), n_aux=10, aux_l=(0, 6), aux_k=(1, 3),
                 exp_range=(0.1, 200.0), layout="orbital_pairs_on_A"):
    """Three-index (a b a~) workload from random atom clusters.

    Each atom carries n_orb orbital shells (l uniform in orb_l, K uniform in
    orb_k) and n_aux auxiliary shells (l uniform in aux_l, K uniform in aux_k).
    Atom pairs (A, B), A != B, are drawn with replacement over all clusters.

    layout "orbital_pairs_on_A": a <= a~ run over the orbital shells on A, b
    over the auxiliary shells on B (n_orb (n_orb+1)/2 * n_aux triples per pair).
    layout "aux_on_A": a over the orbital shells on A, a~ over the auxiliary
    shells on A, b over the orbital shells on B (n_orb * n_aux * n_orb triples).
    """
    rng = np.random.default_rng(seed)
    centers = np.concatenate([_cluster(rng, n_atoms, box, dmin) for _ in range(n_clusters)])
    n_atoms_total = len(centers)
    per_atom = n_orb + n_aux
    n_sh = n_atoms_total * per_atom
    is_orb = np.tile(np.r_[np.ones(n_orb, bool), np.zeros(n_aux, bool)], n_atoms_total)
    l = np.where(is_orb, rng.integers(orb_l[0], orb_l[1] + 1, size=n_sh),
                 rng.integers(aux_l[0], aux_l[1] + 1, size=n_sh)).astype(np.int32)
    nprim = np.where(is_orb, rng.integers(orb_k[0], orb_k[1] + 1, size=n_sh),
                     rng.integers(aux_k[0], aux_k[1] + 1, size=n_sh)).astype(np.int32)
    nprim_total = int(nprim.sum())
    exps = _log_uniform(rng, exp_range[0], exp_range[1], nprim_total)
    coefs = rng.uniform(-1.0, 1.0, size=nprim_total)
    center_of = np.repeat(np.arange(n_atoms_total, dtype=np.int32), per_atom)
    shells = dict(l=l, nprim=nprim, exps=exps, coefs=coefs, centers=centers, center_of=center_of)

    cl = rng.integers(0, n_clusters, size=n_atom_pairs)
    ia = rng.integers(0, n_atoms, size=n_atom_pairs)
    ib = (ia + rng.integers(1, n_atoms, size=n_atom_pairs)) % n_atoms
    atom_a = cl * n_atoms + ia
    atom_b = cl * n_atoms + ib
    orb = np.arange(n_orb)
    aux = np.arange(n_orb, per_atom)
    if layout == "orbital_pairs_on_A":
        ii, jj = np.triu_indices(n_orb)
        la_loc, lt_loc = orb[ii], orb[jj]
        a_loc = np.repeat(la_loc, n_aux)
        t_loc = np.repeat(lt_loc, n_aux)
        b_loc = np.tile(aux, len(la_loc))
    elif layout == "aux_on_A":
        a_loc = np.repeat(orb, n_aux * n_orb)
        t_loc = np.tile(np.repeat(aux, n_orb), n_orb)
        b_loc = np.tile(orb, n_orb * n_aux)
    else:
        raise ValueError(layout)
    per_pair = len(a_loc)
    t_a = (atom_a[:, None] * per_atom + a_loc[None, :]).reshape(-1).astype(np.int32)
    t_t = (atom_a[:, None] * per_atom + t_loc[None, :]).reshape(-1).astype(np.int32)
    t_b = (atom_b[:, None] * per_atom + b_loc[None, :]).reshape(-1).astype(np.int32)
    return shells, t_a, t_t, t_b, per_pair


def molecule_workload(n_atoms, seed, box=None, dmin=1.8, exp_range=(0.05, 60.0), k_family=7):
    """A random molecule with family basis sets (MOLOPT-like structure: all
    shells of an element share one exponent set of k_family primitives).

    Two element kinds alternate: a light one with shells (s, s, p) and a
    heavy one with (s, s, p, p, d); exponents log-uniform in exp_range per
    element, contraction coefficients uniform in [-1, 1] per shell.  Atoms are
    placed by rejection sampling with minimum distance dmin in a cube of side
    `box` (default: sized for ~0.1 atoms per bohr^3).  Returns
    (coords[n_atoms, 3], elements[n_atoms], basis_sets)."""
    rng = np.random.default_rng(seed)
    if box is None:
        box = (n_atoms / 0.1) ** (1.0 / 3.0)
    coords = _cluster(rng, n_atoms, box, dmin)
    elements = ["X" if i % 3 == 0 else "H" for i in range(n_atoms)]
    basis_sets = {}
    for el, ls in (("H", (0, 0, 1)), ("X", (0, 0, 1, 1, 2))):
        e = np.sort(_log_uniform(rng, exp_range[0], exp_range[1], k_family))[::-1].copy()
        basis_sets[el] = [(l, e, rng.uniform(-1.0, 1.0, size=k_family)) for l in ls]
    return coords, elements, basis_sets


def subset_pairs(shells, pair_a, pair_b, idx):
    """Pairs idx of a per-pair-geometry workload (both shells copied)."""
    idx = np.asarray(idx)
    sel = np.concatenate([pair_a[idx], pair_b[idx]])
    order = np.argsort(sel, kind="stable")
    sel_sorted = sel[order]
    uniq, inv = np.unique(sel_sorted, return_inverse=True)
    off = np.zeros(len(shells["l"]) + 1, dtype=np.int64)
    off[1:] = np.cumsum(shells["nprim"])
    prim_idx = np.concatenate([np.arange(off[s], off[s + 1]) for s in uniq]) if len(uniq) else np.zeros(0, np.int64)
    sub = dict(l=shells["l"][uniq], nprim=shells["nprim"][uniq], exps=shells["exps"][prim_idx],
               coefs=shells["coefs"][prim_idx], centers=shells["centers"],
               center_of=shells["center_of"][uniq])
    new_index = np.empty(len(sel), dtype=np.int32)
    new_index[order] = inv
    n = len(idx)
    return sub, new_index[:n], new_index[n:]


# The synthetic stand-ins for the paper's test bases (TESTBAS-L0..L5 and the
# MOLOPT sets); the paper prints no exponents for TESTBAS, so these draws
# cover its l and K ranges instead.
WORKLOADS = {
    "c1_2k_l3_k4": dict(kind="2c", n=2_000, l=_uniform_l(3), k=_k_uniform(4, 4), exp=(0.1, 100.0),
                        d=(0.0, 6.0), seed=0, ops=[("overlap", 0.0), ("coulomb", 0.0)]),
    "c2_200k_l4_k8": dict(kind="2c", n=200_000, l=_uniform_l(4), k=_k_uniform(1, 8), exp=(0.05, 500.0),
                          d=(0.0, 10.0), seed=1,
                          ops=[("overlap", 0.0), ("coulomb", 0.0), ("erfc", 0.11), ("erf", 0.11),
                               ("gauss", 1.0)]),
    "c3_2m_l6_k20": dict(kind="2c", n=2_000_000, l=_geometric_l(6), k=_k_c3, exp=(0.03, 5000.0),
                         d=(0.0, 10.0), seed=2, ops=[("coulomb", 0.0), ("erfc", 0.11)]),
    "c4_aab_20k": dict(kind="aab", n=20_000, seed=3),
    "c5_grad_500k_l5_k12": dict(kind="2c", n=500_000, l=_uniform_l(5), k=_k_uniform(1, 12),
                                exp=(0.05, 500.0), d=(0.0, 10.0), seed=4,
                                ops=[("coulomb", 0.0), ("erfc", 0.11)]),
}


def make(name, n=None):
    """Build a named workload; `n` overrides the number of pairs (atom pairs
    for the (aab) workload) to get a smaller case with the same recipe."""
    w = WORKLOADS[name]
    n = w["n"] if n is None else n
    if w["kind"] == "aab":
        return aab_workload(n, w["seed"])
    return two_center_workload(n, w["l"][0], w["l"][1], w["k"], w["exp"], w["d"], w["seed"])
