"""Accuracy bookkeeping shared by the plain-bar tests and the per-class error
table (tests/error_table.py): runs the library's two-center forms on a pair
list and compares them element by element with the oracle.

Only the oracle (through tests.parity) and the library's public API are used.
"""
import numpy as np

from tests.parity import reference_2c_parts

# well-conditioned elements: C_e = S_e + G_e (tests/parity.py) within this
# factor of |ref_e|
KAPPA_WC = 1e3


def same_sign(shells):
    """The shell set with |c| for every contraction coefficient: no cancellation
    in the contraction over primitives (S_e = |ref_e| for every operator but erfc)."""
    return dict(shells, coefs=np.abs(np.asarray(shells["coefs"], dtype=np.float64)))


def c3_stratified(per_class=20, pool=200_000, seed=6):
    """Up to per_class pairs of every (la, lb) class of the 2M-pair recipe
    (P(l) ~ 2^-l up to l = 6, K 1..20 with 30% heavy shells), drawn from the
    first `pool` pairs of the same recipe."""
    from paper_1701_06588_gb300 import workloads as W
    sh, pa, pb = W.make("c3_2m_l6_k20", n=pool)
    l = sh["l"]
    rng = np.random.default_rng(seed)
    idx = []
    for la in range(7):
        for lb in range(7):
            sel = np.where((l[pa] == la) & (l[pb] == lb))[0]
            if len(sel):
                idx.append(rng.choice(sel, min(per_class, len(sel)), replace=False))
    idx = np.sort(np.concatenate(idx))
    return W.subset_pairs(sh, pa, pb, idx)


def run_forms(api, shells, pa, pb, ops, forms):
    """Blocks of every operator in every form.

    ops: [(name, op id, omega)]; forms: subset of "fp64", "mixed" (one pass per
    operator) and "fp64_fused", "mixed_fused" (all ops in one pass).
    Returns {form: {name: numpy blocks}}."""
    import torch
    b = api.Basis(shells)
    off, total = b.pair_offsets(pa, pb)
    d_off = torch.from_numpy(off).cuda()
    plan = api.Plan2c(b, pa, pb)
    res = {}
    for form in forms:
        prec = "fp64" if form.startswith("fp64") else "mixed"
        outs = [torch.full((max(total, 1),), float("nan"), dtype=torch.float64, device="cuda") for _ in ops]
        if form.endswith("_fused"):
            plan.exec_fused([o[0] for o in ops], d_off, outs, omegas=[o[2] for o in ops], precision=prec)
        else:
            for (name, _, om), o in zip(ops, outs):
                plan.exec(name, d_off, o, omega=om, precision=prec)
        torch.cuda.synchronize()
        res[form] = {name: o[:total].cpu().numpy() for (name, _, _), o in zip(ops, outs)}
    plan.close()
    b.close()
    return res


def references(shells, pa, pb, ops):
    return {name: reference_2c_parts(shells, pa, pb, op, om) for name, op, om in ops}


def element_stats(got, r, tol, kappa=KAPPA_WC, rel_floor=None):
    """Statistics of one set of elements against its oracle parts r.

    max_excess      max |x - ref| / (rtol |ref| + atol + gamma C) over all elements
    wc_fraction     fraction of elements with C <= kappa |ref|
    max_rel_wc      max |x - ref| / |ref| over the well-conditioned elements whose
                    |ref| is above rel_floor (default: the bar's atol)
    max_plain_wc    max |x - ref| / (rtol |ref| + atol) over the well-conditioned
                    elements: the plain bar, no conditioning term (<= 1 passes)
    """
    rtol, atol, gamma = tol
    ref = r["ref"]
    C = r["S"] + r["G"]
    d = np.abs(np.asarray(got, dtype=np.float64) - ref)
    if not np.all(np.isfinite(got)):
        d = np.where(np.isfinite(got), d, np.inf)
    out = {"elements": int(ref.size)}
    if ref.size == 0:
        out.update(max_excess=0.0, wc_fraction=1.0, max_rel_wc=0.0, max_plain_wc=0.0)
        return out
    out["max_excess"] = float(np.max(d / (rtol * np.abs(ref) + atol + gamma * C)))
    wc = C <= kappa * np.abs(ref)
    out["wc_fraction"] = float(wc.mean())
    floor = atol if rel_floor is None else rel_floor
    big = wc & (np.abs(ref) > floor)
    out["max_rel_wc"] = float(np.max(d[big] / np.abs(ref[big]))) if big.any() else None
    out["max_plain_wc"] = float(np.max(d[wc] / (rtol * np.abs(ref[wc]) + atol))) if wc.any() else 0.0
    return out


def class_elements(shells, pa, pb, off):
    """{(la, lb): element indices} of a pair list."""
    l = np.asarray(shells["l"]).astype(np.int64)
    sizes = (2 * l[pa] + 1) * (2 * l[pb] + 1)
    out = {}
    for la in range(7):
        for lb in range(7):
            sel = np.where((l[pa] == la) & (l[pb] == lb))[0]
            if len(sel):
                out[(la, lb)] = (len(sel), np.concatenate([np.arange(off[p], off[p] + sizes[p]) for p in sel]))
    return out
