#!/usr/bin/env python3
"""Per-(la, lb, operator) error table of the two-center forms against the oracle.

    python tests/error_table.py [--md tests/error_table.md] [--json PATH]

Needs a CUDA device and the built library; the expected values come from the
oracle only (tests.parity.reference_2c_parts).  Two workloads:

  c2  the first 3,000 pairs of the 200,000-pair recipe (l 0..4, K 1..8), all
      six operators of the library's two-center passes (overlap, 1/r,
      erfc(0.11r)/r, erf(0.11r)/r, exp(-r^2), exp(-0.3r^2)/r; the fused pass
      takes the first five)
  c3  up to 20 pairs of each of the 49 (la, lb) classes of the 2M-pair recipe
      (l 0..6 with P(l) ~ 2^-l, K 1..20), 1/r and erfc(0.11r)/r

and four forms: FP64 and double-float (mixed), each as one pass per operator
and as the fused multi-operator pass.  Per class and form the table gives

  max rel   the largest |x - ref| / |ref| over the well-conditioned elements
            (S_e + G_e <= 1e3 |ref_e|, tests/parity.py) where the relative term
            of the bar binds, |ref| >= atol / rtol (FP64 1e-2, mixed 1e-4);
            below that the absolute floor is the bar
  excess    the largest |x - ref| / bar over every element, with the
            element-wise conditioned bar of tests/parity.py (<= 1 passes)

and the fraction of well-conditioned elements.
"""
import argparse
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

FORMS = ["fp64", "fp64_fused", "mixed", "mixed_fused"]


def collect(api, name, sh, pa, pb, ops):
    from tests.accuracy import class_elements, element_stats, references, run_forms
    from tests.parity import TOL_FP64, TOL_MIXED
    refs = references(sh, pa, pb, ops)
    res = run_forms(api, sh, pa, pb, ops, ["fp64", "mixed"])
    fused_ops = [o for o in ops if o[1] <= 4]
    res.update(run_forms(api, sh, pa, pb, fused_ops, ["fp64_fused", "mixed_fused"]))
    off = refs[ops[0][0]]["off"]
    classes = class_elements(sh, pa, pb, off)
    rows = []
    for opname, _, om in ops:
        r = refs[opname]
        for (la, lb), (npairs, idx) in sorted(classes.items()):
            sub = {k: r[k][idx] for k in ("ref", "S", "G")}
            row = {"workload": name, "operator": opname, "omega": om, "la": la, "lb": lb, "pairs": npairs}
            for form in FORMS:
                if opname not in res[form]:
                    continue
                tol = TOL_FP64 if form.startswith("fp64") else TOL_MIXED
                st = element_stats(res[form][opname][idx], sub, tol, rel_floor=tol[1] / tol[0])
                row["elements"] = st["elements"]
                row["wc_fraction"] = st["wc_fraction"]
                row[form] = {"max_rel_wc": st["max_rel_wc"], "max_excess": st["max_excess"]}
            rows.append(row)
    return rows


def fmt(x, digits=1):
    if x is None:
        return "-"
    return ("%." + str(digits) + "e") % x


def markdown(rows, meta):
    out = ["# Per-class error of the two-center forms against the oracle", "",
           "Written by `python tests/error_table.py` (%s).  max rel: largest relative error on the "
           "well-conditioned elements (S_e + G_e <= 1e3 |ref_e|) where the relative term of the bar binds (|ref| >= atol/rtol: 1e-2 FP64, 1e-4 mixed); excess: largest "
           "ratio of the error to the element-wise bar of tests/parity.py over every element (<= 1 passes; FP64 "
           "rtol 1e-12, atol 1e-14, gamma 1e-15; mixed rtol 1e-10, atol 1e-14, gamma 2e-13).  wc: fraction of "
           "well-conditioned elements." % meta["gpu"], ""]
    for wl in ("c2", "c3"):
        sel = [r for r in rows if r["workload"] == wl]
        if not sel:
            continue
        worst = {f: max((r[f]["max_excess"] for r in sel if f in r), default=0.0) for f in FORMS}
        worst_rel = {f: max((r[f]["max_rel_wc"] or 0.0 for r in sel if f in r), default=0.0) for f in FORMS}
        out += ["## %s" % meta["workloads"][wl], "",
                "Largest over all classes: " + ", ".join(
                    "%s max rel %s excess %.3g" % (f, fmt(worst_rel[f]), worst[f]) for f in FORMS), "",
                "| operator | la | lb | pairs | elements | wc | FP64 max rel | FP64 fused max rel | mixed max rel | "
                "mixed fused max rel | FP64 excess | FP64 fused excess | mixed excess | mixed fused excess |",
                "|---|---|---|---|---|---|---|---|---|---|---|---|---|---|"]
        for r in sel:
            cells = [r["operator"], str(r["la"]), str(r["lb"]), str(r["pairs"]), str(r["elements"]),
                     "%.3f" % r["wc_fraction"]]
            cells += [fmt(r[f]["max_rel_wc"]) if f in r else "-" for f in FORMS]
            cells += ["%.3f" % r[f]["max_excess"] if f in r else "-" for f in FORMS]
            out.append("| " + " | ".join(cells) + " |")
        out.append("")
    return "\n".join(out)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--md", default=os.path.join(HERE, "error_table.md"))
    ap.add_argument("--json", default=None)
    ap.add_argument("--c2-pairs", type=int, default=3000)
    ap.add_argument("--c3-per-class", type=int, default=20)
    a = ap.parse_args()
    import torch
    from paper_1701_06588_gb300 import api, build, workloads as W
    from tests.accuracy import c3_stratified
    build.build()
    torch.cuda.init()
    rows = []
    sh, pa, pb = W.make("c2_200k_l4_k8", n=a.c2_pairs)
    rows += collect(api, "c2", sh, pa, pb, [("overlap", 0, 0.0), ("coulomb", 1, 0.0), ("erfc", 2, 0.11),
                                            ("erf", 3, 0.11), ("gauss", 4, 1.0), ("gauss_coulomb", 5, 0.3)])
    sh, pa, pb = c3_stratified(per_class=a.c3_per_class)
    rows += collect(api, "c3", sh, pa, pb, [("coulomb", 1, 0.0), ("erfc", 2, 0.11)])
    meta = {"gpu": torch.cuda.get_device_name(),
            "workloads": {"c2": "200,000-pair recipe (l 0..4, K 1..8, seed 1): first %d pairs, six operators"
                                % a.c2_pairs,
                          "c3": "2M-pair recipe (l 0..6, P(l) ~ 2^-l, K 1..20, seed 2): up to %d pairs per "
                                "(la, lb) class, 1/r and erfc(0.11 r)/r" % a.c3_per_class}}
    md = markdown(rows, meta)
    with open(a.md, "w") as f:
        f.write(md)
    if a.json:
        with open(a.json, "w") as f:
            json.dump({"meta": meta, "rows": rows}, f, indent=1)
    bad = [r for r in rows for f in FORMS if f in r and not r[f]["max_excess"] <= 1.0]
    print("%d rows, %d over the bar" % (len(rows), len(bad)))
    return 1 if bad else 0


if __name__ == "__main__":
    sys.exit(main())
