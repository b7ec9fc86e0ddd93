"""ctypes binding of libshg_gb300.so: one Python function per C-ABI entry point
(same names, argument marshalling only; every step of the computation runs in
the library's CUDA kernels).

The library must have been built (paper_1701_06588_gb300.build.build());
there is no fallback of any kind: a missing library raises at first use.
"""
import ctypes
import os
import threading

from . import build as _build

SHG_OK, SHG_EINVAL, SHG_ENOMEM, SHG_ECUDA, SHG_ETIMEOUT, SHG_ERANGE = 0, -1, -2, -3, -4, -5
SHG_OP_OVERLAP, SHG_OP_COULOMB, SHG_OP_ERFC, SHG_OP_ERF, SHG_OP_GAUSS, SHG_OP_GAUSS_COULOMB, SHG_OP_RA2N = range(7)
SHG_PREC_FP64, SHG_PREC_MIXED = 0, 1
SHG_SCHED_PER_CLASS, SHG_SCHED_PERSISTENT = 0, 1

OPERATORS = {"overlap": SHG_OP_OVERLAP, "coulomb": SHG_OP_COULOMB, "erfc": SHG_OP_ERFC, "erf": SHG_OP_ERF,
             "gauss": SHG_OP_GAUSS, "gauss_coulomb": SHG_OP_GAUSS_COULOMB, "ra2n": SHG_OP_RA2N}
PRECISIONS = {"fp64": SHG_PREC_FP64, "mixed": SHG_PREC_MIXED}
SCHEDULES = {"per_class": SHG_SCHED_PER_CLASS, "persistent": SHG_SCHED_PERSISTENT}

# (name, restype, argtypes) of every symbol declared in include/shg.h
_P = ctypes.c_void_p
_I = ctypes.c_int
_L = ctypes.c_int64
_D = ctypes.c_double
SIGNATURES = [
    ("shg_basis_create", _I, [_I, _P, _P, _P, _P, _I, _P, _P, _I, ctypes.POINTER(_P)]),
    ("shg_basis_set_centers", _I, [_P, _P]),
    ("shg_basis_destroy", None, [_P]),
    ("shg_basis_nshells", _L, [_P]),
    ("shg_basis_nprims", _L, [_P]),
    ("shg_pair_offsets", _L, [_P, _L, _P, _P, _P]),
    ("shg_triple_offsets", _L, [_P, _P, _L, _P, _P, _P, _P]),
    ("shg_eval_2c", _I, [_P, _L, _P, _P, _I, _D, _D, _I, _P, _P, _P]),
    ("shg_plan_2c_create", _I, [_P, _L, _P, _P, _I, _P, ctypes.POINTER(_P)]),
    ("shg_plan_2c_exec", _I, [_P, _I, _D, _D, _I, _P, _P, _P]),
    ("shg_plan_launches", _I, [_P]),
    ("shg_plan_launches_prec", _I, [_P, _I]),
    ("shg_plan_2c_set_variant", _I, [_P, _I]),
    ("shg_plan_destroy", None, [_P]),
    ("shg_family_plan_create", _I, [_P, _L, _P, _P, _P, ctypes.POINTER(_P)]),
    ("shg_family_plan_exec", _I, [_P, _I, _D, _P, _P, _P]),
    ("shg_family_plan_counts", _L, [_P, ctypes.POINTER(_L), ctypes.POINTER(_L)]),
    ("shg_family_plan_destroy", None, [_P]),
    ("shg_plan_2c_set_launch", _I, [_P, _I, _I]),
    ("shg_graph_2c_create", _I, [_P, _I, _P, _P, _I, _P, _P, ctypes.POINTER(_P)]),
    ("shg_plan_2c_exec_fused", _I, [_P, _I, _P, _P, _I, _P, _P, _P]),
    ("shg_graph_2c_create_fused", _I, [_P, _I, _P, _P, _I, _P, _P, ctypes.POINTER(_P)]),
    ("shg_graph_launch", _I, [_P, _P]),
    ("shg_graph_destroy", None, [_P]),
    ("shg_eval_3c_aab", _I, [_P, _P, _L, _P, _P, _P, _I, _D, _P, _P, _P]),
    ("shg_eval_2c_grad", _I, [_P, _L, _P, _P, _I, _D, _I, _P, _P, _P, _P, _P]),
    ("shg_eval_3c_aab_grad", _I, [_P, _P, _L, _P, _P, _P, _I, _P, _P, _P, _P, _P]),
    ("shg_eval_2c_noalloc", _I, [_P, _L, _P, _P, _I, _D, _I, _P, _P, _P]),
    ("shg_scatter_2c", _I, [_P, _L, _P, _P, _P, _P, _P, _L, _I, _P, _P]),
    ("shg_gather_2c", _I, [_P, _L, _P, _P, _P, _P, _P, _L, _I, _P, _P]),
    ("shg_reduce_centers", _I, [_P, _L, _P, _P, _P, _P, _P, _P]),
    ("shg_debug_boys", _I, [_L, _P, _I, _P, _P]),
    ("shg_measure_alu_peak", _I, [_I, _I, ctypes.POINTER(_D), _P]),
    ("shg_last_error", ctypes.c_char_p, []),
    ("shg_version", ctypes.c_char_p, []),
]

_lock = threading.Lock()
_lib = None


class ShgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("shg error %d: %s" % (code, msg))
        self.code = code


def library_path():
    return _build.LIB


def load(path=None):
    """Load the shared library (no build, no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or _build.LIB
            if not os.path.exists(p):
                raise RuntimeError("libshg_gb300.so not found at %s: run paper_1701_06588_gb300.build.build()" % p)
            lib = ctypes.CDLL(p)
            for name, res, args in SIGNATURES:
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
        return _lib


def check(rc):
    if rc < 0:
        raise ShgError(int(rc), load().shg_last_error().decode(errors="replace"))
    return rc


def _ptr(x):
    """Address of a numpy array, torch tensor, int or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


def shg_basis_create(n_shells, l, nprim, exps, coefs, n_centers, centers, center_of_shell, normalize):
    h = _P()
    check(load().shg_basis_create(n_shells, _ptr(l), _ptr(nprim), _ptr(exps), _ptr(coefs), n_centers, _ptr(centers),
                                  _ptr(center_of_shell), int(normalize), ctypes.byref(h)))
    return h.value


def shg_basis_set_centers(basis, centers):
    return check(load().shg_basis_set_centers(basis, _ptr(centers)))


def shg_basis_destroy(basis):
    load().shg_basis_destroy(basis)


def shg_pair_offsets(basis, n_pairs, pair_a, pair_b, offsets):
    return check(load().shg_pair_offsets(basis, n_pairs, _ptr(pair_a), _ptr(pair_b), _ptr(offsets)))


def shg_triple_offsets(orb, aux, n, t_a, t_atilde, t_b, offsets):
    return check(load().shg_triple_offsets(orb, aux, n, _ptr(t_a), _ptr(t_atilde), _ptr(t_b), _ptr(offsets)))


def shg_eval_2c(basis, n_pairs, d_pair_a, d_pair_b, op, omega, screen_thresh, precision, d_out_offsets, d_out,
                stream):
    return check(load().shg_eval_2c(basis, n_pairs, _ptr(d_pair_a), _ptr(d_pair_b), op, omega, screen_thresh,
                                    precision, _ptr(d_out_offsets), _ptr(d_out), stream))


def shg_plan_2c_create(basis, n_pairs, d_pair_a, d_pair_b, schedule, stream):
    h = _P()
    check(load().shg_plan_2c_create(basis, n_pairs, _ptr(d_pair_a), _ptr(d_pair_b), schedule, stream,
                                    ctypes.byref(h)))
    return h.value


def shg_plan_2c_exec(plan, op, omega, screen_thresh, precision, d_out_offsets, d_out, stream):
    return check(load().shg_plan_2c_exec(plan, op, omega, screen_thresh, precision, _ptr(d_out_offsets),
                                         _ptr(d_out), stream))


def shg_family_plan_create(basis, n_pairs, d_pair_a, d_pair_b, stream):
    h = _P()
    check(load().shg_family_plan_create(basis, n_pairs, _ptr(d_pair_a), _ptr(d_pair_b), stream, ctypes.byref(h)))
    return h.value


def shg_family_plan_exec(plan, op, omega, d_out_offsets, d_out, stream):
    return check(load().shg_family_plan_exec(plan, op, omega, _ptr(d_out_offsets), _ptr(d_out), stream))


def shg_family_plan_counts(plan):
    nf, ng = _L(), _L()
    n = load().shg_family_plan_counts(plan, ctypes.byref(nf), ctypes.byref(ng))
    return int(n), int(nf.value), int(ng.value)


def shg_family_plan_destroy(plan):
    load().shg_family_plan_destroy(plan)


def shg_plan_launches(plan):
    return load().shg_plan_launches(plan)


def shg_plan_2c_set_variant(plan, variant):
    return check(load().shg_plan_2c_set_variant(plan, variant))


def shg_plan_launches_prec(plan, precision):
    return check(load().shg_plan_launches_prec(plan, precision))


def shg_plan_destroy(plan):
    load().shg_plan_destroy(plan)


def shg_plan_2c_set_launch(plan, threads_per_cta, ctas_per_sm):
    return check(load().shg_plan_2c_set_launch(plan, threads_per_cta, ctas_per_sm))


def shg_graph_2c_create(plan, ops, omegas, precision, d_out_offsets, d_outs):
    import numpy as _np
    n = len(ops)
    ops_a = _np.ascontiguousarray(ops, dtype=_np.int32)
    om_a = _np.ascontiguousarray(omegas, dtype=_np.float64)
    outs_a = (ctypes.c_void_p * n)(*[_ptr(o) for o in d_outs])
    h = _P()
    check(load().shg_graph_2c_create(plan, n, _ptr(ops_a), _ptr(om_a), precision, _ptr(d_out_offsets),
                                     ctypes.cast(outs_a, ctypes.c_void_p), ctypes.byref(h)))
    return h.value


def _op_arrays(ops, omegas, d_outs):
    import numpy as _np
    n = len(ops)
    ops_a = _np.ascontiguousarray(ops, dtype=_np.int32)
    om_a = _np.ascontiguousarray(omegas, dtype=_np.float64)
    outs_a = (ctypes.c_void_p * n)(*[_ptr(o) for o in d_outs])
    return n, ops_a, om_a, outs_a


def shg_plan_2c_exec_fused(plan, ops, omegas, precision, d_out_offsets, d_outs, stream):
    n, ops_a, om_a, outs_a = _op_arrays(ops, omegas, d_outs)
    return check(load().shg_plan_2c_exec_fused(plan, n, _ptr(ops_a), _ptr(om_a), precision, _ptr(d_out_offsets),
                                               ctypes.cast(outs_a, ctypes.c_void_p), stream))


def shg_graph_2c_create_fused(plan, ops, omegas, precision, d_out_offsets, d_outs):
    n, ops_a, om_a, outs_a = _op_arrays(ops, omegas, d_outs)
    h = _P()
    check(load().shg_graph_2c_create_fused(plan, n, _ptr(ops_a), _ptr(om_a), precision, _ptr(d_out_offsets),
                                           ctypes.cast(outs_a, ctypes.c_void_p), ctypes.byref(h)))
    return h.value


def shg_graph_launch(graph, stream):
    return check(load().shg_graph_launch(graph, stream))


def shg_graph_destroy(graph):
    load().shg_graph_destroy(graph)


def shg_eval_3c_aab(orb, aux, n, d_a, d_atilde, d_b, precision, screen_thresh, d_out_offsets, d_out, stream):
    return check(load().shg_eval_3c_aab(orb, aux, n, _ptr(d_a), _ptr(d_atilde), _ptr(d_b), precision, screen_thresh,
                                        _ptr(d_out_offsets), _ptr(d_out), stream))


def shg_eval_2c_grad(basis, n, d_pair_a, d_pair_b, op, omega, precision, d_w_offsets, d_w, d_grad_a, d_grad_b,
                     stream):
    return check(load().shg_eval_2c_grad(basis, n, _ptr(d_pair_a), _ptr(d_pair_b), op, omega, precision,
                                         _ptr(d_w_offsets), _ptr(d_w), _ptr(d_grad_a), _ptr(d_grad_b), stream))


def shg_eval_3c_aab_grad(orb, aux, n, d_a, d_atilde, d_b, precision, d_w_offsets, d_w, d_grad_a, d_grad_b, stream):
    return check(load().shg_eval_3c_aab_grad(orb, aux, n, _ptr(d_a), _ptr(d_atilde), _ptr(d_b), precision,
                                             _ptr(d_w_offsets), _ptr(d_w), _ptr(d_grad_a), _ptr(d_grad_b), stream))


def shg_eval_2c_noalloc(basis, n_pairs, d_pair_a, d_pair_b, op, omega, precision, d_out_offsets, d_out, stream):
    return check(load().shg_eval_2c_noalloc(basis, n_pairs, _ptr(d_pair_a), _ptr(d_pair_b), op, omega, precision,
                                            _ptr(d_out_offsets), _ptr(d_out), stream))


def shg_scatter_2c(basis, n, d_pa, d_pb, d_block_off, d_blocks, d_ao_off, ld, symmetric, d_matrix, stream):
    return check(load().shg_scatter_2c(basis, n, _ptr(d_pa), _ptr(d_pb), _ptr(d_block_off), _ptr(d_blocks),
                                       _ptr(d_ao_off), ld, int(symmetric), _ptr(d_matrix), stream))


def shg_gather_2c(basis, n, d_pa, d_pb, d_block_off, d_matrix, d_ao_off, ld, symmetric, d_blocks, stream):
    return check(load().shg_gather_2c(basis, n, _ptr(d_pa), _ptr(d_pb), _ptr(d_block_off), _ptr(d_matrix),
                                      _ptr(d_ao_off), ld, int(symmetric), _ptr(d_blocks), stream))


def shg_reduce_centers(basis, n, d_pa, d_pb, d_grad_a, d_grad_b, d_center_grad, stream):
    return check(load().shg_reduce_centers(basis, n, _ptr(d_pa), _ptr(d_pb), _ptr(d_grad_a), _ptr(d_grad_b),
                                           _ptr(d_center_grad), stream))


def shg_debug_boys(n, d_T, nmax, d_F, stream):
    return check(load().shg_debug_boys(n, _ptr(d_T), nmax, _ptr(d_F), stream))


def shg_measure_alu_peak(kind, iters, stream):
    v = _D()
    check(load().shg_measure_alu_peak(kind, iters, ctypes.byref(v), stream))
    return v.value


def shg_last_error():
    return load().shg_last_error().decode(errors="replace")


def shg_version():
    return load().shg_version().decode()
