"""User-facing Python API over the C ABI, on PyTorch CUDA tensors.

PyTorch supplies device memory and streams only; the integrals are computed by
the library's CUDA kernels.  There is no CPU path: on a machine without the
built library or without a CUDA device every call raises.
"""
import numpy as np
import torch

from . import _lib as L


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _op(op):
    return L.OPERATORS[op] if isinstance(op, str) else int(op)


def _prec(p):
    return L.PRECISIONS[p] if isinstance(p, str) else int(p)


def _sched(s):
    return L.SCHEDULES[s] if isinstance(s, str) else int(s)


class Basis:
    """A shell set uploaded to the current CUDA device.

    shells: dict with l, nprim, exps, coefs, centers (n_centers x 3),
    center_of (see paper_1701_06588_gb300.workloads).  Raw coefficients are
    multiplied by the closed-form N_l when normalize is true.
    """

    def __init__(self, shells, normalize=True):
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.l = np.ascontiguousarray(shells["l"], dtype=np.int32)
        self.nprim = np.ascontiguousarray(shells["nprim"], dtype=np.int32)
        exps = np.ascontiguousarray(shells["exps"], dtype=np.float64)
        coefs = np.ascontiguousarray(shells["coefs"], dtype=np.float64)
        self.centers = np.ascontiguousarray(shells["centers"], dtype=np.float64).reshape(-1, 3)
        self.center_of = np.ascontiguousarray(shells["center_of"], dtype=np.int32)
        self.device = torch.cuda.current_device()
        self.handle = L.shg_basis_create(len(self.l), self.l, self.nprim, exps, coefs, len(self.centers),
                                         self.centers, self.center_of, bool(normalize))

    def set_centers(self, centers):
        c = np.ascontiguousarray(centers, dtype=np.float64).reshape(-1, 3)
        L.shg_basis_set_centers(self.handle, c)
        self.centers = c

    def close(self):
        if getattr(self, "handle", None):
            L.shg_basis_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def pair_offsets(self, pair_a, pair_b):
        pa = np.ascontiguousarray(pair_a, dtype=np.int32)
        pb = np.ascontiguousarray(pair_b, dtype=np.int32)
        off = np.zeros(len(pa), dtype=np.int64)
        total = L.shg_pair_offsets(self.handle, len(pa), pa, pb, off)
        return off, int(total)

    def triple_offsets(self, aux, t_a, t_atilde, t_b):
        ta, tt, tb = (np.ascontiguousarray(x, dtype=np.int32) for x in (t_a, t_atilde, t_b))
        off = np.zeros(len(ta), dtype=np.int64)
        total = L.shg_triple_offsets(self.handle, aux.handle, len(ta), ta, tt, tb, off)
        return off, int(total)


def _dev_i32(x):
    if isinstance(x, torch.Tensor):
        return x.to(device="cuda", dtype=torch.int32).contiguous()
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.int32)).cuda()


def _dev_i64(x):
    if isinstance(x, torch.Tensor):
        return x.to(device="cuda", dtype=torch.int64).contiguous()
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.int64)).cuda()


class Plan2c:
    """A bucketed pair list (device); reusable for any operator and geometry."""

    def __init__(self, basis, pair_a, pair_b, schedule="persistent", stream=None):
        self.basis = basis
        self.pair_a = _dev_i32(pair_a)
        self.pair_b = _dev_i32(pair_b)
        self.n = int(self.pair_a.numel())
        self.handle = L.shg_plan_2c_create(basis.handle, self.n, self.pair_a, self.pair_b, _sched(schedule),
                                           _stream(stream))
        self.launches = L.shg_plan_launches(self.handle)

    def exec(self, op, out_offsets, out, omega=0.0, precision="fp64", screen_thresh=0.0, stream=None):
        L.shg_plan_2c_exec(self.handle, _op(op), float(omega), float(screen_thresh), _prec(precision),
                           out_offsets, out, _stream(stream))
        return out

    def close(self):
        if getattr(self, "handle", None):
            L.shg_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def eval_2c(basis, pair_a, pair_b, op, omega=0.0, precision="fp64", screen_thresh=0.0, stream=None):
    """All blocks (a|O|b) of a pair list as one flat float64 CUDA tensor plus
    the int64 offsets (numpy) of each block."""
    off, total = basis.pair_offsets(pair_a, pair_b)
    out = torch.empty(max(total, 1), dtype=torch.float64, device="cuda")
    d_off = _dev_i64(off)
    L.shg_eval_2c(basis.handle, len(off), _dev_i32(pair_a), _dev_i32(pair_b), _op(op), float(omega),
                  float(screen_thresh), _prec(precision), d_off, out, _stream(stream))
    return out[:total], off
