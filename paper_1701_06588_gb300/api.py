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

    def launches_for(self, precision):
        """Kernel launches one execution of this plan issues in `precision`."""
        return L.shg_plan_launches_prec(self.handle, _prec(precision))

    def exec(self, op, out_offsets, out, omega=0.0, precision="fp64", screen_thresh=0.0, stream=None):
        L.shg_plan_2c_exec(self.handle, _op(op), float(omega), float(screen_thresh), _prec(precision),
                           out_offsets, out, _stream(stream))
        return out

    def exec_fused(self, ops, out_offsets, outs, omegas=None, precision="fp64", stream=None):
        """Several operators (overlap, coulomb, erfc, erf, gauss; each at most
        once) in one pass sharing the geometry-only angular part; outs[i]
        receives operator ops[i] in the layout of exec."""
        omegas = [0.0] * len(ops) if omegas is None else [float(w) for w in omegas]
        L.shg_plan_2c_exec_fused(self.handle, [_op(o) for o in ops], omegas, _prec(precision), out_offsets,
                                 list(outs), _stream(stream))
        return outs

    def close(self):
        if getattr(self, "handle", None):
            L.shg_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FamilyPlan:
    """Pair list grouped by family pair (shells on one center sharing one
    exponent set): radial terms once per primitive pair of each family pair,
    contracted per shell pair, then the class-tiled angular kernel.  FP64;
    reusable for any operator but (a|r_a^{2n}|b) and any geometry."""

    def __init__(self, basis, pair_a, pair_b, stream=None):
        self.basis = basis
        self.pair_a = _dev_i32(pair_a)
        self.pair_b = _dev_i32(pair_b)
        self.n = int(self.pair_a.numel())
        self.handle = L.shg_family_plan_create(basis.handle, self.n, self.pair_a, self.pair_b, _stream(stream))
        _, self.n_family_pairs, self.n_groups = L.shg_family_plan_counts(self.handle)

    def exec(self, op, out_offsets, out, omega=0.0, stream=None):
        L.shg_family_plan_exec(self.handle, _op(op), float(omega), out_offsets, out, _stream(stream))

    def close(self):
        if getattr(self, "handle", None):
            L.shg_family_plan_destroy(self.handle)
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


def eval_3c_aab(orb, aux, t_a, t_atilde, t_b, precision="fp64", screen_thresh=0.0, stream=None):
    """Three-index overlaps (a b a~) of a triple list (a, a~ in `orb` on one
    center, b in `aux`) as one flat float64 CUDA tensor plus block offsets."""
    off, total = orb.triple_offsets(aux, t_a, t_atilde, t_b)
    out = torch.empty(max(total, 1), dtype=torch.float64, device="cuda")
    L.shg_eval_3c_aab(orb.handle, aux.handle, len(off), _dev_i32(t_a), _dev_i32(t_atilde), _dev_i32(t_b),
                      _prec(precision), float(screen_thresh), _dev_i64(off), out, _stream(stream))
    return out[:total], off


def eval_2c_grad(basis, pair_a, pair_b, op, upstream, offsets=None, omega=0.0, precision="fp64", stream=None):
    """Vector-Jacobian product of the two-center blocks with upstream weights
    (flat float64 CUDA tensor in the layout of eval_2c): returns per-pair
    gradients with respect to R_a and R_b, each (n_pairs, 3) CUDA tensors."""
    if offsets is None:
        offsets, _ = basis.pair_offsets(pair_a, pair_b)
    n = len(offsets)
    ga = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    gb = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    L.shg_eval_2c_grad(basis.handle, n, _dev_i32(pair_a), _dev_i32(pair_b), _op(op), float(omega), _prec(precision),
                       _dev_i64(offsets), upstream.contiguous(), ga, gb, _stream(stream))
    return ga, gb


class TwoCenterIntegrals(torch.autograd.Function):
    """Blocks (a|O|b) as a differentiable function of the center coordinates.

    forward(centers[n_centers, 3] float64, basis, pair_a, pair_b, op, omega)
    returns the flat block tensor; backward calls the library's gradient
    kernel (radial terms recomputed, nothing stored) and scatters the per-pair
    gradients onto the centers with index_add_.
    """

    @staticmethod
    def forward(ctx, centers, basis, pair_a, pair_b, op, omega):
        basis.set_centers(centers.detach().cpu().numpy())
        out, off = eval_2c(basis, pair_a, pair_b, op, omega=omega)
        ctx.basis, ctx.pair_a, ctx.pair_b, ctx.op, ctx.omega, ctx.off = basis, pair_a, pair_b, op, omega, off
        ctx.n_centers = centers.shape[0]
        ctx.device = centers.device
        return out

    @staticmethod
    def backward(ctx, grad_out):
        ga, gb = eval_2c_grad(ctx.basis, ctx.pair_a, ctx.pair_b, ctx.op, grad_out.to("cuda", torch.float64),
                              offsets=ctx.off, omega=ctx.omega)
        ca = torch.from_numpy(ctx.basis.center_of[np.asarray(ctx.pair_a)].astype(np.int64)).cuda()
        cb = torch.from_numpy(ctx.basis.center_of[np.asarray(ctx.pair_b)].astype(np.int64)).cuda()
        g = torch.zeros((ctx.n_centers, 3), dtype=torch.float64, device="cuda")
        g.index_add_(0, ca, ga)
        g.index_add_(0, cb, gb)
        return g.to(ctx.device), None, None, None, None, None


class ThreeIndexOverlap(torch.autograd.Function):
    """Blocks (a b a~) as a differentiable function of the center coordinates.

    forward(centers[n_centers, 3] float64, orb, aux, t_a, t_atilde, t_b): `orb`
    and `aux` index one common list of centers (atoms), which is set on both;
    returns the flat block tensor.  backward calls the library's (aab)
    gradient kernel and scatters the per-triple gradients onto the centers of
    a (= a~) and b with index_add_.
    """

    @staticmethod
    def forward(ctx, centers, orb, aux, t_a, t_atilde, t_b):
        c = centers.detach().cpu().numpy()
        orb.set_centers(c)
        if aux is not orb:
            aux.set_centers(c)
        out, off = eval_3c_aab(orb, aux, t_a, t_atilde, t_b)
        ctx.orb, ctx.aux, ctx.t = orb, aux, (t_a, t_atilde, t_b)
        ctx.off, ctx.n_centers, ctx.device = off, centers.shape[0], centers.device
        return out

    @staticmethod
    def backward(ctx, grad_out):
        t_a, t_atilde, t_b = ctx.t
        ga, gb = eval_3c_aab_grad(ctx.orb, ctx.aux, t_a, t_atilde, t_b, grad_out.to("cuda", torch.float64),
                                  offsets=ctx.off)
        ca = torch.from_numpy(ctx.orb.center_of[np.asarray(t_a)].astype(np.int64)).cuda()
        cb = torch.from_numpy(ctx.aux.center_of[np.asarray(t_b)].astype(np.int64)).cuda()
        g = torch.zeros((ctx.n_centers, 3), dtype=torch.float64, device="cuda")
        g.index_add_(0, ca, ga)
        g.index_add_(0, cb, gb)
        return g.to(ctx.device), None, None, None, None, None


class Graph2c:
    """A CUDA graph replaying one plan for several operators (C ABI
    shg_graph_2c_create / shg_graph_launch; fused=True captures one
    shg_plan_2c_exec_fused pass instead of one pass per operator)."""

    def __init__(self, plan, ops, omegas, out_offsets, outs, precision="fp64", fused=False):
        self.plan = plan
        self.outs = list(outs)
        self.out_offsets = out_offsets
        if fused:
            self.handle = L.shg_graph_2c_create_fused(plan.handle, [_op(o) for o in ops],
                                                      [float(w) for w in omegas], _prec(precision), out_offsets,
                                                      self.outs)
        else:
            self.handle = L.shg_graph_2c_create(plan.handle, [_op(o) for o in ops], [float(w) for w in omegas],
                                                _prec(precision), out_offsets, self.outs)

    def launch(self, stream=None):
        L.shg_graph_launch(self.handle, _stream(stream))

    def close(self):
        if getattr(self, "handle", None):
            L.shg_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HostPipeline2c:
    """Two-center blocks from host pair lists into host output arrays, with
    the copies and the planning overlapped with the computation.

    The pair list is split into n_chunks contiguous slices (default:
    default_chunks(precision)).  For slice k: its pair lists and offsets are
    copied to the device on an upload stream, planned there
    (shg_plan_2c_create, whose one synchronisation waits for that stream
    only), evaluated by one fused pass (shg_plan_2c_exec_fused) on one of
    two compute streams (alternating, so that consecutive passes overlap at
    their tails), and its blocks (a contiguous range of every output,
    since the offsets are the prefix sums of the block sizes) are copied to
    the host on a copy stream.  The host plans slice k+1 while the GPU
    computes slice k, and the read-back of slice k overlaps the computation
    of slice k+1.  Inputs: pinned host tensors pair_a, pair_b (int32),
    offsets (int64) and centers; outputs: pinned host float64 tensors, one
    per operator.  Device buffers are kept between calls.
    """

    def __init__(self, basis, n_chunks=None, launch=None, schedule="persistent"):
        self.basis = basis
        self.n_chunks = None if n_chunks is None else max(1, int(n_chunks))
        self.launch = launch
        self.schedule = schedule
        self.copy_stream = torch.cuda.Stream()
        self.upload_stream = torch.cuda.Stream()
        # chunks alternate between two compute streams, so that chunk k+1's pass
        # fills the tail of chunk k's (each ends with its slowest tile)
        self.compute_streams = [torch.cuda.Stream(), torch.cuda.Stream()]
        self._dev = {}

    @staticmethod
    def default_chunks(precision):
        """Measured on the 2M-pair workload (1/r and erfc), median ms per
        call: FP64 18.7, 18.1-18.8, 18.5 and 19.3 for 1, 2, 4 and 8 chunks
        (4 varies least); mixed 8.3, 8.4, 9.9 and 12.7, so one chunk (every
        chunk of a mixed pass also waits for its own FP64 launch of the classes
        with both l >= 4, whose slowest tile sets a fixed time per chunk)."""
        return 1 if precision == "mixed" else 4

    def _buf(self, name, n, dtype):
        t = self._dev.get(name)
        if t is None or t.numel() < n or t.dtype != dtype:
            t = torch.empty(max(n, 1), dtype=dtype, device="cuda")
            self._dev[name] = t
        return t[:n]

    def run(self, pair_a, pair_b, offsets, ops, outs, omegas=None, precision="fp64", centers=None):
        n = int(pair_a.numel())
        total = int(outs[0].numel())
        omegas = [0.0] * len(ops) if omegas is None else list(omegas)
        stream = torch.cuda.current_stream()
        up = self.upload_stream
        d_pa = self._buf("pa", n, torch.int32)
        d_pb = self._buf("pb", n, torch.int32)
        d_off = self._buf("off", n, torch.int64)
        d_out = [self._buf("out%d" % i, total, torch.float64) for i in range(len(ops))]
        if centers is not None:
            self.basis.set_centers(centers)
        # earlier work on the caller's stream (a previous run's use of the
        # buffers) comes before the uploads and the passes
        start = torch.cuda.Event()
        start.record(stream)
        up.wait_event(start)
        for cs in self.compute_streams:
            cs.wait_event(start)
        off_h = offsets.numpy()
        chunks = self.n_chunks or self.default_chunks(precision)
        bounds = [n * k // chunks for k in range(chunks + 1)]
        plans = []
        for k in range(chunks):
            lo, hi = bounds[k], bounds[k + 1]
            if hi <= lo:
                continue
            torch.cuda.nvtx.range_push("shg:h2d")
            with torch.cuda.stream(up):
                d_pa[lo:hi].copy_(pair_a[lo:hi], non_blocking=True)
                d_pb[lo:hi].copy_(pair_b[lo:hi], non_blocking=True)
                d_off[lo:hi].copy_(offsets[lo:hi], non_blocking=True)
            torch.cuda.nvtx.range_pop()
            plan = Plan2c(self.basis, d_pa[lo:hi], d_pb[lo:hi], schedule=self.schedule, stream=up)
            plans.append(plan)
            if self.launch:
                set_launch(plan, self.launch["threads_per_cta"], self.launch["ctas_per_sm"],
                           self.launch.get("variant", 1))
            planned = torch.cuda.Event()
            planned.record(up)
            cs = self.compute_streams[len(plans) % 2]
            cs.wait_event(planned)
            plan.exec_fused(ops, d_off[lo:hi], d_out, omegas=omegas, precision=precision, stream=cs)
            e0 = int(off_h[lo])
            e1 = int(off_h[hi]) if hi < n else total
            done = torch.cuda.Event()
            done.record(cs)
            self.copy_stream.wait_event(done)
            torch.cuda.nvtx.range_push("shg:d2h")
            with torch.cuda.stream(self.copy_stream):
                for o_h, o_d in zip(outs, d_out):
                    o_h[e0:e1].copy_(o_d[e0:e1], non_blocking=True)
            torch.cuda.nvtx.range_pop()
        # the copy stream waited for every pass: fin orders all of them
        fin = torch.cuda.Event()
        fin.record(self.copy_stream)
        stream.wait_event(fin)
        # the plans' memory is released in the order of the upload stream, after
        # every pass that used it
        up.wait_event(fin)
        for plan in plans:
            plan.close()
        return outs


def set_launch(plan, threads_per_cta=128, ctas_per_sm=0, variant=1):
    """Launch shape of later executions of a plan: threads per CTA, persistent
    CTAs per SM (0 = occupancy limit) and the compiled variant of the
    fused kernel (0, 1 or 2, see shg_plan_2c_set_variant)."""
    L.shg_plan_2c_set_launch(plan.handle, int(threads_per_cta), int(ctas_per_sm))
    L.shg_plan_2c_set_variant(plan.handle, int(variant))


def eval_3c_aab_grad(orb, aux, t_a, t_atilde, t_b, upstream, offsets=None, precision="fp64", stream=None):
    """Vector-Jacobian product of the (a b a~) blocks with upstream weights (flat
    tensor in the layout of eval_3c_aab): per-triple gradients with respect to
    R_a (the common center of a and a~) and R_b, each (n, 3) CUDA tensors."""
    if offsets is None:
        offsets, _ = orb.triple_offsets(aux, t_a, t_atilde, t_b)
    n = len(offsets)
    ga = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    gb = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    L.shg_eval_3c_aab_grad(orb.handle, aux.handle, n, _dev_i32(t_a), _dev_i32(t_atilde), _dev_i32(t_b),
                           _prec(precision), _dev_i64(offsets), upstream.contiguous(), ga, gb, _stream(stream))
    return ga, gb
