"""World-size-2 gloo test of the sharded molecular assembly (CPU only): the
ranks' pair slices cover the molecule's pair list exactly once, and summing
the per-rank partial matrices and forces with the module's all-reduce gives
the full ones.  The blocks and Jacobians come from the oracle and are placed
by a test-local host scatter; the GPU kernels are covered by the -m gpu
tests."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_1701_06588_gb300 import molecule, workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _host_assemble(shells, ao_off, nao, pa, pb, sym, wm):
    """Host stand-in for the scatter kernel (oracle Coulomb blocks) and the
    force path (oracle Jacobians, weights wm)."""
    l = shells["l"]
    M = np.zeros((nao, nao))
    F = np.zeros((len(shells["centers"]), 3))
    if len(pa) == 0:
        return M, F
    v, off, sz = oracle.eval_2c(shells, pa, pb, 1, 0.0, nthreads=2)
    ja, _, _ = oracle.eval_2c_grad(shells, pa, pb, 1, 0.0, center="A", nthreads=2)
    jb, _, _ = oracle.eval_2c_grad(shells, pa, pb, 1, 0.0, center="B", nthreads=2)
    for p in range(len(pa)):
        a, b = pa[p], pb[p]
        na, nb = 2 * l[a] + 1, 2 * l[b] + 1
        blk = v[off[p]:off[p] + sz[p]].reshape(na, nb)
        M[ao_off[a]:ao_off[a] + na, ao_off[b]:ao_off[b] + nb] = blk
        u = wm[ao_off[a]:ao_off[a] + na, ao_off[b]:ao_off[b] + nb].copy()
        if sym and a != b:
            M[ao_off[b]:ao_off[b] + nb, ao_off[a]:ao_off[a] + na] = blk.T
            u += wm[ao_off[b]:ao_off[b] + nb, ao_off[a]:ao_off[a] + na].T
        F[shells["center_of"][a]] += ja[3 * off[p]:3 * (off[p] + sz[p])].reshape(3, sz[p]) @ u.ravel()
        F[shells["center_of"][b]] += jb[3 * off[p]:3 * (off[p] + sz[p])].reshape(3, sz[p]) @ u.ravel()
    return M, F


def _setup():
    coords, el, bs = W.molecule_workload(6, seed=12)
    shells, ao_off, nao = molecule.molecule_shells(coords, el, bs)
    wm = np.random.default_rng(1).uniform(-1, 1, (nao, nao))
    return shells, ao_off, nao, 0.5 * (wm + wm.T)


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    shells, ao_off, nao, wm = _setup()
    a, b = molecule.local_pairs(shells, rank, world, "coulomb")
    M, F = _host_assemble(shells, ao_off, nao, a, b, True, wm)
    tm = molecule.allreduce_sum(torch.from_numpy(M))
    tf = molecule.allreduce_sum(torch.from_numpy(F))
    n = molecule.allreduce_sum(torch.tensor([float(len(a))], dtype=torch.float64))
    if rank == 0:
        q.put((tm.numpy(), tf.numpy(), float(n.item()), [int(x) for x in a[:1]] + [int(x) for x in b[:1]]))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_assembly_over_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    M, F, n, _ = q.get(timeout=600)
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    shells, ao_off, nao, wm = _setup()
    pa, pb = molecule.shell_pairs(len(shells["l"]), True)
    assert n == len(pa)
    Mf, Ff = _host_assemble(shells, ao_off, nao, pa, pb, True, wm)
    np.testing.assert_allclose(M, Mf, rtol=0, atol=1e-14 * np.abs(Mf).max())
    np.testing.assert_allclose(F, Ff, rtol=1e-12, atol=1e-14 * np.abs(Ff).max())
    np.testing.assert_allclose(M, M.T, rtol=0, atol=1e-15 * np.abs(M).max())   # a = b blocks: oracle rounding
