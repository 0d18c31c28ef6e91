"""The multi-GPU shard path on CPU: the partition of a graph into
contiguous factor slices, and the exchange protocol run as world-size-2
gloo ranks.  The ranks' arithmetic is a stand-in (each rank adds fixed terms
onto the running sums, in order), so these tests check what the protocol
must guarantee whatever the kernels compute: the chain hands the sums over
in rank order (the result equals one rank holding every term), every rank
ends with the same sums and takes the same stop decision, the gather
exchange adds the ranks' sums in rank order, and a rank that never takes
part makes the others fail with a timeout instead of waiting for ever.  The
GPU kernels behind the same protocol are compared with the one-GPU run and
the oracle in tests/test_gpu_shard.py."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_1603_02526_gb300 import inputs
from paper_1603_02526_gb300.shard import split_problem


# ---------------------------------------------------------------------------
# partition
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("G", [1, 2, 3, 7])
def test_split_keeps_creation_order_and_balances_edges(G):
    p = inputs.packing_problem(20)
    shards, first = split_problem(p, G)
    assert len(shards) == G and first[0] == 0
    dims = p.var_dims()

    def edges(q):
        return sum(int(dims[b.var_ids].sum()) for b in q.factor_blocks)
    # the slices, taken in rank order, are the original factors in order
    for attr in ("var_ids", "params"):
        whole = np.concatenate([getattr(b, attr).reshape(len(b.var_ids), -1) for b in p.factor_blocks
                                if b.ftype == inputs.PACK_PAIR])
        got = np.concatenate([getattr(b, attr).reshape(len(b.var_ids), -1) for q in shards for b in q.factor_blocks
                              if b.ftype == inputs.PACK_PAIR])
        assert np.array_equal(whole, got)
    # the factor types appear in the original order
    types = [b.ftype for q in shards for b in q.factor_blocks]
    assert types == sorted(types, key=[b.ftype for b in p.factor_blocks].index)
    E = p.num_edges
    assert sum(edges(q) for q in shards) == E
    assert first == list(np.cumsum([0] + [edges(q) for q in shards])[:-1])
    for q in shards:                      # within one factor (6 edges) of E / G
        assert abs(edges(q) - E / G) <= 6
        assert q.var_blocks == p.var_blocks and q.z0 is p.z0


def test_split_rejects_more_shards_than_factors():
    with pytest.raises(ValueError):
        split_problem(inputs.packing_problem(1), 10)


# ---------------------------------------------------------------------------
# a stand-in for one rank's kernels
# ---------------------------------------------------------------------------
class FakeShard:
    """Holds, per variable, a list of terms (this rank's share); the x-step
    adds them one by one onto the incoming sums, z = S / R; residual sums
    are fixed functions of z.  Enough to check the protocol's order."""

    def __init__(self, terms, rho):
        self.terms = terms            # (k, nz) float64: k terms per variable, in order
        self.rho = rho                # (k, nz)
        self.nz = terms.shape[1]
        self.s_out = torch.zeros(self.nz, dtype=torch.float64)
        self.total = torch.zeros(self.nz, dtype=torch.float64)
        self.z = np.zeros(self.nz)
        self.step = 0

    def new_sums(self, n=1):
        return torch.zeros((n, self.nz), dtype=torch.float64)

    def rho_chain(self, a, b):
        a = np.zeros(self.nz) if a is None else a.copy()
        b = np.zeros(self.nz) if b is None else b.copy()
        for r in self.rho:
            a += r
            b += r * r
        return a, b

    def begin(self, srho, srho2):
        self.srho, self.srho2 = srho, srho2

    def init(self):
        self.z[:] = 0.0
        self.step = 0

    def xstep(self, check_prev, s_in, s_out):
        S = np.zeros(self.nz) if s_in is None else s_in.numpy().copy()
        scale = 1.0 / (1.0 + self.step)           # terms shrink: the run converges
        for t in self.terms:
            S += t * scale
        s_out.copy_(torch.from_numpy(S))
        return torch.tensor([float(((self.terms * scale) ** 2).sum()) * scale], dtype=torch.float64) if check_prev else None

    def add_parts(self, parts, total):
        S = parts[0].clone()
        for r in range(1, parts.shape[0]):
            S += parts[r]
        total.copy_(S)

    def zstep(self, total, check_):
        zn = total.numpy() / self.srho
        d = float((self.srho2 * (zn - self.z) ** 2).sum())
        self.z = zn
        self.step += 1
        return torch.tensor([d], dtype=torch.float64) if check_ else None

    def finish(self):
        return torch.tensor([float(((self.terms / (1.0 + self.step)) ** 2).sum()) / (1.0 + self.step)], dtype=torch.float64)

    def sync(self):
        pass


def _terms(seed, nz=7, k_total=12):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((k_total, nz)), rng.uniform(0.5, 2.0, (k_total, nz))


def _slices(G, k_total=12):
    cut = np.linspace(0, k_total, G + 1).astype(int)
    return [(cut[r], cut[r + 1]) for r in range(G)]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _run_local(G, exchange, iters, tol, ce):
    from paper_1603_02526_gb300.shard import LocalGroup, ShardedSweep
    T, R = _terms(7)
    shards = [FakeShard(T[a:b], R[a:b]) for a, b in _slices(G)]
    sw = ShardedSweep(LocalGroup(shards), num_edges=12 * 7, exchange=exchange)
    sw.init()
    r = sw.iterate(iters, tol, tol, ce)
    return r, shards[0].z.copy()


def _dist_worker(rank, port, q, exchange, iters, tol, ce, vanish):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import datetime
    import torch.distributed as dist
    from paper_1603_02526_gb300 import _lib
    from paper_1603_02526_gb300.shard import DistGroup, ShardedSweep
    dist.init_process_group("gloo", rank=rank, world_size=2, timeout=datetime.timedelta(seconds=20))
    T, R = _terms(7)
    a, b = _slices(2)[rank]
    sh = FakeShard(T[a:b], R[a:b])
    try:
        if vanish and rank == 1:
            q.put((rank, "left", None))
            q.close()
            q.join_thread()                      # the message is out before the process ends
            os._exit(0)                          # never takes part in any exchange
        grp = DistGroup(sh, timeout_s=3.0)
        sw = ShardedSweep(grp, num_edges=12 * 7, exchange=exchange)
        sw.init()
        r = sw.iterate(iters, tol, tol, ce)
        q.put((rank, r, sh.z.tolist()))
    except _lib.FgaError as e:
        q.put((rank, "error", e.code))
    dist.destroy_process_group() if not vanish else None


def _run_dist(exchange, iters, tol, ce, vanish=False):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dist_worker, args=(r, port, q, exchange, iters, tol, ce, vanish))
             for r in range(2)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=120) for _ in range(2)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
    return out


@pytest.mark.parametrize("exchange", ["chain", "gather"])
def test_two_gloo_ranks_equal_one_process(exchange):
    """Same iterations, residuals, stop decision and z on both ranks as the
    two shards run in one process; for the chain also as one rank holding
    every term (the hand-over keeps the serial order)."""
    want, zw = _run_local(2, exchange, 200, 1e-2, 3)
    out = _run_dist(exchange, 200, 1e-2, 3)
    for rank, r, z in out:
        assert r == want, (rank, r, want)
        assert np.array_equal(np.array(z), zw)
    assert 0 < want["iters"] < 200 and want["iters"] % 3 == 0 and want["status"] == 0
    if exchange == "chain":
        # one rank holding every term: the same z bit for bit (the chain keeps
        # the serial order); the primal residual sums its ranks' partials, so
        # it may differ in the last bits
        one, z1 = _run_local(1, exchange, 200, 1e-2, 3)
        assert np.array_equal(z1, zw)
        assert (one["iters"], one["status"], one["r_dual"]) == (want["iters"], want["status"], want["r_dual"])
        assert abs(one["r_pri"] - want["r_pri"]) <= 1e-12 * want["r_pri"]


def test_budget_status_over_ranks():
    out = _run_dist("chain", 5, 1e-12, 1)
    for rank, r, z in out:
        assert r["iters"] == 5 and r["status"] == -7     # FGA_EBUDGET


def test_a_rank_that_never_takes_part_times_out():
    out = _run_dist("chain", 50, 0.0, 1, vanish=True)
    assert out[1][1] == "left"
    assert out[0][1] == "error" and out[0][2] == -5      # FGA_ETIMEOUT
