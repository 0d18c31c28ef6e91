"""Shards: one factor graph split across GPUs, one process per GPU.

The paper names multi-GPU execution as future work (Sec. VI).  In
Algorithm 2 the only step that couples factors is the z-update, through the
per-variable sums S_b = sum rho m and R_b = sum rho over the variable's edges
(Sec. II).  So the factors are cut into contiguous slices in creation order,
one per rank; every rank holds all variables, runs the x-, m-, u- and
n-updates of its own factors, and the ranks exchange only the sums (the
fga_shard_* calls of include/fgadmm.h; this module is their binding and the
exchange protocol around them -- every update runs in the library's
kernels).

Two exchanges:
  * "chain" (canonical z-order): rank r adds its terms one by one onto rank
    r-1's running sums and passes them on; the last rank's sums are the
    serial creation-order sums of the whole graph, bit for bit, and are
    broadcast.  FP64 shards therefore reproduce the one-GPU canonical run
    and the serial oracle exactly.
  * "gather" (any z-order): every rank sums its own terms, the sums are
    all-gathered and added in rank order on the device.

Transports: `LocalGroup` runs the shards of one process one after another
(several shards on one GPU; nothing waits on anything else), `DistGroup`
runs one shard per process over torch.distributed (NCCL on GPUs, gloo on
CPU), with a time limit on every exchange.
"""
import ctypes
import datetime

import numpy as np

from . import _lib
from ._lib import check
from .inputs import FactorBlock, Problem


# ---------------------------------------------------------------------------
# partition
# ---------------------------------------------------------------------------
def split_problem(problem, n_shards):
    """Cuts the factors of `problem` (creation order) into `n_shards`
    contiguous slices with about equal numbers of scalar edges.  Every slice
    keeps all variables, the start point and rho/alpha.  Returns the list
    of shard problems and each shard's first edge in the whole graph."""
    if n_shards < 1:
        raise ValueError("n_shards must be >= 1")
    dims = problem.var_dims()
    per_factor = []                       # (block index, row, edges)
    for bi, blk in enumerate(problem.factor_blocks):
        arity = int(dims[blk.var_ids].sum(axis=1)[0]) if blk.var_ids.size else 0
        per_factor.append((bi, blk.var_ids.shape[0], arity))
    total = sum(n * a for _, n, a in per_factor)
    # cut points in edges -> (block, row) boundaries
    cuts = [round(total * k / n_shards) for k in range(n_shards + 1)]
    shards = [Problem(problem.name + "_shard%d" % r, rho=problem.rho, alpha=problem.alpha,
                      meta=dict(problem.meta)) for r in range(n_shards)]
    for s in shards:
        s.var_blocks = list(problem.var_blocks)
        s.z0 = problem.z0
    first_edge = [0] * n_shards
    e = 0
    r = 0
    for bi, n, a in per_factor:
        blk = problem.factor_blocks[bi]
        row = 0
        while row < n:
            while r < n_shards - 1 and e >= cuts[r + 1]:
                r += 1
                first_edge[r] = e
            # rows of this block that fit before the next cut
            room = n - row if r == n_shards - 1 else max(1, -(-(cuts[r + 1] - e) // max(a, 1)))
            take = min(n - row, room)
            prm = blk.params[row:row + take] if blk.params.size else np.zeros((take, 0))
            shards[r].factor_blocks.append(FactorBlock(blk.ftype, blk.var_ids[row:row + take], prm))
            row += take
            e += take * a
    for k in range(r + 1, n_shards):
        first_edge[k] = e
    if any(not s.factor_blocks for s in shards):
        raise ValueError("more shards than factors")
    return shards, first_edge


# ---------------------------------------------------------------------------
# one shard's graph (binding of fga_shard_*)
# ---------------------------------------------------------------------------
def _declare(lib):
    P = ctypes.c_void_p
    i32, i64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    pdbl = ctypes.POINTER(ctypes.c_double)
    for name, args in {"fga_shard_rho_chain": [P, P, P, P, P], "fga_shard_begin": [P, P, P],
                       "fga_shard_xstep": [P, i32, P, P, P], "fga_shard_add_parts": [P, P, i32, P],
                       "fga_shard_zstep": [P, P, i32, P], "fga_shard_finish": [P, P],
                       "fga_shard_stop_rule": [P, i32, dbl, i64, dbl, dbl, pdbl, pdbl,
                                               ctypes.POINTER(ctypes.c_int32)]}.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int


def _vp(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return ctypes.c_void_p(a.ctypes.data)


class ShardGraph:
    """One rank's slice of the graph on its GPU: a FactorGraph in shard mode
    with device buffers for the exchanged sums (torch tensors)."""

    def __init__(self, shard_problem, precision="f64", zorder=0, device=0, stream=None):
        import torch
        from .graph import graph_from_problem
        self.lib = _lib.load()
        _declare(self.lib)
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        opts = {_lib.FGA_OPT_ZORDER: zorder, _lib.FGA_OPT_STORE_M: 1}
        self.g = graph_from_problem(shard_problem, precision, device=device, stream=self.stream, options=opts,
                                    init=False)
        self.z0 = shard_problem.z0
        self.nz = self.g.num_scalar_vars
        self.ne = self.g.num_edges
        self.dtype = torch.float32 if precision == "f32" else torch.float64
        dev = torch.device("cuda", device)
        self.s_out = torch.empty(self.nz, dtype=self.dtype, device=dev)
        self.total = torch.empty(self.nz, dtype=self.dtype, device=dev)
        self.pri = torch.zeros(1, dtype=torch.float64, device=dev)
        self.dual = torch.zeros(1, dtype=torch.float64, device=dev)

    def new_sums(self, n=1):
        import torch
        return torch.empty((n, self.nz), dtype=self.dtype, device=torch.device("cuda", self.device))

    def rho_chain(self, srho_in, srho2_in):
        out, out2 = np.empty(self.nz), np.empty(self.nz)
        check(self.lib.fga_shard_rho_chain(self.g._g, _vp(srho_in), _vp(srho2_in), _vp(out), _vp(out2)),
              "fga_shard_rho_chain")
        return out, out2

    def begin(self, srho, srho2):
        srho = np.ascontiguousarray(srho, dtype=np.float64)
        srho2 = np.ascontiguousarray(srho2, dtype=np.float64)
        check(self.lib.fga_shard_begin(self.g._g, _vp(srho), _vp(srho2)), "fga_shard_begin")

    def init(self, z0=None):
        self.g.fga_init(self.z0 if z0 is None else z0)

    def xstep(self, check_prev, s_in, s_out):
        check(self.lib.fga_shard_xstep(self.g._g, 1 if check_prev else 0, _vp(s_in), _vp(s_out),
                                       _vp(self.pri) if check_prev else None), "fga_shard_xstep")
        return self.pri if check_prev else None

    def add_parts(self, parts, total):
        check(self.lib.fga_shard_add_parts(self.g._g, _vp(parts), int(parts.shape[0]), _vp(total)),
              "fga_shard_add_parts")

    def zstep(self, total, check_):
        check(self.lib.fga_shard_zstep(self.g._g, _vp(total), 1 if check_ else 0, _vp(self.dual) if check_
                                       else None), "fga_shard_zstep")
        return self.dual if check_ else None

    def finish(self):
        check(self.lib.fga_shard_finish(self.g._g, _vp(self.pri)), "fga_shard_finish")
        return self.pri

    def sync(self):
        self.stream.synchronize()

    def read_z(self):
        return self.g.fga_read_z()

    def read_edges(self, which):
        return self.g.fga_read_edge_state(which)


def stop_rule(pri_parts, dual, num_edges, tol_pri, tol_dual):
    """fga_shard_stop_rule on host values (rank-ordered primal partial sums,
    the graph-wide dual sum)."""
    lib = _lib.load()
    _declare(lib)
    p = np.ascontiguousarray(pri_parts, dtype=np.float64)
    rp, rd, st = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
    check(lib.fga_shard_stop_rule(_vp(p), int(p.size), float(dual), int(num_edges), float(tol_pri),
                                  float(tol_dual), ctypes.byref(rp), ctypes.byref(rd), ctypes.byref(st)),
          "fga_shard_stop_rule")
    return rp.value, rd.value, bool(st.value)


# ---------------------------------------------------------------------------
# transports
# ---------------------------------------------------------------------------
class LocalGroup:
    """All shards in this process, run one after another (several shards on
    one GPU).  Every exchange is a hand-over in rank order."""

    def __init__(self, shards):
        self.shards = list(shards)

    def each(self):
        return list(enumerate(self.shards))

    def rho_chain(self):
        a = b = None
        for s in self.shards:
            a, b = s.rho_chain(a, b)
        return a, b

    def chain_sums(self, check_prev):
        """x-steps in rank order, each adding onto the previous rank's sums;
        returns the graph-wide sums (on the last shard) and the primal
        partials (one per rank, host floats) when check_prev."""
        s_in, pri = None, []
        for s in self.shards:
            p = s.xstep(check_prev, s_in, s.s_out)
            if check_prev:
                pri.append(p)
            s_in = s.s_out
        total = s_in
        for s in self.shards:
            s.total.copy_(total)
        return [float(p.item()) for p in pri] if check_prev else None

    def gather_sums(self, check_prev):
        parts = self.shards[0].new_sums(len(self.shards))
        pri = []
        for r, s in enumerate(self.shards):
            p = s.xstep(check_prev, None, parts[r])
            if check_prev:
                pri.append(p)
        for s in self.shards:
            s.add_parts(parts, s.total)
        return [float(p.item()) for p in pri] if check_prev else None

    def zsteps(self, check_):
        duals = [s.zstep(s.total, check_) for s in self.shards]
        return float(duals[0].item()) if check_ else None

    def finish(self):
        return [float(s.finish().item()) for s in self.shards]


class DistGroup:
    """One shard per process over torch.distributed.  `timeout_s` bounds
    every exchange: a rank that does not take part makes the others' next
    exchange fail with a timeout (FgaError FGA_ETIMEOUT) instead of waiting
    for ever."""

    def __init__(self, shard, timeout_s=60.0):
        import torch.distributed as dist
        self.dist = dist
        self.shard = shard
        self.rank = dist.get_rank()
        self.world = dist.get_world_size()
        self.timeout = datetime.timedelta(seconds=timeout_s)
        self.shards = [shard]

    def each(self):
        return [(self.rank, self.shard)]

    def _guard(self, fn, what):
        try:
            return fn()
        except Exception as e:   # a collective that ran out of time or lost its peer
            raise _lib.FgaError(_lib.FGA_ETIMEOUT, "shard exchange (%s)" % what, str(e)) from e

    def _wait(self, work, what):
        self._guard(lambda: work.wait(self.timeout), what)

    def rho_chain(self):
        """R and sum rho^2 through the ranks in rank order (host arrays, sent
        as FP64 tensors on the shard's transport device)."""
        import torch
        dev = self._dev()
        a = b = None
        buf = torch.empty((2, self.shard.nz), dtype=torch.float64, device=dev)
        if self.rank > 0:
            self._wait(self.dist.irecv(buf, self.rank - 1), "rho chain recv")
            h = buf.cpu().numpy()
            a, b = h[0].copy(), h[1].copy()
        a, b = self.shard.rho_chain(a, b)
        if self.rank < self.world - 1:
            out = torch.from_numpy(np.stack([a, b])).to(dev)
            self._wait(self.dist.isend(out, self.rank + 1), "rho chain send")
        res = torch.from_numpy(np.stack([a, b])).to(dev)
        self._wait(self.dist.broadcast(res, self.world - 1, async_op=True), "rho broadcast")
        h = res.cpu().numpy()
        return h[0].copy(), h[1].copy()

    def _dev(self):
        import torch
        return self.shard.s_out.device if self.dist.get_backend() == "nccl" else torch.device("cpu")

    def _to(self, t):
        return t if t.device == self._dev() else t.to(self._dev())

    def _gather_scalar(self, p):
        import torch
        mine = self._to(p.reshape(1).to(torch.float64))
        allv = torch.empty(self.world, dtype=torch.float64, device=mine.device)
        self._wait(self.dist.all_gather_into_tensor(allv, mine, async_op=True), "residual gather")
        return [float(v) for v in allv.cpu()]

    def chain_sums(self, check_prev):
        s = self.shard
        s_in = None
        if self.rank > 0:
            buf = self._to(s.new_sums(1)[0])
            self._wait(self.dist.irecv(buf, self.rank - 1), "chain recv")
            s_in = buf if buf.device == s.s_out.device else buf.to(s.s_out.device)
        p = s.xstep(check_prev, s_in, s.s_out)
        if self.rank < self.world - 1:
            s.sync()
            self._wait(self.dist.isend(self._to(s.s_out), self.rank + 1), "chain send")
        tot = self._to(s.s_out.clone())
        s.sync()
        self._wait(self.dist.broadcast(tot, self.world - 1, async_op=True), "sums broadcast")
        s.total.copy_(tot)
        return self._gather_scalar(p) if check_prev else None

    def gather_sums(self, check_prev):
        import torch
        s = self.shard
        p = s.xstep(check_prev, None, s.s_out)
        s.sync()
        parts = torch.empty(self.world * s.nz, dtype=s.s_out.dtype, device=self._dev())
        self._wait(self.dist.all_gather_into_tensor(parts, self._to(s.s_out), async_op=True), "sums gather")
        s.add_parts(parts.view(self.world, s.nz).to(s.s_out.device), s.total)
        return self._gather_scalar(p) if check_prev else None

    def zsteps(self, check_):
        d = self.shard.zstep(self.shard.total, check_)
        return float(d.item()) if check_ else None

    def finish(self):
        return self._gather_scalar(self.shard.finish())


# ---------------------------------------------------------------------------
# the sharded run (the protocol of fga_iterate, spread over the ranks)
# ---------------------------------------------------------------------------
class ShardedSweep:
    """Algorithm 2 over the shards of `group` (LocalGroup or DistGroup);
    `exchange` is "chain" (canonical order: bit-exact with the one-GPU run)
    or "gather"."""

    def __init__(self, group, num_edges, exchange="chain"):
        if exchange not in ("chain", "gather"):
            raise ValueError(exchange)
        self.group = group
        self.E = int(num_edges)
        self.exchange = exchange
        srho, srho2 = group.rho_chain()
        for _, s in group.each():
            s.begin(srho, srho2)
        self.iters_done = 0

    def init(self):
        for _, s in self.group.each():
            s.init()
        self.iters_done = 0

    def iterate(self, max_iters, tol_pri=0.0, tol_dual=0.0, check_every=1):
        """Runs up to max_iters iterations with the stop rule of fga_iterate
        (first checked iteration whose RMS residuals meet both tolerances;
        checks every check_every-th iteration and at the last one).  Returns
        dict(iters, r_pri, r_dual, status)."""
        g = self.group
        sums = g.chain_sums if self.exchange == "chain" else g.gather_sums
        it, dual, pending = 0, None, False
        while it < max_iters:
            pri = sums(pending)
            if pending:
                rp, rd, stop = stop_rule(pri, dual, self.E, tol_pri, tol_dual)
                if stop:
                    return self._result(it, rp, rd, budget=False)
            it += 1
            self.iters_done += 1
            chk = (self.iters_done % check_every == 0) or it == max_iters
            dual = g.zsteps(chk)
            pending = chk
        if max_iters <= 0:
            return dict(iters=0, r_pri=float("nan"), r_dual=float("nan"), status=_lib.FGA_OK)
        pri = g.finish()
        rp, rd, _ = stop_rule(pri, dual, self.E, tol_pri, tol_dual)
        met = rp <= tol_pri and rd <= tol_dual
        return self._result(it, rp, rd, budget=(tol_pri > 0 or tol_dual > 0) and not met)

    def _result(self, it, rp, rd, budget):
        for _, s in self.group.each():
            s.sync()
        st = _lib.FGA_OK
        if not (np.isfinite(rp) and np.isfinite(rd)):
            st = _lib.FGA_ENONFINITE
        elif budget:
            st = _lib.FGA_EBUDGET
        return dict(iters=it, r_pri=rp, r_dual=rd, status=st)
