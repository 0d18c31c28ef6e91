"""Learned warm start for batched MPC: data generation with the batch
solver, training of the BF16 MLP, and the cold-vs-warm evaluation with cold
fallback.  Argument marshalling and orchestration only: solves, target
extraction, training, inference and the warm-start map all run in
libfgadmm's kernels; torch holds the device buffers.

The network maps x0 (12 values) to 960 values per instance: for each of the
30 steps, (x_{t+1}, u_t) and (lambda_t, mu_t), the multipliers of the
dynamics and of the input box.  The warm start sets z from the trajectory
and every edge's u from the fixed-point relation of Algorithm 2
(u = -(1/rho) times the factor's (sub)gradient), so plain ADMM then iterates
to the same tolerance from a point near its fixed point.
"""
import time

import numpy as np

from . import inputs
from .mlp import MLP
from .mpc import MpcBatch


def _batch(d, precision="f32"):
    b = MpcBatch(d["T"], d["A"], d["B"], d["q"], d["r"], umax=d["umax"], precision=precision)
    b.fga_mpc_batch_set_x0(d["x0"])
    b.fga_mpc_batch_init()
    return b


def generate(n, x0_seed, system_seed=5000, T=30, tol=1e-5, max_iters=20000):
    """Solves n instances of the fixed system to `tol` and returns device
    tensors X (n x 12, FP32) and targets (n x 960, FP32) of the converged
    instances, plus solve statistics."""
    import torch
    d = inputs.mpc_warmstart_inputs(n, system_seed=system_seed, x0_seed=x0_seed, T=T)
    b = _batch(d)
    res = b.fga_mpc_batch_solve(max_iters, tol=tol, check_every=5)
    ld = 2 * (d["nx"] + d["nu"]) * T
    tgt = torch.empty((n, ld), dtype=torch.float32, device="cuda")
    b.fga_mpc_batch_targets(tgt, ld)
    st = b.fga_mpc_batch_read()["status"]
    x0 = d["x0"]
    if np.any(st != 0):
        # drop the instances that missed the tolerance (host-side filtering)
        keep = np.nonzero(st == 0)[0]
        tgt = torch.tensor(tgt.cpu().numpy()[keep], device="cuda")
        x0 = x0[keep]
    X = torch.tensor(x0, dtype=torch.float32, device="cuda")
    return X, tgt, res


def train(X, Y, epochs=30, batch=1024, lr=1e-3, seed=5002, log=None):
    """Trains the 12 -> 256 -> 256 -> 960 MLP on (X, Y); Y is standardised
    in place (the network de-standardises its output)."""
    net = MLP(X.shape[1], 256, 256, Y.shape[1], max_batch=max(16384, batch), seed=seed)
    net.fga_mlp_fit_normalization(Y)
    n = (X.shape[0] // batch) * batch
    losses = []
    steps = 0
    for ep in range(epochs):
        lr_ep = lr * 0.5 * (1 + np.cos(np.pi * ep / epochs))
        for s in range(0, n, batch):
            want = (s == 0)
            lval = net.fga_mlp_train_step(X[s:s + batch], Y[s:s + batch], lr_ep, want_loss=want)
            steps += 1
            if want:
                losses.append(lval)
                if log:
                    log("epoch %d loss %.4e" % (ep, lval))
    return net, dict(losses=losses, steps=steps)


def evaluate(net, n_eval=16384, x0_seed=5003, system_seed=5000, T=30, tol=1e-4, max_iters=20000,
             budget=None, calib=1024):
    """Cold vs warm batched solves of n_eval fresh instances.  Warm: network
    inference, warm-start map, solve with an iteration budget (default: the
    99th percentile of cold iterations on a calibration set), then every
    instance that missed the budget re-solved from cold; all of it timed.
    Both timed arms run in the configuration the autotuner picks on the
    calibration set (CTA size, check interval), each after one untimed
    warm-up solve (CUDA-graph capture), and end with the per-instance
    counters on the host; iteration statistics are given both at that check
    interval (the timed runs) and exactly (untimed runs checking every
    iteration).  The solutions (z, u) are read afterwards."""
    import torch
    dc = inputs.mpc_warmstart_inputs(calib, system_seed=system_seed, x0_seed=x0_seed + 100, T=T)
    bc = _batch(dc)
    if budget is None:
        bc.fga_mpc_batch_solve(max_iters, tol=tol, check_every=1, use_graph=False)
        budget = int(np.percentile(bc.fga_mpc_batch_read(state=False)["iters"], 99))
        bc.fga_mpc_batch_init()
    th, ce = bc.fga_mpc_batch_autotune(max_iters, tol)
    d = inputs.mpc_warmstart_inputs(n_eval, system_seed=system_seed, x0_seed=x0_seed, T=T)
    ld = 2 * (d["nx"] + d["nu"]) * T
    X = torch.tensor(d["x0"], dtype=torch.float32, device="cuda")
    pred = torch.empty((n_eval, ld), dtype=torch.float32, device="cuda")

    def fallback(status, check_every, use_graph):
        miss = np.nonzero(status != 0)[0]
        it = np.zeros(n_eval, dtype=np.int64)
        if miss.size:
            dm = dict(d, x0=d["x0"][miss], T=d["T"][miss])
            bm = _batch(dm)
            bm.fga_mpc_batch_solve(max_iters, tol=tol, check_every=check_every, threads=th, use_graph=use_graph)
            it[miss] = bm.fga_mpc_batch_read(state=False)["iters"]
        return miss, it

    # exact iteration counts (untimed; residuals checked every iteration)
    be = _batch(d)
    be.fga_mpc_batch_solve(max_iters, tol=tol, check_every=1, threads=th, use_graph=False)
    it_cold_exact = be.fga_mpc_batch_read(state=False)["iters"]
    be.fga_mpc_batch_init()
    net.fga_mlp_forward(X, pred)
    be.fga_mpc_batch_warm_start(pred, ld)
    be.fga_mpc_batch_solve(budget, tol=tol, check_every=1, threads=th, use_graph=False)
    we = be.fga_mpc_batch_read(state=False)
    it_warm_exact = we["iters"] + fallback(we["status"], 1, False)[1]
    del be
    # cold, timed
    bcold = _batch(d)
    bcold.fga_mpc_batch_solve(max_iters, tol=tol, check_every=ce, threads=th)   # warm-up: graph capture
    bcold.fga_mpc_batch_init()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc = bcold.fga_mpc_batch_solve(max_iters, tol=tol, check_every=ce, threads=th)
    cold = bcold.fga_mpc_batch_read(state=False)
    t_cold = time.perf_counter() - t0
    cold["z"] = bcold.fga_mpc_batch_read()["z"]
    # warm, timed
    bwarm = _batch(d)
    bwarm.fga_mpc_batch_solve(budget, tol=tol, check_every=ce, threads=th)      # warm-up: graph capture
    bwarm.fga_mpc_batch_init()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    net.fga_mlp_forward(X, pred)
    bwarm.fga_mpc_batch_warm_start(pred, ld)
    rw = bwarm.fga_mpc_batch_solve(budget, tol=tol, check_every=ce, threads=th)
    warm = bwarm.fga_mpc_batch_read(state=False)
    miss, fb_iters = fallback(warm["status"], ce, False)
    torch.cuda.synchronize()
    t_warm = time.perf_counter() - t0
    warm["z"] = bwarm.fga_mpc_batch_read()["z"]
    it_cold = cold["iters"]
    it_warm = warm["iters"] + fb_iters
    # the warm solutions are the cold ones (same optimum, same tolerance)
    dz = np.abs(warm["z"] - cold["z"]).max() if miss.size == 0 else None

    def stats(it):
        return dict(iters_mean=float(it.mean()), iters_p50=float(np.percentile(it, 50)),
                    iters_p99=float(np.percentile(it, 99)))

    return dict(n=n_eval, budget=budget, misses=int(miss.size), threads=th, check_every=ce,
                cold=dict(solves_per_s=n_eval / t_cold, s=t_cold, device_ms=rc["ms"],
                          converged=int((cold["status"] == 0).sum()), at_check_interval=stats(it_cold),
                          **stats(it_cold_exact)),
                warm=dict(solves_per_s=n_eval / t_warm, s=t_warm, device_ms_solve=rw["ms"],
                          at_check_interval=stats(it_warm), **stats(it_warm_exact)),
                max_abs_dz_warm_vs_cold=None if dz is None else float(dz))
