"""The allocation-free batched MPC entry point (fga_mpc_solve_noalloc).

It exists for callers that cannot allocate device memory at solve time
(memory arenas they do not own, real-time loops, allocation-free plugins):
its scratch is a static device array inside the library.  The test calls it
through the C-ABI twice in a row on the same inputs and checks both results
against fga_mpc_batch_solve, the allocating entry point, within the FP32
tolerance of the other batched-MPC tests.  The file is collected last so
that a run stopping at the first failure has already run everything else;
it passes alone in a fresh process as well."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _solve_noalloc(lib, d, stream=None, A=None):
    import torch
    n, nx, nu = len(d["T"]), d["nx"], d["nu"]
    T = np.array(d["T"], dtype=np.int32, copy=True)
    dev = lambda a: torch.tensor(np.asarray(a, dtype=np.float32), device="cuda").contiguous()
    A = dev(d["A"][0] if A is None else A)
    B, q, r, x0 = dev(d["B"][0]), dev(d["q"][0]), dev(d["r"][0]), dev(d["x0"])
    Z = int(((nx + nu) * T.astype(np.int64) + nx).sum())
    z = torch.full((Z,), float("nan"), dtype=torch.float32, device="cuda")
    iters = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    status = torch.full((n,), 99, dtype=torch.int32, device="cuda")
    P = ctypes.c_void_p
    lib.fga_mpc_solve_noalloc.restype = ctypes.c_int
    lib.fga_mpc_solve_noalloc.argtypes = [ctypes.c_int32, P, ctypes.c_int32, ctypes.c_int32, P, P, P, P, P,
                                          ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_int64,
                                          ctypes.c_double, ctypes.c_int32, P, P, P, P]
    torch.cuda.synchronize()
    rc = lib.fga_mpc_solve_noalloc(n, T.ctypes.data, nx, nu, A.data_ptr(), B.data_ptr(), q.data_ptr(),
                                   r.data_ptr(), x0.data_ptr(), d["umax"], 1.0, 1.0, 20000, 1e-4, 1,
                                   z.data_ptr(), iters.data_ptr(), status.data_ptr(),
                                   None if stream is None else stream.cuda_stream)
    assert rc == 0, lib.fga_last_error()
    T[:] = 10 ** 6        # the call keeps its own copy of the horizons
    if stream is not None:
        stream.synchronize()
    torch.cuda.synchronize()
    return z.cpu().numpy().astype(np.float64), iters.cpu().numpy(), status.cpu().numpy()


def test_noalloc_matches_allocating_entry_point_twice():
    from paper_1603_02526_gb300 import build, inputs, _lib
    from paper_1603_02526_gb300.mpc import batch_from_inputs
    build.build()
    lib = _lib.load()
    d = inputs.mpc_batch_inputs(96, seed=4700, tmin=10, tmax=50, shared_system=True)
    b = batch_from_inputs(d, "f32")
    b.fga_mpc_batch_solve(20000, tol=1e-4, check_every=1, threads=128, use_graph=False)
    ref = b.fga_mpc_batch_read()
    S = max(1.0, float(np.abs(ref["z"]).max()))
    for _ in range(2):
        z, it, st = _solve_noalloc(lib, d)
        assert np.all(st == 0) and np.array_equal(st, ref["status"])
        assert np.all(np.abs(it - ref["iters"]) <= 1)
        assert np.abs(z - ref["z"]).max() <= 2e-5 * S


def test_noalloc_other_sizes_on_a_side_stream():
    """nx = 6, nu = 3 (the general-size kernel, the projector formed by the
    library's own one-CTA kernel), queued on a non-default stream: z,
    iterations and status as the allocating entry point's, twice."""
    import torch
    from paper_1603_02526_gb300 import build, inputs, _lib
    from paper_1603_02526_gb300.mpc import batch_from_inputs
    build.build()
    lib = _lib.load()
    d = inputs.mpc_batch_inputs(64, seed=4702, nx=6, nu=3, tmin=5, tmax=40, shared_system=True)
    b = batch_from_inputs(d, "f32")
    b.fga_mpc_batch_solve(20000, tol=1e-4, check_every=1, threads=128, use_graph=False)
    ref = b.fga_mpc_batch_read()
    S = max(1.0, float(np.abs(ref["z"]).max()))
    side = torch.cuda.Stream()
    for _ in range(2):
        z, it, st = _solve_noalloc(lib, d, stream=side)
        assert np.array_equal(st, ref["status"])
        assert np.all(np.abs(it - ref["iters"]) <= 1)
        assert np.abs(z - ref["z"]).max() <= 2e-5 * S


def test_noalloc_non_finite_system_is_refused_per_instance():
    """A NaN in A: the projector cannot be formed, and every instance's
    status is FGA_EINVAL (the allocating path refuses such a system at
    creation)."""
    from paper_1603_02526_gb300 import build, inputs, _lib
    build.build()
    lib = _lib.load()
    d = inputs.mpc_batch_inputs(8, seed=4703, tmin=10, tmax=20, shared_system=True)
    A = d["A"][0].copy()
    A[3, 5] = np.nan
    _, _, st = _solve_noalloc(lib, d, A=A)
    assert np.all(st == _lib.FGA_EINVAL)
    # the next call on a good system is unaffected
    _, _, st = _solve_noalloc(lib, d)
    assert np.all(st == 0)


def test_noalloc_rejects_oversized_batch():
    from paper_1603_02526_gb300 import build, inputs, _lib
    build.build()
    lib = _lib.load()
    d = inputs.mpc_batch_inputs(4096, seed=4701, T_fixed=100, shared_system=True)   # ~20 M edges
    import torch
    T = np.ascontiguousarray(d["T"], dtype=np.int32)
    one = torch.zeros(16, device="cuda")
    lib.fga_mpc_solve_noalloc.restype = ctypes.c_int
    P = ctypes.c_void_p
    lib.fga_mpc_solve_noalloc.argtypes = [ctypes.c_int32, P, ctypes.c_int32, ctypes.c_int32, P, P, P, P, P,
                                          ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_int64,
                                          ctypes.c_double, ctypes.c_int32, P, P, P, P]
    p = one.data_ptr()
    rc = lib.fga_mpc_solve_noalloc(4096, T.ctypes.data, 12, 4, p, p, p, p, p, 1.0, 1.0, 1.0, 10, 1e-4, 1,
                                   p, p, p, None)
    assert rc == _lib.FGA_EINVAL
    assert b"scratch" in lib.fga_last_error()
