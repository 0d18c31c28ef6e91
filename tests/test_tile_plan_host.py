"""Host logic of the disk-tile sweep: the planner (csrc/fga_tile.cpp) that
cuts the pair matrix of a circle packing into 32 x 8 units, gives the units
to CTAs, builds each CTA's z table and the list of staged contributions
every variable sums (Sec. V-A's packing graph; the z-update of Algorithm 2).

The planner is compiled on the host with tests/tile_plan_check.cpp, which
builds the same graph as inputs.packing_problem and writes the plan's tables
out.  The checks are the plan's contract with the kernel, each stated from
the graph itself: every disk pair sits in exactly one register slot of one
unit, with its two disks in that CTA's z table; every staged partial of a
unit or a wall / reward is summed by exactly the slot-variable it belongs
to and by no other; every variable's holder count, owner and degree are
right; the CTA tables fit the kernel's shared-memory and 16-bit limits.
No GPU is needed."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1603_02526_gb300", "csrc")
ROWS, COLS = 32, 8
STAGE = 3 * ROWS + 3 * COLS          # staged partials of one unit
SMEM_MAX = 227 * 1024                # shared memory of one CTA
OWNER = np.int32(-2 ** 31)           # the owner flag in a slot-variable's last field


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    nvcc = shutil.which("nvcc")
    if nvcc:
        d = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "include")
        if os.path.exists(os.path.join(d, "cuda_runtime.h")):
            return d
    return None


@pytest.fixture(scope="module")
def planner(tmp_path_factory):
    inc = _cuda_include()
    if shutil.which("g++") is None or inc is None:
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("plan") / "tile_plan_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I", CSRC, "-I", inc,
                    os.path.join(ROOT, "tests", "tile_plan_check.cpp"), os.path.join(CSRC, "fga_tile.cpp"),
                    "-o", exe], check=True)
    return exe


def _run(planner, tmp_path, N, sms=152, wmax=16):
    out = str(tmp_path)
    os.makedirs(out, exist_ok=True)
    subprocess.run([planner, str(N), str(sms), str(wmax), out], check=True)
    meta = {}
    with open(os.path.join(out, "meta.txt")) as fh:
        for line in fh:
            k, v = line.rstrip("\n").split(" ", 1)
            meta[k] = v if k == "why" else int(v)
    if meta["rc"]:
        return meta, None
    rd = lambda name, dt: np.fromfile(os.path.join(out, name), dtype=dt)
    t = dict(pair_pos=rd("pair_pos.i32", np.int32), rowslot=rd("rowslot.u16", np.uint16).astype(np.int64),
             colslot=rd("colslot.u16", np.uint16).astype(np.int64), mask=rd("mask.u8", np.uint8),
             cta=rd("cta.i32", np.int32).reshape(-1, 6).astype(np.int64), sv=rd("sv.i32", np.int32).reshape(-1, 4),
             zden=rd("zden.f32", np.float32), cptr=rd("cptr.i32", np.int32).astype(np.int64),
             clist=rd("clist.i32", np.int32).astype(np.int64), loc=rd("loc.i32", np.int32).reshape(-1, 3),
             loc_member=rd("loc_member.i64", np.int64), loc_type=rd("loc_type.i32", np.int32))
    return meta, t


def _check_plan(N, meta, t, sms, wmax):
    U, W, G = meta["U"], meta["W"], meta["G"]
    cta, sv = t["cta"], t["sv"]
    unit0, nunit, sv0, nsv, loc0, nloc = cta.T
    nslotvar = sv.shape[0]
    # launch shape
    assert G <= sms and G == -(-U // W) and W == -(-U // sms)
    assert meta["warps"] == min(W, wmax)
    assert np.array_equal(unit0, np.arange(G) * W) and nunit.sum() == U and np.all(nunit >= 1)
    assert np.all(nsv % 3 == 0) and np.array_equal(sv0, np.concatenate([[0], np.cumsum(nsv)[:-1]]))
    assert np.array_equal(loc0, np.concatenate([[0], np.cumsum(nloc)[:-1]])) and nloc.sum() == 4 * N
    assert sv0[-1] + nsv[-1] == nslotvar
    assert meta["smem"] <= SMEM_MAX and meta["stgmax"] <= 65535
    assert meta["smax"] == (nsv // 3).max() and meta["svmax"] == nsv.max()

    # every disk pair (i < j, row-major) in exactly one register slot
    i, j = np.triu_indices(N, k=1)
    pos = t["pair_pos"].astype(np.int64)
    assert pos.size == i.size == meta["npairs"]
    assert np.unique(pos).size == pos.size and pos.min() >= 0 and pos.max() < 256 * U
    unit, slot, lane = pos // 256, (pos // 32) % 8, pos % 32
    col = slot ^ ((lane >> 2) & 7)
    assert np.array_equal(lane, i % ROWS) and np.array_equal(col, j % COLS)
    mask = t["mask"].reshape(U, ROWS)
    assert np.all((mask[unit, lane] >> slot) & 1)
    bits = np.unpackbits(mask[..., None], axis=-1, bitorder="little")      # (U, 32, 8): bit j of lane l
    assert bits.sum() == pos.size                                           # no empty slot marked
    g = unit // W
    rows = t["rowslot"].reshape(U, ROWS)
    cols = t["colslot"].reshape(U, COLS)
    rsv = sv0[g] + 3 * rows[unit, lane]
    csv = sv0[g] + 3 * cols[unit, col]
    for q in range(3):
        assert np.array_equal(sv[rsv + q, 0], 3 * i + q)
        assert np.array_equal(sv[csv + q, 0], 3 * j + q)

    # staged partials: (CTA, staging position) -> the slot-variable that sums it
    idx = (np.arange(COLS)[None, :] ^ ((np.arange(ROWS)[:, None] >> 2) & 7))    # lane l, column c -> slot
    used_col = bits[:, np.arange(ROWS)[:, None], idx].any(axis=1)                # (U, 8)
    used_row = mask != 0                                                         # (U, 32)
    ug = np.arange(U) // W
    uw = np.arange(U) - unit0[ug]
    keys, owners = [], []
    r_u, r_l = np.nonzero(used_row)
    c_u, c_c = np.nonzero(used_col)
    for q in range(3):
        keys.append(ug[r_u] * 2 ** 17 + uw[r_u] * STAGE + q * ROWS + r_l)
        owners.append(sv0[ug[r_u]] + 3 * rows[r_u, r_l] + q)
        keys.append(ug[c_u] * 2 ** 17 + uw[c_u] * STAGE + 3 * ROWS + q * COLS + c_c)
        owners.append(sv0[ug[c_u]] + 3 * cols[c_u, c_c] + q)
    loc = t["loc"].astype(np.int64)
    lg = np.repeat(np.arange(G), nloc)
    ltype, lslot, lstg = loc.T
    wall = ltype == 1
    assert np.all((ltype == 1) | (ltype == 2))
    for q in range(3):
        keys.append(lg[wall] * 2 ** 17 + lstg[wall] + q)
        owners.append(sv0[lg[wall]] + 3 * lslot[wall] + q)
    keys.append(lg[~wall] * 2 ** 17 + lstg[~wall])
    owners.append(sv0[lg[~wall]] + 3 * lslot[~wall] + 2)
    keys, owners = np.concatenate(keys), np.concatenate(owners)
    cptr, clist = t["cptr"], t["clist"]
    assert cptr.size == nslotvar + 1 and cptr[0] == 0 and cptr[-1] == clist.size and np.all(np.diff(cptr) >= 0)
    cnt = np.diff(cptr)
    svi = np.repeat(np.arange(nslotvar), cnt)
    sg = np.searchsorted(sv0, svi, side="right") - 1
    akeys = sg * 2 ** 17 + clist
    assert np.unique(akeys).size == akeys.size                              # each partial summed once
    o1, o2 = np.argsort(keys), np.argsort(akeys)
    assert np.array_equal(keys[o1], akeys[o2])                               # and every one of them
    assert np.array_equal(owners[o1], svi[o2])                               # by its own variable
    # the locals' staging ranges follow the units' and do not overlap
    assert np.all(lstg >= nunit[lg] * STAGE)

    # walls and rewards: each once, at a slot holding its own disk
    wall_disk = t["loc_member"][wall] // 3
    rew_disk = t["loc_member"][~wall]
    assert np.array_equal(np.sort(t["loc_member"][wall]), np.arange(3 * N))
    assert np.array_equal(np.sort(rew_disk), np.arange(N))
    assert np.array_equal(sv[sv0[lg[wall]] + 3 * lslot[wall], 0], 3 * wall_disk)
    assert np.array_equal(sv[sv0[lg[~wall]] + 3 * lslot[~wall] + 2, 0], 3 * rew_disk + 2)
    assert np.array_equal(t["loc_type"], ltype)

    # variables: holders, one owner each, degrees
    v = sv[:, 0].astype(np.int64)
    holders = np.bincount(v, minlength=3 * N)
    assert np.all(holders >= 1) and holders.max() <= 255
    assert np.array_equal(sv[:, 1], holders[v])
    assert np.array_equal(np.bincount(v[sv[:, 3] == OWNER], minlength=3 * N), np.ones(3 * N, np.int64))
    assert np.all((sv[:, 3] == OWNER) | (sv[:, 3] == 0))
    deg = np.where(v % 3 == 2, N + 3, N + 2)
    assert np.array_equal(t["zden"], deg.astype(np.float32))
    for gg in range(G):                                                     # one slot per disk per CTA
        vv = v[sv0[gg]: sv0[gg] + nsv[gg]]
        assert np.unique(vv).size == vv.size


@pytest.mark.parametrize("N", [2, 5, 20, 33, 200, 1000, 2000, 3000])
def test_plan_contract(planner, tmp_path, N):
    meta, t = _run(planner, tmp_path, N)
    assert meta["rc"] == 0, meta["why"]
    _check_plan(N, meta, t, 152, 16)
    if N == 1000:
        assert (meta["U"], meta["W"], meta["warps"]) == (2016, 14, 14)   # one unit per warp
    if N >= 2000:
        assert meta["W"] > 16 and meta["warps"] == 16                    # several units per warp


def test_plan_with_fewer_warps_is_the_same_plan(planner, tmp_path):
    """A smaller block (FGA_OPT_BLOCK) changes only how many warps share the
    units, not the units, their CTAs or the tables."""
    a_meta, a = _run(planner, tmp_path / "a", 1000)
    b_meta, b = _run(planner, tmp_path / "b", 1000, wmax=2)
    _check_plan(1000, b_meta, b, 152, 2)
    assert b_meta["warps"] == 2
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_plan_refusals(planner, tmp_path):
    meta, _ = _run(planner, tmp_path, 1)
    assert meta["rc"] == 1 and "no disk pairs" in meta["why"]
    meta, _ = _run(planner, tmp_path, 20, sms=0)
    assert meta["rc"] == 1 and "launch shape" in meta["why"]
