"""FP32 emulation of Algorithm 2 on circle-packing graphs (test checker).

A plain NumPy restatement, in single precision, of the iteration of Sec. II
(x = Prox(n) per factor, m = x + u, z = sum rho m / sum rho, u += alpha (x - z),
n = z - u) with the Appendix A operators as the FP64 oracle reads them (the
no-collision operator with the radii moved down, walls with unit inward
normals, the linear radius reward x = n + w / rho, the area reward
x = rho n / (rho - 1) written as n + n / (rho - 1)).  Every value is rounded
to FP32 after each operation (NumPy float32 arithmetic); z sums each
variable's terms one by one in creation order in FP32.  Uniform rho and
alpha only.

It exists to measure what FP32 rounding alone does to the iterates of a
graph -- its distance from the FP64 oracle is the yardstick for the GPU's
FP32 message tolerances.  It is not the oracle and the library never uses
it."""
import numpy as np

from paper_1603_02526_gb300 import inputs

f32 = np.float32


class PackingFP32:
    """State of one packing problem (inputs.packing_problem) in FP32."""

    def __init__(self, p, sums="serial"):
        if sums not in ("serial", "tree", "exact"):
            raise ValueError(sums)
        self.sums = sums
        blocks = {b.ftype: b for b in p.factor_blocks}
        pair = blocks.get(inputs.PACK_PAIR)
        wall = blocks[inputs.PACK_WALL]
        self.area = inputs.PACK_RADIUS_QUAD in blocks
        rew = blocks[inputs.PACK_RADIUS_QUAD if self.area else inputs.PACK_RADIUS_LIN]
        if len(p.factor_blocks) != (3 if pair is not None else 2):
            raise ValueError("packing graphs only (pairs, walls, one kind of radius reward)")
        self.rho = f32(p.rho)
        self.alpha = f32(p.alpha)
        dims = p.var_dims()
        first = np.concatenate([[0], np.cumsum(dims)[:-1]])
        # scalar variable of each edge, creation order
        svar = []
        self.npair = 0 if pair is None else pair.var_ids.shape[0]
        if pair is not None:
            v = pair.var_ids
            cols = [first[v[:, 0]], first[v[:, 0]] + 1, first[v[:, 1]], first[v[:, 2]], first[v[:, 2]] + 1,
                    first[v[:, 3]]]
            svar.append(np.stack(cols, 1).ravel())
        v = wall.var_ids
        svar.append(np.stack([first[v[:, 0]], first[v[:, 0]] + 1, first[v[:, 1]]], 1).ravel())
        svar.append(first[rew.var_ids[:, 0]])
        self.svar = np.concatenate(svar).astype(np.int64)
        self.E = self.svar.size
        self.nz = int(dims.sum())
        self.nwall = wall.var_ids.shape[0]
        self.wQ = wall.params[:, 0:2].astype(f32)
        self.wV = wall.params[:, 2:4].astype(f32)
        self.w = None if self.area else rew.params[:, 0].astype(f32)
        self.e_wall = 6 * self.npair
        self.e_rew = self.e_wall + 3 * self.nwall
        self.z = p.z0.astype(f32)
        self.u = np.zeros(self.E, f32)
        self.n = self.z[self.svar] - self.u
        self.x = np.zeros(self.E, f32)
        self.m = np.zeros(self.E, f32)
        # creation-ordered edges of each variable (stable sort keeps the
        # order), as a padded variable x position table: column j holds the
        # j-th edge of every variable (-1 past a row's end)
        order = np.argsort(self.svar, kind="stable")
        deg = np.bincount(self.svar, minlength=self.nz)
        rowp = np.concatenate([[0], np.cumsum(deg)])
        self.slots = np.full((self.nz, max(1, int(deg.max()))), -1, np.int64)
        col = np.arange(self.E) - rowp[self.svar[order]]
        self.slots[self.svar[order], col] = order
        self.has_edges = deg > 0

    def _prox(self):
        n, x = self.n, self.x
        if self.npair:
            q = n[:self.e_wall].reshape(-1, 6)
            dx = q[:, 3] - q[:, 0]
            dy = q[:, 4] - q[:, 1]
            d = np.sqrt(dx * dx + dy * dy)
            D = np.maximum(f32(0), q[:, 2] + q[:, 5] - d)
            act = D > 0
            safe = np.where(d > 0, d, f32(1))
            hx = np.where(d > 0, dx / safe, f32(1))
            hy = np.where(d > 0, dy / safe, f32(0))
            t = D * f32(0.25)           # one rho: each of the four blocks takes D / 4
            o = q.copy()
            o[:, 0] = q[:, 0] - t * hx
            o[:, 1] = q[:, 1] - t * hy
            o[:, 2] = q[:, 2] - t
            o[:, 3] = q[:, 3] + t * hx
            o[:, 4] = q[:, 4] + t * hy
            o[:, 5] = q[:, 5] - t
            x[:self.e_wall] = np.where(act[:, None], o, q).ravel()
        q = n[self.e_wall:self.e_rew].reshape(-1, 3)
        qx, qy = self.wQ[:, 0], self.wQ[:, 1]
        h = qx * (q[:, 0] - self.wV[:, 0]) + qy * (q[:, 1] - self.wV[:, 1]) - q[:, 2]
        lam = np.where(h < 0, -h * f32(0.5), f32(0))   # one rho, |Q| = 1
        o = np.stack([q[:, 0] + lam * qx, q[:, 1] + lam * qy, q[:, 2] - lam], 1)
        x[self.e_wall:self.e_rew] = o.ravel()
        if self.area:
            q = n[self.e_rew:]
            x[self.e_rew:] = q + q * f32(1.0 / (float(self.rho) - 1.0))
        else:
            x[self.e_rew:] = n[self.e_rew:] + self.w / self.rho

    def iterate(self, k=1):
        for _ in range(k):
            self._prox()
            self.m = self.x + self.u
            rm = np.append(self.rho * self.m, f32(0))      # index -1: a zero
            rr = np.append(np.full(self.E, self.rho, f32), f32(0))
            if self.sums == "exact":
                # each sum of FP32 terms exact, rounded once to FP32
                S = rm[self.slots].astype(np.float64).sum(1).astype(f32)
                R = rr[self.slots].astype(np.float64).sum(1).astype(f32)
            elif self.sums == "tree":
                # FP32 pairwise sums of each row (NumPy's reduction)
                S = rm[self.slots].sum(1, dtype=f32)
                R = rr[self.slots].sum(1, dtype=f32)
            else:
                S = np.zeros(self.nz, f32)
                R = np.zeros(self.nz, f32)
                for j in range(self.slots.shape[1]):          # one term per variable at a time
                    S = S + rm[self.slots[:, j]]
                    R = R + rr[self.slots[:, j]]
            self.z = np.where(self.has_edges, S / np.where(self.has_edges, R, f32(1)), self.z)
            zb = self.z[self.svar]
            self.u = self.u + self.alpha * (self.x - zb)
            self.n = zb - self.u
