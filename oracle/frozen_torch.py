"""Plain PyTorch (CPU, float64) restatement of one SSP-RK3 step of GP-MOOD
with the per-stage GP radii and the time step held fixed, for reference
gradients through autograd.

TEST INFRASTRUCTURE ONLY (the oracle side): it takes the GP prediction
vectors from the C oracle and shares nothing with the CUDA path.  Its forward
is pinned to the C oracle's step; its gradient to finite differences.

Definitions (same as the C oracle): ghost fill (periodic / outflow /
reflect / Dirichlet), EDP1 face radii min(r_L, r_R) with periodic ghosts
carrying the radius of the cell they copy and other ghosts the top radius,
GP reconstruction z . q at the Gauss points of each face's radius (FOG: the
cell average), HLLC with S_L = min(u_L-c_L, u_R-c_R), S_R = max(u_L+c_L,
u_R+c_R), the flux difference of eq. fvm_F and SSP-RK3 (eq. rk3).
"""
from __future__ import annotations

import numpy as np
import torch

from . import gauss_rule, gp_weights, stencil

BC = {"periodic": 0, "outflow": 1, "reflect": 2, "dirichlet": 3}


def _prim_to_cons(P, gamma):
    r, u, v, p = P
    return [r, r * u, r * v, p / (gamma - 1.0) + 0.5 * r * (u * u + v * v)]


class FrozenStep:
    """Frozen-radius SSP-RK3 step of one 2D problem (dict from ``inputs``)."""

    def __init__(self, prob):
        self.p = prob
        self.nx, self.ny = int(prob["nx"]), int(prob["ny"])
        self.top = int(prob["cascade"][0])
        self.H = max(self.top + 1, 2)
        self.dx = (prob["x1"] - prob["x0"]) / self.nx
        self.dy = (prob["y1"] - prob["y0"]) / self.ny
        self.gamma = prob["gamma"]
        for s in prob["bc"]:
            if s not in BC:
                raise ValueError(f"boundary {s} not supported here")
        self.w = {}
        self.off = {}
        lx, ly = prob["ell"] / self.dx, prob["ell"] / self.dy
        for R in prob["cascade"]:
            if R == 0:
                continue
            self.w[R] = torch.tensor(gp_weights(2, R, lx, ly), dtype=torch.float64)
            self.off[R] = stencil(2, R)
        self.gw = {q: torch.tensor(gauss_rule(q)[1]) for q in (1, 2, 3, 4)}

    # ---- ghost cells: x pass over interior rows, then y pass over all columns
    def ghost(self, U):
        H, nx, ny, g = self.H, self.nx, self.ny, self.gamma
        bc = self.p["bc"]
        # x pass
        cols = []
        for k in range(H, 0, -1):  # west ghosts, outermost first
            cols.append(self._xghost(U, 0, k))
        west = torch.stack(cols, dim=2)
        cols = [self._xghost(U, 1, k) for k in range(1, H + 1)]
        east = torch.stack(cols, dim=2)
        Ux = torch.cat([west, U, east], dim=2)  # (4, ny, nx+2H)
        rows = [self._yghost(Ux, 0, k) for k in range(H, 0, -1)]
        south = torch.stack(rows, dim=1)
        rows = [self._yghost(Ux, 1, k) for k in range(1, H + 1)]
        north = torch.stack(rows, dim=1)
        return torch.cat([south, Ux, north], dim=1)  # (4, ny+2H, nx+2H)

    def _xghost(self, U, side, k):
        kind = BC[self.p["bc"][side]]
        nx = self.nx
        if kind == 3:
            S = _prim_to_cons(self.p["bc_prim"][side], self.gamma)
            return torch.stack([torch.full((self.ny,), float(s), dtype=U.dtype) for s in S])
        if kind == 0:
            src = (-k) % nx if side == 0 else (nx - 1 + k) % nx
        elif kind == 2:
            src = k - 1 if side == 0 else nx - k
        else:
            src = 0 if side == 0 else nx - 1
        col = U[:, :, src]
        if kind == 2:
            col = torch.stack([col[0], -col[1], col[2], col[3]])
        return col

    def _yghost(self, Ux, side, k):
        kind = BC[self.p["bc"][2 + side]]
        ny = self.ny
        if kind == 3:
            S = _prim_to_cons(self.p["bc_prim"][2 + side], self.gamma)
            return torch.stack([torch.full((Ux.shape[2],), float(s), dtype=Ux.dtype) for s in S])
        if kind == 0:
            src = (-k) % ny if side == 0 else (ny - 1 + k) % ny
        elif kind == 2:
            src = k - 1 if side == 0 else ny - k
        else:
            src = 0 if side == 0 else ny - 1
        row = Ux[:, src, :]
        if kind == 2:
            row = torch.stack([row[0], row[1], -row[2], row[3]])
        return row

    # ---- radii of possibly-ghost cells
    def _radius(self, ordm, i, j):
        """radii of cells (i, j) given as index arrays (may be ghosts)"""
        ii, jj = i.copy(), j.copy()
        top = np.full(i.shape, self.top, dtype=np.int64)
        px = self.p["bc"][0] == "periodic"
        py = self.p["bc"][2] == "periodic"
        outx = (ii < 0) | (ii >= self.nx)
        outy = (jj < 0) | (jj >= self.ny)
        ii = ii % self.nx
        jj = jj % self.ny
        r = ordm[jj, ii].astype(np.int64)
        r = np.where(outx & ~np.bool_(px), top, r)
        r = np.where(outy & ~np.bool_(py), top, r)
        return r

    def _hllc(self, UL, UR):
        g = self.gamma
        rL, rR = UL[0], UR[0]
        uL, vL = UL[1] / rL, UL[2] / rL
        uR, vR = UR[1] / rR, UR[2] / rR
        pL = (g - 1.0) * (UL[3] - 0.5 * (UL[1] * UL[1] + UL[2] * UL[2]) / rL)
        pR = (g - 1.0) * (UR[3] - 0.5 * (UR[1] * UR[1] + UR[2] * UR[2]) / rR)
        cL = torch.sqrt(g * pL / rL)
        cR = torch.sqrt(g * pR / rR)
        SL = torch.where(uL - cL < uR - cR, uL - cL, uR - cR)
        SR = torch.where(uL + cL > uR + cR, uL + cL, uR + cR)
        num = pR - pL + rL * uL * (SL - uL) - rR * uR * (SR - uR)
        den = rL * (SL - uL) - rR * (SR - uR)
        Ss = num / den
        FL = [rL * uL, rL * uL * uL + pL, rL * uL * vL, uL * (UL[3] + pL)]
        FR = [rR * uR, rR * uR * uR + pR, rR * uR * vR, uR * (UR[3] + pR)]
        # branches: S_L >= 0 -> F_L; else S* >= 0 -> F*_L; else S_R > 0 -> F*_R;
        # else F_R.  The star state is formed on the contact side K only, with
        # its denominators replaced by 1 where the star flux is not used (so
        # the unused branch contributes exact zeros to the gradient)
        left = Ss >= 0
        useL = SL >= 0
        useS = (~useL) & (left | (SR > 0))
        sel = lambda a, b: torch.where(left, a, b)
        r, u, v, E, p, S = sel(rL, rR), sel(uL, uR), sel(vL, vR), sel(UL[3], UR[3]), sel(pL, pR), sel(SL, SR)
        D = torch.where(useS, S - Ss, torch.ones_like(Ss))
        dS = torch.where(useS, S - u, torch.ones_like(Ss))
        f = r * dS / D
        Us = [f, f * Ss, f * v, f * (E / r + (Ss - u) * (Ss + p / (r * dS)))]
        out = []
        for k in range(4):
            FK = sel(FL[k], FR[k])
            UK = sel(UL[k], UR[k])
            Fs = FK + S * (Us[k] - UK)
            out.append(torch.where(useL, FL[k], torch.where(useS, Fs, FR[k])))
        return out

    def _recon(self, Xg, R, face, gi, ci, cj):
        """state of cells (ci, cj) at Gauss point gi of face (0 E, 1 W, 2 N, 3 S), radius R"""
        H = self.H
        if R == 0:
            return [Xg[v][cj + H, ci + H] for v in range(4)]
        z = self.w[R][face, gi]
        out = []
        for v in range(4):
            s = 0.0
            for m, (a, b) in enumerate(self.off[R]):
                s = s + z[m] * Xg[v][cj + b + H, ci + a + H]
            out.append(s)
        return out

    def residual(self, X, ordm):
        """F_nabla of the interior state X (4, ny, nx) at per-cell radii ordm."""
        nx, ny = self.nx, self.ny
        Xg = self.ghost(X)
        # x faces: between (i-1, j) and (i, j), i = 0..nx
        I, J = np.meshgrid(np.arange(nx + 1), np.arange(ny), indexing="xy")
        kf = np.minimum(self._radius(ordm, I - 1, J), self._radius(ordm, I, J))
        Fx = self._faces(Xg, kf, I - 1, J, I, J, 0)
        I, J = np.meshgrid(np.arange(nx), np.arange(ny + 1), indexing="xy")
        kf = np.minimum(self._radius(ordm, I, J - 1), self._radius(ordm, I, J))
        Fy = self._faces(Xg, kf, I, J - 1, I, J, 1)
        out = []
        for v in range(4):
            out.append((Fx[v][:, 1:] - Fx[v][:, :-1]) / self.dx + (Fy[v][1:, :] - Fy[v][:-1, :]) / self.dy)
        return torch.stack(out)

    def _faces(self, Xg, kf, iL, jL, iR, jR, d):
        """face-averaged fluxes; every face is reconstructed at its own radius
        only (no masked-out evaluations, which could be non-physical)"""
        shape = kf.shape
        F = [torch.zeros(shape, dtype=torch.float64) for _ in range(4)]
        for R in sorted(set(kf.ravel().tolist())):
            sel = np.nonzero(kf == R)
            q = 1 if R == 0 else R + 1
            acc = [0.0] * 4
            for gi in range(q):
                UL = self._recon(Xg, R, 0 if d == 0 else 2, gi, iL[sel], jL[sel])
                UR = self._recon(Xg, R, 1 if d == 0 else 3, gi, iR[sel], jR[sel])
                if d == 0:
                    f = self._hllc(UL, UR)
                else:
                    h = self._hllc([UL[0], UL[2], UL[1], UL[3]], [UR[0], UR[2], UR[1], UR[3]])
                    f = [h[0], h[2], h[1], h[3]]
                for v in range(4):
                    acc[v] = acc[v] + self.gw[q][gi] * f[v]
            idx = (torch.as_tensor(sel[0]), torch.as_tensor(sel[1]))
            for v in range(4):
                F[v] = F[v].index_put(idx, acc[v])
        return F

    def step(self, U, ords, dt):
        """One SSP-RK3 step with radii ords[s] (ny, nx) per stage and a given dt."""
        Y1 = U - dt * self.residual(U, ords[0])
        Y2 = Y1 - dt * self.residual(Y1, ords[1])
        X3 = 0.25 * (3.0 * U + Y2)
        Y3 = X3 - dt * self.residual(X3, ords[2])
        return (U + 2.0 * Y3) / 3.0
