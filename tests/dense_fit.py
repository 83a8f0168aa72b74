"""Dense brute-force FIT operators for tiny grids (test helper).

Independent of the oracle's stencil code: the discrete gradient G, curl C and
divergence S are built from their combinatorial definitions (Sec. II, eqs.
maxwell_grid1-2) -- oriented edges between points, faces bounded by
counter-clockwise vertex loops, cells bounded by outward faces -- over the
full canonical index space (component a of point q at a*Np + P(q)).

The degrees of freedom are chosen geometrically: an edge or face that lies
in a wall of the box is not one (PEC: tangential e = 0, normal b = 0).
"""
from __future__ import annotations

import itertools

import numpy as np


class DenseFIT:
    def __init__(self, dims):
        self.n = tuple(int(v) for v in dims)
        nx, ny, nz = self.n
        self.Np = (nx + 1) * (ny + 1) * (nz + 1)
        self.N = 3 * self.Np
        self._build()

    def pidx(self, q):
        nx, ny, _ = self.n
        return q[0] + (nx + 1) * (q[1] + (ny + 1) * q[2])

    def _points(self):
        nx, ny, nz = self.n
        return itertools.product(range(nx + 1), range(ny + 1), range(nz + 1))

    def _in_box(self, q):
        return all(0 <= q[t] <= self.n[t] for t in range(3))

    def _on_wall(self, verts):
        """True when all vertices share one wall plane of the box."""
        for t in range(3):
            for side in (0, self.n[t]):
                if all(v[t] == side for v in verts):
                    return True
        return False

    def _edge_of(self, v, w):
        """Edge index and orientation sign for the segment v -> w."""
        diff = [w[t] - v[t] for t in range(3)]
        axis = [t for t in range(3) if diff[t] != 0]
        assert len(axis) == 1 and abs(diff[axis[0]]) == 1
        a = axis[0]
        start = v if diff[a] > 0 else w
        return a * self.Np + self.pidx(start), (1 if diff[a] > 0 else -1)

    def _build(self):
        N, Np = self.N, self.Np
        unit = [(1, 0, 0), (0, 1, 0), (0, 0, 1)]
        add = lambda q, u, s=1: tuple(q[t] + s * u[t] for t in range(3))
        self.G = np.zeros((N, Np))          # edges x points
        self.C = np.zeros((N, N))           # faces x edges
        self.S = np.zeros((Np, N))          # cells x faces (cell index = its lowest point)
        self.edge_exists = np.zeros(N, bool)
        self.face_exists = np.zeros(N, bool)
        self.edge_dof = np.zeros(N, bool)
        self.face_dof = np.zeros(N, bool)
        self.cell_exists = np.zeros(Np, bool)
        self.node_interior = np.zeros(Np, bool)
        for q in self._points():
            p = self.pidx(q)
            self.node_interior[p] = all(0 < q[t] < self.n[t] for t in range(3))
            for a in range(3):
                # edge q -> q + u_a
                w = add(q, unit[a])
                if self._in_box(w):
                    r = a * Np + p
                    self.edge_exists[r] = True
                    self.edge_dof[r] = not self._on_wall([q, w])
                    self.G[r, self.pidx(q)] -= 1.0
                    self.G[r, self.pidx(w)] += 1.0
                # face normal a with corner q: loop q, q+u_b, q+u_b+u_c, q+u_c
                b, c = (a + 1) % 3, (a + 2) % 3
                loop = [q, add(q, unit[b]), add(add(q, unit[b]), unit[c]), add(q, unit[c])]
                if all(self._in_box(v) for v in loop):
                    r = a * Np + p
                    self.face_exists[r] = True
                    self.face_dof[r] = not self._on_wall(loop)
                    for s in range(4):
                        col, sign = self._edge_of(loop[s], loop[(s + 1) % 4])
                        self.C[r, col] += sign
            # cell with lowest corner q: outward faces
            top = add(q, (1, 1, 1))
            if self._in_box(top):
                self.cell_exists[p] = True
                for a in range(3):
                    self.S[p, a * Np + p] -= 1.0
                    self.S[p, a * Np + self.pidx(add(q, unit[a]))] += 1.0

    # ---- one leapfrog step as a dense matrix over the dofs ----
    def propagator(self, ca, cb, ch):
        """Dense one-step map of (e^n, h^{n-1/2}) -> (e^{n+1}, h^{n+1/2}),
        restricted to the degrees of freedom.  ca, cb, ch: flat length-N."""
        ie = np.flatnonzero(self.edge_dof)
        ih = np.flatnonzero(self.face_dof)
        Cr = self.C[np.ix_(ih, ie)]                  # faces(dof) x edges(dof)
        A = np.diag(ca[ie])
        B = np.diag(cb[ie])
        Dh = np.diag(ch[ih])
        top = np.hstack([A - B @ Cr.T @ Dh @ Cr, B @ Cr.T])
        bot = np.hstack([-Dh @ Cr, np.eye(len(ih))])
        return np.vstack([top, bot]), ie, ih
