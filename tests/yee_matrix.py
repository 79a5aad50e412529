"""Dense Yee operators assembled from grid positions alone (brute force for tiny cavities).

Nothing here restates the oracle's update loops.  Every unknown is identified by
its position on the doubled lattice (coordinates 2x, 2y, 2z): a point with one
odd coordinate carries the E component along that axis (an edge midpoint); a
point with two odd coordinates carries the H component along the remaining even
axis (a face centre); three odd coordinates is a cell centre and none is a node.
The curl of a field G at point q is, for each cyclic (a, b, c),

    (curl G)_a(q) = [G_c(q + e_b) - G_c(q - e_b)] - [G_b(q + e_c) - G_b(q - e_c)]

with one doubled-lattice step being half a cell, so each difference spans one
cell (dx = 1).  PEC: E points on a face tangential to it are not unknowns and
read as zero.

order=4 builds the fourth-order differences instead,
    c1 [G(q + e) - G(q - e)] + c2 [G(q + 3e) - G(q - 3e)],   c1 = 9/8, c2 = -1/24,
where a tap past a wall is the mirror point across it, with sign -1 for an E
point and +1 for an H point (tangential E odd, tangential H even about a PEC
wall); the divergences mirror normal components with the opposite parities.
"""
from __future__ import annotations

import itertools

import numpy as np

import cavity_inputs as ci

AXES = 3
CYCLIC = ((0, 1, 2), (1, 2, 0), (2, 0, 1))


C1_4, C2_4 = 9.0 / 8.0, -1.0 / 24.0


class YeeSpace:
    def __init__(self, nx: int, ny: int, nz: int, order: int = 2):
        self.n = (nx, ny, nz)
        self.taps = ((1, 1.0),) if order == 2 else ((1, C1_4), (3, C2_4))
        self.e_pts, self.h_pts = [], []
        lim = (2 * nx, 2 * ny, 2 * nz)
        for q in itertools.product(*(range(L + 1) for L in lim)):
            odd = [v % 2 for v in q]
            if sum(odd) == 1:
                a = odd.index(1)
                # tangential to a face: on a boundary plane of an axis other than a
                on_face = any(q[b] in (0, lim[b]) for b in range(AXES) if b != a)
                if not on_face:
                    self.e_pts.append(q)
            elif sum(odd) == 2:
                self.h_pts.append(q)
        self.e_idx = {q: n for n, q in enumerate(self.e_pts)}
        self.h_idx = {q: n for n, q in enumerate(self.h_pts)}
        self.lim = lim

    @staticmethod
    def comp_of(q) -> int:
        odd = [v % 2 for v in q]
        return odd.index(1) if sum(odd) == 1 else odd.index(0)

    def _inside(self, q):
        return all(0 <= q[a] <= self.lim[a] for a in range(AXES))

    def _mirror(self, p, axis, odd_sign):
        """The point p, with its coordinate along axis reflected into the box, and the image's sign."""
        p = list(p)
        if p[axis] < 0:
            p[axis] = -p[axis]
        elif p[axis] > self.lim[axis]:
            p[axis] = 2 * self.lim[axis] - p[axis]
        else:
            return tuple(p), 1.0
        assert self._inside(p), f"tap reaches more than one wall image at {p}"
        return tuple(p), odd_sign

    def _curl(self, rows, src_idx, src_is_e):
        strict = not src_is_e   # every H point exists; tangential E points on a face are not unknowns
        M = np.zeros((len(rows), len(src_idx)))
        for r, q in enumerate(rows):
            a = self.comp_of(q)
            for (aa, b, c) in CYCLIC:
                if aa != a:
                    continue
                for comp_axis, diff_axis, sign in ((c, b, +1.0), (b, c, -1.0)):
                    for dist, w in self.taps:
                        for step, s2 in ((+dist, +w), (-dist, -w)):
                            p = list(q)
                            p[diff_axis] += step
                            p = tuple(p)
                            if len(self.taps) == 1 and not self._inside(p):
                                raise AssertionError(f"stencil leaves the box at {p}")
                            # tangential E: odd image; tangential H: even image
                            p, img = self._mirror(p, diff_axis, -1.0 if src_is_e else 1.0)
                            assert self.comp_of(p) == comp_axis
                            col = src_idx.get(p)
                            if col is None:
                                if strict:
                                    raise AssertionError(f"missing unknown at {p}")
                                continue  # tangential PEC edge: E = 0
                            M[r, col] += sign * s2 * img
        return M

    def curl_e(self):
        """(H points) x (E unknowns): curl E evaluated at every H point."""
        return self._curl(self.h_pts, self.e_idx, src_is_e=True)

    def curl_h(self):
        """(E unknowns) x (H points): curl H evaluated at every interior E point."""
        return self._curl(self.e_pts, self.h_idx, src_is_e=False)

    def div_nodes(self):
        """Interior nodes x E unknowns: sum_a E_a(q + e_a) - E_a(q - e_a)."""
        nodes = [q for q in itertools.product(*(range(L + 1) for L in self.lim))
                 if all(v % 2 == 0 for v in q) and all(0 < q[a] < self.lim[a] for a in range(AXES))]
        D = np.zeros((len(nodes), len(self.e_pts)))
        for r, q in enumerate(nodes):
            for a in range(AXES):
                for dist, w in self.taps:
                    for step, s in ((+dist, w), (-dist, -w)):
                        p = list(q); p[a] += step
                        p, img = self._mirror(p, a, 1.0)    # normal E: even image
                        D[r, self.e_idx[p]] += s * img
        return D

    def div_cells(self):
        """Cells x H points: sum_a H_a(q + e_a) - H_a(q - e_a)."""
        cells = [q for q in itertools.product(*(range(L + 1) for L in self.lim)) if all(v % 2 == 1 for v in q)]
        D = np.zeros((len(cells), len(self.h_pts)))
        for r, q in enumerate(cells):
            for a in range(AXES):
                for dist, w in self.taps:
                    for step, s in ((+dist, w), (-dist, -w)):
                        p = list(q); p[a] += step
                        p, img = self._mirror(p, a, -1.0)   # normal H: odd image
                        D[r, self.h_idx[p]] += s * img
        return D

    # --- mapping between unknown vectors and canonical (nz+1, ny+1, nx+1) arrays ---
    @staticmethod
    def canon_index(q):
        # canonical index (i, j, k) of the point: floor of the half-cell coordinate
        return q[0] // 2, q[1] // 2, q[2] // 2

    def gather(self, fields, pts, offset):
        v = np.zeros(len(pts))
        for n, q in enumerate(pts):
            i, j, k = self.canon_index(q)
            v[n] = fields[offset + self.comp_of(q)][k, j, i]
        return v

    def scatter(self, v, fields, pts, offset):
        for n, q in enumerate(pts):
            i, j, k = self.canon_index(q)
            fields[offset + self.comp_of(q)][k, j, i] = v[n]

    def diag(self, coef3, pts):
        d = np.zeros(len(pts))
        for n, q in enumerate(pts):
            i, j, k = self.canon_index(q)
            d[n] = coef3[self.comp_of(q)][k, j, i]
        return d


def one_step_matrix(space: YeeSpace, ce3, ch3):
    """Dense M acting on x = [H; E]: H' = H - Ch CE E; E' = E + Ce CH H'."""
    CE, CH = space.curl_e(), space.curl_h()
    Ch = np.diag(space.diag(ch3, space.h_pts))
    Ce = np.diag(space.diag(ce3, space.e_pts))
    nh, ne = len(space.h_pts), len(space.e_pts)
    A = np.block([[np.eye(nh), -Ch @ CE], [np.zeros((ne, nh)), np.eye(ne)]])   # H half-step
    B = np.block([[np.eye(nh), np.zeros((nh, ne))], [Ce @ CH, np.eye(ne)]])    # E half-step
    return B @ A, CE, CH


def sigma(m, n, order=2):
    """Symbol of the staggered difference on the standing wave sin(pi m x / n): D -> 2 sigma."""
    if order == 2:
        return np.sin(np.pi * m / (2 * n))
    return C1_4 * np.sin(np.pi * m / (2 * n)) + C2_4 * np.sin(3 * np.pi * m / (2 * n))


def mode_frequencies(nx, ny, nz, ce, ch, dt, order=2):
    """omega*dt of every discrete cavity mode, with TE/TM multiplicity."""
    out = []
    for m, n, p in itertools.product(range(nx), range(ny), range(nz)):
        nz_count = (m > 0) + (n > 0) + (p > 0)
        if nz_count < 2:
            continue
        s = sigma(m, nx, order) ** 2 + sigma(n, ny, order) ** 2 + sigma(p, nz, order) ** 2
        w = 2.0 * np.arcsin(np.sqrt(ce * ch * s))
        out += [w] * (2 if nz_count == 3 else 1)
    return np.sort(np.array(out))
