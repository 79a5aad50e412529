"""Multi-rank host logic on CPU ranks (gloo, world size 2, 127.0.0.1).

1. The bench's N > 1 aggregation: every rank's units over the slowest rank's time.
2. z-slab domain decomposition (the multi-GPU design for one cavity): each rank steps its own planes
   in FP64 and exchanges one ghost plane per half step (E at its upper face before the H update, H at its
   lower face before the E update); gathered, the result equals the single-domain restatement bit for
   bit and the oracle to rounding.
3. The same for the fourth-order scheme: two ghost planes per side (E: two above, one below before the H
   update; H: two below, one above before the E update), wall images along x, y and at the global z walls;
   gathered, equal to the one-slab restatement bit for bit and to the oracle's step4 to rounding.
4. Temporal blocking across ranks (T = 2): two ghost planes of all six fields per side, exchanged once per
   two steps, both steps then taken locally; gathered, equal to the single-domain restatement bit for bit,
   and dropping one exchange shows.
"""
import os
import socket

import numpy as np
import pytest

import cavity_inputs as ci

WORLD = 2


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run(fn, *args):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_entry, args=(fn, port) + args, nprocs=WORLD, join=True)


def _entry(rank, fn, port, *args):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(WORLD),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        fn(rank, *args)
    finally:
        dist.destroy_process_group()


# ------------------------------------------------------------------ 1. bench aggregation
def _agg(rank, out_dir):
    import bench
    ws, r, local = bench.dist_env()
    assert (ws, r, local) == (WORLD, rank, rank)
    t = bench.max_over_ranks(10.0 + 3.0 * rank, ws)       # rank 1 is the slow one
    rate = bench.job_rate(1000.0, ws, t)
    np.save(os.path.join(out_dir, f"agg{rank}.npy"), np.array([t, rate]))


def test_bench_max_over_ranks_and_job_rate(tmp_path):
    _run(_agg, str(tmp_path))
    for rank in range(WORLD):
        t, rate = np.load(tmp_path / f"agg{rank}.npy")
        assert t == 13.0 and rate == pytest.approx(2000.0 / 13.0)


# ------------------------------------------------------------------ 2. z-slab decomposition
def _owned(nz, rank):
    """Cell planes [k0, k1) of a rank (the last rank also owns the node plane nz)."""
    b = [nz * q // WORLD for q in range(WORLD + 1)]
    return b[rank], b[rank + 1]


def _slab_step(loc, ce, ch, k0, k1, nz, rank):
    """One leapfrog step on a slab.  `loc` holds planes k0-1 .. k1 (local index k - k0 + 1) of the six
    canonical arrays; ce/ch hold the same planes.  Plane arithmetic follows the whole-array restatement
    of Eq. 2 (Listing 3 style), restricted to owned planes."""
    import torch.distributed as dist
    Ex, Ey, Ez, Hx, Hy, Hz = loc
    cex, cey, cez = ce
    chx, chy, chz = ch
    ny, nx = Ex.shape[1] - 1, Ex.shape[2] - 1

    def L(k):   # local plane index
        return k - k0 + 1

    last = rank == WORLD - 1
    # E at plane k1 (upper ghost) for the H update: from the next rank's first owned plane
    if rank + 1 < WORLD:
        recv = np.empty((2,) + Ex.shape[1:])
        dist_recv(recv, rank + 1)
    if rank > 0:
        dist_send(np.stack([Ex[L(k0)], Ey[L(k0)]]), rank - 1)
    if rank + 1 < WORLD:
        Ex[L(k1)], Ey[L(k1)] = recv[0], recv[1]
    s = np.s_
    kc = s[L(k0):L(k1)]                      # owned cell planes (Hx, Hy, Ez)
    kn = s[L(k0):L(k1) + (1 if last else 0)]  # owned node planes (Hz, Ex, Ey)
    up = s[L(k0) + 1:L(k1) + 1]
    Hx[kc, :ny, :] -= chx[kc, :ny, :] * ((Ez[kc, 1:, :] - Ez[kc, :ny, :]) - (Ey[up, :ny, :] - Ey[kc, :ny, :]))
    Hy[kc, :, :nx] -= chy[kc, :, :nx] * ((Ex[up, :, :nx] - Ex[kc, :, :nx]) - (Ez[kc, :, 1:] - Ez[kc, :, :nx]))
    Hz[kn, :ny, :nx] -= chz[kn, :ny, :nx] * ((Ey[kn, :ny, 1:] - Ey[kn, :ny, :nx]) - (Ex[kn, 1:, :nx] - Ex[kn, :ny, :nx]))
    # H at plane k0-1 (lower ghost) for the E update: from the previous rank's last owned plane
    if rank > 0:
        recv = np.empty((2,) + Hx.shape[1:])
        dist_recv(recv, rank - 1)
    if rank + 1 < WORLD:
        dist_send(np.stack([Hx[L(k1 - 1)], Hy[L(k1 - 1)]]), rank + 1)
    if rank > 0:
        Hx[L(k0 - 1)], Hy[L(k0 - 1)] = recv[0], recv[1]
    # interior Ex, Ey planes 1 .. nz-1 that this rank owns: [max(k0, 1), k1)
    e_lo, e_hi = max(k0, 1), k1
    ke = s[L(e_lo):L(e_hi)]
    dn = s[L(e_lo) - 1:L(e_hi) - 1]
    Ex[ke, 1:ny, :nx] += cex[ke, 1:ny, :nx] * ((Hz[ke, 1:ny, :nx] - Hz[ke, :ny - 1, :nx]) - (Hy[ke, 1:ny, :nx] - Hy[dn, 1:ny, :nx]))
    Ey[ke, :ny, 1:nx] += cey[ke, :ny, 1:nx] * ((Hx[ke, :ny, 1:nx] - Hx[dn, :ny, 1:nx]) - (Hz[ke, :ny, 1:nx] - Hz[ke, :ny, :nx - 1]))
    kz = s[L(k0):L(k1)]
    Ez[kz, 1:ny, 1:nx] += cez[kz, 1:ny, 1:nx] * ((Hy[kz, 1:ny, 1:nx] - Hy[kz, 1:ny, :nx - 1]) - (Hx[kz, 1:ny, 1:nx] - Hx[kz, :ny - 1, 1:nx]))


def dist_send(a, dst):
    import torch
    import torch.distributed as dist
    dist.send(torch.from_numpy(np.ascontiguousarray(a)), dst)


def dist_recv(a, src):
    import torch
    import torch.distributed as dist
    t = torch.from_numpy(a)
    dist.recv(t, src)


def _slabs(rank, dims, steps, seed, out_dir):
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    sh = (nz + 1, ny + 1, nx + 1)
    ce = [rng.uniform(0.2, 0.28, sh) for _ in range(3)]
    ch = [rng.uniform(0.2, 0.28, sh) for _ in range(3)]
    f = [np.asarray(a, np.float64) for a in ci.random_fields(seed, nx, ny, nz)]
    k0, k1 = _owned(nz, rank)
    lo, hi = k0 - 1, k1 + 1                  # local planes, one ghost on each side (clipped at 0 / nz)

    def cut(a):
        out = np.zeros((hi - lo + 1,) + a.shape[1:])
        a_lo, a_hi = max(lo, 0), min(hi, nz)
        out[a_lo - lo:a_hi - lo + 1] = a[a_lo:a_hi + 1]
        return out
    loc = [cut(a) for a in f]
    lce = [cut(a) for a in ce]
    lch = [cut(a) for a in ch]
    for _ in range(steps):
        _slab_step(loc, lce, lch, k0, k1, nz, rank)
    own_hi = k1 + (1 if rank == WORLD - 1 else 0)
    np.save(os.path.join(out_dir, f"slab{rank}.npy"),
            np.stack([a[k0 - lo:own_hi - lo] for a in loc]))


@pytest.mark.parametrize("dims,steps", [((9, 7, 10), 6), ((6, 11, 5), 9)])
def test_zslab_decomposition_matches_single_domain(tmp_path, dims, steps):
    import oracle
    from tests.test_oracle_pins import numpy_step
    nx, ny, nz = dims
    seed = 5
    _run(_slabs, dims, steps, seed, str(tmp_path))
    parts = [np.load(tmp_path / f"slab{r}.npy") for r in range(WORLD)]
    got = np.concatenate(parts, axis=1)      # [component, k, j, i]
    rng = np.random.default_rng(seed)
    sh = (nz + 1, ny + 1, nx + 1)
    ce = [rng.uniform(0.2, 0.28, sh) for _ in range(3)]
    ch = [rng.uniform(0.2, 0.28, sh) for _ in range(3)]
    f = [np.asarray(a, np.float64) for a in ci.random_fields(seed, nx, ny, nz)]
    ref = [a.copy() for a in f]
    for _ in range(steps):
        numpy_step(ref, ce, ch)
    orc = oracle.as_f64(ci.random_fields(seed, nx, ny, nz))
    oracle.step(orc, ce, ch, steps)
    for c, name in enumerate(ci.COMPONENTS):
        m = ci.extent_mask(name, nx, ny, nz)
        assert np.array_equal(got[c][m], ref[c][m]), name
        assert np.max(np.abs(got[c][m] - orc[c][m])) <= 1e-13, name


# ------------------------------------------------------------------ 3. z-slabs for the fourth-order scheme
# The (2,4) differences reach two positions: H at plane m reads E at planes m-1 .. m+2, E at plane k reads
# H at planes k-2 .. k+1.  A slab therefore keeps two ghost planes on each side; before the H update it
# receives E at its two planes above from the next rank (or takes the odd image about the wall at nz), and
# before the E update H at its two planes below from the previous rank (or the even image about the wall at
# 0).  Along x and y, taps past a wall are the images as well.  Written here as a ghost-cell restatement:
# one slab covering every plane is the single-domain scheme, which the oracle's step4 must match.
C1, C2 = 9.0 / 8.0, -1.0 / 24.0


def _ext(a, axis, n, odd):
    """a extended by two image layers on each side along axis: index q of the result is q - 2.
    odd: node-aligned (0..n, zero on both walls) with odd images; else half-aligned (0..n-1), even images."""
    t = lambda q: np.take(a, [q], axis=axis)
    if odd:
        parts = [-t(2), -t(1), np.take(a, range(n + 1), axis=axis), -t(n - 1), -t(n - 2)]
    else:
        parts = [t(1), t(0), np.take(a, range(n), axis=axis), t(n - 1), t(n - 2)]
    return np.concatenate(parts, axis=axis)


def _d4(a, axis, lo_tap, count):
    """c1 (a[p+1] - a[p]) + c2 (a[p+2] - a[p-1]) for p = lo_tap .. lo_tap + count - 1 along axis."""
    g = lambda o: np.take(a, range(lo_tap + o, lo_tap + o + count), axis=axis)
    return C1 * (g(1) - g(0)) + C2 * (g(2) - g(-1))


def _swap(rank, world, up, down):
    """Send `up` to rank + 1 and `down` to rank - 1; return (what rank - 1 sent up, what rank + 1 sent
    down), None at the ends.  Non-blocking pairs, so any world size works."""
    import torch
    import torch.distributed as dist
    ops, from_below, from_above = [], None, None
    if rank > 0:
        from_below = torch.empty(up.shape, dtype=torch.float64)
        ops += [dist.irecv(from_below, rank - 1), dist.isend(torch.from_numpy(np.ascontiguousarray(down)), rank - 1)]
    if rank + 1 < world:
        from_above = torch.empty(down.shape, dtype=torch.float64)
        ops += [dist.irecv(from_above, rank + 1), dist.isend(torch.from_numpy(np.ascontiguousarray(up)), rank + 1)]
    for op in ops:
        op.wait()
    return (None if from_below is None else from_below.numpy()), (None if from_above is None else from_above.numpy())


def _step4_slab(loc, ce, ch, k0, k1, nz, rank, world):
    """One (2,4) step on a slab whose arrays hold planes k0-2 .. k1+2 (local index k - k0 + 2).  Owned
    planes: [k0, k1) (the last rank also the node plane nz); each rank owns at least two.  Canonical
    [k, j, i] arrays.  With world == 1 the slab is the whole cavity (images on both z walls)."""
    Ex, Ey, Ez, Hx, Hy, Hz = loc
    ny, nx = Ex.shape[1] - 1, Ex.shape[2] - 1
    L = lambda k: k - k0 + 2
    first, last = rank == 0, rank == world - 1
    # ---- E ghost planes: k0 - 1 below, k1 and k1 + 1 above
    if world > 1:
        below, above = _swap(rank, world, np.stack([Ex[L(k1) - 1:L(k1)], Ey[L(k1) - 1:L(k1)]]),
                             np.stack([Ex[L(k0):L(k0) + 2], Ey[L(k0):L(k0) + 2]]))
        if below is not None:
            Ex[L(k0) - 1], Ey[L(k0) - 1] = below[0, 0], below[1, 0]
        if above is not None:
            Ex[L(k1):L(k1) + 2], Ey[L(k1):L(k1) + 2] = above[0], above[1]
    if first:   # odd images about the wall at 0: E(-1) = -E(1), E(-2) = -E(2)
        for a in (Ex, Ey):
            a[L(-1)], a[L(-2)] = -a[L(1)], -a[L(2)]
    if last:    # E(nz) = 0 (tangential), E(nz + 1) = -E(nz - 1)
        for a in (Ex, Ey):
            a[L(nz)], a[L(nz) + 1] = 0.0, -a[L(nz) - 1]
    kc = slice(L(k0), L(k1))                       # owned cell planes (Hx, Hy, Ez)
    kn = slice(L(k0), L(k1) + (1 if last else 0))  # owned node planes (Hz)
    ncz = L(k1) - L(k0)
    dyEz = _d4(_ext(Ez[kc], 1, ny, True), 1, 2, ny)
    dzEy = _d4(Ey, 0, L(k0), ncz)[:, :ny, :]
    Hx[kc, :ny, :] -= ch[0][kc, :ny, :] * (dyEz - dzEy)
    dzEx = _d4(Ex, 0, L(k0), ncz)[:, :, :nx]
    dxEz = _d4(_ext(Ez[kc], 2, nx, True), 2, 2, nx)
    Hy[kc, :, :nx] -= ch[1][kc, :, :nx] * (dzEx - dxEz)
    dxEy = _d4(_ext(Ey[kn, :ny, :], 2, nx, True), 2, 2, nx)
    dyEx = _d4(_ext(Ex[kn, :, :nx], 1, ny, True), 1, 2, ny)
    Hz[kn, :ny, :nx] -= ch[2][kn, :ny, :nx] * (dxEy - dyEx)
    # ---- H ghost planes: k0 - 2 and k0 - 1 below, k1 above
    if world > 1:
        below, above = _swap(rank, world, np.stack([Hx[L(k1) - 2:L(k1)], Hy[L(k1) - 2:L(k1)]]),
                             np.stack([Hx[L(k0):L(k0) + 1], Hy[L(k0):L(k0) + 1]]))
        if below is not None:
            Hx[L(k0) - 2:L(k0)], Hy[L(k0) - 2:L(k0)] = below[0], below[1]
        if above is not None:
            Hx[L(k1)], Hy[L(k1)] = above[0, 0], above[1, 0]
    if first:   # even images about the wall at 0: H(-1) = H(0), H(-2) = H(1)
        for a in (Hx, Hy):
            a[L(-1)], a[L(-2)] = a[L(0)], a[L(1)]
    if last:    # H(nz) = H(nz - 1)
        for a in (Hx, Hy):
            a[L(nz)] = a[L(nz) - 1]
    # ---- E update on non-tangential entries: D of H at node k uses planes k-2 .. k+1 (taps p-1 .. p+2
    # with p = k - 1), in x and y the extended arrays (index q + 2) with p = i + 1
    e_lo = max(k0, 1)
    ke = slice(L(e_lo), L(k1))
    nke = L(k1) - L(e_lo)
    if nke > 0:
        dyHz = _d4(_ext(Hz[ke, :ny, :nx], 1, ny, False), 1, 1, ny + 1)[:, 1:ny, :]
        dzHy = _d4(Hy, 0, L(e_lo) - 1, nke)[:, 1:ny, :nx]
        Ex[ke, 1:ny, :nx] += ce[0][ke, 1:ny, :nx] * (dyHz - dzHy)
        dzHx = _d4(Hx, 0, L(e_lo) - 1, nke)[:, :ny, 1:nx]
        dxHz = _d4(_ext(Hz[ke, :ny, :nx], 2, nx, False), 2, 1, nx + 1)[:, :, 1:nx]
        Ey[ke, :ny, 1:nx] += ce[1][ke, :ny, 1:nx] * (dzHx - dxHz)
    kz = slice(L(k0), L(k1))
    dxHy = _d4(_ext(Hy[kz, :, :nx], 2, nx, False), 2, 1, nx + 1)[:, 1:ny, 1:nx]
    dyHx = _d4(_ext(Hx[kz, :ny, :], 1, ny, False), 1, 1, ny + 1)[:, 1:ny, 1:nx]
    Ez[kz, 1:ny, 1:nx] += ce[2][kz, 1:ny, 1:nx] * (dxHy - dyHx)


def _slabs4(rank, dims, steps, seed, out_dir, world=WORLD):
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    sh = (nz + 1, ny + 1, nx + 1)
    ce = [rng.uniform(0.2, 0.28, sh) for _ in range(3)]
    ch = [rng.uniform(0.2, 0.28, sh) for _ in range(3)]
    f = [np.asarray(a, np.float64) for a in ci.random_fields(seed, nx, ny, nz)]
    b = [nz * q // world for q in range(world + 1)]
    k0, k1 = b[rank], b[rank + 1]
    lo, hi = k0 - 2, k1 + 2

    def cut(a):
        out = np.zeros((hi - lo + 1,) + a.shape[1:])
        a_lo, a_hi = max(lo, 0), min(hi, nz)
        out[a_lo - lo:a_hi - lo + 1] = a[a_lo:a_hi + 1]
        return out
    loc = [cut(a) for a in f]
    lce = [cut(a) for a in ce]
    lch = [cut(a) for a in ch]
    for _ in range(steps):
        _step4_slab(loc, lce, lch, k0, k1, nz, rank, world)
    own_hi = k1 + (1 if rank == world - 1 else 0)
    out = np.stack([a[k0 - lo:own_hi - lo] for a in loc])
    if out_dir is None:
        return out
    np.save(os.path.join(out_dir, f"slab4_{rank}.npy"), out)


@pytest.mark.parametrize("dims,steps", [((9, 7, 10), 6), ((6, 11, 7), 9)])
def test_zslab_fourth_order_matches_single_domain_and_oracle(tmp_path, dims, steps):
    import oracle
    nx, ny, nz = dims
    seed = 7
    _run(_slabs4, dims, steps, seed, str(tmp_path))
    got = np.concatenate([np.load(tmp_path / f"slab4_{r}.npy") for r in range(WORLD)], axis=1)
    whole = _slabs4(0, dims, steps, seed, None, world=1)   # one slab: the single-domain restatement
    rng = np.random.default_rng(seed)
    sh = (nz + 1, ny + 1, nx + 1)
    ce = [rng.uniform(0.2, 0.28, sh) for _ in range(3)]
    ch = [rng.uniform(0.2, 0.28, sh) for _ in range(3)]
    orc = oracle.as_f64(ci.random_fields(seed, nx, ny, nz))
    oracle.step4(orc, ce, ch, steps)
    for c, name in enumerate(ci.COMPONENTS):
        m = ci.extent_mask(name, nx, ny, nz)
        assert np.array_equal(got[c][m], whole[c][m]), name
        assert np.max(np.abs(got[c][m] - orc[c][m])) <= 1e-13, name


# ------------------------------------------------------------------ 4. z-slabs with temporal blocking (T = 2)
# The two-step kernel's counterpart across ranks: each rank keeps two ghost planes of all six fields on each
# side, exchanges them once per two steps, and then takes both steps locally, recomputing the ghost planes
# it needs (their outermost values go stale, which the owned planes never read: two steps reach two planes).
def _local_step(loc, ce, ch, g0, nz):
    """One step on local planes 0 .. P-1 (global g0 + p), each value updated wherever the local arrays
    hold its inputs; E on the global z walls and cell-centred components at the node plane nz are never
    written.  Per value the arithmetic of the whole-array restatement of Eq. 2."""
    Ex, Ey, Ez, Hx, Hy, Hz = loc
    cex, cey, cez = ce
    chx, chy, chz = ch
    P = Ex.shape[0]
    ny, nx = Ex.shape[1] - 1, Ex.shape[2] - 1
    cell = [p for p in range(P) if g0 + p < nz]                          # Hx, Hy, Ez planes that exist
    hc = np.array([p for p in cell if p + 1 < P], int)                  # Hx, Hy: need E at p + 1
    Hx[hc, :ny, :] -= chx[hc, :ny, :] * ((Ez[hc, 1:, :] - Ez[hc, :ny, :]) - (Ey[hc + 1, :ny, :] - Ey[hc, :ny, :]))
    Hy[hc, :, :nx] -= chy[hc, :, :nx] * ((Ex[hc + 1, :, :nx] - Ex[hc, :, :nx]) - (Ez[hc, :, 1:] - Ez[hc, :, :nx]))
    Hz[:, :ny, :nx] -= chz[:, :ny, :nx] * ((Ey[:, :ny, 1:] - Ey[:, :ny, :nx]) - (Ex[:, 1:, :nx] - Ex[:, :ny, :nx]))
    en = np.array([p for p in range(1, P) if 0 < g0 + p < nz], int)     # Ex, Ey: need H at p - 1; not walls
    Ex[en, 1:ny, :nx] += cex[en, 1:ny, :nx] * ((Hz[en, 1:ny, :nx] - Hz[en, :ny - 1, :nx]) - (Hy[en, 1:ny, :nx] - Hy[en - 1, 1:ny, :nx]))
    Ey[en, :ny, 1:nx] += cey[en, :ny, 1:nx] * ((Hx[en, :ny, 1:nx] - Hx[en - 1, :ny, 1:nx]) - (Hz[en, :ny, 1:nx] - Hz[en, :ny, :nx - 1]))
    ez = np.array(cell, int)
    Ez[ez, 1:ny, 1:nx] += cez[ez, 1:ny, 1:nx] * ((Hy[ez, 1:ny, 1:nx] - Hy[ez, 1:ny, :nx - 1]) - (Hx[ez, 1:ny, 1:nx] - Hx[ez, :ny - 1, 1:nx]))


def _slabs_t2(rank, dims, pairs, seed, out_dir, skip_pair):
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    sh = (nz + 1, ny + 1, nx + 1)
    ce = [rng.uniform(0.2, 0.28, sh) for _ in range(3)]
    ch = [rng.uniform(0.2, 0.28, sh) for _ in range(3)]
    f = [np.asarray(a, np.float64) for a in ci.random_fields(seed, nx, ny, nz)]
    k0, k1 = _owned(nz, rank)
    own_hi = k1 + (1 if rank == WORLD - 1 else 0)      # owned planes [k0, own_hi)
    lo, hi = max(k0 - 2, 0), min(own_hi + 1, nz)        # local planes lo .. hi
    loc = [a[lo:hi + 1].copy() for a in f]
    lce = [a[lo:hi + 1] for a in ce]
    lch = [a[lo:hi + 1] for a in ch]
    exchanges = 0
    for pair in range(pairs):
        if pair != skip_pair:
            # two owned planes go to each neighbour: the first two down, the last two up
            up = np.stack([a[k1 - 2 - lo:k1 - lo] for a in loc])
            down = np.stack([a[k0 - lo:k0 + 2 - lo] for a in loc])
            below, above = _swap(rank, WORLD, up, down)
            if below is not None:
                for a, b in zip(loc, below):
                    a[k0 - 2 - lo:k0 - lo] = b
            if above is not None:
                for a, b in zip(loc, above):
                    a[k1 - lo:hi + 1 - lo] = b[:hi + 1 - k1]
            exchanges += 1
        _local_step(loc, lce, lch, lo, nz)
        _local_step(loc, lce, lch, lo, nz)
    np.save(os.path.join(out_dir, f"t2slab{rank}.npy"), np.stack([a[k0 - lo:own_hi - lo] for a in loc]))
    assert exchanges == pairs - (1 if 0 <= skip_pair < pairs else 0)


@pytest.mark.parametrize("dims,pairs", [((9, 7, 10), 3), ((6, 11, 9), 5)])
def test_zslab_two_step_halo_matches_single_domain(tmp_path, dims, pairs):
    from tests.test_oracle_pins import numpy_step
    nx, ny, nz = dims
    seed = 8
    rng = np.random.default_rng(seed)
    sh = (nz + 1, ny + 1, nx + 1)
    ce = [rng.uniform(0.2, 0.28, sh) for _ in range(3)]
    ch = [rng.uniform(0.2, 0.28, sh) for _ in range(3)]
    ref = [np.asarray(a, np.float64) for a in ci.random_fields(seed, nx, ny, nz)]
    for _ in range(2 * pairs):
        numpy_step(ref, ce, ch)
    for skip in (-1, 1):      # -1: every exchange; 1: the second pair's exchange dropped, which must show
        _run(_slabs_t2, dims, pairs, seed, str(tmp_path), skip)
        got = np.concatenate([np.load(tmp_path / f"t2slab{r}.npy") for r in range(WORLD)], axis=1)
        same = all(np.array_equal(got[c][ci.extent_mask(n, nx, ny, nz)], ref[c][ci.extent_mask(n, nx, ny, nz)])
                   for c, n in enumerate(ci.COMPONENTS))
        assert same == (skip < 0)
