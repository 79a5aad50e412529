"""Multi-rank host logic on CPU ranks (gloo, world size 2, 127.0.0.1).

1. The bench's N > 1 aggregation: every rank's units over the slowest rank's time.
2. z-slab domain decomposition (the multi-GPU design for one cavity): each rank steps its own planes
   in FP64 and exchanges one ghost plane per half step (E at its upper face before the H update, H at its
   lower face before the E update); gathered, the result equals the single-domain restatement bit for
   bit and the oracle to rounding.
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
